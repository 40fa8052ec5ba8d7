// Discrete adjoint of one FP64 ADER-DG step (predictor + corrector).
//
// The forward step is u' = u + dt (rvol(u) - lift(F*(traces(u)))), with the
// predictor (Picard sweeps, Sec. 3) local to each cell and the corrector
// coupling neighbours through the face traces.  Given lam' = dJ/du', the
// adjoint returns lam = dJ/du = lam' + (d(rvol, traces)/du)^T (rvol_bar,
// trace_bar), in two kernels:
//
//  k_corrector_adj_fp64  per cell and face: the adjoint of the face flux F*
//      (lift rows of both cells sharing the face), then of the Rusanov-type
//      flux and, on walls, of the ghost state, giving trace_bar of the cell's
//      own traces (no scatter: each face record belongs to one cell).
//  k_predictor_adj_fp64  per cell: recompute the Picard iterates q^(0..n)
//      into shared memory, then run the predictor backwards: face
//      extrapolation and wave speed, weak volume residual, time averages and
//      final evaluation, and the n sweeps, each through the hand-written
//      reverse of the point-wise flux (ns_flux_adj).
//
// Non-smooth points take one-sided derivatives: max(s_L, s_R) differentiates
// into s_L on ties, |v.n| into sign(v.n) (0 at 0).
#include <cuda_runtime.h>

#include "adg_internal.h"
#include "adg_physics.cuh"

namespace adg {

template <int N>
struct AdjCfg {
    static constexpr int n = N + 1;
    static constexpr int cpb = N <= 2 ? 4 : N <= 4 ? 2 : 1;
    static constexpr int threads = cpb * n * n;
    static constexpr int SL = 4 * n * n;
    // iterates q^(1..n) (n slices each) + q^(0) (one slice) + QB, RB, QXB, QYB
    static constexpr int per_cell = (n * n + 1) * SL + 4 * n * SL;
    static constexpr size_t smem = (size_t)cpb * per_cell * sizeof(double);
};

// ------------------------------------------------------------------ corrector
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_adj_fp64(const double* __restrict__ lam, const double* __restrict__ trace,
                     double* __restrict__ trace_bar, int cells, double dt, const Basis B, const Phys P,
                     const Background bg) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int cell_raw = blockIdx.x * CPB + cl;
    if (cell_raw >= cells) return;  // no barriers in this kernel
    const int cell = cell_raw;
    const int ix = cell % P.nx, iy = cell / P.nx;
    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const bool wall = xface ? (P.bc_x == ADG_BC_WALL && ((f == 0 && ix == P.nx - 1) || (f == 1 && ix == 0)))
                                : (P.bc_y == ADG_BC_WALL && ((f == 2 && iy == P.ny - 1) || (f == 3 && iy == 0)));
        int nb = -1, nf = -1;
        if (f == 0) { nb = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1); nf = 1; }
        else if (f == 1) { nb = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1); nf = 0; }
        else if (f == 2) { nb = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix; nf = 3; }
        else { nb = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix; nf = 2; }
        // adjoint of the face value F*: lift rows of the own cell and, on an
        // interior face, of the neighbour that uses the same value
        const double* lo = lam + (size_t)cell * SL;
        double Fb[4];
        auto lift_row = [&](const double* L, int face, double out[4], double sign_acc) {
            // contribution of cell L's use of its face `face` at node m
            const double* w = (face == 0 || face == 2) ? B.lift1 : B.lift0;
            const double sgn = (face == 0 || face == 2) ? -1.0 : 1.0;
            const double h = (face < 2) ? P.inv_hx : P.inv_hy;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double s = 0.0;
#pragma unroll
                for (int p = 0; p < n; ++p) s += w[p] * (face < 2 ? L[v * n2 + m * n + p] : L[v * n2 + p * n + m]);
                out[v] += sign_acc * sgn * dt * h * s;
            }
        };
#pragma unroll
        for (int v = 0; v < 4; ++v) Fb[v] = 0.0;
        lift_row(lo, f, Fb, 1.0);
        if (!wall) lift_row(lam + (size_t)nb * SL, nf, Fb, 1.0);

        const double* own = trace + ((size_t)cell * 4 + f) * TR;
        double rec[kTraceComps];
#pragma unroll
        for (int c = 0; c < kTraceComps; ++c) rec[c] = own[c * n + m];
        double qo[4] = {rec[0], rec[1], rec[2], rec[3]};
        double qn[4], fn[4], sn;
        double z = 0.0, pb = 0.0, rb = 0.0;
        if (wall) {
            if (xface) {
                z = P.y0 + (iy + B.xi[m]) * P.hy;
                pb = bg.pbar_node[iy * n + m];
                rb = bg.rhobar_node[iy * n + m];
            } else {
                const int fi = iy + (f == 2 ? 1 : 0);
                z = P.y0 + fi * P.hy;
                pb = bg.pbar_face[fi];
                rb = bg.rhobar_face[fi];
            }
            // ghost (as in the forward wall_ghost)
            const double nx = f == 0 ? 1.0 : f == 1 ? -1.0 : 0.0;
            const double ny = f == 2 ? 1.0 : f == 3 ? -1.0 : 0.0;
            const double mn = rec[1] * nx + rec[2] * ny;
            qn[1] = rec[1] - 2.0 * mn * nx;
            qn[2] = rec[2] - 2.0 * mn * ny;
            qn[0] = P.gravity ? rb : rec[0];
            qn[3] = P.gravity ? pb / P.gm1 + rb * P.g * z : rec[3];
            Flux4 fl;
            ns_flux(qn, rec + 8, rec + 12, z, pb, rb, P, fl, true, 0.0, P.gravity ? -P.g / P.cp : 0.0);
#pragma unroll
            for (int v = 0; v < 4; ++v) fn[v] = xface ? fl.F[v] : fl.G[v];
            sn = wave_speed(qn, z, xface, P);
        } else {
            const double* ot = trace + ((size_t)nb * 4 + nf) * TR;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qn[v] = ot[v * n + m];
                fn[v] = ot[(4 + v) * n + m];
            }
            sn = ot[16 * n + m];
        }
        const bool own_left = (f == 0 || f == 2);
        const double sL = own_left ? rec[16] : sn, sR = own_left ? sn : rec[16];
        const double* qL = own_left ? qo : qn;
        const double* qR = own_left ? qn : qo;
        const double s = fmax(sL, sR);
        // Rusanov adjoint
        double s_b = 0.0;
        double q_own_b[4], f_own_b[4], q_oth_b[4], f_oth_b[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            s_b += -0.5 * (qR[v] - qL[v]) * Fb[v];
            f_own_b[v] = 0.5 * Fb[v];
            f_oth_b[v] = 0.5 * Fb[v];
            const double qR_b = -0.5 * s * Fb[v], qL_b = 0.5 * s * Fb[v];
            q_own_b[v] = own_left ? qL_b : qR_b;
            q_oth_b[v] = own_left ? qR_b : qL_b;
        }
        const bool left_wins = sL >= sR;
        double s_own_b = ((left_wins && own_left) || (!left_wins && !own_left)) ? s_b : 0.0;
        const double s_oth_b = s_b - s_own_b;
        double gxb[4] = {0, 0, 0, 0}, gyb[4] = {0, 0, 0, 0};
        if (wall) {
            // ghost flux, ghost speed and ghost state back to the own trace
            double qGb[4] = {0, 0, 0, 0};
            wave_speed_adj(qn, z, xface, P, s_oth_b, qGb);
            const double zero4[4] = {0, 0, 0, 0};
            ns_flux_adj(qn, rec + 8, rec + 12, z, P, xface ? f_oth_b : zero4, xface ? zero4 : f_oth_b, zero4, qGb,
                        gxb, gyb, true);
#pragma unroll
            for (int v = 0; v < 4; ++v) qGb[v] += q_oth_b[v];
            const double nx = f == 0 ? 1.0 : f == 1 ? -1.0 : 0.0;
            const double ny = f == 2 ? 1.0 : f == 3 ? -1.0 : 0.0;
            // qG1 = q1 - 2 (q1 nx + q2 ny) nx, qG2 = q2 - 2 (q1 nx + q2 ny) ny
            const double mnb = -2.0 * (qGb[1] * nx + qGb[2] * ny);
            q_own_b[1] += qGb[1] + mnb * nx;
            q_own_b[2] += qGb[2] + mnb * ny;
            if (!P.gravity) {
                q_own_b[0] += qGb[0];
                q_own_b[3] += qGb[3];
            }
        }
        double* ob = trace_bar + ((size_t)cell * 4 + f) * TR;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            ob[v * n + m] = q_own_b[v];
            ob[(4 + v) * n + m] = f_own_b[v];
            ob[(8 + v) * n + m] = gxb[v];
            ob[(12 + v) * n + m] = gyb[v];
        }
        ob[16 * n + m] = s_own_b;
    }
}

// ------------------------------------------------------------------ predictor
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_adj_fp64(const double* __restrict__ u, const double* __restrict__ lam,
                     const double* __restrict__ trace, const double* __restrict__ trace_bar,
                     double* __restrict__ lam_out, int cells, double dt, const Basis B, const Phys P,
                     const Background bg) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    double* IT = sm + (size_t)cl * AdjCfg<N>::per_cell;  // q^(r) at IT + ((r-1) n + k) SL, r = 1..n
    double* U0 = IT + n * n * SL;                        // q^(0) = u (one slice)
    double* QB = U0 + SL;
    double* RB = QB + n * SL;
    double* QXB = RB + n * SL;
    double* QYB = QXB + n * SL;
    const int ix = cell % P.nx, iy = cell / P.nx;
    const double x = P.x0 + (ix + B.xi[i]) * P.hx;
    const double z = P.y0 + (iy + B.xi[j]) * P.hy;
    const double pbar = bg.pbar_node[iy * n + j];
    const double rhobar = bg.rhobar_node[iy * n + j];
    double Sm[4] = {0.0, 0.0, 0.0, 0.0};
    if (P.source == ADG_SRC_STEADY) steady_source(x, z, P, Sm);
    auto iter = [&](int r, int k) -> double* { return r == 0 ? U0 : IT + ((r - 1) * n + k) * SL; };

    double uu[4];
    const double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uu[v] = uc[v * n2 + node];
        U0[v * n2 + node] = uu[v];
    }
    __syncthreads();

    auto grads = [&](const double* Qk, double q[4], double qx[4], double qy[4]) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const double* Qv = Qk + v * n2;
            q[v] = Qv[node];
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.D[i][p] * Qv[j * n + p];
                sy += B.D[j][p] * Qv[p * n + i];
            }
            qx[v] = sx * P.inv_hx;
            qy[v] = sy * P.inv_hy;
        }
    };
    // F, G of slice k go to RB / QXB as scratch during the forward recompute
    auto divergence = [&](const double* Fk, const double* Gk, int v) {
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sx += B.D[i][p] * Fk[v * n2 + j * n + p];
            sy += B.D[j][p] * Gk[v * n2 + p * n + i];
        }
        return -(sx * P.inv_hx + sy * P.inv_hy);
    };

    // ---------------- forward recompute of the iterates (as k_predictor_fp64)
    {
        double q[4], qx[4], qy[4];
        Flux4 f;
        grads(U0, q, qx, qy);
        ns_flux(q, qx, qy, z, pbar, rhobar, P, f);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            RB[v * n2 + node] = f.F[v];
            QXB[v * n2 + node] = f.G[v];
        }
        __syncthreads();
        double R0[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) R0[v] = f.S[v] + Sm[v] + divergence(RB, QXB, v);
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
            for (int v = 0; v < 4; ++v) iter(1, l)[v * n2 + node] = uu[v] + dt * (B.Kw1[l] * R0[v]);
        }
        __syncthreads();
    }
#pragma unroll 1
    for (int r = 2; r <= n; ++r) {
        double R[n][4];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double q[4], qx[4], qy[4];
            Flux4 f;
            grads(iter(r - 1, k), q, qx, qy);
            ns_flux(q, qx, qy, z, pbar, rhobar, P, f);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                RB[k * SL + v * n2 + node] = f.F[v];
                QXB[k * SL + v * n2 + node] = f.G[v];
                R[k][v] = f.S[v] + Sm[v];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < n; ++k) {
#pragma unroll
            for (int v = 0; v < 4; ++v) R[k][v] += divergence(RB + k * SL, QXB + k * SL, v);
        }
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < n; ++k) acc += B.Kw[l][k] * R[k][v];
                iter(r, l)[v * n2 + node] = uu[v] + dt * acc;
            }
        }
        __syncthreads();
    }

    // ---------------- reverse of the epilogue
    // time-averaged face data of the forward (for the wave-speed adjoint)
    const double* tr = trace + (size_t)cell * 4 * TR;
    const double* tb = trace_bar + (size_t)cell * 4 * TR;
    // adjoint of the face records incl. the wave speed, per face node
    auto face_rec_bar = [&](int f, int m, double out[16]) {
        const double* rb = tb + f * TR;
        const double* rf = tr + f * TR;
#pragma unroll
        for (int c = 0; c < 16; ++c) out[c] = rb[c * n + m];
        const double sb = rb[16 * n + m];
        if (sb != 0.0) {
            double qf[4] = {rf[0 * n + m], rf[1 * n + m], rf[2 * n + m], rf[3 * n + m]};
            const bool xface = f < 2;
            const double zf = xface ? P.y0 + (iy + B.xi[m]) * P.hy : P.y0 + (iy + (f == 2 ? 1 : 0)) * P.hy;
            wave_speed_adj(qf, zf, xface, P, sb, out);
        }
    };
    // slot adjoints at this node: qbar, Fbar, Gbar, qxbar, qybar
    double Aq[4] = {0, 0, 0, 0}, AF[4] = {0, 0, 0, 0}, AG[4] = {0, 0, 0, 0}, Ax[4] = {0, 0, 0, 0},
           Ay[4] = {0, 0, 0, 0};
    {
        double e[16];
        face_rec_bar(0, j, e);  // east: phi1[i]
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Aq[v] += B.phi1[i] * e[v];
            AF[v] += B.phi1[i] * e[4 + v];
            Ax[v] += B.phi1[i] * e[8 + v];
            Ay[v] += B.phi1[i] * e[12 + v];
        }
        face_rec_bar(1, j, e);  // west: phi0[i]
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Aq[v] += B.phi0[i] * e[v];
            AF[v] += B.phi0[i] * e[4 + v];
            Ax[v] += B.phi0[i] * e[8 + v];
            Ay[v] += B.phi0[i] * e[12 + v];
        }
        face_rec_bar(2, i, e);  // north: phi1[j]
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Aq[v] += B.phi1[j] * e[v];
            AG[v] += B.phi1[j] * e[4 + v];
            Ax[v] += B.phi1[j] * e[8 + v];
            Ay[v] += B.phi1[j] * e[12 + v];
        }
        face_rec_bar(3, i, e);  // south: phi0[j]
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Aq[v] += B.phi0[j] * e[v];
            AG[v] += B.phi0[j] * e[4 + v];
            Ax[v] += B.phi0[j] * e[8 + v];
            Ay[v] += B.phi0[j] * e[12 + v];
        }
    }
    // weak volume residual: rvol_bar = dt lam'
    const double* lc = lam + (size_t)cell * SL;
    double Sbar_b[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sx += B.Vx[i][p] * lc[v * n2 + j * n + p];
            sy += B.Vx[j][p] * lc[v * n2 + p * n + i];
        }
        AF[v] += dt * P.inv_hx * sx;
        AG[v] += dt * P.inv_hy * sy;
        Sbar_b[v] = dt * lc[v * n2 + node];
    }
    // final evaluation and time averages: q^(n)_k
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        double q[4], qx[4], qy[4];
        grads(iter(n, k), q, qx, qy);
        const double wk = B.w[k];
        double Fb[4], Gb[4], Sb[4], qb[4], qxb[4], qyb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Fb[v] = wk * AF[v];
            Gb[v] = wk * AG[v];
            Sb[v] = wk * Sbar_b[v];
            qb[v] = wk * Aq[v];
            qxb[v] = wk * Ax[v];
            qyb[v] = wk * Ay[v];
        }
        ns_flux_adj(q, qx, qy, z, P, Fb, Gb, Sb, qb, qxb, qyb);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            QB[k * SL + v * n2 + node] = qb[v];
            QXB[k * SL + v * n2 + node] = qxb[v];
            QYB[k * SL + v * n2 + node] = qyb[v];
        }
    }
    __syncthreads();
    // fold the gradient adjoints back: q_bar(j,p) += (1/h) sum_i' D[i'][p] qx_bar(j,i')
    auto fold = [&]() {
#pragma unroll 1
        for (int k = 0; k < n; ++k) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double sx = 0.0, sy = 0.0;
#pragma unroll
                for (int p = 0; p < n; ++p) {
                    sx += B.D[p][i] * QXB[k * SL + v * n2 + j * n + p];
                    sy += B.D[p][j] * QYB[k * SL + v * n2 + p * n + i];
                }
                QB[k * SL + v * n2 + node] += sx * P.inv_hx + sy * P.inv_hy;
            }
        }
    };
    fold();
    __syncthreads();

    // ---------------- reverse sweeps r = n .. 2
    double ub[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int r = n; r >= 2; --r) {
        // q^(r)_l = u + dt sum_k Kw[l][k] R_k(q^(r-1))
        double Rb[n][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double qbl[n];
#pragma unroll
            for (int l = 0; l < n; ++l) {
                qbl[l] = QB[l * SL + v * n2 + node];
                ub[v] += qbl[l];
            }
#pragma unroll
            for (int k = 0; k < n; ++k) {
                double acc = 0.0;
#pragma unroll
                for (int l = 0; l < n; ++l) acc += B.Kw[l][k] * qbl[l];
                Rb[k][v] = dt * acc;
            }
        }
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < 4; ++v) RB[k * SL + v * n2 + node] = Rb[k][v];
        __syncthreads();
        // R_k = -(1/hx) D_x F_k - (1/hy) D_y G_k + S_k: F_bar(j,p) = -(1/hx) sum_i' D[i'][p] Rb(j,i')
#pragma unroll 1
        for (int k = 0; k < n; ++k) {
            double Fb[4], Gb[4], Sb[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double sx = 0.0, sy = 0.0;
#pragma unroll
                for (int p = 0; p < n; ++p) {
                    sx += B.D[p][i] * RB[k * SL + v * n2 + j * n + p];
                    sy += B.D[p][j] * RB[k * SL + v * n2 + p * n + i];
                }
                Fb[v] = -sx * P.inv_hx;
                Gb[v] = -sy * P.inv_hy;
                Sb[v] = Rb[k][v];
            }
            double q[4], qx[4], qy[4];
            grads(iter(r - 1, k), q, qx, qy);
            double qb[4] = {0, 0, 0, 0}, qxb[4] = {0, 0, 0, 0}, qyb[4] = {0, 0, 0, 0};
            ns_flux_adj(q, qx, qy, z, P, Fb, Gb, Sb, qb, qxb, qyb);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                QXB[k * SL + v * n2 + node] = qxb[v];
                QYB[k * SL + v * n2 + node] = qyb[v];
                Rb[k][v] = qb[v];  // reuse: point-wise part of q^(r-1)_k bar
            }
        }
        __syncthreads();  // all reads of QB (this sweep) and RB done, QXB/QYB complete
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < 4; ++v) QB[k * SL + v * n2 + node] = Rb[k][v];
        fold();
        __syncthreads();
    }
    // ---------------- sweep 1: q^(1)_l = u + dt Kw1[l] R(u)
    {
        double R0b[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < n; ++l) {
                const double b = QB[l * SL + v * n2 + node];
                ub[v] += b;
                acc += B.Kw1[l] * b;
            }
            R0b[v] = dt * acc;
            RB[v * n2 + node] = R0b[v];
        }
        __syncthreads();
        double Fb[4], Gb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.D[p][i] * RB[v * n2 + j * n + p];
                sy += B.D[p][j] * RB[v * n2 + p * n + i];
            }
            Fb[v] = -sx * P.inv_hx;
            Gb[v] = -sy * P.inv_hy;
        }
        double q[4], qx[4], qy[4];
        grads(U0, q, qx, qy);
        double qb[4] = {0, 0, 0, 0}, qxb[4] = {0, 0, 0, 0}, qyb[4] = {0, 0, 0, 0};
        ns_flux_adj(q, qx, qy, z, P, Fb, Gb, R0b, qb, qxb, qyb);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            QXB[v * n2 + node] = qxb[v];
            QYB[v * n2 + node] = qyb[v];
            ub[v] += qb[v];
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.D[p][i] * QXB[v * n2 + j * n + p];
                sy += B.D[p][j] * QYB[v * n2 + p * n + i];
            }
            ub[v] += sx * P.inv_hx + sy * P.inv_hy;
        }
    }
    if (active) {
        double* lo = lam_out + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) lo[v * n2 + node] = lc[v * n2 + node] + ub[v];
    }
}

template <int N>
static int adj_n(const double* u, const double* lam, double* lam_out, const double* trace, double* trace_bar,
                 int cells, double dt, const Basis& B, const Phys& P, const Background& bg, cudaStream_t s) {
    using C = AdjCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_corrector_adj_fp64<N, C::cpb><<<blocks, C::threads, 0, s>>>(lam, trace, trace_bar, cells, dt, B, P, bg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    auto kern = k_predictor_adj_fp64<N, C::cpb>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<blocks, C::threads, C::smem, s>>>(u, lam, trace, trace_bar, lam_out, cells, dt, B, P, bg);
    return (int)cudaGetLastError();
}

int launch_step_adjoint_fp64(int N, const double* u, const double* lam, double* lam_out, const double* trace,
                             double* trace_bar, int cells, double dt, const Basis& B, const Phys& P,
                             const Background& bg, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return adj_n<1>(u, lam, lam_out, trace, trace_bar, cells, dt, B, P, bg, s);
        case 2: return adj_n<2>(u, lam, lam_out, trace, trace_bar, cells, dt, B, P, bg, s);
        case 3: return adj_n<3>(u, lam, lam_out, trace, trace_bar, cells, dt, B, P, bg, s);
        case 4: return adj_n<4>(u, lam, lam_out, trace, trace_bar, cells, dt, B, P, bg, s);
        case 5: return adj_n<5>(u, lam, lam_out, trace, trace_bar, cells, dt, B, P, bg, s);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace adg
