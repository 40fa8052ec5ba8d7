// FP64 ADER-DG predictor and corrector kernels for sm_103a.
//
// Predictor (Sec. 3, ADER-DG of Dumbser et al. 2008): per cell, the
// element-local space-time polynomial q(x, y, tau) on (N+1)^3 Gauss-Legendre
// nodes is found by n = N+1 Picard sweeps
//     q_l = u + dt * sum_k (K1^{-1})_{lk} w_k R_k,
//     R   = -dF/dx - dG/dy + S   (strong form, element-local),
// after which grad q, F, G, S are evaluated once more on the final iterate and
// averaged in time.  The kernel writes the weak volume residual
//     rvol = (1/hx) sum_p (w_p/w_i) D_pi Fbar_pj + (1/hy) sum_p (w_p/w_j) D_pj Gbar_ip + Sbar
// and, per face node, the boundary-extrapolated time averages
// (q-bar, normal flux, grad q-bar) plus the Rusanov speed.
//
// Corrector: per cell, the Rusanov-type viscous flux of Gassner et al. 2008
// on its 4 faces (neighbour traces, or a slip-wall ghost, Eq. 10) and the
// FP64 update u += dt (rvol - lift(F*)).
//
// Thread mapping: CPB cells per block, one thread per spatial node (j, i) of
// a cell; each thread loops over the n time nodes of its node column, so the
// time contraction of the Picard update stays in registers.  The space-time
// tensor of a cell (q, F, G: 3 x n^3 x 4 doubles) lives in shared memory.
// FP64 arithmetic is the binding resource on this part, so the first sweep
// (whose iterate is constant in time) evaluates the fluxes once, not n times.
#include <cuda_runtime.h>

#include "adg_internal.h"
#include "adg_physics.cuh"

namespace adg {

template <int N>
struct Fp64Cfg {
    static constexpr int n = N + 1;
    // cells per block: enough threads per block for small degrees
    static constexpr int cpb = N == 1 ? 32 : N == 2 ? 16 : N == 3 ? 8 : N <= 5 ? 4 : 2;
    static constexpr int threads = cpb * n * n;
    static constexpr size_t smem_pred = (size_t)cpb * 3 * n * 4 * n * n * sizeof(double);
};

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_fp64(const double* __restrict__ u, double* __restrict__ rvol,
                 double* __restrict__ trace, int cells, double dt, double t,
                 const Basis B, const Phys P, const Background bg) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    double* Q = sm + (size_t)cl * (3 * n * SL);
    double* Fs = Q + n * SL;
    double* Gs = Fs + n * SL;
    const int ix = cell % P.nx, iy = cell / P.nx;
    const double x = P.x0 + (ix + B.xi[i]) * P.hx;
    const double z = P.y0 + (iy + B.xi[j]) * P.hy;
    const double pbar = bg.pbar_node[iy * n + j];
    const double rhobar = bg.rhobar_node[iy * n + j];
    (void)t;

    double uu[4];
    const double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uu[v] = uc[v * n2 + node];
        Q[v * n2 + node] = uu[v];
    }
    double Sm[4] = {0.0, 0.0, 0.0, 0.0};
    if (P.source == ADG_SRC_STEADY) steady_source(x, z, P, Sm);
    __syncthreads();

    // gradients of q_k at this node and the point-wise fluxes; F, G to smem
    auto eval_node = [&](const double* Qk, double q[4], double qx[4], double qy[4], Flux4& f) {
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
        ns_flux(q, qx, qy, z, pbar, rhobar, P, f);
    };
    // -dF/dx - dG/dy at this node from the fluxes of time slice k in smem
    auto divergence = [&](int k, int v) {
        const double* Fv = Fs + k * SL + v * n2;
        const double* Gv = Gs + k * SL + v * n2;
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sx += B.D[i][p] * Fv[j * n + p];
            sy += B.D[j][p] * Gv[p * n + i];
        }
        return -(sx * P.inv_hx + sy * P.inv_hy);
    };

    // sweep 1: the iterate is u at every time node, so one flux evaluation
    {
        double q[4], qx[4], qy[4];
        Flux4 f;
        eval_node(Q, q, qx, qy, f);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Fs[v * n2 + node] = f.F[v];
            Gs[v * n2 + node] = f.G[v];
        }
        double R0[4];
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 4; ++v) R0[v] = f.S[v] + Sm[v] + divergence(0, v);
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
            for (int v = 0; v < 4; ++v) Q[l * SL + v * n2 + node] = uu[v] + dt * (B.Kw1[l] * R0[v]);
        }
        __syncthreads();
    }
    // sweeps 2..n
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        double R[n][4];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double q[4], qx[4], qy[4];
            Flux4 f;
            eval_node(Q + k * SL, q, qx, qy, f);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                Fs[k * SL + v * n2 + node] = f.F[v];
                Gs[k * SL + v * n2 + node] = f.G[v];
                R[k][v] = f.S[v] + Sm[v];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < n; ++k) {
#pragma unroll
            for (int v = 0; v < 4; ++v) R[k][v] += divergence(k, v);
        }
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < n; ++k) acc += B.Kw[l][k] * R[k][v];
                Q[l * SL + v * n2 + node] = uu[v] + dt * acc;
            }
        }
        __syncthreads();
    }

    // final evaluation on the converged iterate and time averages
    double qb[4], Fb[4], Gb[4], Sb[4], qxb[4], qyb[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qb[v] = Fb[v] = Gb[v] = Sb[v] = qxb[v] = qyb[v] = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
        double q[4], qx[4], qy[4];
        Flux4 f;
        eval_node(Q + k * SL, q, qx, qy, f);
        const double wk = B.w[k];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            qb[v] += wk * q[v];
            Fb[v] += wk * f.F[v];
            Gb[v] += wk * f.G[v];
            Sb[v] += wk * (f.S[v] + Sm[v]);
            qxb[v] += wk * qx[v];
            qyb[v] += wk * qy[v];
        }
    }
    __syncthreads();
    // time averages to shared memory: slots 0..4 = qbar, Fbar, Gbar, qxbar, qybar
    double* A = Q;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        A[0 * SL + v * n2 + node] = qb[v];
        A[1 * SL + v * n2 + node] = Fb[v];
        A[2 * SL + v * n2 + node] = Gb[v];
        A[3 * SL + v * n2 + node] = qxb[v];
        A[4 * SL + v * n2 + node] = qyb[v];
    }
    __syncthreads();
    if (active) {
        double* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.Vx[p][i] * A[1 * SL + v * n2 + j * n + p];
                sy += B.Vx[p][j] * A[2 * SL + v * n2 + p * n + i];
            }
            rc[v * n2 + node] = sx * P.inv_hx + sy * P.inv_hy + Sb[v];
        }
    }
    // boundary-extrapolated traces: faces E, W (x = const), N, S (y = const)
    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const double* phi = (f == 0 || f == 2) ? B.phi1 : B.phi0;
        double rec[kTraceComps];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int slot = c == 0 ? 0 : c == 1 ? (xface ? 1 : 2) : (c == 2 ? 3 : 4);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double* S = A + slot * SL + v * n2;
                double s = 0.0;
#pragma unroll
                for (int p = 0; p < n; ++p) s += phi[p] * (xface ? S[m * n + p] : S[p * n + m]);
                rec[c * 4 + v] = s;
            }
        }
        const double zf = xface ? P.y0 + (iy + B.xi[m]) * P.hy
                                : P.y0 + (iy + (f == 2 ? 1 : 0)) * P.hy;
        rec[16] = wave_speed(rec, zf, xface, P);
        if (active) {
            double* tr = trace + ((size_t)cell * 4 + f) * kTraceComps * n;
#pragma unroll
            for (int c = 0; c < kTraceComps; ++c) tr[c * n + m] = rec[c];
        }
    }
}

// Slip-wall ghost of face f (0 E, 1 W, 2 N, 3 S) from the interior trace
// record rec at height z (reading of Sec. 4.2, Eq. 10): rho and rhoE of the
// background, momentum reflected, interior gradients, heat flux of the
// background temperature profile.
__device__ __forceinline__ void wall_ghost(const double* rec, int f, double z, double pbar,
                                           double rhobar, const Phys& P, double qG[4],
                                           double fG[4], double& sG) {
    const double nx = f == 0 ? 1.0 : f == 1 ? -1.0 : 0.0;
    const double ny = f == 2 ? 1.0 : f == 3 ? -1.0 : 0.0;
    const double mn = rec[1] * nx + rec[2] * ny;
    qG[1] = rec[1] - 2.0 * mn * nx;
    qG[2] = rec[2] - 2.0 * mn * ny;
    if (P.gravity) {
        qG[0] = rhobar;
        qG[3] = pbar / P.gm1 + rhobar * P.g * z;
    } else {
        qG[0] = rec[0];
        qG[3] = rec[3];
    }
    Flux4 fl;
    const double Tz = P.gravity ? -P.g / P.cp : 0.0;
    ns_flux(qG, rec + 8, rec + 12, z, pbar, rhobar, P, fl, true, 0.0, Tz);
    const bool xdir = f < 2;
#pragma unroll
    for (int v = 0; v < 4; ++v) fG[v] = xdir ? fl.F[v] : fl.G[v];
    sG = wave_speed(qG, z, xdir, P);
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_fp64(double* __restrict__ u, const double* __restrict__ rvol,
                 const double* __restrict__ trace, int cells, double dt, const Basis B,
                 const Phys P, const Background bg) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    __shared__ double Fst[CPB][4][4][n];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int ix = cell % P.nx, iy = cell / P.nx;

    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const bool wall = xface ? (P.bc_x == ADG_BC_WALL && ((f == 0 && ix == P.nx - 1) || (f == 1 && ix == 0)))
                                : (P.bc_y == ADG_BC_WALL && ((f == 2 && iy == P.ny - 1) || (f == 3 && iy == 0)));
        const double* own = trace + ((size_t)cell * 4 + f) * TR;
        double rec[kTraceComps];
#pragma unroll
        for (int c = 0; c < kTraceComps; ++c) rec[c] = own[c * n + m];
        double qo[4] = {rec[0], rec[1], rec[2], rec[3]};
        double fo[4] = {rec[4], rec[5], rec[6], rec[7]};
        const double so = rec[16];
        double qn[4], fn[4], sn;
        if (wall) {
            double z, pb, rb;
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
            wall_ghost(rec, f, z, pb, rb, P, qn, fn, sn);
        } else {
            int nb, nf;
            if (f == 0) { nb = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1); nf = 1; }
            else if (f == 1) { nb = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1); nf = 0; }
            else if (f == 2) { nb = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix; nf = 3; }
            else { nb = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix; nf = 2; }
            const double* ot = trace + ((size_t)nb * 4 + nf) * TR;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qn[v] = ot[v * n + m];
                fn[v] = ot[(4 + v) * n + m];
            }
            sn = ot[16 * n + m];
        }
        double out[4];
        if (f == 0 || f == 2) rusanov(qo, fo, so, qn, fn, sn, out);  // own cell on the - side
        else rusanov(qn, fn, sn, qo, fo, so, out);
#pragma unroll
        for (int v = 0; v < 4; ++v) Fst[cl][f][v][m] = out[v];
    }
    __syncthreads();
    if (!active) return;
    double* uc = u + (size_t)cell * SL;
    const double* rc = rvol + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double face = (B.lift1[i] * Fst[cl][0][v][j] - B.lift0[i] * Fst[cl][1][v][j]) * P.inv_hx +
                            (B.lift1[j] * Fst[cl][2][v][i] - B.lift0[j] * Fst[cl][3][v][i]) * P.inv_hy;
        uc[v * n2 + node] += dt * (rc[v * n2 + node] - face);
    }
}

template <int N>
static int launch_pred(const double* u, double* rvol, double* trace, int cells, double dt,
                       double t, const Basis& B, const Phys& P, const Background& bg,
                       cudaStream_t s) {
    using C = Fp64Cfg<N>;
    auto kern = k_predictor_fp64<N, C::cpb>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_pred);
    if (e != cudaSuccess) return (int)e;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    kern<<<blocks, C::threads, C::smem_pred, s>>>(u, rvol, trace, cells, dt, t, B, P, bg);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_corr(double* u, const double* rvol, const double* trace, int cells, double dt,
                       const Basis& B, const Phys& P, const Background& bg, cudaStream_t s) {
    using C = Fp64Cfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_corrector_fp64<N, C::cpb><<<blocks, C::threads, 0, s>>>(u, rvol, trace, cells, dt, B, P, bg);
    return (int)cudaGetLastError();
}

int launch_predictor_fp64(int N, const double* u, double* rvol, double* trace, int cells,
                          double dt, double t, const Basis& B, const Phys& P,
                          const Background& bg, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return launch_pred<1>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 2: return launch_pred<2>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 3: return launch_pred<3>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 4: return launch_pred<4>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 5: return launch_pred<5>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 6: return launch_pred<6>(u, rvol, trace, cells, dt, t, B, P, bg, s);
        case 7: return launch_pred<7>(u, rvol, trace, cells, dt, t, B, P, bg, s);
    }
    return (int)cudaErrorInvalidValue;
}

int launch_corrector_fp64(int N, double* u, const double* rvol, const double* trace, int cells,
                          double dt, const Basis& B, const Phys& P, const Background& bg,
                          void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return launch_corr<1>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 2: return launch_corr<2>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 3: return launch_corr<3>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 4: return launch_corr<4>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 5: return launch_corr<5>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 6: return launch_corr<6>(u, rvol, trace, cells, dt, B, P, bg, s);
        case 7: return launch_corr<7>(u, rvol, trace, cells, dt, B, P, bg, s);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace adg
