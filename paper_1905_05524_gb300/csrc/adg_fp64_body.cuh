// FP64 predictor body shared by the uniform-mesh kernel (adg_fp64.cu) and the
// adaptive-mesh kernel (adg_amr.cu).  See adg_fp64.cu for the method.
#pragma once
#include "adg_internal.h"
#include "adg_physics.cuh"

namespace adg {

// Predictor body for one cell per group of n^2 threads (CPB groups per
// block).  The cell's geometry arrives as its lower-left corner (xorg, yorg),
// the cell sizes in P (hx, hy and the penalty eta_x, eta_y) and the
// background pressure/density at this thread's node height.  TSRC selects
// the time-dependent manufactured source (evaluated at t + xi_k dt for time
// node k); it is a separate instantiation so that the source-free kernel's
// register allocation is not shaped by the source's arithmetic.
//
// REC (local time stepping, adg_amr.cu): also write the face traces of every
// time node k of the final iterate, ttrace[cell][k][face][16][n] (q, normal
// flux, q_x, q_y extrapolated to the face), from which a finer neighbour
// forms the trace averaged over its own part of this cell's step.
template <int N, int CPB, bool TSRC = false, bool REC = false>
__device__ __forceinline__ void predictor_fp64_body(const double* __restrict__ u, double* __restrict__ rvol,
                                                    double* __restrict__ trace, int cell, bool active, double dt,
                                                    const Basis& B, const Phys& P, double xorg, double yorg,
                                                    double pbar, double rhobar, double* sm, double t = 0.0,
                                                    double* __restrict__ ttrace = nullptr) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    static_assert(!REC || n >= 3, "the per-time-node traces use the flux area (2 n SL >= 5 SL)");
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    double* Q = sm + (size_t)cl * (3 * n * SL);
    double* Fs = Q + n * SL;
    double* Gs = Fs + n * SL;
    const double x = xorg + B.xi[i] * P.hx;
    const double z = yorg + B.xi[j] * P.hy;

    double uu[4];
    const double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uu[v] = uc[v * n2 + node];
        Q[v * n2 + node] = uu[v];
    }
    double Sm[4] = {0.0, 0.0, 0.0, 0.0};
    if (P.source == ADG_SRC_STEADY) steady_source(x, z, P, Sm);
    auto src_k = [&](int k, double S[4]) {
        if constexpr (TSRC) {
            paper_source(x, z, t + B.xi[k] * dt, P, S);
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) S[v] = Sm[v];
        }
    };
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
        if constexpr (!TSRC) {
#pragma unroll
            for (int l = 0; l < n; ++l) {
#pragma unroll
                for (int v = 0; v < 4; ++v) Q[l * SL + v * n2 + node] = uu[v] + dt * (B.Kw1[l] * R0[v]);
            }
        } else {  // the residual differs between time nodes by the source only
            double acc[n][4];
#pragma unroll
            for (int l = 0; l < n; ++l)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[l][v] = B.Kw1[l] * R0[v];
            for (int k = 0; k < n; ++k) {
                double S[4];
                src_k(k, S);
#pragma unroll
                for (int l = 0; l < n; ++l)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[l][v] += B.Kw[l][k] * S[v];
            }
#pragma unroll
            for (int l = 0; l < n; ++l)
#pragma unroll
                for (int v = 0; v < 4; ++v) Q[l * SL + v * n2 + node] = uu[v] + dt * acc[l][v];
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
            double Sk[4];
            src_k(k, Sk);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                Fs[k * SL + v * n2 + node] = f.F[v];
                Gs[k * SL + v * n2 + node] = f.G[v];
                R[k][v] = f.S[v] + Sk[v];
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
        if constexpr (REC) {
            // slots 0..4 = q, F, G, q_x, q_y of time node k in the free flux area (5 SL <= 2 n SL)
            double* T = Fs;
            __syncthreads();  // the previous time node's extrapolation has read T
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T[0 * SL + v * n2 + node] = q[v];
                T[1 * SL + v * n2 + node] = f.F[v];
                T[2 * SL + v * n2 + node] = f.G[v];
                T[3 * SL + v * n2 + node] = qx[v];
                T[4 * SL + v * n2 + node] = qy[v];
            }
            __syncthreads();
            for (int idx = node; idx < 4 * n; idx += n2) {
                const int fc = idx / n, m = idx - fc * n;
                const bool xface = fc < 2;
                const double* phi = (fc == 0 || fc == 2) ? B.phi1 : B.phi0;
                double* tt = ttrace + ((((size_t)cell * n + k) * 4 + fc) * 16) * n;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int slot = c == 0 ? 0 : c == 1 ? (xface ? 1 : 2) : (c == 2 ? 3 : 4);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const double* S = T + slot * SL + v * n2;
                        double sv = 0.0;
#pragma unroll
                        for (int p = 0; p < n; ++p) sv += phi[p] * (xface ? S[m * n + p] : S[p * n + m]);
                        if (active) tt[(c * 4 + v) * n + m] = sv;
                    }
                }
            }
        }
        const double wk = B.w[k];
        double Sk[4];
        src_k(k, Sk);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            qb[v] += wk * q[v];
            Fb[v] += wk * f.F[v];
            Gb[v] += wk * f.G[v];
            Sb[v] += wk * (f.S[v] + Sk[v]);
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
        const double zf = xface ? yorg + B.xi[m] * P.hy : yorg + (f == 2 ? P.hy : 0.0);
        rec[16] = wave_speed(rec, zf, xface, P);
        if (active) {
            double* tr = trace + ((size_t)cell * 4 + f) * kTraceComps * n;
#pragma unroll
            for (int c = 0; c < kTraceComps; ++c) tr[c * n + m] = rec[c];
        }
    }
}

}  // namespace adg
