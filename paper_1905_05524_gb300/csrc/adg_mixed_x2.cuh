// Node-pair mixed-precision predictor body (even n), shared by the per-mesh
// kernel (adg_mixed.cu) and the batched persistent kernel over uniform
// instances (adg_amr.cu); the arithmetic of predictor_mixed_body in the same
// order (Sec. 3; the arithmetic split of adg_mixed.cu).
#pragma once
#include <cuda_runtime.h>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mixed_point.cuh"

namespace adg {

// ---------------------------------------------------------------------------
// Node-pair predictor (even n): each thread carries the two neighbouring
// nodes (j, 2m) and (j, 2m+1) of a row through the same steps as
// predictor_mixed_body, in the same shared-memory layout and with the same
// arithmetic in the same order (bitwise the same results).  What changes is
// what one shared-memory load serves: a 16-byte load of two adjacent slice
// pairs of row j feeds four packed FMAs of the two nodes' x-contractions, and
// a 16-byte load of the pair (p, 2m), (p, 2m+1) of a column feeds the two
// nodes' y-contractions.  With the lanes of a column pair adjacent, a column
// load is one run of equal addresses; the node-per-thread form's column
// loads (lanes n apart sharing an address) cost two wavefronts each.
// Measured on the degree-5 warm bubble: a quarter fewer shared-memory load
// wavefronts, at half the resident warps.
template <int N, int CPB_ = 0>
struct MixCfg2 {
    static constexpr int n = N + 1;
    static_assert(n % 2 == 0, "node pairs need an even number of nodes per row");
    static constexpr int tpc = n * n / 2;  // threads per cell
    // measured at N = 5: 7 cells per block (126 threads, three resident blocks) took 101.7 us on the
    // 81x81 warm bubble against 105.2 (6 cells), 102.5 (5), and 0.791 against 0.834 ms per step on
    // the 243x243 sweep mesh; 4, 8, 10 cells were slower still (0.132, 0.123, 0.113 ms)
    static constexpr int cpb_default = N == 3 ? 16 : N == 5 ? 7 : 4;
    static constexpr int cpb = CPB_ ? CPB_ : cpb_default;
    static constexpr int threads = cpb * tpc;
    static constexpr int npair = n / 2;
    static constexpr int raw = 3 * npair * 4 * n * n * 2;             // q', F, G as float2 pairs
    static constexpr int bank_off = 16;                                // floats, mod 32, between cells
    static constexpr int stride = raw + ((bank_off - raw % 32) + 32) % 32;  // a multiple of 4 floats
    static constexpr size_t smem_pred = (size_t)cpb * stride * sizeof(float);
    // three resident blocks asked of the register allocator: at N = 3 taking the pair's
    // own iterate from its row loads otherwise grows the kernel to 218 registers (two
    // blocks, 0.175 ms per 243x243 step); capped it keeps 167 (0.157 ms)
    static constexpr int minb = (N == 5 || N == 3) ? 3 : 1;
};

template <int N, int CPB>
__device__ __forceinline__ void predictor_mixed_body_x2(const double* __restrict__ u, float* __restrict__ rvol,
                                                        float* __restrict__ trace, int cells, int c0, float dt,
                                                        const BasisF& B, const PhysF& P, const MixedBg& bg,
                                                        float* smf) {
    using C = MixCfg2<N, CPB>;
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TPC = C::tpc;
    constexpr int NP = n, RS = n * NP, SLP = 4 * RS;  // time-average rows (even n: no padding)
    constexpr int NPAIR = C::npair, PS = 4 * n2;      // slice pairs, pair stride (float2)
    const int cl = threadIdx.x / TPC;
    const int loc = threadIdx.x - cl * TPC;
    // column-pair-major: the lanes of one column pair are adjacent, so a
    // column load is one run of equal addresses (a shared-memory load costs
    // a wavefront per run of adjacent lanes with equal addresses, at most 16
    // runs of 8-byte or 8 of 16-byte accesses in one)
    const int ip = loc / n, j = loc - ip * n, i0 = 2 * ip;
    const int nd0 = j * n + i0;  // first node of the pair; the second is nd0 + 1
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    float2* Q2 = reinterpret_cast<float2*>(smf + (size_t)cl * C::stride);  // [h][v][j][i]
    float2* F2 = Q2 + NPAIR * PS;
    float2* G2 = F2 + NPAIR * PS;
    // float4 = the float2 pairs of nodes (a, b) and (a, b+1), b even
    auto ld4 = [](const float2* S, int idx) { return *reinterpret_cast<const float4*>(S + idx); };
    auto st4 = [](float2* S, int idx, float2 a, float2 b) {
        *reinterpret_cast<float4*>(S + idx) = make_float4(a.x, a.y, b.x, b.y);
    };
    const int ix = cell % P.nx, iy = cell / P.nx;
    const int row = iy * n + j;
    const float z = node_coord_f(P.y0, iy, B.xi[j], P.hy);
    const double rb64 = bg.rb[row], Eb64 = bg.Eb[row];
    const float rb = f64_to_f32(rb64), Eb = f64_to_f32(Eb64), pb = bg.pb[row];
    const float dzr = bg.dzr[row], dzE = bg.dzE[row];
    float up[2][4];
    const double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        up[a][0] = f64_to_f32(uc[nd0 + a] - rb64);
        up[a][1] = f64_to_f32(uc[n2 + nd0 + a]);
        up[a][2] = f64_to_f32(uc[2 * n2 + nd0 + a]);
        up[a][3] = f64_to_f32(uc[3 * n2 + nd0 + a] - Eb64);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) st4(Q2, v * n2 + nd0, bc2(up[0][v]), bc2(up[1][v]));
    float Sm[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    if (P.source == ADG_SRC_STEADY) {
#pragma unroll
        for (int a = 0; a < 2; ++a) steady_source_f(node_coord_f(P.x0, ix, B.xi[i0 + a], P.hx), z, P, Sm[a]);
    }
    __syncthreads();

    // the two nodes' rows of D along x and the row's column of D along y, scaled by 1/h
    float dI0[n], dI1[n], dJ[n];
#pragma unroll
    for (int p = 0; p < n; ++p) {
        dI0[p] = B.D[i0][p] * P.inv_hx;
        dI1[p] = B.D[i0 + 1][p] * P.inv_hx;
        dJ[p] = B.D[j][p] * P.inv_hy;
    }
    // x-contractions of row j for both nodes: one 16-byte load per two terms
    auto xdot2 = [&](const float2* S, float2& s0, float2& s1) {
        const float2* r = S + j * n;
        float4 a = ld4(r, 0);
        s0 = fma2(bc2(dI0[1]), make_float2(a.z, a.w), mul2(bc2(dI0[0]), make_float2(a.x, a.y)));
        s1 = fma2(bc2(dI1[1]), make_float2(a.z, a.w), mul2(bc2(dI1[0]), make_float2(a.x, a.y)));
#pragma unroll
        for (int p = 2; p < n; p += 2) {
            a = ld4(r, p);
            s0 = fma2(bc2(dI0[p + 1]), make_float2(a.z, a.w), fma2(bc2(dI0[p]), make_float2(a.x, a.y), s0));
            s1 = fma2(bc2(dI1[p + 1]), make_float2(a.z, a.w), fma2(bc2(dI1[p]), make_float2(a.x, a.y), s1));
        }
    };
    // the same, also returning the pair's own values, which the row loads
    // include (the load at p = i0), so the iterate needs no load of its own
    auto xdot2_own = [&](const float2* S, float2& s0, float2& s1, float2& q0, float2& q1) {
        const float2* r = S + j * n;
        float4 a = ld4(r, 0);
        float4 own = a;
        s0 = fma2(bc2(dI0[1]), make_float2(a.z, a.w), mul2(bc2(dI0[0]), make_float2(a.x, a.y)));
        s1 = fma2(bc2(dI1[1]), make_float2(a.z, a.w), mul2(bc2(dI1[0]), make_float2(a.x, a.y)));
#pragma unroll
        for (int p = 2; p < n; p += 2) {
            a = ld4(r, p);
            if (p == i0) own = a;
            s0 = fma2(bc2(dI0[p + 1]), make_float2(a.z, a.w), fma2(bc2(dI0[p]), make_float2(a.x, a.y), s0));
            s1 = fma2(bc2(dI1[p + 1]), make_float2(a.z, a.w), fma2(bc2(dI1[p]), make_float2(a.x, a.y), s1));
        }
        q0 = make_float2(own.x, own.y);
        q1 = make_float2(own.z, own.w);
    };
    // y-contractions of the column pair (2m, 2m+1): one 16-byte load per term of both nodes
    auto ydot2 = [&](const float2* S, float2& s0, float2& s1) {
        float4 a = ld4(S, i0);
        s0 = mul2(bc2(dJ[0]), make_float2(a.x, a.y));
        s1 = mul2(bc2(dJ[0]), make_float2(a.z, a.w));
#pragma unroll
        for (int p = 1; p < n; ++p) {
            a = ld4(S, p * n + i0);
            s0 = fma2(bc2(dJ[p]), make_float2(a.x, a.y), s0);
            s1 = fma2(bc2(dJ[p]), make_float2(a.z, a.w), s1);
        }
    };
    // both slices of pair h at both nodes; fluxes of node a in f[a]
    auto eval_pair = [&](int h, FluxF2 f[2]) {
        float2 q[2][4], gx[2][4], gy[2][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float2* S = Q2 + h * PS + v * n2;
            xdot2_own(S, gx[0][v], gx[1][v], q[0][v], q[1][v]);
            ydot2(S, gy[0][v], gy[1][v]);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            gy[a][0] = add2(gy[a][0], bc2(dzr));
            gy[a][3] = add2(gy[a][3], bc2(dzE));
            ns_flux_pert2(q[a], gx[a], gy[a], z, rb, Eb, pb, P, f[a]);
        }
    };
    auto store_flux_pair = [&](int h, const FluxF2 f[2]) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            st4(F2, h * PS + v * n2 + nd0, f[0].F[v], f[1].F[v]);
            st4(G2, h * PS + v * n2 + nd0, f[0].G[v], f[1].G[v]);
        }
    };
    // dF/dx + dG/dy of slice pair h at both nodes
    auto divergence2 = [&](int h, int v, float2& d0, float2& d1) {
        float2 x0, x1, y0, y1;
        xdot2(F2 + h * PS + v * n2, x0, x1);
        ydot2(G2 + h * PS + v * n2, y0, y1);
        d0 = add2(x0, y0);
        d1 = add2(x1, y1);
    };

    {  // sweep 1: iterate constant in time (both slices of pair 0 hold it)
        FluxF2 f[2];
        eval_pair(0, f);
        store_flux_pair(0, f);
        __syncthreads();
        float R0[2][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float2 d0, d1;
            divergence2(0, v, d0, d1);
            R0[0][v] = (v == 2 ? f[0].S2.x : 0.f) + Sm[0][v] - d0.x;
            R0[1][v] = (v == 2 ? f[1].S2.x : 0.f) + Sm[1][v] - d1.x;
        }
#pragma unroll
        for (int g = 0; g < NPAIR; ++g) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                float2 a[2];
#pragma unroll
                for (int b = 0; b < 2; ++b)
                    a[b] = make_float2(fmaf(dt, B.Kw1[2 * g] * R0[b][v], up[b][v]),
                                       fmaf(dt, B.Kw1[2 * g + 1] * R0[b][v], up[b][v]));
                st4(Q2, g * PS + v * n2 + nd0, a[0], a[1]);
            }
        }
        __syncthreads();
    }
    // sweeps 2..n on the slice pairs, the residual contracted in time one variable at a time
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        float2 S2h[2][NPAIR];
#pragma unroll
        for (int h = 0; h < NPAIR; ++h) {
            FluxF2 f[2];
            eval_pair(h, f);
            store_flux_pair(h, f);
            S2h[0][h] = f[0].S2;
            S2h[1][h] = f[1].S2;
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float2 R2[2][NPAIR];
#pragma unroll
            for (int h = 0; h < NPAIR; ++h) {
                float2 d[2];
                divergence2(h, v, d[0], d[1]);
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    R2[b][h] = bc2(Sm[b][v]);
                    if (v == 2) R2[b][h] = add2(R2[b][h], S2h[b][h]);
                    R2[b][h] = fma2(bc2(-1.f), d[b], R2[b][h]);
                }
            }
#pragma unroll
            for (int g = 0; g < NPAIR; ++g) {
                const int l0 = 2 * g, l1 = 2 * g + 1;
                float2 o[2];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    float2 a0 = mul2(make_float2(B.Kw[l0][0], B.Kw[l0][1]), R2[b][0]);
                    float2 a1 = mul2(make_float2(B.Kw[l1][0], B.Kw[l1][1]), R2[b][0]);
#pragma unroll
                    for (int h = 1; h < NPAIR; ++h) {
                        a0 = fma2(make_float2(B.Kw[l0][2 * h], B.Kw[l0][2 * h + 1]), R2[b][h], a0);
                        a1 = fma2(make_float2(B.Kw[l1][2 * h], B.Kw[l1][2 * h + 1]), R2[b][h], a1);
                    }
                    o[b] = make_float2(fmaf(dt, a0.x + a0.y, up[b][v]), fmaf(dt, a1.x + a1.y, up[b][v]));
                }
                st4(Q2, g * PS + v * n2 + nd0, o[0], o[1]);
            }
        }
        __syncthreads();
    }

    // final evaluation on the converged iterate and the time averages
    float qb[2][4], Fb[2][4], Gb[2][4], qxb[2][4], qyb[2][4], Sz[2] = {0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int v = 0; v < 4; ++v) qb[b][v] = Fb[b][v] = Gb[b][v] = qxb[b][v] = qyb[b][v] = 0.f;
#pragma unroll
    for (int h = 0; h < NPAIR; ++h) {
        float2 q[2][4], gx[2][4], gy[2][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float2* S = Q2 + h * PS + v * n2;
            xdot2_own(S, gx[0][v], gx[1][v], q[0][v], q[1][v]);
            ydot2(S, gy[0][v], gy[1][v]);
        }
        const float w0 = B.w[2 * h], w1 = B.w[2 * h + 1];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            gy[b][0] = add2(gy[b][0], bc2(dzr));
            gy[b][3] = add2(gy[b][3], bc2(dzE));
            FluxF2 f;
            ns_flux_pert2(q[b], gx[b], gy[b], z, rb, Eb, pb, P, f);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qb[b][v] = fmaf(w1, q[b][v].y, fmaf(w0, q[b][v].x, qb[b][v]));
                Fb[b][v] = fmaf(w1, f.F[v].y, fmaf(w0, f.F[v].x, Fb[b][v]));
                Gb[b][v] = fmaf(w1, f.G[v].y, fmaf(w0, f.G[v].x, Gb[b][v]));
                qxb[b][v] = fmaf(w1, gx[b][v].y, fmaf(w0, gx[b][v].x, qxb[b][v]));
                qyb[b][v] = fmaf(w1, gy[b][v].y, fmaf(w0, gy[b][v].x, qyb[b][v]));
            }
            Sz[b] = fmaf(w1, f.S2.y, fmaf(w0, f.S2.x, Sz[b]));
        }
    }
    __syncthreads();
    // time averages, row-major: slots 0..4 = qbar, Fbar, Gbar, qxbar, qybar
    float* A = reinterpret_cast<float*>(Q2);
    const int rm = j * NP + i0;
    auto st2 = [](float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); };
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        st2(A + 0 * SLP + v * RS + rm, qb[0][v], qb[1][v]);
        st2(A + 1 * SLP + v * RS + rm, Fb[0][v], Fb[1][v]);
        st2(A + 2 * SLP + v * RS + rm, Gb[0][v], Gb[1][v]);
        st2(A + 3 * SLP + v * RS + rm, qxb[0][v], qxb[1][v]);
        st2(A + 4 * SLP + v * RS + rm, qyb[0][v], qyb[1][v]);
    }
    __syncthreads();
    if (active) {
        float* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                const float fr = A[1 * SLP + v * RS + j * NP + p];
                const float2 gc = *reinterpret_cast<const float2*>(A + 2 * SLP + v * RS + p * NP + i0);
                sx0 = fmaf(B.Vx[p][i0], fr, sx0);
                sx1 = fmaf(B.Vx[p][i0 + 1], fr, sx1);
                sy0 = fmaf(B.Vx[p][j], gc.x, sy0);
                sy1 = fmaf(B.Vx[p][j], gc.y, sy1);
            }
            const float sb = Sm[0][v] + (v == 2 ? Sz[0] : 0.f);
            const float sb1 = Sm[1][v] + (v == 2 ? Sz[1] : 0.f);
            st2(rc + v * n2 + nd0, __fadd_rn(__fmaf_rn(sx0, P.inv_hx, __fmul_rn(sy0, P.inv_hy)), sb),
                __fadd_rn(__fmaf_rn(sx1, P.inv_hx, __fmul_rn(sy1, P.inv_hy)), sb1));
        }
    }
    for (int idx = loc; idx < 4 * n; idx += TPC) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const float* phi = (f == 0 || f == 2) ? B.phi1 : B.phi0;
        float rec[kTraceComps];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int slot = c == 0 ? 0 : c == 1 ? (xface ? 1 : 2) : (c == 2 ? 3 : 4);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float* S = A + slot * SLP + v * RS;
                float s = 0.f;
#pragma unroll
                for (int p = 0; p < n; ++p) s = fmaf(phi[p], xface ? S[m * NP + p] : S[p * NP + m], s);
                rec[c * 4 + v] = s;
            }
        }
        float rbf, pbf;
        if (xface) {
            rbf = f64_to_f32(bg.rb[iy * n + m]);
            pbf = bg.pb[iy * n + m];
        } else {
            const float* fb = bg.face + ((size_t)iy * 2 + (f == 2 ? 0 : 1)) * kFaceBg;
            rbf = fb[0];
            pbf = fb[2];
        }
        const float zf = node_coord_f(P.y0, iy, xface ? B.xi[m] : (f == 2 ? 1.f : 0.f), P.hy);
        const float rho = __fadd_rn(rbf, rec[0]);
        const float rinv = __frcp_rn(rho);
        const float pp = trace_pp_f(rec, rinv, zf, P);
        rec[16] = wave_speed_f(rho, rec[1], rec[2], pp, pbf, xface, P);
        if (active) {
            float* tr = trace + ((size_t)cell * 4 + f) * kTraceComps * n;
#pragma unroll
            for (int c = 0; c < kTraceComps; ++c) tr[c * n + m] = rec[c];
        }
    }
}

}  // namespace adg
