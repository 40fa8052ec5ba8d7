// Mixed-precision bodies shared by the per-mesh kernels (adg_mixed.cu) and the
// batched persistent kernels over uniform and adaptive instances
// (adg_amr.cu): the node-per-thread predictor body, the slip-wall ghost and
// Rusanov flux on perturbations, and the corrector body (Sec. 3; the
// arithmetic split of adg_mixed.cu).
#pragma once
#include <cuda_runtime.h>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mixed_point.cuh"
#include "adg_tv_cell.cuh"

namespace adg {

template <int N, int CPB_ = 0>
struct MixCfg {
    static constexpr int n = N + 1;
    static constexpr int cpb_default = tv_cpb(N);
    static constexpr int cpb = CPB_ ? CPB_ : cpb_default;
    static constexpr int threads = cpb * n * n;
    // time averages: rows padded to an even length.  Per-cell shared-memory
    // stride: the slice-pair arrays, padded to a bank offset (mod 32 floats)
    // between neighbouring cells.  Measured per degree: 8 at N = 2 and 18 at
    // N = 4 (where a count of bank conflicts per half-warp of 8-byte accesses
    // predicts fewer than at 16) beat 16 by 5%; at N = 5 the same count
    // favours 8, which measured 2% slower, so 16 stays there and elsewhere
    static constexpr int np = n + (n & 1);
    static constexpr int npair = (n + 1) / 2;
    static constexpr int raw = 3 * npair * 4 * n * n * 2;
    static constexpr int bank_off = cpb != cpb_default ? 16 : N == 2 ? 8 : N == 4 ? 18 : 16;
    static constexpr int stride = raw + ((bank_off - raw % 32) + 32) % 32;
    static constexpr size_t smem_pred = (size_t)cpb * stride * sizeof(float);
    // minimum resident blocks asked of the register allocator (measured: at
    // N = 5 the four blocks that shared memory admits beat three blocks
    // without spills, 0.111 against 0.115 ms; N = 4 asks for the four its
    // 128 registers allow; N = 2 runs 5% faster at four blocks (96
    // registers) than at the allocator's 124; N = 7 1% faster at four
    // blocks (128 registers, 8 bytes spilled) than at three; N = 6 at six
    // blocks spills 120 bytes; elsewhere the allocator's own choice is best)
    static constexpr int minb = (N == 5 && cpb == 4) ? 4 : (N == 4 && cpb == 5) ? 4 : (N == 3 && cpb == 8) ? 5 : (N == 2 && cpb == 16) ? 4 : (N == 6 && cpb == 2) ? 4 : (N == 7 && cpb == 2) ? 4 : (N == 6 && cpb == 3) ? 3 : (N == 6 && cpb == 5) ? 2 : 1;
};

// Predictor body for the tile of CPB cells starting at cell c0 (one thread per
// spatial node); shared by the per-mesh kernel and the batched persistent one.
//
// Shared-memory layout per cell: the iterate q' and the fluxes F and G, each
// row-major [h][v][j][i] of float2 holding time slices (2h, 2h+1) -- the
// pairs the packed FP32x2 flux evaluation works on.  One 8-byte load then
// serves both slices of a contraction term: x-contractions walk a row (the
// lanes of one row read the same entry, a broadcast), y-contractions a column
// (the lanes of one column likewise), with no transposed copies.  For odd n
// the last pair's second slice repeats slice n-1 and meets the zero padding
// of Kw and w.  The shared-memory data path bounds this kernel.
template <int N, int CPB>
__device__ __forceinline__ void predictor_mixed_body(const double* __restrict__ u, float* __restrict__ rvol,
                                                     float* __restrict__ trace, int cells, int c0, float dt,
                                                     const BasisF& B, const PhysF& P, const MixedBg& bg,
                                                     float* smf) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    constexpr int NP = MixCfg<N, CPB>::np, RS = n * NP, SLP = 4 * RS;  // padded row, var and slice strides
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    constexpr int NPAIR = MixCfg<N, CPB>::npair, PS = 4 * n2;  // slice pairs, pair stride (float2)
    float2* Q2 = reinterpret_cast<float2*>(smf + (size_t)cl * MixCfg<N, CPB>::stride);  // [h][v][j][i]
    float2* F2 = Q2 + NPAIR * PS;                                                       // [h][v][j][i]
    float2* G2 = F2 + NPAIR * PS;                                                       // [h][v][j][i]
    const int ix = cell % P.nx, iy = cell / P.nx;
    const int row = iy * n + j;
    const float x = node_coord_f(P.x0, ix, B.xi[i], P.hx);
    const float z = node_coord_f(P.y0, iy, B.xi[j], P.hy);
    (void)x;
    const double rb64 = bg.rb[row], Eb64 = bg.Eb[row];
    const float rb = f64_to_f32(rb64), Eb = f64_to_f32(Eb64), pb = bg.pb[row];
    const float dzr = bg.dzr[row], dzE = bg.dzE[row];
    // FP64 perturbation split, then FP32 from here on
    float up[4];
    const double* uc = u + (size_t)cell * SL;
    up[0] = f64_to_f32(uc[node] - rb64);
    up[1] = f64_to_f32(uc[n2 + node]);
    up[2] = f64_to_f32(uc[2 * n2 + node]);
    up[3] = f64_to_f32(uc[3 * n2 + node] - Eb64);
#pragma unroll
    for (int v = 0; v < 4; ++v) Q2[v * n2 + node] = make_float2(up[v], up[v]);
    float Sm[4] = {0.f, 0.f, 0.f, 0.f};
    if (P.source == ADG_SRC_STEADY) steady_source_f(x, z, P, Sm);
    __syncthreads();

    // This node's rows of D, pre-scaled by 1/h
    float dI[n], dJ[n];
#pragma unroll
    for (int p = 0; p < n; ++p) {
        dI[p] = B.D[i][p] * P.inv_hx;
        dJ[p] = B.D[j][p] * P.inv_hy;
    }
    // scaled D-contraction along the row (x) or the column (y) through this
    // node of one slice pair and variable
    auto xdot = [&](const float2* S) {
        const float2* r = S + j * n;
        float2 s = mul2(bc2(dI[0]), r[0]);
#pragma unroll
        for (int p = 1; p < n; ++p) s = fma2(bc2(dI[p]), r[p], s);
        return s;
    };
    auto ydot = [&](const float2* S) {
        const float2* c = S + i;
        float2 s = mul2(bc2(dJ[0]), c[0]);
#pragma unroll
        for (int p = 1; p < n; ++p) s = fma2(bc2(dJ[p]), c[p * n], s);
        return s;
    };
    // the x-contraction, also returning this node's own value: the row load
    // at p = i, so the iterate needs no load of its own
    auto xdot_own = [&](const float2* S, float2& own) {
        const float2* r = S + j * n;
        float2 a = r[0];
        own = a;
        float2 s = mul2(bc2(dI[0]), a);
#pragma unroll
        for (int p = 1; p < n; ++p) {
            a = r[p];
            if (p == i) own = a;
            s = fma2(bc2(dI[p]), a, s);
        }
        return s;
    };
    // both slices of pair h at this node
    auto eval_pair = [&](int h, float2 q[4], float2 gx[4], float2 gy[4], FluxF2& f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float2* S = Q2 + h * PS + v * n2;
            gx[v] = xdot_own(S, q[v]);
            gy[v] = ydot(S);
        }
        gy[0] = add2(gy[0], bc2(dzr));
        gy[3] = add2(gy[3], bc2(dzE));
        ns_flux_pert2(q, gx, gy, z, rb, Eb, pb, P, f);
    };
    auto store_flux_pair = [&](int h, const FluxF2& f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            F2[h * PS + v * n2 + node] = f.F[v];
            G2[h * PS + v * n2 + node] = f.G[v];
        }
    };
    // dF/dx + dG/dy of slice pair h at this node
    auto divergence = [&](int h, int v) { return add2(xdot(F2 + h * PS + v * n2), ydot(G2 + h * PS + v * n2)); };
    // slices 2g, 2g+1 of variable v (for odd n the slot past the last slice
    // repeats it)
    auto store_q_pair = [&](int g, int v, float a, float b) {
        Q2[g * PS + v * n2 + node] = make_float2(a, 2 * g + 1 < n ? b : a);
    };

    {  // sweep 1: iterate constant in time (both slices of pair 0 hold it)
        float2 q[4], gx[4], gy[4];
        FluxF2 f;
        eval_pair(0, q, gx, gy, f);
        store_flux_pair(0, f);
        __syncthreads();
        float R0[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) R0[v] = (v == 2 ? f.S2.x : 0.f) + Sm[v] - divergence(0, v).x;
#pragma unroll
        for (int g = 0; g < NPAIR; ++g) {
            const int l1 = 2 * g + 1 < n ? 2 * g + 1 : 2 * g;
#pragma unroll
            for (int v = 0; v < 4; ++v)
                store_q_pair(g, v, fmaf(dt, B.Kw1[2 * g] * R0[v], up[v]), fmaf(dt, B.Kw1[l1] * R0[v], up[v]));
        }
        __syncthreads();
    }
    // sweeps 2..n on the slice pairs; the residual is contracted in time one
    // variable at a time, so only the z-momentum source of each pair stays
    // live across the barrier
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        float2 S2h[NPAIR];
#pragma unroll
        for (int h = 0; h < NPAIR; ++h) {
            float2 q[4], gx[4], gy[4];
            FluxF2 f;
            eval_pair(h, q, gx, gy, f);
            store_flux_pair(h, f);
            S2h[h] = f.S2;
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float2 R2[NPAIR];  // slices 2h, 2h+1 of variable v
#pragma unroll
            for (int h = 0; h < NPAIR; ++h) {
                R2[h] = bc2(Sm[v]);
                if (v == 2) R2[h] = add2(R2[h], S2h[h]);
                R2[h] = fma2(bc2(-1.f), divergence(h, v), R2[h]);
            }
#pragma unroll
            for (int g = 0; g < NPAIR; ++g) {
                const int l0 = 2 * g, l1 = 2 * g + 1 < n ? 2 * g + 1 : 2 * g;
                float2 a0 = mul2(make_float2(B.Kw[l0][0], B.Kw[l0][1]), R2[0]);
                float2 a1 = mul2(make_float2(B.Kw[l1][0], B.Kw[l1][1]), R2[0]);
#pragma unroll
                for (int h = 1; h < NPAIR; ++h) {
                    a0 = fma2(make_float2(B.Kw[l0][2 * h], B.Kw[l0][2 * h + 1]), R2[h], a0);
                    a1 = fma2(make_float2(B.Kw[l1][2 * h], B.Kw[l1][2 * h + 1]), R2[h], a1);
                }
                store_q_pair(g, v, fmaf(dt, a0.x + a0.y, up[v]), fmaf(dt, a1.x + a1.y, up[v]));
            }
        }
        __syncthreads();
    }

    // final evaluation on the converged iterate and the time averages
    // (scalar accumulators: half the registers of packed ones, at the
    // register peak of the kernel)
    float qb[4], Fb[4], Gb[4], Sb[4], qxb[4], qyb[4], Sz = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) qb[v] = Fb[v] = Gb[v] = qxb[v] = qyb[v] = 0.f;
#pragma unroll
    for (int h = 0; h < NPAIR; ++h) {
        float2 q[4], gx[4], gy[4];
        FluxF2 f;
        eval_pair(h, q, gx, gy, f);
        const float w0 = B.w[2 * h], w1 = B.w[2 * h + 1];  // w[n] = 0 pads an odd n
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            qb[v] = fmaf(w1, q[v].y, fmaf(w0, q[v].x, qb[v]));
            Fb[v] = fmaf(w1, f.F[v].y, fmaf(w0, f.F[v].x, Fb[v]));
            Gb[v] = fmaf(w1, f.G[v].y, fmaf(w0, f.G[v].x, Gb[v]));
            qxb[v] = fmaf(w1, gx[v].y, fmaf(w0, gx[v].x, qxb[v]));
            qyb[v] = fmaf(w1, gy[v].y, fmaf(w0, gy[v].x, qyb[v]));  // full y-gradient (background included)
        }
        Sz = fmaf(w1, f.S2.y, fmaf(w0, f.S2.x, Sz));
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Sb[v] = Sm[v];  // the time weights sum to one
    Sb[2] += Sz;
    __syncthreads();
    // time averages, row-major with padded rows: slots 0..4 = qbar, Fbar, Gbar, qxbar, qybar
    float* A = reinterpret_cast<float*>(Q2);
    const int rm = j * NP + i;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        A[0 * SLP + v * RS + rm] = qb[v];
        A[1 * SLP + v * RS + rm] = Fb[v];
        A[2 * SLP + v * RS + rm] = Gb[v];
        A[3 * SLP + v * RS + rm] = qxb[v];
        A[4 * SLP + v * RS + rm] = qyb[v];
    }
    __syncthreads();
    if (active) {
        float* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx = fmaf(B.Vx[p][i], A[1 * SLP + v * RS + j * NP + p], sx);
                sy = fmaf(B.Vx[p][j], A[2 * SLP + v * RS + p * NP + i], sy);
            }
            rc[v * n2 + node] = __fadd_rn(__fmaf_rn(sx, P.inv_hx, __fmul_rn(sy, P.inv_hy)), Sb[v]);
        }
    }
    for (int idx = node; idx < 4 * n; idx += n2) {
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
        // background at the face node: nodal values on x-faces, extrapolated on y-faces
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

// Slip-wall ghost (Eq. 10 reading): the background state at the face (rb, Eb,
// pb), momentum reflected, interior gradients, background heat flux.  Its
// flux and wave speed are evaluated on that base with zero perturbation --
// the FP64 path's ghost exactly; for the Rusanov jump the ghost is returned
// as a perturbation (dr, dE) against the base of the interior trace (the
// extrapolated nodal background on y-faces, zero on x-faces).
__device__ __forceinline__ void wall_ghost_f(const float* rec, int f, float z, float rb, float Eb,
                                             float pb, float dr, float dE, const PhysF& P,
                                             float qG[4], float fG[4], float& sG) {
    const float nx = f == 0 ? 1.f : f == 1 ? -1.f : 0.f;
    const float ny = f == 2 ? 1.f : f == 3 ? -1.f : 0.f;
    const float mn = __fmaf_rn(rec[1], nx, __fmul_rn(rec[2], ny));
    qG[0] = P.gravity ? 0.f : rec[0];
    qG[1] = __fmaf_rn(__fmul_rn(-2.f, mn), nx, rec[1]);
    qG[2] = __fmaf_rn(__fmul_rn(-2.f, mn), ny, rec[2]);
    qG[3] = P.gravity ? 0.f : rec[3];
    float gx[4], gy[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        gx[v] = rec[8 + v];
        gy[v] = rec[12 + v];
    }
    FluxF fl;
    ns_flux_pert(qG, gx, gy, z, rb, Eb, pb, P, fl, true, P.gravity ? -P.g / P.cp : 0.f);
    const bool xdir = f < 2;
#pragma unroll
    for (int v = 0; v < 4; ++v) fG[v] = xdir ? fl.F[v] : fl.G[v];
    const float rho = __fadd_rn(rb, qG[0]);
    const float rinv = __frcp_rn(rho);
    const float pp = trace_pp_f(qG, rinv, z, P);
    sG = wave_speed_f(rho, qG[1], qG[2], pp, pb, xdir, P);
    if (P.gravity) {
        qG[0] = dr;
        qG[3] = dE;
    }
}

// Rusanov flux on perturbations.  dRL[v]: base of the right state minus base
// of the left state (the two cells' extrapolated backgrounds differ on
// y-faces), so the jump is that of the full states.  Explicit rounding: the
// two cells of a face obtain bitwise the same flux.
__device__ __forceinline__ void rusanov_f(const float qL[4], const float fL[4], float sL,
                                          const float qR[4], const float fR[4], float sR, const float dRL[4],
                                          float out[4]) {
    const float hs = __fmul_rn(-0.5f, fmaxf(sL, sR));
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float avg = __fmul_rn(0.5f, __fadd_rn(fL[v], fR[v]));
        out[v] = __fmaf_rn(hs, __fadd_rn(__fsub_rn(qR[v], qL[v]), dRL[v]), avg);
    }
}

// Corrector body; with TV the TV indicator of the updated state follows in
// the same kernel (tv_cell, bitwise what k_tv_cells_mixed computes).
template <int N, int CPB, bool TV = false>
__device__ __forceinline__ void corrector_mixed_body(double* __restrict__ u, const float* __restrict__ rvol,
                                                     const float* __restrict__ trace, int cells, int c0,
                                                     double dt, const BasisF& B, const PhysF& P,
                                                     const MixedBg& bg, const TvEpilogue& epi = TvEpilogue{}) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    __shared__ float Fst[CPB][4][4][n];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int ix = cell % P.nx, iy = cell / P.nx;
    // this node's state and residual (and the background row of the TV
    // field), loaded before the face fluxes so their latency overlaps them
    double* uc = u + (size_t)cell * SL;
    const float* rc = rvol + (size_t)cell * SL;
    double uo[4];
    float rv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uo[v] = active ? uc[v * n2 + node] : 0.0;  // padding threads touch no state
        rv[v] = rc[v * n2 + node];
    }
    double rb_row = 0.0, Eb_row = 0.0;
    float pb_row = 0.f;
    if constexpr (TV) {
        const int row = iy * n + j;
        rb_row = bg.rb[row];
        Eb_row = bg.Eb[row];
        pb_row = bg.pb[row];
    }

    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const bool wall = xface ? (P.bc_x == ADG_BC_WALL && ((f == 0 && ix == P.nx - 1) || (f == 1 && ix == 0)))
                                : (P.bc_y == ADG_BC_WALL && ((f == 2 && iy == P.ny - 1) || (f == 3 && iy == 0)));
        const float* own = trace + ((size_t)cell * 4 + f) * TR;
        float rec[kTraceComps];
#pragma unroll
        for (int c = 0; c < kTraceComps; ++c) rec[c] = own[c * n + m];
        float qo[4] = {rec[0], rec[1], rec[2], rec[3]};
        float fo[4] = {rec[4], rec[5], rec[6], rec[7]};
        const float so = rec[16];
        float qn[4], fn[4], sn;
        float dRL[4] = {0.f, 0.f, 0.f, 0.f};
        if (wall) {
            float z, rb, Eb, pb, dr = 0.f, dE = 0.f;
            if (xface) {  // nodal heights: the traces' base is the exact background
                z = node_coord_f(P.y0, iy, B.xi[m], P.hy);
                rb = f64_to_f32(bg.rb[iy * n + m]);
                Eb = f64_to_f32(bg.Eb[iy * n + m]);
                pb = bg.pb[iy * n + m];
            } else {
                z = node_coord_f(P.y0, iy, f == 2 ? 1.f : 0.f, P.hy);
                const float* fb = bg.face + ((size_t)iy * 2 + (f == 2 ? 0 : 1)) * kFaceBg;
                rb = fb[3];
                Eb = fb[4];
                pb = fb[5];
                dr = fb[6];
                dE = fb[7];
            }
            wall_ghost_f(rec, f, z, rb, Eb, pb, dr, dE, P, qn, fn, sn);
        } else {
            int nb, nf;
            if (f == 0) { nb = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1); nf = 1; }
            else if (f == 1) { nb = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1); nf = 0; }
            else if (f == 2) { nb = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix; nf = 3; }
            else { nb = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix; nf = 2; }
            const float* ot = trace + ((size_t)nb * 4 + nf) * TR;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qn[v] = ot[v * n + m];
                fn[v] = ot[(4 + v) * n + m];
            }
            sn = ot[16 * n + m];
            if (!xface) {  // upper cell's base minus lower cell's base at this face
                const float* fb = bg.face + ((size_t)iy * 2 + (f == 2 ? 0 : 1)) * kFaceBg;
                dRL[0] = fb[6];
                dRL[3] = fb[7];
            }
        }
        float out[4];
        if (f == 0 || f == 2) rusanov_f(qo, fo, so, qn, fn, sn, dRL, out);
        else rusanov_f(qn, fn, sn, qo, fo, so, dRL, out);
#pragma unroll
        for (int v = 0; v < 4; ++v) Fst[cl][f][v][m] = out[v];
    }
    __syncthreads();
    double unew[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        // explicit rounding: the per-mesh and the batched corrector agree bitwise
        const float fx = __fsub_rn(__fmul_rn(B.lift1[i], Fst[cl][0][v][j]), __fmul_rn(B.lift0[i], Fst[cl][1][v][j]));
        const float fy = __fsub_rn(__fmul_rn(B.lift1[j], Fst[cl][2][v][i]), __fmul_rn(B.lift0[j], Fst[cl][3][v][i]));
        const float face = __fmaf_rn(fx, P.inv_hx, __fmul_rn(fy, P.inv_hy));
        const float du = __fsub_rn(rv[v], face);
        unew[v] = fma(dt, f32_to_f64(du), uo[v]);  // FP64 accumulation
        if (active) uc[v * n2 + node] = unew[v];
    }
    if constexpr (TV) {
        __shared__ float fs[CPB][n2], red[CPB][n2];
        const int row = iy * n + j;
        const float z = tv_node_z(iy, j, B, P);
        const float f = tv_field_mixed(unew, epi.var, rb_row, Eb_row, pb_row, z, P, (float)epi.theta0,
                                       (float)(1.0 - epi.Rcp));
        static_assert(CPB == tv_cpb(N), "the TV statistics combine blocks of tv_cpb(N) cells");
        const double r = tv_cell<N, float>(f, epi.var == ADG_TV_THETA ? 0.f : bg.dzr[row], node, i, j, B,
                                           P.inv_hx, P.inv_hy, fs[cl], red[cl], active, epi.tv + cell);
        tv_block_triple<CPB>(r, node == 0, cl, min(CPB, cells - c0), epi.part);
    }
}

}  // namespace adg
