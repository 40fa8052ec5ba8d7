// Mixed-precision predictor with the derivative contractions on the tensor
// cores (ADG_PREC_MIXED_TF32): the Picard iteration of Sec. 3 on
// perturbation variables, as in adg_mixed_body.cuh, except that the four
// D-contractions of every sweep -- the x- and y-gradients of the iterate and
// the x-derivative of F and y-derivative of G -- run as warp MMAs
// (mma.sync m16n8k8, TF32 operands, FP32 accumulation) instead of packed
// FP32 FMAs.
//
// Accuracy: every operand a is split into a_hi (its top 11 significant bits,
// exactly a TF32 number) and a_lo = a - a_hi (exact in FP32, |a_lo| < 2^-10
// |a|), likewise D, and each product is accumulated as a_lo D_hi + a_hi D_lo
// + a_hi D_hi (the three-term split).  The dropped a_lo D_lo is below 2^-20
// of the product, and the MMA reads a_lo and D_lo as TF32 (their top 11
// bits), another 2^-21 each: a product is within about 2^-19 of exact in the
// worst case, 2^-22 typically, against 2^-24 for one FP32 rounding.
//
// ADG_PREC_MIXED_BF16X3 runs the same contractions as mma.sync m16n8k16 with
// BF16 operands: every operand is split exactly into three BF16 numbers
// a = a_hi + a_mid + a_lo (each the top 8 significant bits of what remains,
// so |a_mid| < 2^-7 |a| and |a_lo| < 2^-14 |a|), likewise D, and the six
// products of order 1 to 2^-14 -- hi hi, mid hi, hi mid, lo hi, mid mid,
// hi lo -- are accumulated in FP32 by three MMAs, the K = 16 of each
// holding two of them side by side (K = n <= 8 per product):
//   [a_hi | a_mid] x [D_hi ; D_hi],  [a_hi | a_lo] x [D_mid ; D_hi],
//   [a_mid | a_hi] x [D_mid ; D_lo].
// The dropped mid lo, lo mid and lo lo are below 2^-20 of the product: about
// 2^-21 in the worst case, 2^-25 typically (tests/test_split_products.py
// checks both splits and these orders on the host).
//
// Shape: for one cell and direction the contraction is a (rows x n) by
// (n x n) product, rows = (slice pair, variable, line, slice): 16-row tiles,
// K = n padded to 8 (the padding columns of D are zero), N = n padded to 8.
// The MMA's accumulator layout does not hold the four variables and both
// gradients of one node in one lane, so the results go to shared memory
// (gradients X2, Y2; the divergence reuses X2, Y2) and the node threads read
// them for the point-wise flux and the time contraction: four barriers per
// sweep instead of two.
#include <cuda_runtime.h>

#include <cstdint>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mixed_body.cuh"
#include "adg_mixed_point.cuh"

namespace adg {
namespace {

template <int N>
struct TcCfg {
    static constexpr int n = N + 1;
    static_assert(n % 2 == 0 && n <= 8, "even n <= 8: slice pairs without padding, K and N within 8");
    static constexpr int cpb = N == 3 ? 8 : N == 5 ? 4 : 2;
    static constexpr int node_threads = cpb * n * n;
    static constexpr int threads = (node_threads + 31) / 32 * 32;  // whole warps for mma.sync
    static constexpr int npair = n / 2;
    static constexpr int arr = npair * 4 * n * n * 2;  // floats of one [h][v][j][i] float2 array
    static constexpr int raw = 5 * arr;                // Q2, F2, G2, X2, Y2
    static constexpr int stride = raw + ((16 - raw % 32) + 32) % 32;
    static constexpr size_t smem = (size_t)cpb * stride * sizeof(float);
};

__device__ __forceinline__ uint32_t tf32_hi(float a) { return __float_as_uint(a) & 0xffffe000u; }

// Exact three-way BF16 split of a: the FP32 bit patterns of hi, mid, lo (the
// low 16 bits zero, so the top 16 are the BF16 numbers), hi + mid + lo = a.
__device__ __forceinline__ void bf16_split3(float a, uint32_t& h, uint32_t& m, uint32_t& l) {
    h = __float_as_uint(a) & 0xffff0000u;
    const float r1 = __fsub_rn(a, __uint_as_float(h));  // exact: the low 16 significant bits of a
    m = __float_as_uint(r1) & 0xffff0000u;
    const float r2 = __fsub_rn(r1, __uint_as_float(m));  // exact, at most 8 significant bits
    l = __float_as_uint(r2) & 0xffff0000u;              // = r2
}

// two BF16 numbers (FP32 patterns with zero low halves) in one register, the
// first in the low half
__device__ __forceinline__ uint32_t bf16_pack(uint32_t lo_elem, uint32_t hi_elem) {
    return (lo_elem >> 16) | hi_elem;
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a0, const uint32_t a1, const uint32_t a2,
                                         const uint32_t a3, const uint32_t b0, const uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 16-row tile of the contraction out(r, k') = sum_k in(r, k) Dh[k'][k]
// of one cell: row r = 2 R + s (s the slice of the float2 pair), R = hv n +
// line; x-direction: in(r, k) at ((hv n + line) n + k) 2 + s (line = j, k
// along the row); y-direction: at ((hv n + k) n + line) 2 + s (line = i, k
// along the column).  The output uses the same index map with k'.  bf: the
// lane's B fragments -- TF32: hi {bf[0], bf[1]}, lo {bf[2], bf[3]} (rows k =
// t, t + 4); BF16: hi, mid, lo pairs (rows k = 2t, 2t + 1) in bf[0..2].
template <int n, bool YDIR, bool BF16>
__device__ __forceinline__ void mma_tile(const float* __restrict__ S, float* __restrict__ Dst, int m0,
                                         const uint32_t bf[4], int lane) {
    const int g = lane >> 2, t = lane & 3;
    auto idx = [](int r, int k) {
        const int R = r >> 1, s = r & 1;
        const int hv = R / n, line = R - hv * n;
        return YDIR ? ((hv * n + k) * n + line) * 2 + s : ((hv * n + line) * n + k) * 2 + s;
    };
    const int r0 = m0 + g, r1 = m0 + g + 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (BF16) {
        // A: row g (r0) and g + 8 (r1), columns k = 2t, 2t + 1 of each K half
        const int ka = 2 * t, kb = 2 * t + 1;
        const float a00 = ka < n ? S[idx(r0, ka)] : 0.f, a01 = kb < n ? S[idx(r0, kb)] : 0.f;
        const float a10 = ka < n ? S[idx(r1, ka)] : 0.f, a11 = kb < n ? S[idx(r1, kb)] : 0.f;
        uint32_t h00, m00, l00, h01, m01, l01, h10, m10, l10, h11, m11, l11;
        bf16_split3(a00, h00, m00, l00);
        bf16_split3(a01, h01, m01, l01);
        bf16_split3(a10, h10, m10, l10);
        bf16_split3(a11, h11, m11, l11);
        const uint32_t H0 = bf16_pack(h00, h01), M0 = bf16_pack(m00, m01), L0 = bf16_pack(l00, l01);
        const uint32_t H1 = bf16_pack(h10, h11), M1 = bf16_pack(m10, m11), L1 = bf16_pack(l10, l11);
        mma_bf16(c, H0, H1, M0, M1, bf[0], bf[0]);  // a_hi D_hi + a_mid D_hi
        mma_bf16(c, H0, H1, L0, L1, bf[1], bf[0]);  // a_hi D_mid + a_lo D_hi
        mma_bf16(c, M0, M1, H0, H1, bf[1], bf[2]);  // a_mid D_mid + a_hi D_lo
    } else {
        float a[4];
        a[0] = S[idx(r0, t)];
        a[1] = S[idx(r1, t)];
        a[2] = t + 4 < n ? S[idx(r0, t + 4)] : 0.f;
        a[3] = t + 4 < n ? S[idx(r1, t + 4)] : 0.f;
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ah[q] = tf32_hi(a[q]);
            al[q] = __float_as_uint(__fsub_rn(a[q], __uint_as_float(ah[q])));
        }
        const uint32_t bh[2] = {bf[0], bf[1]}, bl[2] = {bf[2], bf[3]};
        mma_tf32(c, al, bh);
        mma_tf32(c, ah, bl);
        mma_tf32(c, ah, bh);
    }
    const int k0 = 2 * t, k1 = 2 * t + 1;
    if (k0 < n) {
        Dst[idx(r0, k0)] = c[0];
        Dst[idx(r1, k0)] = c[2];
    }
    if (k1 < n) {
        Dst[idx(r0, k1)] = c[1];
        Dst[idx(r1, k1)] = c[3];
    }
}

// all tiles of the block's cells for slice pairs [0, hcount): src -> dst along x or y
template <int N, int CPB, bool YDIR, bool BF16>
__device__ __forceinline__ void contract_all(float* smf, int src_off, int dst_off, int hcount, const uint32_t bf[4]) {
    using C = TcCfg<N>;
    constexpr int n = N + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = C::threads / 32;
    const int tiles_per_cell = hcount * 4 * n * 2 / 16;
    for (int tt = warp; tt < CPB * tiles_per_cell; tt += nwarps) {
        const int cl = tt / tiles_per_cell, m0 = (tt - cl * tiles_per_cell) * 16;
        float* base = smf + (size_t)cl * C::stride;
        mma_tile<n, YDIR, BF16>(base + src_off, base + dst_off, m0, bf, lane);
    }
}

template <int N, int CPB, bool BF16>
__global__ void __launch_bounds__(TcCfg<N>::threads)
k_predictor_mixed_tc(const double* __restrict__ u, float* __restrict__ rvol, float* __restrict__ trace, int cells,
                     float dt, const BasisF B, const PhysF P, const MixedBg bg) {
    using C = TcCfg<N>;
    extern __shared__ float smf[];
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    constexpr int NPAIR = C::npair, PS = 4 * n2, NP = n, RS = n * NP, SLP = 4 * RS;
    constexpr int OQ = 0, OF = C::arr, OG = 2 * C::arr, OX = 3 * C::arr, OY = 4 * C::arr;  // float offsets
    const bool node_thread = threadIdx.x < C::node_threads;
    const int tid = node_thread ? threadIdx.x : 0;  // the spare lanes of the last warp mirror thread 0 and write nothing
    const int cl = tid / n2;
    const int node = tid - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = node_thread && cell_raw < cells;
    const int cell = cell_raw < cells ? cell_raw : cells - 1;
    float* base = smf + (size_t)cl * C::stride;
    float2* Q2 = reinterpret_cast<float2*>(base + OQ);
    float2* F2 = reinterpret_cast<float2*>(base + OF);
    float2* G2 = reinterpret_cast<float2*>(base + OG);
    const float2* X2 = reinterpret_cast<const float2*>(base + OX);
    const float2* Y2 = reinterpret_cast<const float2*>(base + OY);
    const int ix = cell % P.nx, iy = cell / P.nx;
    const int row = iy * n + j;
    const float x = node_coord_f(P.x0, ix, B.xi[i], P.hx);
    const float z = node_coord_f(P.y0, iy, B.xi[j], P.hy);
    const double rb64 = bg.rb[row], Eb64 = bg.Eb[row];
    const float rb = f64_to_f32(rb64), Eb = f64_to_f32(Eb64), pb = bg.pb[row];
    const float dzr = bg.dzr[row], dzE = bg.dzE[row];

    // B fragments of the two contractions: b[k][k'] = D[k'][k] / h (column k' = g),
    // split in TF32 hi + lo (rows k = t, t + 4) or in BF16 hi + mid + lo (rows k = 2t, 2t + 1)
    uint32_t bx[4], by[4];
    {
        const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
        if constexpr (BF16) {
            uint32_t xs[2][3], ys[2][3];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = 2 * t + q;
                const float dx = (g < n && k < n) ? __fmul_rn(B.D[g][k], P.inv_hx) : 0.f;
                const float dy = (g < n && k < n) ? __fmul_rn(B.D[g][k], P.inv_hy) : 0.f;
                bf16_split3(dx, xs[q][0], xs[q][1], xs[q][2]);
                bf16_split3(dy, ys[q][0], ys[q][1], ys[q][2]);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                bx[p] = bf16_pack(xs[0][p], xs[1][p]);
                by[p] = bf16_pack(ys[0][p], ys[1][p]);
            }
            bx[3] = by[3] = 0u;
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = t + 4 * q;
                const float dx = (g < n && k < n) ? __fmul_rn(B.D[g][k], P.inv_hx) : 0.f;
                const float dy = (g < n && k < n) ? __fmul_rn(B.D[g][k], P.inv_hy) : 0.f;
                bx[q] = tf32_hi(dx);
                bx[2 + q] = __float_as_uint(__fsub_rn(dx, __uint_as_float(bx[q])));
                by[q] = tf32_hi(dy);
                by[2 + q] = __float_as_uint(__fsub_rn(dy, __uint_as_float(by[q])));
            }
        }
    }

    float up[4];
    const double* uc = u + (size_t)cell * SL;
    up[0] = f64_to_f32(uc[node] - rb64);
    up[1] = f64_to_f32(uc[n2 + node]);
    up[2] = f64_to_f32(uc[2 * n2 + node]);
    up[3] = f64_to_f32(uc[3 * n2 + node] - Eb64);
    if (node_thread) {
#pragma unroll
        for (int v = 0; v < 4; ++v) Q2[v * n2 + node] = make_float2(up[v], up[v]);
    }
    float Sm[4] = {0.f, 0.f, 0.f, 0.f};
    if (P.source == ADG_SRC_STEADY) steady_source_f(x, z, P, Sm);
    __syncthreads();

    auto gradients = [&](int hcount) {
        contract_all<N, CPB, false, BF16>(smf, OQ, OX, hcount, bx);
        contract_all<N, CPB, true, BF16>(smf, OQ, OY, hcount, by);
    };
    auto divergences = [&](int hcount) {
        contract_all<N, CPB, false, BF16>(smf, OF, OX, hcount, bx);
        contract_all<N, CPB, true, BF16>(smf, OG, OY, hcount, by);
    };
    // both slices of pair h at this node from the contraction outputs
    auto eval_pair = [&](int h, float2 q[4], float2 gx[4], float2 gy[4], FluxF2& f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            q[v] = Q2[h * PS + v * n2 + node];
            gx[v] = X2[h * PS + v * n2 + node];
            gy[v] = Y2[h * PS + v * n2 + node];
        }
        gy[0] = add2(gy[0], bc2(dzr));
        gy[3] = add2(gy[3], bc2(dzE));
        ns_flux_pert2(q, gx, gy, z, rb, Eb, pb, P, f);
    };
    auto divergence = [&](int h, int v) { return add2(X2[h * PS + v * n2 + node], Y2[h * PS + v * n2 + node]); };

    {  // sweep 1: iterate constant in time (pair 0 holds it)
        gradients(1);
        __syncthreads();
        FluxF2 f;
        if (node_thread) {
            float2 q[4], gx[4], gy[4];
            eval_pair(0, q, gx, gy, f);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                F2[v * n2 + node] = f.F[v];
                G2[v * n2 + node] = f.G[v];
            }
        }
        __syncthreads();
        divergences(1);
        __syncthreads();
        if (node_thread) {
            float R0[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) R0[v] = (v == 2 ? f.S2.x : 0.f) + Sm[v] - divergence(0, v).x;
#pragma unroll
            for (int g = 0; g < NPAIR; ++g)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    Q2[g * PS + v * n2 + node] = make_float2(fmaf(dt, B.Kw1[2 * g] * R0[v], up[v]),
                                                             fmaf(dt, B.Kw1[2 * g + 1] * R0[v], up[v]));
        }
        __syncthreads();
    }
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        gradients(NPAIR);
        __syncthreads();
        float2 S2h[NPAIR];
        if (node_thread) {
#pragma unroll
            for (int h = 0; h < NPAIR; ++h) {
                float2 q[4], gx[4], gy[4];
                FluxF2 f;
                eval_pair(h, q, gx, gy, f);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    F2[h * PS + v * n2 + node] = f.F[v];
                    G2[h * PS + v * n2 + node] = f.G[v];
                }
                S2h[h] = f.S2;
            }
        }
        __syncthreads();
        divergences(NPAIR);
        __syncthreads();
        if (node_thread) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                float2 R2[NPAIR];
#pragma unroll
                for (int h = 0; h < NPAIR; ++h) {
                    R2[h] = bc2(Sm[v]);
                    if (v == 2) R2[h] = add2(R2[h], S2h[h]);
                    R2[h] = fma2(bc2(-1.f), divergence(h, v), R2[h]);
                }
#pragma unroll
                for (int g = 0; g < NPAIR; ++g) {
                    const int l0 = 2 * g, l1 = 2 * g + 1;
                    float2 a0 = mul2(make_float2(B.Kw[l0][0], B.Kw[l0][1]), R2[0]);
                    float2 a1 = mul2(make_float2(B.Kw[l1][0], B.Kw[l1][1]), R2[0]);
#pragma unroll
                    for (int h = 1; h < NPAIR; ++h) {
                        a0 = fma2(make_float2(B.Kw[l0][2 * h], B.Kw[l0][2 * h + 1]), R2[h], a0);
                        a1 = fma2(make_float2(B.Kw[l1][2 * h], B.Kw[l1][2 * h + 1]), R2[h], a1);
                    }
                    Q2[g * PS + v * n2 + node] = make_float2(fmaf(dt, a0.x + a0.y, up[v]), fmaf(dt, a1.x + a1.y, up[v]));
                }
            }
        }
        __syncthreads();
    }

    // final evaluation on the converged iterate and the time averages
    gradients(NPAIR);
    __syncthreads();
    float qb[4], Fb[4], Gb[4], Sb[4], qxb[4], qyb[4], Sz = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) qb[v] = Fb[v] = Gb[v] = qxb[v] = qyb[v] = 0.f;
    if (node_thread) {
#pragma unroll
        for (int h = 0; h < NPAIR; ++h) {
            float2 q[4], gx[4], gy[4];
            FluxF2 f;
            eval_pair(h, q, gx, gy, f);
            const float w0 = B.w[2 * h], w1 = B.w[2 * h + 1];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qb[v] = fmaf(w1, q[v].y, fmaf(w0, q[v].x, qb[v]));
                Fb[v] = fmaf(w1, f.F[v].y, fmaf(w0, f.F[v].x, Fb[v]));
                Gb[v] = fmaf(w1, f.G[v].y, fmaf(w0, f.G[v].x, Gb[v]));
                qxb[v] = fmaf(w1, gx[v].y, fmaf(w0, gx[v].x, qxb[v]));
                qyb[v] = fmaf(w1, gy[v].y, fmaf(w0, gy[v].x, qyb[v]));
            }
            Sz = fmaf(w1, f.S2.y, fmaf(w0, f.S2.x, Sz));
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Sb[v] = Sm[v];
    Sb[2] += Sz;
    __syncthreads();
    // time averages, row-major: slots 0..4 = qbar, Fbar, Gbar, qxbar, qybar
    float* A = base + OQ;
    const int rm = j * NP + i;
    if (node_thread) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            A[0 * SLP + v * RS + rm] = qb[v];
            A[1 * SLP + v * RS + rm] = Fb[v];
            A[2 * SLP + v * RS + rm] = Gb[v];
            A[3 * SLP + v * RS + rm] = qxb[v];
            A[4 * SLP + v * RS + rm] = qyb[v];
        }
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
    for (int idx = node; node_thread && idx < 4 * n; idx += n2) {
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
    pdl_trigger();  // the corrector (launched programmatically) may be scheduled
}

template <int N>
int launch_tc_n(const double* u, float* rvol, float* trace, int cells, float dt, const BasisF& B, const PhysF& P,
                const MixedBg& bg, bool bf16, cudaStream_t s) {
    using C = TcCfg<N>;
    auto kern = bf16 ? k_predictor_mixed_tc<N, C::cpb, true> : k_predictor_mixed_tc<N, C::cpb, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<(cells + C::cpb - 1) / C::cpb, C::threads, C::smem, s>>>(u, rvol, trace, cells, dt, B, P, bg);
    return (int)cudaGetLastError();
}

}  // namespace

bool tc_degree_supported(int N) { return N == 3 || N == 5 || N == 7; }

int launch_predictor_mixed_tc(int N, const double* u, float* rvol, float* trace, int cells, double dt,
                              const BasisF& B, const PhysF& P, const MixedBg& bg, bool bf16, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const float dtf = (float)dt;
    switch (N) {
        case 3: return launch_tc_n<3>(u, rvol, trace, cells, dtf, B, P, bg, bf16, s);
        case 5: return launch_tc_n<5>(u, rvol, trace, cells, dtf, B, P, bg, bf16, s);
        case 7: return launch_tc_n<7>(u, rvol, trace, cells, dtf, B, P, bg, bf16, s);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace adg
