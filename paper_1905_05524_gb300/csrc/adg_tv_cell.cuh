// Per-cell total variation (Sec. 3, Eq. 6), shared by the TV kernels
// (adg_tv.cu) and the corrector epilogues that evaluate the indicator on the
// freshly updated state (adg_fp64.cu, adg_mixed.cu), so both give bitwise the
// same TV.  One thread per node, CPB cells per block.
//
//   TV = sum_ij w_i w_j (|df/dx| + |df/dy|),
//
// f the indicator field at the nodes (theta or rho), derivatives by the nodal
// derivative matrix.
#pragma once
#include "adg_convert.cuh"
#include "adg_internal.h"

namespace adg {

// Everything below rounds explicitly (no contraction left to the compiler):
// the TV kernels and the corrector epilogues inline these routines into
// different kernels and must still agree bitwise.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// height of node row j of cell row iy
__device__ __forceinline__ double tv_node_z(int iy, int j, const Basis& B, const Phys& P) {
    return __dadd_rn(P.y0, __dmul_rn(__dadd_rn((double)iy, B.xi[j]), P.hy));
}
__device__ __forceinline__ float tv_node_z(int iy, int j, const BasisF& B, const PhysF& P) {
    return __fadd_rn(P.y0, __fmul_rn(__fadd_rn((float)iy, B.xi[j]), P.hy));
}

__device__ __forceinline__ double theta_of(const double q[4], double z, const Phys& P) {
    const double rinv = __ddiv_rn(1.0, q[0]);
    const double gz = P.gravity ? __dmul_rn(P.g, z) : 0.0;
    const double ke = __dmul_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(q[1], q[1]), __dmul_rn(q[2], q[2]))), rinv);
    const double p = __dmul_rn(P.gm1, __dsub_rn(__dsub_rn(q[3], ke), __dmul_rn(q[0], gz)));
    const double T = __dmul_rn(__dmul_rn(p, rinv), P.invR);
    return __dmul_rn(T, pow(__ddiv_rn(P.p0, p), P.Rcp));
}

// Mixed-precision indicator field from the FP64 state at one node: the FP64
// perturbation split (rho' = rho - rhobar, E' = rhoE - Ebar), then FP32.  For
// theta the perturbation is evaluated without the 300 K offset,
//     theta'/theta0 = (1 + p'/pbar)^(1-R/cp) / (1 + rho'/rhobar) - 1
//                   = expm1((1 - R/cp) log1p(p'/pbar) - log1p(rho'/rhobar)),
// (theta = p^(1-R/cp) p0^(R/cp) / (rho R), theta0 the same expression at the
// background), so no FP32 value carries theta ~ 300 K.  For rho the field is
// rho' (the caller adds d rhobar/dz to the y-derivative).
__device__ __forceinline__ float tv_field_mixed(const double q[4], int var, double rb64, double Eb64, float pb,
                                                float z, const PhysF& P, float theta0, float one_m_kappa) {
    const float rp = f64_to_f32(__dsub_rn(q[0], rb64));
    if (var != ADG_TV_THETA) return rp;
    const float Ep = f64_to_f32(__dsub_rn(q[3], Eb64));
    const float mx = f64_to_f32(q[1]), my = f64_to_f32(q[2]);
    const float rb = f64_to_f32(rb64);
    const float rho = __fadd_rn(rb, rp);
    const float ke = __fdividef(__fmul_rn(0.5f, __fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my))), rho);
    const float pp = __fmul_rn(P.gm1, __fsub_rn(__fsub_rn(Ep, ke), __fmul_rn(__fmul_rn(P.g, z), rp)));
    const float arg = __fsub_rn(__fmul_rn(one_m_kappa, log1pf(__fdividef(pp, pb))), log1pf(__fdividef(rp, rb)));
    return __fmul_rn(theta0, expm1f(arg));
}

__device__ __forceinline__ double tv_abs(double x) { return fabs(x); }
__device__ __forceinline__ float tv_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double tv_to_f64(double x) { return x; }
__device__ __forceinline__ double tv_to_f64(float x) { return f32_to_f64(x); }

// TV of this thread's cell from the field value f at its node.  fs, red: this
// cell's two n^2 scratch rows in shared memory; fy_add is added to the
// y-derivative (background gradient).  Every thread of the block must call
// it (three barriers); node 0 of an active cell writes *out and gets the
// value back (zero elsewhere).  Sums run over rows first (one thread per
// row), then over the row sums.
template <int N, typename T, typename BT>
__device__ __forceinline__ double tv_cell(T f, T fy_add, int node, int i, int j, const BT& B, T inv_hx, T inv_hy,
                                          T* fs, T* red, bool active, double* out) {
    constexpr int n = N + 1;
    fs[node] = f;
    __syncthreads();
    T fx = T(0), fy = T(0);
#pragma unroll
    for (int p = 0; p < n; ++p) {
        fx = rfma(B.D[i][p], fs[j * n + p], fx);
        fy = rfma(B.D[j][p], fs[p * n + i], fy);
    }
    fx = rmul(fx, inv_hx);
    fy = radd(rmul(fy, inv_hy), fy_add);
    red[node] = rmul(rmul(B.w[i], B.w[j]), radd(tv_abs(fx), tv_abs(fy)));
    __syncthreads();
    if (i == 0) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < n; ++a) s = radd(s, red[j * n + a]);
        fs[j] = s;  // every thread has read fs before the barrier above
    }
    __syncthreads();
    double r = 0.0;
    if (node == 0 && active) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < n; ++a) s = radd(s, fs[a]);
        r = tv_to_f64(s);
        *out = r;
    }
    return r;
}

// The (count, mean, M2) triple of this block's TV values into part[3 b ..]:
// the first step of the statistics (Chan et al.'s pairwise combination
// starts from exact per-block triples).  tvc: the cell's TV on node 0 (from
// tv_cell); ncell: active cells of the block.  Exact two-pass over at most
// CPB values by one thread (a full block's mean is a multiplication where
// CPB is a power of two).  Every thread of the block calls it (one barrier).
template <int CPB>
__device__ __forceinline__ void tv_block_triple(double tvc, bool node0, int cl, int ncell, double* part) {
    __shared__ double ctv[CPB];
    if (node0 && cl < ncell) ctv[cl] = tvc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int a = 0; a < ncell; ++a) s = __dadd_rn(s, ctv[a]);
        const double mean = (ncell == CPB && (CPB & (CPB - 1)) == 0) ? __dmul_rn(s, 1.0 / CPB)
                                                                     : __ddiv_rn(s, (double)ncell);
        double q = 0.0;
        for (int a = 0; a < ncell; ++a) {
            const double d = __dsub_rn(ctv[a], mean);
            q = __fma_rn(d, d, q);
        }
        double* p = part + 3 * (size_t)blockIdx.x;
        p[0] = (double)ncell;
        p[1] = mean;
        p[2] = q;
    }
}

}  // namespace adg
