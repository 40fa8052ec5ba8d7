// Total-variation refinement indicator (Sec. 3, Eqs. 6-8), scenario
// initialisation (Sec. 4.1, 4.2), stable time step and finiteness scan.
//
// TV per cell: TV = sum_ij w_i w_j (|df/dx| + |df/dy|) with f = theta
// (potential temperature, Sec. 4.2) or rho at the nodes, derivatives by the
// nodal derivative matrix (adg_tv_cell.cuh).  Mean and population standard
// deviation over all cells follow Chan, Golub and LeVeque's pairwise update
// (cited by the paper for a parallel, stable evaluation): every block that
// produces TV values reduces its own cells exactly (two-pass), then the
// block triples are combined in a fixed order, so the result is
// deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_physics.cuh"
#include "adg_tv_cell.cuh"

namespace adg {

template <int N>
struct TvCfg {
    static constexpr int n = N + 1;
    static constexpr int cpb = tv_cpb(N);
};

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_tv_cells(const double* __restrict__ u, double* __restrict__ tv, double* __restrict__ part, int cells, int var,
           const Basis B, const Phys P) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    __shared__ double fs[CPB][n2];
    __shared__ double red[CPB][n2];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int iy = cell / P.nx;
    const double* uc = u + (size_t)cell * SL;
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = uc[v * n2 + node];
    const double z = tv_node_z(iy, j, B, P);
    const double f = var == ADG_TV_THETA ? theta_of(q, z, P) : q[0];
    const double r = tv_cell<N, double>(f, 0.0, node, i, j, B, P.inv_hx, P.inv_hy, fs[cl], red[cl], active,
                                        tv + cell);
    tv_block_triple<CPB>(r, node == 0, cl, min(CPB, cells - (int)blockIdx.x * CPB), part);
}

// Mixed-precision TV: FP64 perturbation split, FP32 field and sums
// (tv_field_mixed).
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_tv_cells_mixed(const double* __restrict__ u, double* __restrict__ tv, double* __restrict__ part, int cells,
                 int var, const BasisF B, const PhysF P, const MixedBg bg, float theta0, float one_m_kappa) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    __shared__ float fs[CPB][n2];
    __shared__ float red[CPB][n2];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int iy = cell / P.nx;
    const int row = iy * n + j;
    const double* uc = u + (size_t)cell * SL;
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = uc[v * n2 + node];
    const float z = tv_node_z(iy, j, B, P);
    const float f = tv_field_mixed(q, var, bg.rb[row], bg.Eb[row], bg.pb[row], z, P, theta0, one_m_kappa);
    const double r = tv_cell<N, float>(f, var == ADG_TV_THETA ? 0.f : bg.dzr[row], node, i, j, B, P.inv_hx,
                                       P.inv_hy, fs[cl], red[cl], active, tv + cell);
    tv_block_triple<CPB>(r, node == 0, cl, min(CPB, cells - (int)blockIdx.x * CPB), part);
}

// Statistics of the TV values and the flags, one launch.  The TV-producing
// kernels have left one exact (count, mean, M2) triple per block of cells.
// Every block of this kernel combines all of them with Chan et al.'s
// pairwise update in the same fixed order -- thread t folds triples
// [t per, (t+1) per) left to right, then a binary tree joins the thread
// results (warp shuffles within each warp, then across the warp results;
// sigma once per block) -- so every block holds bitwise the same mean and
// sigma without
// waiting on any other block; then it flags its own cells.  The weights
// n_b/(n_a+n_b) and n_a n_b/(n_a+n_b) of every combine depend only on the
// cell count and come divided out by the host (tv_stats_prepare, the same
// IEEE quotients): the device runs multiplies and adds, since FP64 division
// is a long dependent chain on this part.
constexpr int kPartThreads = kTvThreads;

// Flag decision: refine if TV >= mean + T_r sigma, coarsen if
// TV < mean + T_c sigma, keep all when sigma <= 1e-12 |mean| (reading F1).
// The thresholds round product and sum separately (no contraction), as
// mean + T * sigma is usually written, and are formed once per block; the
// per-cell comparisons use the IEEE-754 order of non-negative doubles as
// 64-bit integers (TV >= 0): exact, and off the narrow FP64 pipe.  NaN
// compares false both ways.
struct TvThresholds {
    long long br, bc;  // encodings of the thresholds
    bool r_all, c_none, flat;
};

__device__ __forceinline__ TvThresholds tv_thresholds(double mu, double sig, double T_r, double T_c) {
    const double thr_r = __dadd_rn(mu, __dmul_rn(T_r, sig)), thr_c = __dadd_rn(mu, __dmul_rn(T_c, sig));
    TvThresholds h;
    h.flat = sig <= 1e-12 * fabs(mu) || !(thr_r == thr_r) || !(thr_c == thr_c);
    h.r_all = thr_r <= 0.0;   // a threshold <= 0 lies at or below every TV
    h.c_none = thr_c <= 0.0;
    h.br = __double_as_longlong(thr_r);
    h.bc = __double_as_longlong(thr_c);
    return h;
}

__device__ __forceinline__ int8_t tv_flag_of(double x, const TvThresholds& h) {
    const long long bx = __double_as_longlong(x);
    const bool nan = (bx & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
    const bool ref = h.r_all || bx >= h.br;
    const bool coa = !h.c_none && bx < h.bc;
    return (h.flat || nan) ? (int8_t)0 : ref ? (int8_t)1 : (coa ? (int8_t)-1 : (int8_t)0);
}

// Chan et al.'s combine of (mean m, M2 m2) with (mb, m2b) under the
// host-divided weights g1 = n_b/(n_a+n_b), g2 = n_a n_b/(n_a+n_b); every
// operation rounds explicitly, so each code path below forms the same bits.
__device__ __forceinline__ void chan_combine(double& m, double& m2, double mb, double m2b, double g1, double g2) {
    const double d = __dsub_rn(mb, m);
    m = __fma_rn(d, g1, m);
    m2 = __fma_rn(__dmul_rn(d, d), g2, __dadd_rn(m2, m2b));
}

constexpr int kFoldMax = 8;  // folds up to this length load all their triples in one batch

__global__ void __launch_bounds__(kTvThreads)
k_tv_stats_flags(const double* __restrict__ tv, const TvStatsArgs st, double T_r, double T_c,
                 double* __restrict__ stats, int8_t* __restrict__ flags) {
    __shared__ double wm[kTvThreads / 32], w2[kTvThreads / 32];
    __shared__ TvThresholds thr;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int k0 = t * st.per, k1 = min(k0 + st.per, st.nblk);
    const bool batch = st.per <= kFoldMax;
    // this thread's tree and fold weights (host-prepared), loaded ahead of
    // the dependent chain and of the wait for the kernel before this one
    double f1[kTvLevels], f2[kTvLevels], g1[kFoldMax], g2[kFoldMax];
#pragma unroll
    for (int l = 0; l < kTvLevels; ++l) {
        const int pos = l < 5 ? t : lane;
        f1[l] = st.wtree[2 * (l * kTvThreads + pos)];
        f2[l] = st.wtree[2 * (l * kTvThreads + pos) + 1];
    }
#pragma unroll
    for (int q = 1; q < kFoldMax; ++q) {
        const bool in = batch && k0 + q < k1;
        g1[q] = in ? st.wfold[2 * (k0 + q)] : 0.0;
        g2[q] = in ? st.wfold[2 * (k0 + q) + 1] : 0.0;
    }
    // the block triples and the TV values come from the kernel before this
    // one (programmatic launch)
    pdl_wait();
    const int c_first = blockIdx.x * kTvThreads + t;
    const double tv_first = (flags && c_first < st.cells) ? tv[c_first] : 0.0;
    // left fold of this thread's block triples
    double m = 0.0, m2 = 0.0;
    if (batch) {
        double mb[kFoldMax], m2b[kFoldMax];
#pragma unroll
        for (int q = 0; q < kFoldMax; ++q) {
            const bool in = k0 + q < k1;
            mb[q] = in ? st.part[3 * (k0 + q) + 1] : 0.0;
            m2b[q] = in ? st.part[3 * (k0 + q) + 2] : 0.0;
        }
        if (k0 < k1) {
            m = mb[0];
            m2 = m2b[0];
        }
#pragma unroll
        for (int q = 1; q < kFoldMax; ++q)
            if (k0 + q < k1) chan_combine(m, m2, mb[q], m2b[q], g1[q], g2[q]);
    } else if (k0 < k1) {  // long folds: loads batched four at a time
        m = st.part[3 * k0 + 1];
        m2 = st.part[3 * k0 + 2];
        for (int k = k0 + 1; k < k1; k += 4) {
            double mb[4], m2b[4], h1[4], h2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = min(k + q, k1 - 1);
                mb[q] = st.part[3 * kk + 1];
                m2b[q] = st.part[3 * kk + 2];
                h1[q] = st.wfold[2 * kk];
                h2[q] = st.wfold[2 * kk + 1];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k + q < k1) chan_combine(m, m2, mb[q], m2b[q], h1[q], h2[q]);
        }
    }
    // tree: strides 16..1 within each warp, then 4..1 across the warp results
    // (weights are zero where the right-hand entry holds no cells)
#pragma unroll
    for (int l = 0, s = 16; s > 0; ++l, s >>= 1) {
        const double mo = __shfl_down_sync(0xffffffffu, m, s), m2o = __shfl_down_sync(0xffffffffu, m2, s);
        if (lane < s) chan_combine(m, m2, mo, m2o, f1[l], f2[l]);
    }
    if (lane == 0) {
        wm[w] = m;
        w2[w] = m2;
    }
    __syncthreads();
    if (w == 0) {
        m = lane < kTvThreads / 32 ? wm[lane] : 0.0;
        m2 = lane < kTvThreads / 32 ? w2[lane] : 0.0;
#pragma unroll
        for (int l = 5, s = kTvThreads / 64; s > 0; ++l, s >>= 1) {
            const double mo = __shfl_down_sync(0xffffffffu, m, s), m2o = __shfl_down_sync(0xffffffffu, m2, s);
            if (lane < s) chan_combine(m, m2, mo, m2o, f1[l], f2[l]);
        }
        if (lane == 0) {
            const double sig = sqrt(m2 / (double)st.cells);
            if (blockIdx.x == 0 && stats) {
                stats[0] = m;
                stats[1] = sig;
            }
            thr = tv_thresholds(m, sig, T_r, T_c);
        }
    }
    __syncthreads();
    if (!flags) return;
    const TvThresholds h = thr;
    if (c_first < st.cells) flags[c_first] = tv_flag_of(tv_first, h);
    for (int c = c_first + gridDim.x * kTvThreads; c < st.cells; c += gridDim.x * kTvThreads)
        flags[c] = tv_flag_of(tv[c], h);
}

// Flags from (mean, sigma) held in device memory, one cell per thread.
__global__ void __launch_bounds__(kPartThreads)
k_tv_flag_cells(const double* __restrict__ tv, int cells, const double* __restrict__ stats, double T_r,
                double T_c, int8_t* __restrict__ flags) {
    const int c = blockIdx.x * kPartThreads + threadIdx.x;
    if (c < cells) flags[c] = tv_flag_of(tv[c], tv_thresholds(stats[0], stats[1], T_r, T_c));
}

// ---------------------------------------------------------------- scenarios
__device__ double cosine_bubble(double x, double z, double A, double a, double xc, double zc) {
    const double r = sqrt((x - xc) * (x - xc) + (z - zc) * (z - zc));
    return r <= a ? 0.5 * A * (1.0 + cos(3.14159265358979323846 * r / a)) : 0.0;
}

__device__ double gauss_bubble(double x, double z, double A, double a, double s, double xc,
                               double zc) {
    const double r = sqrt((x - xc) * (x - xc) + (z - zc) * (z - zc));
    return r <= a ? A : A * exp(-((r - a) * (r - a)) / (s * s));
}

template <int N>
__global__ void k_init(double* __restrict__ u, int cells, int kind, double A, double a,
                       double xc, double zc, const Basis B, const Phys P) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2;
    const int j = node / n, i = node - j * n;
    const int ix = cell % P.nx, iy = cell / P.nx;
    const double x = P.x0 + (ix + B.xi[i]) * P.hx;
    const double z = P.y0 + (iy + B.xi[j]) * P.hy;
    double q[4];
    if (kind == ADG_SCEN_STEADY) {
        const double k = 2.0 * 3.14159265358979323846 / P.sL;
        const double rho = 1.0 + P.sa * sin(k * (x + z));
        q[0] = rho;
        q[1] = rho * P.sU;
        q[2] = rho * P.sU;
        q[3] = P.sp / P.gm1 + 0.5 * rho * (2.0 * P.sU * P.sU);
    } else if (kind == ADG_SCEN_TAYLOR_GREEN || kind == ADG_SCEN_CAVITY) {  // Sec. 4.1 CFD scenarios
        double u = 0.0, v = 0.0, p = 100.0 / P.gamma;
        if (kind == ADG_SCEN_TAYLOR_GREEN) {
            u = sin(x) * cos(z);
            v = -cos(x) * sin(z);
            p += 0.25 * (cos(2.0 * x) + cos(2.0 * z));
        }
        q[0] = 1.0;
        q[1] = u;
        q[2] = v;
        q[3] = p / P.gm1 + 0.5 * (u * u + v * v);
    } else if (kind == ADG_SCEN_PAPER) {  // Eq. 8 at t = 0
        double s, c;
        sincos(2.0 * 3.14159265358979323846 / P.sL * (x + z), &s, &c);
        const double rho = 1.0 + 0.5 * s, vel = 0.25 * s;
        q[0] = rho;
        q[1] = rho * vel;
        q[2] = rho * vel;
        q[3] = (0.1 * c + 1.0 / P.gamma) / P.gm1 + rho * vel * vel;
    } else {
        double th = 0.0;
        if (kind == ADG_SCEN_COSINE) th = cosine_bubble(x, z, A, a, xc, zc);
        else if (kind == ADG_SCEN_TWO_BUBBLES)
            th = gauss_bubble(x, z, 0.5, 150.0, 50.0, 500.0, 300.0) +
                 gauss_bubble(x, z, -0.15, 0.0, 50.0, 560.0, 640.0);
        // isentropic background: Exner pi = 1 - g z / (cp theta0), pbar = p0 pi^(cp/R)
        const double ex = 1.0 - P.g * z / (P.cp * P.theta0);
        const double pb = P.p0 * pow(ex, 1.0 / P.Rcp);
        const double T = (P.theta0 + th) * ex;
        const double rho = pb / (P.R * T);
        q[0] = rho;
        q[1] = 0.0;
        q[2] = 0.0;
        q[3] = pb / P.gm1 + rho * P.g * z;
    }
    double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) uc[v * n2 + node] = q[v];
}

// per-block maximum of |v| + c + 2 eta lambda_v (eta on the smaller cell size)
template <int N>
__global__ void k_max_speed(const double* __restrict__ u, double* __restrict__ partial, int cells,
                            const Basis B, const Phys P) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    __shared__ double red[256];
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (gid < cells * n2) {
        const int cell = gid / n2, node = gid - cell * n2;
        const int j = node / n;
        const int iy = cell / P.nx;
        const double z = P.y0 + (iy + B.xi[j]) * P.hy;
        const double* uc = u + (size_t)cell * SL;
        const double rho = uc[node], mx = uc[n2 + node], my = uc[2 * n2 + node], E = uc[3 * n2 + node];
        const double gz = P.gravity ? P.g * z : 0.0;
        const double p = P.gm1 * (E - 0.5 * (mx * mx + my * my) / rho - rho * gz);
        const double c = sqrt(P.gamma * p / rho);
        const double eta = fmax(P.eta_x, P.eta_y);
        s = sqrt(mx * mx + my * my) / rho + c + 2.0 * eta * P.lamv / rho;
        if (!(s == s)) s = 1e300;  // NaN: report as unstable
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_check_finite(const double* __restrict__ u, size_t count, int* flag) {
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < count;
         a += (size_t)gridDim.x * blockDim.x) {
        if (!isfinite(u[a])) {
            atomicOr(flag, 1);
            return;
        }
    }
}

// ------------------------------------------------------------------ launchers
template <int N>
static int tv_cells_n(const double* u, double* tv, double* part, int cells, int var, const Basis& B,
                      const Phys& P, cudaStream_t s) {
    using C = TvCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_tv_cells<N, C::cpb><<<blocks, C::cpb * C::n * C::n, 0, s>>>(u, tv, part, cells, var, B, P);
    return (int)cudaGetLastError();
}

int launch_tv_cells(int N, const double* u, double* tv, double* part, int cells, int var, const Basis& B,
                    const Phys& P, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return tv_cells_n<1>(u, tv, part, cells, var, B, P, s);
        case 2: return tv_cells_n<2>(u, tv, part, cells, var, B, P, s);
        case 3: return tv_cells_n<3>(u, tv, part, cells, var, B, P, s);
        case 4: return tv_cells_n<4>(u, tv, part, cells, var, B, P, s);
        case 5: return tv_cells_n<5>(u, tv, part, cells, var, B, P, s);
        case 6: return tv_cells_n<6>(u, tv, part, cells, var, B, P, s);
        case 7: return tv_cells_n<7>(u, tv, part, cells, var, B, P, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <int N>
static int init_n(double* u, int cells, int kind, double A, double a, double xc, double zc,
                  const Basis& B, const Phys& P, cudaStream_t s) {
    const int total = cells * (N + 1) * (N + 1);
    k_init<N><<<(total + 255) / 256, 256, 0, s>>>(u, cells, kind, A, a, xc, zc, B, P);
    return (int)cudaGetLastError();
}

int launch_init_scenario(int N, double* u, int cells, int kind, double A, double a, double xc,
                         double zc, const Basis& B, const Phys& P, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return init_n<1>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 2: return init_n<2>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 3: return init_n<3>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 4: return init_n<4>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 5: return init_n<5>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 6: return init_n<6>(u, cells, kind, A, a, xc, zc, B, P, s);
        case 7: return init_n<7>(u, cells, kind, A, a, xc, zc, B, P, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <int N>
static int speed_n(const double* u, double* partial, int cells, const Basis& B, const Phys& P,
                   int* nb, cudaStream_t s) {
    const int total = cells * (N + 1) * (N + 1);
    const int blocks = (total + 255) / 256;
    *nb = blocks;
    if (!partial) return 0;
    k_max_speed<N><<<blocks, 256, 0, s>>>(u, partial, cells, B, P);
    return (int)cudaGetLastError();
}

int launch_max_speed(int N, const double* u, double* partial, int cells, const Basis& B,
                     const Phys& P, int* nblocks_out, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return speed_n<1>(u, partial, cells, B, P, nblocks_out, s);
        case 2: return speed_n<2>(u, partial, cells, B, P, nblocks_out, s);
        case 3: return speed_n<3>(u, partial, cells, B, P, nblocks_out, s);
        case 4: return speed_n<4>(u, partial, cells, B, P, nblocks_out, s);
        case 5: return speed_n<5>(u, partial, cells, B, P, nblocks_out, s);
        case 6: return speed_n<6>(u, partial, cells, B, P, nblocks_out, s);
        case 7: return speed_n<7>(u, partial, cells, B, P, nblocks_out, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <int N>
static int tv_cells_mixed_n(const double* u, double* tv, double* part, int cells, int var, const BasisF& B,
                            const PhysF& P, const MixedBg& bg, float theta0, float omk, cudaStream_t s) {
    using C = TvCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_tv_cells_mixed<N, C::cpb>
        <<<blocks, C::cpb * C::n * C::n, 0, s>>>(u, tv, part, cells, var, B, P, bg, theta0, omk);
    return (int)cudaGetLastError();
}

int launch_tv_cells_mixed(int N, const double* u, double* tv, double* part, int cells, int var,
                          const BasisF& B, const PhysF& P, const MixedBg& bg, double theta0, double Rcp,
                          void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const float t0 = (float)theta0, omk = (float)(1.0 - Rcp);
    switch (N) {
        case 1: return tv_cells_mixed_n<1>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 2: return tv_cells_mixed_n<2>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 3: return tv_cells_mixed_n<3>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 4: return tv_cells_mixed_n<4>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 5: return tv_cells_mixed_n<5>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 6: return tv_cells_mixed_n<6>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
        case 7: return tv_cells_mixed_n<7>(u, tv, part, cells, var, B, P, bg, t0, omk, s);
    }
    return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------- statistics setup
int tv_stats_blocks(int N, int cells) { return (cells + tv_cpb(N) - 1) / tv_cpb(N); }

size_t tv_stats_scratch_doubles(int N, int cells) {
    return 5 * (size_t)tv_stats_blocks(N, cells) + 2 * (size_t)kTvLevels * kTvThreads;
}

static int tv_fold_per(int nblk) { return (nblk + kTvThreads - 1) / kTvThreads; }

TvStatsArgs tv_stats_args(int N, int cells, const double* part) {
    TvStatsArgs a;
    a.nblk = tv_stats_blocks(N, cells);
    a.per = tv_fold_per(a.nblk);
    a.cells = cells;
    a.part = part;
    a.wfold = part + 3 * (size_t)a.nblk;
    a.wtree = part + 5 * (size_t)a.nblk;
    return a;
}

// Weights n_b/(n_a+n_b) and n_a n_b/(n_a+n_b) of every combine of
// k_tv_stats_flags, from the block cell counts alone (IEEE division here).
int tv_stats_prepare(int N, int cells, double* part, void* stream) {
    static_assert(kTvThreads == 256 && kTvLevels == 8, "tree shape: 8 warps of 32");
    const int cpb = tv_cpb(N), nblk = tv_stats_blocks(N, cells), per = tv_fold_per(nblk);
    std::vector<double> w(2 * (size_t)nblk + 2 * (size_t)kTvLevels * kTvThreads, 0.0);
    double* wfold = w.data();
    double* wtree = w.data() + 2 * (size_t)nblk;
    auto put = [&](int level, int pos, double na, double nb) {
        wtree[2 * ((size_t)level * kTvThreads + pos)] = nb / (na + nb);
        wtree[2 * ((size_t)level * kTvThreads + pos) + 1] = na * nb / (na + nb);
    };
    std::vector<double> tcnt(kTvThreads, 0.0);
    for (int t = 0; t < kTvThreads; ++t) {
        const int k0 = t * per, k1 = std::min(k0 + per, nblk);
        double na = 0.0;
        for (int k = k0; k < k1; ++k) {
            const double nb = (double)std::min(cpb, cells - k * cpb);
            if (k > k0) {
                wfold[2 * k] = nb / (na + nb);
                wfold[2 * k + 1] = na * nb / (na + nb);
            }
            na += nb;
        }
        tcnt[t] = na;
    }
    // levels 0..4: lane l of each warp takes lane l + s, s = 16, 8, 4, 2, 1
    for (int l = 0, s = 16; s > 0; ++l, s >>= 1)
        for (int wp = 0; wp < kTvThreads / 32; ++wp)
            for (int lane = 0; lane < s; ++lane) {
                const int a = 32 * wp + lane, b = a + s;
                if (tcnt[b] > 0.0) {
                    put(l, a, tcnt[a], tcnt[b]);
                    tcnt[a] += tcnt[b];
                }
            }
    // levels 5..7: warp results, entry l takes entry l + s, s = 4, 2, 1
    std::vector<double> wc(kTvThreads / 32);
    for (int wp = 0; wp < kTvThreads / 32; ++wp) wc[wp] = tcnt[32 * wp];
    for (int l = 5, s = kTvThreads / 64; s > 0; ++l, s >>= 1)
        for (int a = 0; a < s; ++a)
            if (wc[a + s] > 0.0) {
                put(l, a, wc[a], wc[a + s]);
                wc[a] += wc[a + s];
            }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(part + 3 * (size_t)nblk, w.data(), w.size() * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host table must outlive the copy
    return (int)e;
}

int launch_tv_stats_flags(const double* tv, const TvStatsArgs& st, double T_r, double T_c, double* stats_dev,
                          int8_t* flags, void* stream) {
    // with flags: enough blocks for one cell per thread, at most one per SM
    // (every block repeats the combine); without: a single block
    int nb = 1;
    if (flags) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        nb = std::max(1, std::min((st.cells + kTvThreads - 1) / kTvThreads, sms));
    }
    // programmatic launch: scheduled while the TV-producing kernel drains,
    // waits for it in pdl_wait() before reading the TV values and triples
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kTvThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tv_stats_flags, tv, st, T_r, T_c, stats_dev, flags);
    return e != cudaSuccess ? (int)e : (int)cudaGetLastError();
}

int launch_tv_flags_given(const double* tv, int cells, const double* stats_dev, double T_r, double T_c,
                          int8_t* flags, void* stream) {
    const int nb = (cells + kPartThreads - 1) / kPartThreads;
    k_tv_flag_cells<<<nb, kPartThreads, 0, (cudaStream_t)stream>>>(tv, cells, stats_dev, T_r, T_c, flags);
    return (int)cudaGetLastError();
}

int launch_check_finite(const double* u, size_t count, int* flag, void* stream) {
    k_check_finite<<<1216, 256, 0, (cudaStream_t)stream>>>(u, count, flag);
    return (int)cudaGetLastError();
}

}  // namespace adg
