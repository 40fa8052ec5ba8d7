// Total-variation refinement indicator (Sec. 3, Eqs. 6-8), scenario
// initialisation (Sec. 4.1, 4.2), stable time step and finiteness scan.
//
// TV per cell: TV = sum_ij w_i w_j (|df/dx| + |df/dy|) with f = theta
// (potential temperature, Sec. 4.2) or rho at the nodes, derivatives by the
// nodal derivative matrix.  Mean and population standard deviation over all
// cells follow Chan, Golub and LeVeque's pairwise update (cited by the paper
// for a parallel, stable evaluation): contiguous chunks are reduced exactly
// (two-pass) per block, then the partial (count, mean, M2) triples are
// combined in a fixed binary tree, so the result is deterministic.
#include <cuda_runtime.h>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_physics.cuh"

namespace adg {

template <int N>
struct TvCfg {
    static constexpr int n = N + 1;
    static constexpr int cpb = N == 1 ? 32 : N == 2 ? 16 : N == 3 ? 8 : N <= 5 ? 4 : 2;
};

__device__ __forceinline__ double theta_of(const double q[4], double z, const Phys& P) {
    const double rinv = 1.0 / q[0];
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) * rinv - q[0] * gz);
    const double T = p * rinv * P.invR;
    return T * pow(P.p0 / p, P.Rcp);
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_tv_cells(const double* __restrict__ u, double* __restrict__ tv, int cells, int var,
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
    const double z = P.y0 + (iy + B.xi[j]) * P.hy;
    fs[cl][node] = var == ADG_TV_THETA ? theta_of(q, z, P) : q[0];
    __syncthreads();
    double fx = 0.0, fy = 0.0;
#pragma unroll
    for (int p = 0; p < n; ++p) {
        fx += B.D[i][p] * fs[cl][j * n + p];
        fy += B.D[j][p] * fs[cl][p * n + i];
    }
    red[cl][node] = B.w[i] * B.w[j] * (fabs(fx * P.inv_hx) + fabs(fy * P.inv_hy));
    __syncthreads();
    if (node == 0 && active) {
        double s = 0.0;
        for (int a = 0; a < n2; ++a) s += red[cl][a];
        tv[cell] = s;
    }
}

// Mixed-precision TV: the indicator field is formed from the FP64 state by
// the FP64 perturbation split (rho' = rho - rhobar, E' = rhoE - Ebar) and then
// in FP32.  For theta the potential-temperature perturbation is evaluated
// without the 300 K offset,
//     theta'/theta0 = (1 + p'/pbar)^(1-R/cp) / (1 + rho'/rhobar) - 1
//                   = expm1((1 - R/cp) log1p(p'/pbar) - log1p(rho'/rhobar)),
// (theta = p^(1-R/cp) p0^(R/cp) / (rho R) and theta0 is the same expression
// at the background), so no FP32 value carries theta ~ 300 K.  For rho the
// field is rho' and the background gradient d rhobar/dz is added.
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_tv_cells_mixed(const double* __restrict__ u, double* __restrict__ tv, int cells, int var,
                 const BasisF B, const PhysF P, const MixedBg bg, float theta0, float one_m_kappa) {
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
    const double rb64 = bg.rb[row];
    const float rp = f64_to_f32(uc[node] - rb64);
    float f;
    if (var == ADG_TV_THETA) {
        const float Ep = f64_to_f32(uc[3 * n2 + node] - bg.Eb[row]);
        const float mx = f64_to_f32(uc[n2 + node]), my = f64_to_f32(uc[2 * n2 + node]);
        const float rb = f64_to_f32(rb64);
        const float rho = rb + rp;
        const float z = P.y0 + (iy + B.xi[j]) * P.hy;
        const float pp = P.gm1 * (Ep - 0.5f * (mx * mx + my * my) / rho - P.g * z * rp);
        f = theta0 * expm1f(one_m_kappa * log1pf(pp / bg.pb[row]) - log1pf(rp / rb));
    } else {
        f = rp;
    }
    fs[cl][node] = f;
    __syncthreads();
    float fx = 0.f, fy = 0.f;
#pragma unroll
    for (int p = 0; p < n; ++p) {
        fx = fmaf(B.D[i][p], fs[cl][j * n + p], fx);
        fy = fmaf(B.D[j][p], fs[cl][p * n + i], fy);
    }
    fx *= P.inv_hx;
    fy *= P.inv_hy;
    if (var != ADG_TV_THETA) fy += bg.dzr[row];
    red[cl][node] = B.w[i] * B.w[j] * (fabsf(fx) + fabsf(fy));
    __syncthreads();
    if (node == 0 && active) {
        float s = 0.f;  // FP32 sum of n^2 positive terms: relative error ~n^2 * 6e-8
        for (int a = 0; a < n2; ++a) s += red[cl][a];
        tv[cell] = f32_to_f64(s);
    }
}

// Multi-block statistics.  Block b owns the contiguous chunk of cells
// [b*chunk, min((b+1)*chunk, cells)); it forms the chunk's count, mean and M2
// by an exact two-pass reduction in a fixed tree and writes the triple to
// part[b] (scratch).  k_tv_flags then combines the partial triples with Chan
// et al.'s pairwise update in a fixed binary tree (deterministic) and writes
// the flags.
constexpr int kPartThreads = 256;

__device__ __forceinline__ double block_sum_256(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = kPartThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kPartThreads)
k_tv_partials(const double* __restrict__ tv, int cells, int chunk, double* __restrict__ part) {
    __shared__ double sh[kPartThreads];
    const int b = blockIdx.x;
    const int lo = b * chunk;
    const int hi = min(cells, lo + chunk);
    double s = 0.0;
    for (int c = lo + threadIdx.x; c < hi; c += kPartThreads) s += tv[c];
    const double cnt = (double)max(0, hi - lo);
    const double sum = block_sum_256(s, sh);
    const double mean = cnt > 0.0 ? sum / cnt : 0.0;
    double q = 0.0;
    for (int c = lo + threadIdx.x; c < hi; c += kPartThreads) {
        const double d = tv[c] - mean;
        q += d * d;
    }
    const double m2 = block_sum_256(q, sh);
    if (threadIdx.x == 0) {
        part[3 * b + 0] = cnt;
        part[3 * b + 1] = mean;
        part[3 * b + 2] = m2;
    }
}

constexpr int kMaxPartials = 1024;

// Every block combines all partial triples in the same fixed binary tree
// (so every block obtains bitwise the same mean and sigma), block 0 writes
// them out, and each block flags its own chunk of cells.  Spreading the FP64
// flag comparisons over many SMs matters on a part with 2 FP64 FMA per clock
// per SM.
__global__ void __launch_bounds__(kPartThreads)
k_tv_flags(const double* __restrict__ part, int nparts, const double* __restrict__ tv, int cells, int chunk,
           double T_r, double T_c, double* __restrict__ stats, int8_t* __restrict__ flags) {
    __shared__ double sc[kMaxPartials], smean[kMaxPartials], sm2[kMaxPartials];
    const int t = threadIdx.x;
    for (int a = t; a < kMaxPartials; a += kPartThreads) {
        sc[a] = a < nparts ? part[3 * a] : 0.0;
        smean[a] = a < nparts ? part[3 * a + 1] : 0.0;
        sm2[a] = a < nparts ? part[3 * a + 2] : 0.0;
    }
    __syncthreads();
    int top = 1;
    while (top < nparts) top <<= 1;
    for (int stride = top / 2; stride > 0; stride >>= 1) {
        for (int a = t; a < stride; a += kPartThreads) {
            const double na = sc[a], nb = sc[a + stride];
            const double nn = na + nb;
            if (nb > 0.0) {
                const double d = smean[a + stride] - smean[a];
                smean[a] = smean[a] + d * (nb / nn);
                sm2[a] = sm2[a] + sm2[a + stride] + d * d * (na * nb / nn);
                sc[a] = nn;
            }
        }
        __syncthreads();
    }
    const double mu = smean[0];
    const double sig = sc[0] > 0.0 ? sqrt(sm2[0] / sc[0]) : 0.0;
    if (blockIdx.x == 0 && t == 0 && stats) {
        stats[0] = mu;
        stats[1] = sig;
    }
    if (!flags) return;
    const double thr_r = mu + T_r * sig;
    const double thr_c = mu + T_c * sig;
    const bool flat = sig <= 1e-12 * fabs(mu);  // reading F1: keep all
    const int lo = blockIdx.x * chunk, hi = min(cells, lo + chunk);
    for (int c = lo + t; c < hi; c += kPartThreads) {
        const double x = tv[c];
        flags[c] = flat ? (int8_t)0 : x >= thr_r ? (int8_t)1 : (x < thr_c ? (int8_t)-1 : (int8_t)0);
    }
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
static int tv_cells_n(const double* u, double* tv, int cells, int var, const Basis& B,
                      const Phys& P, cudaStream_t s) {
    using C = TvCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_tv_cells<N, C::cpb><<<blocks, C::cpb * C::n * C::n, 0, s>>>(u, tv, cells, var, B, P);
    return (int)cudaGetLastError();
}

int launch_tv_cells(int N, const double* u, double* tv, int cells, int var, const Basis& B,
                    const Phys& P, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return tv_cells_n<1>(u, tv, cells, var, B, P, s);
        case 2: return tv_cells_n<2>(u, tv, cells, var, B, P, s);
        case 3: return tv_cells_n<3>(u, tv, cells, var, B, P, s);
        case 4: return tv_cells_n<4>(u, tv, cells, var, B, P, s);
        case 5: return tv_cells_n<5>(u, tv, cells, var, B, P, s);
        case 6: return tv_cells_n<6>(u, tv, cells, var, B, P, s);
        case 7: return tv_cells_n<7>(u, tv, cells, var, B, P, s);
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
static int tv_cells_mixed_n(const double* u, double* tv, int cells, int var, const BasisF& B,
                            const PhysF& P, const MixedBg& bg, float theta0, float omk, cudaStream_t s) {
    using C = TvCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    k_tv_cells_mixed<N, C::cpb><<<blocks, C::cpb * C::n * C::n, 0, s>>>(u, tv, cells, var, B, P, bg, theta0, omk);
    return (int)cudaGetLastError();
}

int launch_tv_cells_mixed(int N, const double* u, double* tv, int cells, int var, const BasisF& B,
                          const PhysF& P, const MixedBg& bg, double theta0, double Rcp, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const float t0 = (float)theta0, omk = (float)(1.0 - Rcp);
    switch (N) {
        case 1: return tv_cells_mixed_n<1>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 2: return tv_cells_mixed_n<2>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 3: return tv_cells_mixed_n<3>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 4: return tv_cells_mixed_n<4>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 5: return tv_cells_mixed_n<5>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 6: return tv_cells_mixed_n<6>(u, tv, cells, var, B, P, bg, t0, omk, s);
        case 7: return tv_cells_mixed_n<7>(u, tv, cells, var, B, P, bg, t0, omk, s);
    }
    return (int)cudaErrorInvalidValue;
}

int tv_stats_partials(int cells) {
    const int chunk = tv_stats_chunk(cells);
    return (cells + chunk - 1) / chunk;
}

int tv_stats_chunk(int cells) {
    int chunk = 256;
    while ((cells + chunk - 1) / chunk > kMaxPartials) chunk *= 2;
    return chunk;
}

int launch_tv_stats_multi(const double* tv, int cells, double T_r, double T_c, double* part,
                          double* stats_dev, int8_t* flags, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = tv_stats_chunk(cells);
    const int np = (cells + chunk - 1) / chunk;
    k_tv_partials<<<np, kPartThreads, 0, s>>>(tv, cells, chunk, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    k_tv_flags<<<np, kPartThreads, 0, s>>>(part, np, tv, cells, chunk, T_r, T_c, stats_dev, flags);
    return (int)cudaGetLastError();
}

int launch_tv_flags_given(const double* tv, int cells, const double* part1, double T_r, double T_c,
                          int8_t* flags, void* stream) {
    const int chunk = tv_stats_chunk(cells);
    const int nb = (cells + chunk - 1) / chunk;
    k_tv_flags<<<nb, kPartThreads, 0, (cudaStream_t)stream>>>(part1, 1, tv, cells, chunk, T_r, T_c, nullptr, flags);
    return (int)cudaGetLastError();
}

int launch_check_finite(const double* u, size_t count, int* flag, void* stream) {
    k_check_finite<<<1216, 256, 0, (cudaStream_t)stream>>>(u, count, flag);
    return (int)cudaGetLastError();
}

}  // namespace adg
