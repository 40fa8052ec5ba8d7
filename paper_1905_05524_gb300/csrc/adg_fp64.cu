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
#include "adg_fp64_body.cuh"
#include "adg_tv_cell.cuh"

namespace adg {

template <int N>
struct Fp64Cfg {
    static constexpr int n = N + 1;
    // cells per block: enough threads per block for small degrees
    static constexpr int cpb = tv_cpb(N);
    static constexpr int threads = cpb * n * n;
    static constexpr size_t smem_pred = (size_t)cpb * 3 * n * 4 * n * n * sizeof(double);
};

template <int N, int CPB, bool TSRC>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_fp64(const double* __restrict__ u, double* __restrict__ rvol,
                 double* __restrict__ trace, int cells, double dt, double t,
                 const Basis B, const Phys P, const Background bg) {
    constexpr int n = N + 1, n2 = n * n;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int j = (threadIdx.x - cl * n2) / n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int ix = cell % P.nx, iy = cell / P.nx;
    predictor_fp64_body<N, CPB, TSRC>(u, rvol, trace, cell, active, dt, B, P, P.x0 + ix * P.hx,
                                      P.y0 + iy * P.hy, bg.pbar_node[iy * n + j], bg.rhobar_node[iy * n + j],
                                      sm, t);
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

// No-slip wall (ADG_BC_NOSLIP): ghost density and pressure of the interior
// trace, velocity 2 v_wall - v (v_wall = (lid_u, 0) on the north wall, zero
// elsewhere), interior gradients, adiabatic (zero ghost heat flux).
__device__ __forceinline__ void noslip_ghost(const double* rec, int f, double z, const Phys& P, double qG[4],
                                             double fG[4], double& sG) {
    const double rho = rec[0], mx = rec[1], my = rec[2];
    const double wu = f == 2 ? P.lid_u : 0.0;
    const double rinv = 1.0 / rho;
    qG[0] = rho;
    qG[1] = 2.0 * rho * wu - mx;
    qG[2] = -my;
    // same pressure: only the kinetic energy changes
    qG[3] = rec[3] + 0.5 * ((qG[1] * qG[1] + qG[2] * qG[2]) - (mx * mx + my * my)) * rinv;
    Flux4 fl;
    ns_flux(qG, rec + 8, rec + 12, z, 0.0, 0.0, P, fl, true, 0.0, 0.0);
    const bool xdir = f < 2;
#pragma unroll
    for (int v = 0; v < 4; ++v) fG[v] = xdir ? fl.F[v] : fl.G[v];
    sG = wave_speed(qG, z, xdir, P);
}

// The Taylor-Green field (Sec. 4.1) and its x- and y-derivatives at (x, y, t):
// rho = 1, v = a (sin x cos y, -cos x sin y), p = b (cos 2x + cos 2y)/4 + 100/gamma,
// a = exp(-2 mu t), b = exp(-4 mu t).
__device__ __forceinline__ void taylor_green(double x, double y, double t, const Phys& P, double Q[4],
                                             double Qx[4], double Qy[4]) {
    const double a = exp(-2.0 * P.mu * t), b = exp(-4.0 * P.mu * t);
    double sx, cx, sy, cy, s2x, c2x, s2y, c2y;
    sincos(x, &sx, &cx);
    sincos(y, &sy, &cy);
    sincos(2.0 * x, &s2x, &c2x);
    sincos(2.0 * y, &s2y, &c2y);
    const double u = a * sx * cy, v = -a * cx * sy;
    const double ux = a * cx * cy, uy = -a * sx * sy, vx = a * sx * sy, vy = -a * cx * cy;
    const double p = 0.25 * b * (c2x + c2y) + 100.0 / P.gamma;
    const double px = -0.5 * b * s2x, py = -0.5 * b * s2y;
    Q[0] = 1.0;
    Q[1] = u;
    Q[2] = v;
    Q[3] = p / P.gm1 + 0.5 * (u * u + v * v);
    Qx[0] = 0.0;
    Qx[1] = ux;
    Qx[2] = vx;
    Qx[3] = px / P.gm1 + u * ux + v * vx;
    Qy[0] = 0.0;
    Qy[1] = uy;
    Qy[2] = vy;
    Qy[3] = py / P.gm1 + u * uy + v * vy;
}

// Analytic boundary (ADG_BC_ANALYTIC): the ghost is the field's state and
// normal flux at the face node (x, y), averaged over [t, t + dt] at the
// Gauss-Legendre time nodes like the interior traces.
__device__ __forceinline__ void analytic_ghost(double x, double y, int f, double t, double dt, const Basis& B,
                                               const Phys& P, int n, double qG[4], double fG[4], double& sG) {
    const bool xdir = f < 2;
#pragma unroll
    for (int v = 0; v < 4; ++v) qG[v] = fG[v] = 0.0;
    for (int k = 0; k < n; ++k) {
        double Q[4], Qx[4], Qy[4];
        taylor_green(x, y, t + B.xi[k] * dt, P, Q, Qx, Qy);
        Flux4 fl;
        ns_flux(Q, Qx, Qy, y, 0.0, 0.0, P, fl);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            qG[v] += B.w[k] * Q[v];
            fG[v] += B.w[k] * (xdir ? fl.F[v] : fl.G[v]);
        }
    }
    sG = wave_speed(qG, y, xdir, P);
}

// With TV the TV indicator of the updated state follows in the same kernel
// (tv_cell, bitwise what k_tv_cells computes).
template <int N, int CPB, bool TV>
__device__ __forceinline__ void corrector_fp64_body(double* __restrict__ u, const double* __restrict__ rvol,
                                                    const double* __restrict__ trace, int cells, int c0, double dt,
                                                    const Basis& B, const Phys& P, const Background& bg,
                                                    const TvEpilogue& epi, double t) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    __shared__ double Fst[CPB][4][4][n];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int ix = cell % P.nx, iy = cell / P.nx;

    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, m = idx - f * n;
        const bool xface = f < 2;
        const bool top = f == 2 && iy == P.ny - 1, bot = f == 3 && iy == 0;
        const bool wall = xface ? (P.bc_x == ADG_BC_WALL && ((f == 0 && ix == P.nx - 1) || (f == 1 && ix == 0)))
                                : ((P.bc_y == ADG_BC_WALL && (top || bot)) ||
                                   (P.bc_y == ADG_BC_WALL_EXCHANGE && bot) || (P.bc_y == ADG_BC_EXCHANGE_WALL && top));
        const bool halo = !xface && ((P.bc_y == ADG_BC_EXCHANGE && (top || bot)) ||
                                     (P.bc_y == ADG_BC_WALL_EXCHANGE && top) || (P.bc_y == ADG_BC_EXCHANGE_WALL && bot));
        // no-slip and analytic sides (Sec. 4.1 CFD scenarios)
        const bool edge = xface ? ((f == 0 && ix == P.nx - 1) || (f == 1 && ix == 0)) : (top || bot);
        const int side_bc = xface ? P.bc_x : P.bc_y;
        const bool noslip = edge && side_bc == ADG_BC_NOSLIP;
        const bool analytic = edge && side_bc == ADG_BC_ANALYTIC;
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
        } else if (noslip || analytic) {
            const double xf = xface ? P.x0 + (ix + (f == 0 ? 1 : 0)) * P.hx : P.x0 + (ix + B.xi[m]) * P.hx;
            const double yf = xface ? P.y0 + (iy + B.xi[m]) * P.hy : P.y0 + (iy + (f == 2 ? 1 : 0)) * P.hy;
            if (noslip) noslip_ghost(rec, f, yf, P, qn, fn, sn);
            else analytic_ghost(xf, yf, f, t, dt, B, P, n, qn, fn, sn);
        } else {
            int nb, nf;
            if (f == 0) { nb = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1); nf = 1; }
            else if (f == 1) { nb = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1); nf = 0; }
            else if (f == 2) { nb = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix; nf = 3; }
            else { nb = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix; nf = 2; }
            const double* ot = halo ? (f == 2 ? bg.halo_n : bg.halo_s) + (size_t)ix * TR
                                    : trace + ((size_t)nb * 4 + nf) * TR;
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
    double* uc = u + (size_t)cell * SL;
    const double* rc = rvol + (size_t)cell * SL;
    double unew[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double face = (B.lift1[i] * Fst[cl][0][v][j] - B.lift0[i] * Fst[cl][1][v][j]) * P.inv_hx +
                            (B.lift1[j] * Fst[cl][2][v][i] - B.lift0[j] * Fst[cl][3][v][i]) * P.inv_hy;
        if (active) {  // padding threads touch no state
            unew[v] = uc[v * n2 + node] + dt * (rc[v * n2 + node] - face);
            uc[v * n2 + node] = unew[v];
        } else {
            unew[v] = 1.0;
        }
    }
    if constexpr (TV) {
        __shared__ double fs[CPB][n2], red[CPB][n2];
        const double z = tv_node_z(iy, j, B, P);
        const double f = epi.var == ADG_TV_THETA ? theta_of(unew, z, P) : unew[0];
        static_assert(CPB == tv_cpb(N), "the TV statistics combine blocks of tv_cpb(N) cells");
        const double r =
            tv_cell<N, double>(f, 0.0, node, i, j, B, P.inv_hx, P.inv_hy, fs[cl], red[cl], active, epi.tv + cell);
        tv_block_triple<CPB>(r, node == 0, cl, min(CPB, cells - c0), epi.part);
    }
}

template <int N, int CPB, bool TV>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_fp64(double* __restrict__ u, const double* __restrict__ rvol,
                 const double* __restrict__ trace, int cells, double dt, const Basis B,
                 const Phys P, const Background bg, const TvEpilogue epi, double t) {
    corrector_fp64_body<N, CPB, TV>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P, bg, epi, t);
}

// Batched persistent FP64 kernels over uniform instances (tile = instance,
// first cell; tile t goes to block t mod grid): the per-mesh bodies.
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_batch_fp64(const Fp64Inst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                       const Basis B) {
    constexpr int n = N + 1, n2 = n * n;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int j = (threadIdx.x - cl * n2) / n;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const BatchTile tl = tiles[tt];
        const Fp64Inst& I = insts[tl.inst];
        const Phys P = I.P;
        const int cell_raw = tl.c0 + cl;
        const bool active = cell_raw < I.cells;
        const int cell = active ? cell_raw : I.cells - 1;
        const int ix = cell % P.nx, iy = cell / P.nx;
        predictor_fp64_body<N, CPB>(I.u, I.rvol, I.trace, cell, active, I.dt, B, P, P.x0 + ix * P.hx,
                                    P.y0 + iy * P.hy, I.bg.pbar_node[iy * n + j], I.bg.rhobar_node[iy * n + j], sm);
        __syncthreads();
    }
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_batch_fp64(const Fp64Inst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                       const Basis B) {
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const BatchTile tl = tiles[tt];
        const Fp64Inst& I = insts[tl.inst];
        const Phys P = I.P;
        const Background bg = I.bg;
        corrector_fp64_body<N, CPB, false>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dt, B, P, bg, TvEpilogue{}, 0.0);
        __syncthreads();
    }
}

template <int N>
static int batch_fp64_n(int phase, const Fp64Inst* insts, const BatchTile* tiles, int ntiles, const Basis& B,
                        int* cpb_out, int* blocks_io, cudaStream_t s) {
    using C = Fp64Cfg<N>;
    if (cpb_out) *cpb_out = C::cpb;
    if (!tiles) {  // query: smem limit and persistent grid (not during capture)
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e;
        if (phase == 0) {
            e = cudaFuncSetAttribute(k_predictor_batch_fp64<N, C::cpb>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)C::smem_pred);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_predictor_batch_fp64<N, C::cpb>,
                                                                  C::threads, C::smem_pred);
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_corrector_batch_fp64<N, C::cpb>, C::threads,
                                                              0);
        }
        if (e != cudaSuccess) return (int)e;
        if (blocks_io) *blocks_io = per_sm > 0 ? per_sm * sms : sms;
        return 0;
    }
    if (phase == 0)
        k_predictor_batch_fp64<N, C::cpb><<<*blocks_io, C::threads, C::smem_pred, s>>>(insts, tiles, ntiles, B);
    else
        k_corrector_batch_fp64<N, C::cpb><<<*blocks_io, C::threads, 0, s>>>(insts, tiles, ntiles, B);
    return (int)cudaGetLastError();
}

int launch_batch_fp64(int N, int phase, const Fp64Inst* insts, const BatchTile* tiles, int ntiles, const Basis& B,
                      int* cpb_out, int* blocks_out, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return batch_fp64_n<1>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 2: return batch_fp64_n<2>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 3: return batch_fp64_n<3>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 4: return batch_fp64_n<4>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 5: return batch_fp64_n<5>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 6: return batch_fp64_n<6>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
        case 7: return batch_fp64_n<7>(phase, insts, tiles, ntiles, B, cpb_out, blocks_out, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <int N>
static int launch_pred(const double* u, double* rvol, double* trace, int cells, double dt,
                       double t, const Basis& B, const Phys& P, const Background& bg,
                       cudaStream_t s) {
    using C = Fp64Cfg<N>;
    auto kern = P.source == ADG_SRC_PAPER ? k_predictor_fp64<N, C::cpb, true> : k_predictor_fp64<N, C::cpb, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_pred);
    if (e != cudaSuccess) return (int)e;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    kern<<<blocks, C::threads, C::smem_pred, s>>>(u, rvol, trace, cells, dt, t, B, P, bg);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_corr(double* u, const double* rvol, const double* trace, int cells, double dt,
                       const Basis& B, const Phys& P, const Background& bg, const TvEpilogue* epi,
                       double t, cudaStream_t s) {
    using C = Fp64Cfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    if (epi)
        k_corrector_fp64<N, C::cpb, true>
            <<<blocks, C::threads, 0, s>>>(u, rvol, trace, cells, dt, B, P, bg, *epi, t);
    else
        k_corrector_fp64<N, C::cpb, false>
            <<<blocks, C::threads, 0, s>>>(u, rvol, trace, cells, dt, B, P, bg, TvEpilogue{}, t);
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
                          void* stream, const TvEpilogue* epi, double t) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return launch_corr<1>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 2: return launch_corr<2>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 3: return launch_corr<3>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 4: return launch_corr<4>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 5: return launch_corr<5>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 6: return launch_corr<6>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
        case 7: return launch_corr<7>(u, rvol, trace, cells, dt, B, P, bg, epi, t, s);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace adg
