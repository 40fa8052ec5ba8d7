// MUSCL-Hancock finite-volume scheme with the van Albada limiter for the
// inviscid equations of Sec. 2 (the paper's second scheme, Sec. 3; run
// without viscosity on the colliding bubbles, Sec. 4.2).  Unsplit MUSCL-
// Hancock on cell averages of (rho, rho u, rho v, rho E), FP64:
//
//  1. k_fv_half, one thread per cell: perturbations U' = U - Ubar(z_centre)
//     of the hydrostatic background (zero without gravity), van Albada
//     slopes a b (a + b) / (a^2 + b^2) of U' per direction (zero next to a
//     wall in its direction), face states Ubar(z_face) + U' +- slope/2 (the
//     background at rest is reproduced exactly at every face), their
//     half-step evolution with the cell's own flux differences and the
//     source -g rho' at the centre; writes the four face states and the
//     half-step rho' of the cell.
//  2. k_fv_update, one thread per cell: Rusanov fluxes (s = max |v.n| + c)
//     on its four faces from its own and its neighbours' face states (a
//     slip-wall ghost with the background rho, rhoE and reflected momentum
//     on walls), then U -= dt/h (flux differences) and the source at the
//     half-step mean.  Each face is computed by both its cells with the
//     same operands in the same order, so both see bitwise the same flux.
//
// Momentum fluxes carry p' = p - pbar(z) at the height where they are
// evaluated (Eq. 7).  State layout: u[v][iy][ix] (structure of arrays).
//
// Mixed precision (k_fv_step_mixed): the same scheme as one fused kernel per
// step on shared-memory tiles, FP32 arithmetic on perturbations of the
// background, FP64 state and accumulation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mesh.h"

struct adg_fv {
    adg_mesh_desc d;
    int cells = 0;
    double hx = 0, hy = 0, gm1 = 0;
    double* u = nullptr;       // [4][cells]
    double* half = nullptr;    // [17][cells]: UE, UW, UN, US (4 each), rho' at the half step
    double* bg = nullptr;      // [6][ny] centre rhobar, Ebar, pbar; [3][ny + 1] face rhobar, Ebar, pbar
    double* part = nullptr;    // stable-dt block maxima
    int part_blocks = 0;
    // mixed precision: second state buffer (the fused step reads u, writes
    // u2, then the two swap) and the FP32 background tables
    double* u2 = nullptr;
    float4* pert = nullptr;    // FP32 perturbations of u (kept current by the step; ping-pong with pert2)
    float4* pert2 = nullptr;
    bool pert_stale = true;    // u was changed outside the step
    float* bgf = nullptr;      // [ny] centre (rhobar, pbar, Ebar + pbar, g z), [ny + 1] faces
                               // (rhobar, pbar, 0, g z), [ny] face minus centre Ebar + pbar (north, south)
};

namespace adg {
namespace {

struct FvPhys {
    double gamma, gm1, g, hx, hy, x0, y0;
    int nx, ny, cells, wall_x, wall_y, gravity;
    const double* rbc;  // [ny] background at cell centres
    const double* Ebc;
    const double* pbc;
    const double* rbf;  // [ny + 1] background at horizontal faces
    const double* Ebf;
    const double* pbf;
};

__device__ __forceinline__ double van_albada(double a, double b) {
    const double ab = a * b;
    return ab > 0.0 ? ab * (a + b) / (a * a + b * b) : 0.0;
}

// inviscid flux along x (xdir) or y with p' = p - pbar at height z
__device__ __forceinline__ void euler_flux(const double q[4], double z, double pbar, bool xdir, const FvPhys& P,
                                           double f[4]) {
    const double rinv = 1.0 / q[0];
    const double u = q[1] * rinv, v = q[2] * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v) - q[0] * gz);
    const double vn = xdir ? u : v;
    f[0] = xdir ? q[1] : q[2];
    f[1] = q[1] * vn + (xdir ? p - pbar : 0.0);
    f[2] = q[2] * vn + (xdir ? 0.0 : p - pbar);
    f[3] = vn * (q[3] + p);
}

__device__ __forceinline__ double euler_speed(const double q[4], double z, bool xdir, const FvPhys& P) {
    const double rinv = 1.0 / q[0];
    const double u = q[1] * rinv, v = q[2] * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v) - q[0] * gz);
    return fabs(xdir ? u : v) + sqrt(P.gamma * p * rinv);
}

// F* = (F_L + F_R)/2 - max(s_L, s_R)(q_R - q_L)/2 with explicit rounding
__device__ __forceinline__ void rusanov_fv(const double qL[4], const double qR[4], double z, double pbar, bool xdir,
                                           const FvPhys& P, double out[4]) {
    double fL[4], fR[4];
    euler_flux(qL, z, pbar, xdir, P, fL);
    euler_flux(qR, z, pbar, xdir, P, fR);
    const double hs = __dmul_rn(-0.5, fmax(euler_speed(qL, z, xdir, P), euler_speed(qR, z, xdir, P)));
#pragma unroll
    for (int v = 0; v < 4; ++v)
        out[v] = __fma_rn(hs, __dsub_rn(qR[v], qL[v]), __dmul_rn(0.5, __dadd_rn(fL[v], fR[v])));
}

// slip-wall ghost of a face state (background rho, rhoE at height z with gravity)
__device__ __forceinline__ void wall_ghost_fv(const double q[4], double nx, double ny, double rbf, double Ebf,
                                              const FvPhys& P, double g[4]) {
    const double mn = q[1] * nx + q[2] * ny;
    g[0] = P.gravity ? rbf : q[0];
    g[1] = q[1] - 2.0 * mn * nx;
    g[2] = q[2] - 2.0 * mn * ny;
    g[3] = P.gravity ? Ebf : q[3];
}

__global__ void __launch_bounds__(256) k_fv_half(const double* __restrict__ u, double* __restrict__ half,
                                                 double dt, const FvPhys P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.cells) return;
    const int ix = c % P.nx, iy = c / P.nx;
    const int e = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1), w = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1);
    const int nn = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix, s = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix;
    const int iyn = iy + 1 == P.ny ? 0 : iy + 1, iys = iy == 0 ? P.ny - 1 : iy - 1;
    const bool flat_x = P.wall_x && (ix == 0 || ix == P.nx - 1);
    const bool flat_y = P.wall_y && (iy == 0 || iy == P.ny - 1);
    const double bc[4] = {P.rbc[iy], 0.0, 0.0, P.Ebc[iy]};
    const double bn[4] = {P.rbc[iyn], 0.0, 0.0, P.Ebc[iyn]};
    const double bs[4] = {P.rbc[iys], 0.0, 0.0, P.Ebc[iys]};
    const double bfn[4] = {P.rbf[iy + 1], 0.0, 0.0, P.Ebf[iy + 1]};
    const double bfs[4] = {P.rbf[iy], 0.0, 0.0, P.Ebf[iy]};
    double UE[4], UW[4], UN[4], US[4], U[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const size_t o = (size_t)v * P.cells;
        U[v] = u[o + c];
        const double up = U[v] - bc[v];
        const double sx = flat_x ? 0.0 : van_albada(up - (u[o + w] - bc[v]), (u[o + e] - bc[v]) - up);
        const double sy = flat_y ? 0.0 : van_albada(up - (u[o + s] - bs[v]), (u[o + nn] - bn[v]) - up);
        UE[v] = U[v] + 0.5 * sx;
        UW[v] = U[v] - 0.5 * sx;
        UN[v] = bfn[v] + up + 0.5 * sy;
        US[v] = bfs[v] + up - 0.5 * sy;
    }
    const double zc = P.y0 + (iy + 0.5) * P.hy;
    const double zn = P.y0 + (iy + 1) * P.hy, zs = P.y0 + iy * P.hy;
    double fE[4], fW[4], gN[4], gS[4];
    euler_flux(UE, zc, P.pbc[iy], true, P, fE);
    euler_flux(UW, zc, P.pbc[iy], true, P, fW);
    euler_flux(UN, zn, P.pbf[iy + 1], false, P, gN);
    euler_flux(US, zs, P.pbf[iy], false, P, gS);
    const double ax = 0.5 * dt / P.hx, ay = 0.5 * dt / P.hy;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        double d = -ax * (fE[v] - fW[v]) - ay * (gN[v] - gS[v]);
        if (v == 2 && P.gravity) d += 0.5 * dt * (-P.g * (U[0] - bc[0]));
        half[(size_t)(0 + v) * P.cells + c] = UE[v] + d;
        half[(size_t)(4 + v) * P.cells + c] = UW[v] + d;
        half[(size_t)(8 + v) * P.cells + c] = UN[v] + d;
        half[(size_t)(12 + v) * P.cells + c] = US[v] + d;
        if (v == 0) half[(size_t)16 * P.cells + c] = (U[0] + d) - bc[0];  // rho' of the half-step mean
    }
}

__global__ void __launch_bounds__(256) k_fv_update(double* __restrict__ u, const double* __restrict__ half,
                                                   double dt, const FvPhys P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.cells) return;
    const int ix = c % P.nx, iy = c / P.nx;
    const int e = iy * P.nx + (ix + 1 == P.nx ? 0 : ix + 1), w = iy * P.nx + (ix == 0 ? P.nx - 1 : ix - 1);
    const int nn = (iy + 1 == P.ny ? 0 : iy + 1) * P.nx + ix, s = (iy == 0 ? P.ny - 1 : iy - 1) * P.nx + ix;
    auto ld = [&](int slot, int cell, double q[4]) {
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = half[(size_t)(slot + v) * P.cells + cell];
    };
    const double zc = P.y0 + (iy + 0.5) * P.hy;
    const double zn = P.y0 + (iy + 1) * P.hy, zs = P.y0 + iy * P.hy;
    double own[4], nb[4], FE[4], FW[4], GN[4], GS[4];
    // east face: own E state (left), east neighbour's W state (right)
    ld(0, c, own);
    if (P.wall_x && ix == P.nx - 1) wall_ghost_fv(own, 1.0, 0.0, P.rbc[iy], P.Ebc[iy], P, nb);
    else ld(4, e, nb);
    rusanov_fv(own, nb, zc, P.pbc[iy], true, P, FE);
    // west face: west neighbour's E state (left), own W state (right)
    ld(4, c, own);
    if (P.wall_x && ix == 0) wall_ghost_fv(own, -1.0, 0.0, P.rbc[iy], P.Ebc[iy], P, nb);
    else ld(0, w, nb);
    rusanov_fv(nb, own, zc, P.pbc[iy], true, P, FW);
    // north face: own N state (below), north neighbour's S state (above)
    ld(8, c, own);
    if (P.wall_y && iy == P.ny - 1) wall_ghost_fv(own, 0.0, 1.0, P.rbf[iy + 1], P.Ebf[iy + 1], P, nb);
    else ld(12, nn, nb);
    rusanov_fv(own, nb, zn, P.pbf[iy + 1], false, P, GN);
    // south face: south neighbour's N state (below), own S state (above)
    ld(12, c, own);
    if (P.wall_y && iy == 0) wall_ghost_fv(own, 0.0, -1.0, P.rbf[iy], P.Ebf[iy], P, nb);
    else ld(8, s, nb);
    rusanov_fv(nb, own, zs, P.pbf[iy], false, P, GS);
    const double rp = half[(size_t)16 * P.cells + c];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const size_t o = (size_t)v * P.cells + c;
        double du = -dt / P.hx * (FE[v] - FW[v]) - dt / P.hy * (GN[v] - GS[v]);
        if (v == 2 && P.gravity) du += dt * (-P.g * rp);
        u[o] += du;
    }
}

// per-block maxima of (|u| + c) and (|v| + c) at cell centres
__global__ void __launch_bounds__(256) k_fv_speed(const double* __restrict__ u, double* __restrict__ part,
                                                  const FvPhys P) {
    __shared__ double sx[256], sy[256];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double ax = 0.0, ay = 0.0;
    if (c < P.cells) {
        const int iy = c / P.nx;
        double q[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = u[(size_t)v * P.cells + c];
        const double zc = P.y0 + (iy + 0.5) * P.hy;
        ax = euler_speed(q, zc, true, P);
        ay = euler_speed(q, zc, false, P);
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            sx[threadIdx.x] = fmax(sx[threadIdx.x], sx[threadIdx.x + k]);
            sy[threadIdx.x] = fmax(sy[threadIdx.x], sy[threadIdx.x + k]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sx[0];
        part[2 * blockIdx.x + 1] = sy[0];
    }
}

__device__ double fv_bubble(double x, double z, double A, double a, double s, double xc, double zc) {
    const double r = sqrt((x - xc) * (x - xc) + (z - zc) * (z - zc));
    return r <= a ? A : A * exp(-((r - a) * (r - a)) / (s * s));
}

// ---------------------------------------------------------------------------
// Mixed precision: one fused kernel per step on tiles of kFvTx x kFvTy cells.
// The FP64 state is split once per loaded cell into FP32 perturbations of the
// row's centre background (rho' = rho - rhobar, E' = rhoE - Ebar: two FP64
// subtractions, integer-pipe conversions); everything after that is FP32:
//   phase 1  perturbations of the tile plus a 2-cell halo into shared memory;
//   phase 2  van Albada slopes, face states and their half-step evolution for
//            the tile plus a 1-cell halo (face states stay perturbations: the
//            x-faces of the row's centre background, the y-faces of the
//            background at the face height, so both states of a face share
//            one base and the Rusanov jump is a jump of perturbations);
//   phase 3  one Rusanov flux per face of the tile (a face on a tile edge is
//            computed by both tiles with the same operands and instructions);
//   phase 4  du in FP32, accumulated in FP64: uo = u + du.
// The flux of a perturbation state over the base (rhobar, pbar, g z) uses
// rho = rhobar + rho' and p' = (gamma - 1)(E' - |m|^2/(2 rho) - g z rho').
// The energy flux v.n (Hbar + h'), h' = E' + p', Hbar = Ebar + pbar, is kept
// in two parts, v.n and v.n h', and Hbar enters only as products with
// velocity differences: Hbar_c (v_E - v_W) for x-faces and, for y-faces,
// Hbar_c (v_N - v_S) + dN v_N - dS v_S with dN, dS the face enthalpies minus
// the centre one formed in FP64.  The sum Hbar + h' (h' is five orders of
// magnitude smaller) and the face enthalpies themselves are never rounded
// to FP32.  Reads u, writes uo (the state is double-buffered).
constexpr int kFvTx = 32, kFvTy = 8, kFvThreads = kFvTx * kFvTy;
constexpr int kFvPw = kFvTx + 4, kFvPh = kFvTy + 4;  // perturbation tile (halo 2)
constexpr int kFvHw = kFvTx + 2, kFvHh = kFvTy + 2;  // half-step tile (halo 1)
constexpr int kFvFx = (kFvTx + 1) * kFvTy;           // x-faces of a tile
constexpr int kFvFy = kFvTx * (kFvTy + 1);           // y-faces of a tile
constexpr int kFvShared = (kFvFx + kFvFy) > kFvPw * kFvPh ? (kFvFx + kFvFy) : kFvPw * kFvPh;
// dynamic shared memory: perturbations / face fluxes, four half-step face
// states, half-step rho', face velocity factors
constexpr size_t kFvSmemBytes =
    sizeof(float4) * ((size_t)kFvShared + 4 * (size_t)kFvHh * kFvHw) + sizeof(float) * ((size_t)kFvThreads + kFvFx + kFvFy);

struct FvMixed {
    const double* rbc;  // [ny] centre rhobar (FP64, for the split)
    const double* Ebc;  // [ny] centre Ebar
    const float4* cb;   // [ny] centre (rhobar, pbar, Hbar, g z)
    const float4* fb;   // [ny + 1] faces (rhobar, pbar, 0, g z)
    const float2* dh;   // [ny] Hbar(north face) - Hbar_c, Hbar(south face) - Hbar_c
    float gamma, gm1;
    float hdtx, hdty, hdtg;  // dt/(2 hx), dt/(2 hy), dt g/2
    float dtx, dty, dtg;     // dt/hx, dt/hy, dt g
    int nx, ny, cells, wall_x, wall_y, gravity;
};

__device__ __forceinline__ int fv_wrap(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// van Albada in FP32; differences below ~1e-15 (squares outside the normal
// range, where the fast division is not defined) give a zero slope, an
// absolute change below 1e-15
__device__ __forceinline__ float va_f(float a, float b) {
    const float ab = a * b;
    const float den = a * a + b * b;
    return (ab > 0.0f && den > 1e-30f) ? __fdividef(ab * (a + b), den) : 0.0f;
}

__device__ __forceinline__ float fv_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// hardware square root approximation (relative error ~2^-23): it only scales
// the Rusanov dissipation
__device__ __forceinline__ float fv_sqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// flux of a perturbation state q over the base b = (rhobar, pbar, -, g z)
// along x (xdir) or y, without the energy flux's Hbar part: f.w = v.n h';
// vn = v.n (the factor of Hbar); returns the wave speed |v.n| + c
__device__ __forceinline__ float fv_flux_f(const float4 q, const float4 b, bool xdir, const FvMixed& M, float4& f,
                                           float& vn) {
    const float rho = b.x + q.x;
    const float rinv = fv_rcp(rho);
    const float u = q.y * rinv, v = q.z * rinv;
    const float pp = M.gm1 * (q.w - 0.5f * (q.y * u + q.z * v) - b.w * q.x);
    vn = xdir ? u : v;
    f.x = xdir ? q.y : q.z;
    f.y = q.y * vn + (xdir ? pp : 0.0f);
    f.z = q.z * vn + (xdir ? 0.0f : pp);
    f.w = vn * (q.w + pp);
    return fabsf(vn) + fv_sqrt(M.gamma * (b.y + pp) * rinv);
}

// Rusanov flux of two perturbation states over one base; the energy flux is
// Hbar a + F.w with a = (v.n_L + v.n_R)/2
__device__ __forceinline__ float4 fv_rusanov_f(const float4 qL, const float4 qR, const float4 b, bool xdir,
                                               const FvMixed& M, float& a) {
    float4 fL, fR;
    float vL, vR;
    const float sL = fv_flux_f(qL, b, xdir, M, fL, vL);
    const float sR = fv_flux_f(qR, b, xdir, M, fR, vR);
    const float hs = 0.5f * fmaxf(sL, sR);
    a = 0.5f * (vL + vR);
    return make_float4(0.5f * (fL.x + fR.x) - hs * (qR.x - qL.x), 0.5f * (fL.y + fR.y) - hs * (qR.y - qL.y),
                       0.5f * (fL.z + fR.z) - hs * (qR.z - qL.z), 0.5f * (fL.w + fR.w) - hs * (qR.w - qL.w));
}

// slip-wall ghost of a perturbation face state: the background rho and rhoE
// (zero perturbation) with gravity, the interior ones without; normal momentum
// reflected
__device__ __forceinline__ float4 fv_ghost_f(const float4 q, bool xwall, const FvMixed& M) {
    return make_float4(M.gravity ? 0.0f : q.x, xwall ? -q.y : q.y, xwall ? q.z : -q.z, M.gravity ? 0.0f : q.w);
}

__device__ __forceinline__ float4 f4_add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 f4_axpy(float s, float4 a, float4 b) {  // b + s a
    return make_float4(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z), fmaf(s, a.w, b.w));
}

__global__ void __launch_bounds__(kFvThreads) k_fv_step_mixed(const double* __restrict__ u, double* __restrict__ uo,
                                                              const float4* __restrict__ pin,
                                                              float4* __restrict__ pout, const FvMixed M) {
    extern __shared__ float4 fv_smem[];
    float4* sp = fv_smem;                                // phase 1-2: perturbations; phase 3-4: face fluxes
    float4 (*sh)[kFvHh * kFvHw] = reinterpret_cast<float4 (*)[kFvHh * kFvHw]>(fv_smem + kFvShared);
                                                         // half-step face states E, W, N, S
    float* srp = reinterpret_cast<float*>(fv_smem + kFvShared + 4 * kFvHh * kFvHw);  // half-step rho'
    float* sa = srp + kFvThreads;                        // face velocity factor of Hbar in the energy flux
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kFvTx, y0 = blockIdx.y * kFvTy;
    // phase 1: the FP32 perturbations of the tile plus a 2-cell halo (wrapped
    // indices; wall-side halo values are never used), split from the FP64
    // state by the previous step's phase 4 (or by k_fv_split)
    for (int k = tid; k < kFvPw * kFvPh; k += kFvThreads) {
        const int r = k / kFvPw, c = k - r * kFvPw;
        const int gy = fv_wrap(y0 - 2 + r, M.ny), gx = fv_wrap(x0 - 2 + c, M.nx);
        sp[k] = pin[(size_t)gy * M.nx + gx];
    }
    __syncthreads();
    // phase 2: slopes, face states, half-step evolution (tile plus 1-cell halo,
    // corners unused)
    for (int k = tid; k < kFvHw * kFvHh; k += kFvThreads) {
        const int r = k / kFvHw, c = k - r * kFvHw;
        if ((r == 0 || r == kFvHh - 1) && (c == 0 || c == kFvHw - 1)) continue;
        const int gy = fv_wrap(y0 - 1 + r, M.ny), gx = fv_wrap(x0 - 1 + c, M.nx);
        const bool flat_x = M.wall_x && (gx == 0 || gx == M.nx - 1);
        const bool flat_y = M.wall_y && (gy == 0 || gy == M.ny - 1);
        const int p = (r + 1) * kFvPw + (c + 1);
        const float4 up = sp[p], pw = sp[p - 1], pe = sp[p + 1], ps = sp[p - kFvPw], pn = sp[p + kFvPw];
        float4 sx = make_float4(0.f, 0.f, 0.f, 0.f), sy = sx;
        if (!flat_x)
            sx = make_float4(va_f(up.x - pw.x, pe.x - up.x), va_f(up.y - pw.y, pe.y - up.y),
                             va_f(up.z - pw.z, pe.z - up.z), va_f(up.w - pw.w, pe.w - up.w));
        if (!flat_y)
            sy = make_float4(va_f(up.x - ps.x, pn.x - up.x), va_f(up.y - ps.y, pn.y - up.y),
                             va_f(up.z - ps.z, pn.z - up.z), va_f(up.w - ps.w, pn.w - up.w));
        const float4 qE = f4_axpy(0.5f, sx, up), qW = f4_axpy(-0.5f, sx, up);
        const float4 qN = f4_axpy(0.5f, sy, up), qS = f4_axpy(-0.5f, sy, up);
        const float4 bc = M.cb[gy], bn = M.fb[gy + 1], bs = M.fb[gy];
        const float2 dh = M.dh[gy];
        float4 fE, fW, gN, gS;
        float vE, vW, vN, vS;
        fv_flux_f(qE, bc, true, M, fE, vE);
        fv_flux_f(qW, bc, true, M, fW, vW);
        fv_flux_f(qN, bn, false, M, gN, vN);
        fv_flux_f(qS, bs, false, M, gS, vS);
        const float hx = fmaf(bc.z, vE - vW, fE.w - fW.w);
        const float hy = fmaf(bc.z, vN - vS, fmaf(dh.x, vN, fmaf(-dh.y, vS, gN.w - gS.w)));
        float4 d;
        d.x = -M.hdtx * (fE.x - fW.x) - M.hdty * (gN.x - gS.x);
        d.y = -M.hdtx * (fE.y - fW.y) - M.hdty * (gN.y - gS.y);
        d.z = -M.hdtx * (fE.z - fW.z) - M.hdty * (gN.z - gS.z) - M.hdtg * up.x;
        d.w = -M.hdtx * hx - M.hdty * hy;
        sh[0][k] = f4_add(qE, d);
        sh[1][k] = f4_add(qW, d);
        sh[2][k] = f4_add(qN, d);
        sh[3][k] = f4_add(qS, d);
        if (r >= 1 && r <= kFvTy && c >= 1 && c <= kFvTx) srp[(r - 1) * kFvTx + (c - 1)] = up.x + d.x;
    }
    __syncthreads();
    // phase 3: Rusanov fluxes, x-faces [r][j] (west face of tile column j),
    // then y-faces [k][c] (south face of tile row k)
    float4* fxs = sp;
    float4* fys = sp + kFvFx;
    for (int k = tid; k < kFvFx + kFvFy; k += kFvThreads) {
        if (k < kFvFx) {
            const int r = k / (kFvTx + 1), j = k - r * (kFvTx + 1);
            const int gy = y0 + r, gf = x0 + j;
            if (gy >= M.ny || gf > M.nx) continue;
            const int h = (r + 1) * kFvHw + j;  // half-tile cell left of the face
            float4 qL = sh[0][h], qR = sh[1][h + 1];
            if (M.wall_x && gf == 0) qL = fv_ghost_f(qR, true, M);
            if (M.wall_x && gf == M.nx) qR = fv_ghost_f(qL, true, M);
            fxs[k] = fv_rusanov_f(qL, qR, M.cb[gy], true, M, sa[k]);
        } else {
            const int kk = k - kFvFx;
            const int r = kk / kFvTx, c = kk - r * kFvTx;
            const int gf = y0 + r, gx = x0 + c;
            if (gf > M.ny || gx >= M.nx) continue;
            const int h = r * kFvHw + (c + 1);  // half-tile cell below the face
            float4 qL = sh[2][h], qR = sh[3][h + kFvHw];
            if (M.wall_y && gf == 0) qL = fv_ghost_f(qR, false, M);
            if (M.wall_y && gf == M.ny) qR = fv_ghost_f(qL, false, M);
            fys[kk] = fv_rusanov_f(qL, qR, M.fb[gf], false, M, sa[k]);
        }
    }
    __syncthreads();
    // phase 4: FP32 increment, FP64 accumulation
    const int ty = tid / kFvTx, tx = tid - ty * kFvTx;
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy >= M.ny || gx >= M.nx) return;
    const float4 FW = fxs[ty * (kFvTx + 1) + tx], FE = fxs[ty * (kFvTx + 1) + tx + 1];
    const float4 GS = fys[ty * kFvTx + tx], GN = fys[(ty + 1) * kFvTx + tx];
    const float aW = sa[ty * (kFvTx + 1) + tx], aE = sa[ty * (kFvTx + 1) + tx + 1];
    const float aS = sa[kFvFx + ty * kFvTx + tx], aN = sa[kFvFx + (ty + 1) * kFvTx + tx];
    const float Hc = M.cb[gy].z;
    const float2 dh = M.dh[gy];
    const float rp = srp[tid];
    const float du0 = -M.dtx * (FE.x - FW.x) - M.dty * (GN.x - GS.x);
    const float du1 = -M.dtx * (FE.y - FW.y) - M.dty * (GN.y - GS.y);
    const float du2 = -M.dtx * (FE.z - FW.z) - M.dty * (GN.z - GS.z) - M.dtg * rp;
    const float ex = fmaf(Hc, aE - aW, FE.w - FW.w);
    const float ey = fmaf(Hc, aN - aS, fmaf(dh.x, aN, fmaf(-dh.y, aS, GN.w - GS.w)));
    const float du3 = -M.dtx * ex - M.dty * ey;
    const size_t i = (size_t)gy * M.nx + gx;
    const double r1 = __dadd_rn(u[i], f32_to_f64(du0));
    const double m1 = __dadd_rn(u[(size_t)M.cells + i], f32_to_f64(du1));
    const double n1 = __dadd_rn(u[(size_t)2 * M.cells + i], f32_to_f64(du2));
    const double E1 = __dadd_rn(u[(size_t)3 * M.cells + i], f32_to_f64(du3));
    uo[i] = r1;
    uo[(size_t)M.cells + i] = m1;
    uo[(size_t)2 * M.cells + i] = n1;
    uo[(size_t)3 * M.cells + i] = E1;
    // the next step's FP32 perturbations (the same split phase 1 would make)
    pout[i] = make_float4(f64_to_f32(__dsub_rn(r1, M.rbc[gy])), f64_to_f32(m1), f64_to_f32(n1),
                          f64_to_f32(__dsub_rn(E1, M.Ebc[gy])));
}

// FP32 perturbations of the whole FP64 state (after the state is set or
// initialised; the step keeps them current afterwards)
__global__ void __launch_bounds__(256) k_fv_split(const double* __restrict__ u, float4* __restrict__ p,
                                                  const FvMixed M) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= M.cells) return;
    const int gy = c / M.nx;
    p[c] = make_float4(f64_to_f32(__dsub_rn(u[c], M.rbc[gy])), f64_to_f32(u[(size_t)M.cells + c]),
                       f64_to_f32(u[(size_t)2 * M.cells + c]),
                       f64_to_f32(__dsub_rn(u[(size_t)3 * M.cells + c], M.Ebc[gy])));
}

// point values at cell centres: background atmosphere with theta' (Sec. 4.2)
__global__ void k_fv_init(double* __restrict__ u, int kind, double A, double a, double xc, double zc,
                          double R, double cp, double p0, double theta0, const FvPhys P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.cells) return;
    const int ix = c % P.nx, iy = c / P.nx;
    const double x = P.x0 + (ix + 0.5) * P.hx, z = P.y0 + (iy + 0.5) * P.hy;
    double th = 0.0;
    if (kind == ADG_SCEN_COSINE) {
        const double r = sqrt((x - xc) * (x - xc) + (z - zc) * (z - zc));
        th = r <= a ? 0.5 * A * (1.0 + cos(3.14159265358979323846 * r / a)) : 0.0;
    } else if (kind == ADG_SCEN_TWO_BUBBLES) {
        th = fv_bubble(x, z, 0.5, 150.0, 50.0, 500.0, 300.0) + fv_bubble(x, z, -0.15, 0.0, 50.0, 560.0, 640.0);
    }
    const double ex = 1.0 - P.g * z / (cp * theta0);
    const double pb = p0 * pow(ex, cp / R);
    const double rho = pb / (R * (theta0 + th) * ex);
    u[c] = rho;
    u[(size_t)P.cells + c] = 0.0;
    u[(size_t)2 * P.cells + c] = 0.0;
    u[(size_t)3 * P.cells + c] = pb / P.gm1 + rho * P.g * z;
}

FvPhys fv_phys(const adg_fv* f) {
    FvPhys P;
    P.gamma = f->d.gamma;
    P.gm1 = f->gm1;
    P.g = f->d.gravity ? f->d.g : 0.0;
    P.hx = f->hx;
    P.hy = f->hy;
    P.x0 = f->d.x0;
    P.y0 = f->d.y0;
    P.nx = f->d.nx;
    P.ny = f->d.ny;
    P.cells = f->cells;
    P.wall_x = f->d.bc_x == ADG_BC_WALL;
    P.wall_y = f->d.bc_y == ADG_BC_WALL;
    P.gravity = f->d.gravity ? 1 : 0;
    const int ny = f->d.ny;
    P.rbc = f->bg;
    P.Ebc = f->bg + ny;
    P.pbc = f->bg + 2 * ny;
    P.rbf = f->bg + 3 * ny;
    P.Ebf = f->bg + 3 * ny + (ny + 1);
    P.pbf = f->bg + 3 * ny + 2 * (ny + 1);
    return P;
}

FvMixed fv_mixed(const adg_fv* f, double dt) {
    FvMixed M;
    const int ny = f->d.ny;
    M.rbc = f->bg;
    M.Ebc = f->bg + ny;
    M.cb = reinterpret_cast<const float4*>(f->bgf);
    M.fb = reinterpret_cast<const float4*>(f->bgf) + ny;
    M.dh = reinterpret_cast<const float2*>(f->bgf + 4 * (size_t)ny + 4 * (size_t)(ny + 1));
    const double g = f->d.gravity ? f->d.g : 0.0;
    M.gamma = (float)f->d.gamma;
    M.gm1 = (float)f->gm1;
    M.hdtx = (float)(0.5 * dt / f->hx);
    M.hdty = (float)(0.5 * dt / f->hy);
    M.hdtg = (float)(0.5 * dt * g);
    M.dtx = (float)(dt / f->hx);
    M.dty = (float)(dt / f->hy);
    M.dtg = (float)(dt * g);
    M.nx = f->d.nx;
    M.ny = ny;
    M.cells = f->cells;
    M.wall_x = f->d.bc_x == ADG_BC_WALL;
    M.wall_y = f->d.bc_y == ADG_BC_WALL;
    M.gravity = f->d.gravity ? 1 : 0;
    return M;
}

int fv_blocks(int cells) { return (cells + 255) / 256; }

}  // namespace
}  // namespace adg

using adg::cuda_fail;
using adg::fail;

static int fv_device(const adg_fv* f) {
    cudaError_t e = cudaSetDevice(f->d.device);
    return e == cudaSuccess ? ADG_OK : cuda_fail(e, "fv: cudaSetDevice");
}

static void fv_free(adg_fv* f) {
    if (!f) return;
    cudaSetDevice(f->d.device);
    cudaFree(f->u);
    cudaFree(f->half);
    cudaFree(f->bg);
    cudaFree(f->part);
    cudaFree(f->u2);
    cudaFree(f->pert);
    cudaFree(f->pert2);
    cudaFree(f->bgf);
    delete f;
}

extern "C" int adg_fv_create(const adg_mesh_desc* d, adg_fv** out) {
    if (!d || !out) return fail(ADG_EINVAL, "fv_create: NULL argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || (long long)d->nx * d->ny > (1LL << 28))
        return fail(ADG_EINVAL, "fv_create: bad mesh size");
    if (!(d->Lx > 0.0) || !(d->Ly > 0.0)) return fail(ADG_EINVAL, "fv_create: Lx, Ly must be > 0");
    if ((d->bc_x != ADG_BC_PERIODIC && d->bc_x != ADG_BC_WALL) || (d->bc_y != ADG_BC_PERIODIC && d->bc_y != ADG_BC_WALL))
        return fail(ADG_EINVAL, "fv_create: boundaries are periodic or slip walls");
    if (!(d->gamma > 1.0) || !(d->R > 0.0)) return fail(ADG_EINVAL, "fv_create: invalid gas constants");
    if (d->mu != 0.0) return fail(ADG_EINVAL, "fv_create: the finite-volume scheme is inviscid (mu = 0)");
    if (d->precision != ADG_PREC_FP64 && d->precision != ADG_PREC_MIXED)
        return fail(ADG_EINVAL, "fv_create: precision must be FP64 or mixed");
    if (d->precision == ADG_PREC_MIXED && d->gravity && d->bc_y == ADG_BC_PERIODIC)
        return fail(ADG_EUNSUPPORTED, "fv_create: mixed precision with gravity needs walls in y");
    if (d->gravity && !(d->theta0 > 0.0 && d->p0 > 0.0))
        return fail(ADG_EINVAL, "fv_create: gravity needs theta0 > 0 and p0 > 0");
    int ndev = 0;
    ADG_CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (d->device < 0 || d->device >= ndev) return fail(ADG_EINVAL, "fv_create: bad device ordinal");
    adg_fv* f = new adg_fv();
    f->d = *d;
    f->cells = d->nx * d->ny;
    f->hx = d->Lx / d->nx;
    f->hy = d->Ly / d->ny;
    f->gm1 = d->gamma - 1.0;
    if (int rc = fv_device(f)) {
        delete f;
        return rc;
    }
    const int ny = d->ny;
    f->part_blocks = adg::fv_blocks(f->cells);
    const size_t nbg = 3 * (size_t)ny + 3 * (size_t)(ny + 1);
    const bool mixed = d->precision == ADG_PREC_MIXED;
    if (mixed) {
        const cudaError_t e = cudaFuncSetAttribute(adg::k_fv_step_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)adg::kFvSmemBytes);
        if (e != cudaSuccess) {
            delete f;
            return cuda_fail(e, "fv_create: shared memory attribute");
        }
    }
    const size_t nbgf = 4 * (size_t)ny + 4 * (size_t)(ny + 1) + 2 * (size_t)ny;
    bool ok = cudaMalloc(&f->u, (size_t)4 * f->cells * 8) == cudaSuccess && cudaMalloc(&f->bg, nbg * 8) == cudaSuccess &&
              cudaMalloc(&f->part, (size_t)2 * f->part_blocks * 8) == cudaSuccess;
    if (ok && mixed)
        ok = cudaMalloc(&f->u2, (size_t)4 * f->cells * 8) == cudaSuccess && cudaMalloc(&f->bgf, nbgf * 4) == cudaSuccess &&
             cudaMalloc(&f->pert, (size_t)f->cells * 16) == cudaSuccess &&
             cudaMalloc(&f->pert2, (size_t)f->cells * 16) == cudaSuccess;
    else if (ok)
        ok = cudaMalloc(&f->half, (size_t)17 * f->cells * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fv_free(f);
        return fail(ADG_ENOMEM, "fv_create: device allocation failed");
    }
    // isentropic background (Eq. 6 reading) at centres and faces; zero without gravity
    std::vector<double> h(nbg, 0.0);
    if (d->gravity) {
        const double cp = d->gamma * d->R / (d->gamma - 1.0);
        auto bgp = [&](double z, double& r, double& E, double& p) {
            const double ex = 1.0 - d->g * z / (cp * d->theta0);
            p = d->p0 * std::pow(ex, cp / d->R);
            r = p / (d->R * d->theta0 * ex);
            E = p / f->gm1 + r * d->g * z;
        };
        for (int iy = 0; iy < ny; ++iy) bgp(d->y0 + (iy + 0.5) * f->hy, h[iy], h[ny + iy], h[2 * ny + iy]);
        for (int k = 0; k <= ny; ++k)
            bgp(d->y0 + k * f->hy, h[3 * ny + k], h[3 * ny + (ny + 1) + k], h[3 * ny + 2 * (ny + 1) + k]);
    }
    // FP32 tables of the mixed path: (rhobar, pbar, Ebar + pbar, g z) at centres, then faces
    std::vector<float> hf(nbgf, 0.0f);
    if (mixed && d->gravity) {
        for (int iy = 0; iy < ny; ++iy) {
            hf[4 * iy + 0] = (float)h[iy];
            hf[4 * iy + 1] = (float)h[2 * ny + iy];
            hf[4 * iy + 2] = (float)(h[ny + iy] + h[2 * ny + iy]);
            hf[4 * iy + 3] = (float)(d->g * (d->y0 + (iy + 0.5) * f->hy));
        }
        auto Hf = [&](int k) { return h[3 * ny + (ny + 1) + k] + h[3 * ny + 2 * (ny + 1) + k]; };
        for (int k = 0; k <= ny; ++k) {
            float* q = hf.data() + 4 * (size_t)ny + 4 * (size_t)k;
            q[0] = (float)h[3 * ny + k];
            q[1] = (float)h[3 * ny + 2 * (ny + 1) + k];
            q[2] = 0.0f;
            q[3] = (float)(d->g * (d->y0 + k * f->hy));
        }
        for (int iy = 0; iy < ny; ++iy) {
            float* q = hf.data() + 4 * (size_t)ny + 4 * (size_t)(ny + 1) + 2 * (size_t)iy;
            const double Hc = h[ny + iy] + h[2 * ny + iy];
            q[0] = (float)(Hf(iy + 1) - Hc);
            q[1] = (float)(Hf(iy) - Hc);
        }
    }
    if (cudaMemcpy(f->bg, h.data(), nbg * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        (mixed && cudaMemcpy(f->bgf, hf.data(), nbgf * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(f->u, 0, (size_t)4 * f->cells * 8) != cudaSuccess) {
        cudaGetLastError();
        fv_free(f);
        return fail(ADG_ECUDA, "fv_create: initialisation failed");
    }
    *out = f;
    return ADG_OK;
}

extern "C" void adg_fv_destroy(adg_fv* f) { fv_free(f); }

extern "C" size_t adg_fv_state_count(const adg_fv* f) { return f ? (size_t)4 * f->cells : 0; }

extern "C" int adg_fv_set_state(adg_fv* f, const double* u, size_t count, int on_device, void* stream) {
    if (!f || !u) return fail(ADG_EINVAL, "fv_set_state: NULL argument");
    if (count != (size_t)4 * f->cells) return fail(ADG_EINVAL, "fv_set_state: count must be 4 * cells");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "bad on_device");
    if (int rc = fv_device(f)) return rc;
    ADG_CK(cudaMemcpyAsync(f->u, u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           (cudaStream_t)stream),
           "fv_set_state");
    if (on_device == 0) ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "fv_set_state sync");
    f->pert_stale = true;
    return ADG_OK;
}

extern "C" int adg_fv_get_state(adg_fv* f, double* u, size_t count, int on_device, void* stream) {
    if (!f || !u) return fail(ADG_EINVAL, "fv_get_state: NULL argument");
    if (count != (size_t)4 * f->cells) return fail(ADG_EINVAL, "fv_get_state: count must be 4 * cells");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "bad on_device");
    if (int rc = fv_device(f)) return rc;
    ADG_CK(cudaMemcpyAsync(u, f->u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           (cudaStream_t)stream),
           "fv_get_state");
    if (on_device == 0) ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "fv_get_state sync");
    return ADG_OK;
}

extern "C" int adg_fv_init_scenario(adg_fv* f, const adg_scenario* s, void* stream) {
    if (!f || !s) return fail(ADG_EINVAL, "fv_init_scenario: NULL argument");
    if (s->kind != ADG_SCEN_COSINE && s->kind != ADG_SCEN_TWO_BUBBLES && s->kind != ADG_SCEN_BACKGROUND)
        return fail(ADG_EINVAL, "fv_init_scenario: cosine bubble, two bubbles or background");
    if (!f->d.gravity) return fail(ADG_EINVAL, "fv_init_scenario: bubble scenarios need gravity");
    if (s->kind == ADG_SCEN_COSINE && !(s->a > 0.0)) return fail(ADG_EINVAL, "fv_init_scenario: radius must be > 0");
    if (int rc = fv_device(f)) return rc;
    const adg::FvPhys P = adg::fv_phys(f);
    const double cp = f->d.gamma * f->d.R / f->gm1;
    adg::k_fv_init<<<adg::fv_blocks(f->cells), 256, 0, (cudaStream_t)stream>>>(
        f->u, s->kind, s->A, s->a, s->xc, s->zc, f->d.R, cp, f->d.p0, f->d.theta0, P);
    ADG_CK(cudaGetLastError(), "fv_init_scenario launch");
    f->pert_stale = true;
    return ADG_OK;
}

extern "C" int adg_fv_step(adg_fv* f, double dt, void* stream) {
    if (!f) return fail(ADG_EINVAL, "fv_step: NULL argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADG_EINVAL, "fv_step: dt must be finite and > 0");
    if (int rc = fv_device(f)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (f->d.precision == ADG_PREC_MIXED) {
        const adg::FvMixed M = adg::fv_mixed(f, dt);
        if (f->pert_stale) {
            adg::k_fv_split<<<adg::fv_blocks(f->cells), 256, 0, s>>>(f->u, f->pert, M);
            ADG_CK(cudaGetLastError(), "fv_step split");
            f->pert_stale = false;
        }
        const dim3 grid((f->d.nx + adg::kFvTx - 1) / adg::kFvTx, (f->d.ny + adg::kFvTy - 1) / adg::kFvTy);
        adg::k_fv_step_mixed<<<grid, adg::kFvThreads, adg::kFvSmemBytes, s>>>(f->u, f->u2, f->pert, f->pert2, M);
        ADG_CK(cudaGetLastError(), "fv_step mixed");
        std::swap(f->u, f->u2);
        std::swap(f->pert, f->pert2);
        return ADG_OK;
    }
    const adg::FvPhys P = adg::fv_phys(f);
    const int nb = adg::fv_blocks(f->cells);
    adg::k_fv_half<<<nb, 256, 0, s>>>(f->u, f->half, dt, P);
    ADG_CK(cudaGetLastError(), "fv_step half");
    adg::k_fv_update<<<nb, 256, 0, s>>>(f->u, f->half, dt, P);
    ADG_CK(cudaGetLastError(), "fv_step update");
    return ADG_OK;
}

extern "C" int adg_fv_stable_dt(adg_fv* f, double cfl, double* dt, void* stream) {
    if (!f || !dt) return fail(ADG_EINVAL, "fv_stable_dt: NULL argument");
    if (!(cfl > 0.0)) return fail(ADG_EINVAL, "fv_stable_dt: cfl must be > 0");
    if (int rc = fv_device(f)) return rc;
    const adg::FvPhys P = adg::fv_phys(f);
    cudaStream_t s = (cudaStream_t)stream;
    adg::k_fv_speed<<<f->part_blocks, 256, 0, s>>>(f->u, f->part, P);
    ADG_CK(cudaGetLastError(), "fv_stable_dt launch");
    std::vector<double> h((size_t)2 * f->part_blocks);
    ADG_CK(cudaMemcpyAsync(h.data(), f->part, h.size() * 8, cudaMemcpyDeviceToHost, s), "fv_stable_dt copy");
    ADG_CK(cudaStreamSynchronize(s), "fv_stable_dt sync");
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < f->part_blocks; ++b) {
        sx = std::max(sx, h[2 * b]);
        sy = std::max(sy, h[2 * b + 1]);
    }
    if (!(sx > 0.0 || sy > 0.0) || !std::isfinite(sx) || !std::isfinite(sy))
        return fail(ADG_ENONFINITE, "fv_stable_dt: non-finite or zero wave speed");
    *dt = cfl / (sx / f->hx + sy / f->hy);
    return ADG_OK;
}
