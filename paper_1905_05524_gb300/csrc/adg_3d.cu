// Three-dimensional FP64 ADER-DG (the ABC flow of Sec. 4.1 and the 3D cosine
// bubble of Sec. 4.2): the scheme of adg_fp64.cu with one more direction.
//
// Predictor (Sec. 3): per cell, the element-local space-time polynomial on
// (N+1)^4 Gauss-Legendre nodes by n = N+1 Picard sweeps
//     q_l = u + dt sum_k (K1^{-1})_{lk} w_k R_k,  R = -dF/dx - dG/dy - dH/dz + S,
// then grad q, F, G, H, S once more on the final iterate, averaged in time.
// It writes the weak volume residual
//     rvol = sum_d (1/h_d) sum_p (w_p / w_i_d) D_p,i_d Fbar_d(.. p ..) + Sbar
// and, per face node, the boundary-extrapolated averages (q-bar, normal
// flux, grad q-bar) and the Rusanov speed.
// Corrector: the Rusanov-type viscous flux on the 6 faces (neighbour traces,
// a slip-wall ghost with the background of Eq. 6 and the heat flux of
// Eq. 10, or the analytic ABC field) and the FP64 update u += dt (rvol - lift).
//
// Thread mapping: CPB cells per block, one thread per spatial node (l, j, i);
// each thread walks the n time nodes of its node, so the Picard update's
// time contraction stays in registers.  Shared memory per cell: the n time
// slices of the iterate and the F, G, H of one time slice (the divergence of
// slice k is taken before slice k+1's fluxes overwrite them); after the last
// sweep the same space holds the seven time-averaged fields the volume term
// and the traces contract.
//
// Layouts: u[c][v][l][j][i], c = (iz ny + iy) nx + ix, v in (rho, rho u,
// rho v, rho w, rho E); traces [c][face E W N S T B][kTr3][n^2], face nodes
// (l, j) on x-faces, (l, i) on y-faces, (j, i) on z-faces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mesh.h"

namespace adg {
namespace {

constexpr int kTr3 = 26;  // q-bar(5), normal flux(5), qx-bar(5), qy-bar(5), qz-bar(5), speed

struct Phys3 {
    double gamma, gm1, R, invR, mu, kappa, g, cp, p0, theta0, lamv, dTdz;
    double eta[3], h[3], inv_h[3], org[3];
    int nc[3], bc[3];
    int gravity, field;
};

// background p, rho at node heights [nz][n] and at horizontal faces [nz + 1]
struct Bg3 {
    const double* pn;
    const double* rn;
    const double* pf;
    const double* rf;
};

// Point-wise fluxes f[b][v] in the three directions and the z-momentum
// source of a state q with gradients g[b][v] at height z.  Momentum fluxes
// carry p' = p - pbar (Eq. 7); heat_wall replaces grad T by (0, 0, dTbar/dz)
// (slip-wall ghost, Eq. 10).
__device__ __forceinline__ void ns_flux3(const double q[5], const double g[3][5], double z, double pbar,
                                         double rhobar, const Phys3& P, bool heat_wall, double f[3][5],
                                         double& src) {
    const double rinv = 1.0 / q[0];
    const double vel[3] = {q[1] * rinv, q[2] * rinv, q[3] * rinv};
    const double kin = 0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    const double gg = P.gravity ? P.g : 0.0;
    const double p = P.gm1 * (q[4] - q[0] * kin - q[0] * gg * z);
    const double pp = p - pbar;
    const double T = p * rinv * P.invR;
    double d[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d[a][b] = (g[b][1 + a] - vel[a] * g[b][0]) * rinv;
    const double div = d[0][0] + d[1][1] + d[2][2];
    double dT[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (heat_wall) {
            dT[b] = b == 2 ? P.dTdz : 0.0;
        } else {
            double s = g[b][4] - (vel[0] * g[b][1] + vel[1] * g[b][2] + vel[2] * g[b][3]) + kin * g[b][0] -
                       gg * z * g[b][0];
            if (b == 2) s -= q[0] * gg;
            dT[b] = (P.gm1 * s - P.R * T * g[b][0]) * rinv * P.invR;
        }
    }
    double sig[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            sig[a][b] = P.mu * ((a == b ? (2.0 / 3.0) * div : 0.0) - (d[a][b] + d[b][a]));
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        f[b][0] = q[1 + b];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[b][1 + a] = q[1 + a] * vel[b] + (a == b ? pp : 0.0) + sig[a][b];
        f[b][4] = vel[b] * (q[4] + p) + vel[0] * sig[0][b] + vel[1] * sig[1][b] + vel[2] * sig[2][b] -
                  P.kappa * dT[b];
    }
    src = P.gravity ? -P.g * (q[0] - rhobar) : 0.0;
}

// Rusanov speed |v_dir| + c + 2 eta_dir lambda_v / rho at height z
__device__ __forceinline__ double wave_speed3(const double q[5], double z, int dir, const Phys3& P) {
    const double rinv = 1.0 / q[0];
    const double gg = P.gravity ? P.g : 0.0;
    const double p = P.gm1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * rinv - q[0] * gg * z);
    const double mn = dir == 0 ? q[1] : dir == 1 ? q[2] : q[3];  // selects keep q in registers
    return fabs(mn * rinv) + sqrt(P.gamma * p * rinv) + 2.0 * P.eta[dir] * P.lamv * rinv;
}

__device__ __forceinline__ void rusanov5(const double qL[5], const double fL[5], double sL, const double qR[5],
                                         const double fR[5], double sR, double out[5]) {
    const double s = fmax(sL, sR);
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * s * (qR[v] - qL[v]);
}

// The ABC field (Sec. 4.1) and its gradient, differentiated by hand:
// a = e^{-mu t}, u = a (sin z + cos y), v = a (sin x + cos z),
// w = a (sin y + cos x), rho = 1, p = -a^2 (cos x sin y + sin x cos z +
// sin z cos y) + 100/gamma.
__device__ __forceinline__ void abc_field(double x, double y, double z, double t, const Phys3& P, double q[5],
                                          double g[3][5]) {
    const double a = exp(-P.mu * t), a2 = a * a;
    const double sx = sin(x), cx = cos(x), sy = sin(y), cy = cos(y), sz = sin(z), cz = cos(z);
    const double vel[3] = {a * (sz + cy), a * (sx + cz), a * (sy + cx)};
    // dvel[a][b] = d vel_a / d x_b
    const double dv[3][3] = {{0.0, -a * sy, a * cz}, {a * cx, 0.0, -a * sz}, {-a * sx, a * cy, 0.0}};
    const double p = -a2 * (cx * sy + sx * cz + sz * cy) + 100.0 / P.gamma;
    const double dp[3] = {-a2 * (-sx * sy + cx * cz), -a2 * (cx * cy - sz * sy), -a2 * (-sx * sz + cz * cy)};
    q[0] = 1.0;
    q[1] = vel[0];
    q[2] = vel[1];
    q[3] = vel[2];
    q[4] = p / P.gm1 + 0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        g[b][0] = 0.0;
        g[b][1] = dv[0][b];
        g[b][2] = dv[1][b];
        g[b][3] = dv[2][b];
        g[b][4] = dp[b] / P.gm1 + vel[0] * dv[0][b] + vel[1] * dv[1][b] + vel[2] * dv[2][b];
    }
}


template <int N>
struct Cfg3 {
    static constexpr int n = N + 1, n2 = n * n, n3 = n * n * n;
    static constexpr int cpb = N == 1 ? 16 : N == 2 ? 8 : N == 3 ? 4 : 2;
    static constexpr int threads = cpb * n3;
    static constexpr int slots = (n + 3) > 7 ? n + 3 : 7;  // iterate + one slice of fluxes, or 7 averages
    static constexpr size_t smem = (size_t)cpb * slots * 5 * n3 * sizeof(double);
};

template <int N>
__global__ void __launch_bounds__(Cfg3<N>::threads)
k3_predictor(const double* __restrict__ u, double* __restrict__ rvol, double* __restrict__ trace, int cells,
             double dt, const Basis B, const Phys3 P, const Bg3 bg) {
    using C = Cfg3<N>;
    constexpr int n = C::n, n2 = C::n2, n3 = C::n3, SL = 5 * n3;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n3;
    const int node = threadIdx.x - cl * n3;
    const int l = node / n2, j = (node / n) % n, i = node % n;
    const int cell_raw = blockIdx.x * C::cpb + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int iz = cell / (P.nc[0] * P.nc[1]);
    double* Q = sm + (size_t)cl * C::slots * SL;  // [n][5][n3]
    double* Fs = Q + n * SL;                      // [3][5][n3]: F, G, H of one time slice
    const double z = P.org[2] + (iz + B.xi[l]) * P.h[2];
    const double pbar = bg.pn[iz * n + l], rhobar = bg.rn[iz * n + l];

    double uu[5];
    const double* uc = u + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        uu[v] = uc[v * n3 + node];
        Q[v * n3 + node] = uu[v];
    }
    __syncthreads();

    // state, gradients and fluxes of time slice Qk at this node
    auto eval = [&](const double* Qk, double q[5], double g[3][5], double f[3][5], double& src) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double* Qv = Qk + v * n3;
            q[v] = Qv[node];
            double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.D[i][p] * Qv[(l * n + j) * n + p];
                sy += B.D[j][p] * Qv[(l * n + p) * n + i];
                sz += B.D[l][p] * Qv[(p * n + j) * n + i];
            }
            g[0][v] = sx * P.inv_h[0];
            g[1][v] = sy * P.inv_h[1];
            g[2][v] = sz * P.inv_h[2];
        }
        ns_flux3(q, g, z, pbar, rhobar, P, false, f, src);
    };
    auto store = [&](const double f[3][5]) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int v = 0; v < 5; ++v) Fs[(b * 5 + v) * n3 + node] = f[b][v];
    };
    // -dF/dx - dG/dy - dH/dz at this node from the slice in Fs
    auto divergence = [&](int v) {
        const double* Fv = Fs + v * n3;
        const double* Gv = Fs + (5 + v) * n3;
        const double* Hv = Fs + (10 + v) * n3;
        double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sx += B.D[i][p] * Fv[(l * n + j) * n + p];
            sy += B.D[j][p] * Gv[(l * n + p) * n + i];
            sz += B.D[l][p] * Hv[(p * n + j) * n + i];
        }
        return -(sx * P.inv_h[0] + sy * P.inv_h[1] + sz * P.inv_h[2]);
    };

    // sweep 1: the iterate is u at every time node: one flux evaluation
    {
        double q[5], g[3][5], f[3][5], src;
        eval(Q, q, g, f, src);
        store(f);
        __syncthreads();
        double R0[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) R0[v] = (v == 3 ? src : 0.0) + divergence(v);
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < 5; ++v) Q[k * SL + v * n3 + node] = uu[v] + dt * (B.Kw1[k] * R0[v]);
        __syncthreads();
    }
    // sweeps 2..n
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        double R[n][5];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double q[5], g[3][5], f[3][5], src;
            eval(Q + k * SL, q, g, f, src);
            __syncthreads();  // the previous slice's divergence has read Fs
            store(f);
            __syncthreads();
#pragma unroll
            for (int v = 0; v < 5; ++v) R[k][v] = (v == 3 ? src : 0.0) + divergence(v);
        }
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                double acc = 0.0;
#pragma unroll
                for (int m = 0; m < n; ++m) acc += B.Kw[k][m] * R[m][v];
                Q[k * SL + v * n3 + node] = uu[v] + dt * acc;
            }
        __syncthreads();
    }

    // final evaluation on the converged iterate: time averages
    double qb[5], fb[3][5], gb[3][5], sb = 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        qb[v] = 0.0;
#pragma unroll
        for (int b = 0; b < 3; ++b) fb[b][v] = gb[b][v] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < n; ++k) {
        double q[5], g[3][5], f[3][5], src;
        eval(Q + k * SL, q, g, f, src);
        const double wk = B.w[k];
        sb += wk * src;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            qb[v] += wk * q[v];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                fb[b][v] += wk * f[b][v];
                gb[b][v] += wk * g[b][v];
            }
        }
    }
    __syncthreads();
    // slots: 0 q-bar, 1..3 F-, G-, H-bar, 4..6 qx-, qy-, qz-bar
    double* A = Q;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        A[v * n3 + node] = qb[v];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            A[(1 + b) * SL + v * n3 + node] = fb[b][v];
            A[(4 + b) * SL + v * n3 + node] = gb[b][v];
        }
    }
    __syncthreads();
    if (active) {
        double* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double* Fv = A + 1 * SL + v * n3;
            const double* Gv = A + 2 * SL + v * n3;
            const double* Hv = A + 3 * SL + v * n3;
            double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx += B.Vx[p][i] * Fv[(l * n + j) * n + p];
                sy += B.Vx[p][j] * Gv[(l * n + p) * n + i];
                sz += B.Vx[p][l] * Hv[(p * n + j) * n + i];
            }
            rc[v * n3 + node] = sx * P.inv_h[0] + sy * P.inv_h[1] + sz * P.inv_h[2] + (v == 3 ? sb : 0.0);
        }
    }
    // boundary-extrapolated traces of faces E, W (x), N, S (y), T, B (z)
    const int ic0 = cell % P.nc[0], ic1 = (cell / P.nc[0]) % P.nc[1];
    for (int idx = node; idx < 6 * n2; idx += n3) {
        const int f = idx / n2, m = idx - f * n2;
        const int a = m / n, b = m - a * n;
        const int dir = f >> 1;
        const double* phi = (f & 1) ? B.phi0 : B.phi1;
        // the gradient components are read only by slip-wall ghosts: written
        // for wall faces alone
        const int icd = dir == 0 ? ic0 : dir == 1 ? ic1 : iz;
        const int ncd = dir == 0 ? P.nc[0] : dir == 1 ? P.nc[1] : P.nc[2];
        const int bcd = dir == 0 ? P.bc[0] : dir == 1 ? P.bc[1] : P.bc[2];
        const bool wallface = bcd == ADG_BC_WALL && ((f & 1) ? icd == 0 : icd == ncd - 1);
        double rec[kTr3];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            if (c >= 2 && !wallface) {
#pragma unroll
                for (int v = 0; v < 5; ++v) rec[c * 5 + v] = 0.0;
                continue;
            }
            const int slot = c == 0 ? 0 : c == 1 ? 1 + dir : 2 + c;  // q, normal flux, qx, qy, qz
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const double* S = A + slot * SL + v * n3;
                double s = 0.0;
#pragma unroll
                for (int p = 0; p < n; ++p) {
                    const int at = dir == 0 ? (a * n + b) * n + p : dir == 1 ? (a * n + p) * n + b : (p * n + a) * n + b;
                    s += phi[p] * S[at];
                }
                rec[c * 5 + v] = s;
            }
        }
        const double zf = dir < 2 ? P.org[2] + (iz + B.xi[a]) * P.h[2] : P.org[2] + (iz + ((f & 1) ? 0 : 1)) * P.h[2];
        rec[25] = wave_speed3(rec, zf, dir, P);
        if (active) {
            double* tr = trace + ((size_t)cell * 6 + f) * kTr3 * n2;
#pragma unroll
            for (int c = 0; c < kTr3; ++c)
                if (c < 10 || c == 25 || wallface) tr[c * n2 + m] = rec[c];
        }
    }    pdl_trigger();
}

struct Phys3f {
    float gamma, gm1, R, invR, mu, kappa, g, lamv, dTdz;
    float inv_h[3], eta[3];
    int gravity;
};

struct Bg3m {
    const double* rb;   // [nz][n] rhobar at nodes (FP64, for the split)
    const double* Eb;   // [nz][n] Ebar = pbar/(gamma-1) + rhobar g z
    const float* rbf;   // [nz][n] rhobar
    const float* pbf;   // [nz][n] pbar
    const float* Hbf;   // [nz][n] Ebar + pbar
    const float* dzr;   // [nz][n] d rhobar/dz of the nodal interpolant
    const float* dzE;   // [nz][n] d Ebar/dz
    const double* ext;  // [nz][2: top, bottom][2: rhobar, Ebar] extrapolated to the z-faces
    const double* zn;   // [nz][n] node heights
    const float* zext;  // [nz][2: top, bottom][2: rhobar, pbar_eff] of the extrapolated z-face base,
                        // pbar_eff = (gamma-1)(Ebar - rhobar g z_face) formed in FP64
};

__device__ __forceinline__ void ns_flux3f(const float q[5], const float g[3][5], float gz, float rb, float pb,
                                          float Hb, const Phys3f& P, float f[3][5], float& src,
                                          bool heat_wall = false, float dTdz = 0.0f) {
    const float rho = rb + q[0];
    const float rinv = __frcp_rn(rho);
    const float vel[3] = {q[1] * rinv, q[2] * rinv, q[3] * rinv};
    const float kin = 0.5f * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    const float pp = P.gm1 * (q[4] - rho * kin - gz * q[0]);
    const float T = (pb + pp) * rinv * P.invR;
    float d[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d[a][b] = (g[b][1 + a] - vel[a] * g[b][0]) * rinv;
    const float div = d[0][0] + d[1][1] + d[2][2];
    float dT[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float s = g[b][4] - (vel[0] * g[b][1] + vel[1] * g[b][2] + vel[2] * g[b][3]) + kin * g[b][0] - gz * g[b][0];
        if (b == 2) s -= rho * P.g;
        dT[b] = heat_wall ? (b == 2 ? dTdz : 0.0f) : (P.gm1 * s - P.R * T * g[b][0]) * rinv * P.invR;
    }
    float sig[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            sig[a][b] = P.mu * ((a == b ? (2.0f / 3.0f) * div : 0.0f) - (d[a][b] + d[b][a]));
    const float h = Hb + (q[4] + pp);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        f[b][0] = q[1 + b];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[b][1 + a] = q[1 + a] * vel[b] + (a == b ? pp : 0.0f) + sig[a][b];
        f[b][4] = vel[b] * h + vel[0] * sig[0][b] + vel[1] * sig[1][b] + vel[2] * sig[2][b] - P.kappa * dT[b];
    }
    src = P.gravity ? -P.g * q[0] : 0.0f;
}

// MX: the mixed-precision form -- Rusanov flux from the FP64 jump of the
// face states converted to FP32, flux average and lifting in FP32, the
// update in FP64 (ghost states stay FP64).
template <int N, bool MX>
__global__ void __launch_bounds__(Cfg3<N>::threads)
k3_corrector(double* __restrict__ u, const double* __restrict__ rvol, const double* __restrict__ trace, int cells,
             double dt, double t, const Basis B, const Phys3 P, const Bg3 bg, const Phys3f Pf) {
    using C = Cfg3<N>;
    using FT = typename std::conditional<MX, float, double>::type;
    constexpr int n = C::n, n2 = C::n2, n3 = C::n3, SL = 5 * n3, TR = kTr3 * n2;
    __shared__ FT Fst[C::cpb][6][5][n2];
    const int cl = threadIdx.x / n3;
    const int node = threadIdx.x - cl * n3;
    const int l = node / n2, j = (node / n) % n, i = node % n;
    const int cell_raw = blockIdx.x * C::cpb + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int ic0 = cell % P.nc[0], ic1 = (cell / P.nc[0]) % P.nc[1], ic2 = cell / (P.nc[0] * P.nc[1]);
    pdl_wait();  // programmatic launch: the predictor's residual and traces are complete and visible

    for (int idx = node; idx < 6 * n2; idx += n3) {
        const int f = idx / n2, m = idx - f * n2;
        const int a = m / n, b = m - a * n;
        const int dir = f >> 1;
        const bool plus = (f & 1) == 0;
        // selects instead of arrays indexed by the face's direction (keeps
        // everything in registers)
        const int icd = dir == 0 ? ic0 : dir == 1 ? ic1 : ic2;
        const int ncd = dir == 0 ? P.nc[0] : dir == 1 ? P.nc[1] : P.nc[2];
        const int bcd = dir == 0 ? P.bc[0] : dir == 1 ? P.bc[1] : P.bc[2];
        const bool edge = plus ? icd == ncd - 1 : icd == 0;
        const double* own = trace + ((size_t)cell * 6 + f) * TR;
        double qo[5], fo[5], g[3][5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            qo[v] = own[v * n2 + m];
            fo[v] = own[(5 + v) * n2 + m];
        }
        const double so = own[25 * n2 + m];
        double qn[5], fn[5], sn;
        if (edge && bcd == ADG_BC_WALL) {
            // slip wall: background rho, rhoE at the face node (interior ones
            // without gravity), reflected normal momentum, interior gradient,
            // background heat flux
            double z, pb, rb;
            if (dir < 2) {
                z = P.org[2] + (ic2 + B.xi[a]) * P.h[2];
                pb = bg.pn[ic2 * n + a];
                rb = bg.rn[ic2 * n + a];
            } else {
                const int fz = ic2 + (plus ? 1 : 0);
                z = P.org[2] + fz * P.h[2];
                pb = bg.pf[fz];
                rb = bg.rf[fz];
            }
            qn[0] = qo[0];
            qn[1] = dir == 0 ? -qo[1] : qo[1];
            qn[2] = dir == 1 ? -qo[2] : qo[2];
            qn[3] = dir == 2 ? -qo[3] : qo[3];
            qn[4] = qo[4];
            if (P.gravity) {
                qn[0] = rb;
                qn[4] = pb / P.gm1 + rb * P.g * z;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int v = 0; v < 5; ++v) g[c][v] = own[((2 + c) * 5 + v) * n2 + m];
            if constexpr (MX) {
                // the ghost's flux and speed in FP32: with gravity the zero
                // perturbation of rho and rhoE over the exact background at the
                // face node (rhobar, pbar, Ebar + pbar), without it the ghost state
                float qg[5], gf[3][5], ff[3][5], src;
                float rbf = 0.0f, pbf = 0.0f, Hbf = 0.0f, gz = 0.0f;
                if (P.gravity) {
                    qg[0] = 0.0f;
                    qg[4] = 0.0f;
                    rbf = f64_to_f32(rb);
                    pbf = f64_to_f32(pb);
                    Hbf = f64_to_f32(qn[4] + pb);
                    gz = f64_to_f32(P.g * z);
                } else {
                    qg[0] = f64_to_f32(qn[0]);
                    qg[4] = f64_to_f32(qn[4]);
                }
                qg[1] = f64_to_f32(qn[1]);
                qg[2] = f64_to_f32(qn[2]);
                qg[3] = f64_to_f32(qn[3]);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int v = 0; v < 5; ++v) gf[c][v] = f64_to_f32(g[c][v]);
                ns_flux3f(qg, gf, gz, rbf, pbf, Hbf, Pf, ff, src, true, Pf.dTdz);
#pragma unroll
                for (int v = 0; v < 5; ++v) fn[v] = f32_to_f64(dir == 0 ? ff[0][v] : dir == 1 ? ff[1][v] : ff[2][v]);
                const float rho = rbf + qg[0];
                const float rinv = __frcp_rn(rho);
                const float pp = Pf.gm1 * (qg[4] - 0.5f * (qg[1] * qg[1] + qg[2] * qg[2] + qg[3] * qg[3]) * rinv -
                                           gz * qg[0]);
                const float mn = dir == 0 ? qg[1] : dir == 1 ? qg[2] : qg[3];
                sn = f32_to_f64(fabsf(mn) * rinv + sqrtf(Pf.gamma * (pbf + pp) * rinv) +
                                2.0f * Pf.eta[dir] * Pf.lamv * rinv);
            } else {
                double ff[3][5], src;
                ns_flux3(qn, g, z, pb, rb, P, true, ff, src);
#pragma unroll
                for (int v = 0; v < 5; ++v) fn[v] = dir == 0 ? ff[0][v] : dir == 1 ? ff[1][v] : ff[2][v];
                sn = wave_speed3(qn, z, dir, P);
            }
        } else if (edge && bcd == ADG_BC_ANALYTIC) {
            // the analytic field averaged over the step at the time nodes
            double xf[3];
            const int icc[3] = {ic0, ic1, ic2};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // along the face: node a (x-, y-faces: z; z-faces: y) and b
                const bool normal = c == dir;
                const int node_c = c == 2 ? a : (c == 1 ? (dir == 2 ? a : (dir == 0 ? b : 0)) : b);
                xf[c] = normal ? P.org[c] + (icc[c] + (plus ? 1 : 0)) * P.h[c]
                               : P.org[c] + (icc[c] + B.xi[node_c]) * P.h[c];
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) qn[v] = fn[v] = 0.0;
            for (int k = 0; k < n; ++k) {
                double q[5], ff[3][5], src;
                abc_field(xf[0], xf[1], xf[2], t + B.xi[k] * dt, P, q, g);
                ns_flux3(q, g, xf[2], 0.0, 0.0, P, false, ff, src);
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    qn[v] += B.w[k] * q[v];
                    fn[v] += B.w[k] * (dir == 0 ? ff[0][v] : dir == 1 ? ff[1][v] : ff[2][v]);
                }
            }
            sn = wave_speed3(qn, xf[2], dir, P);
        } else {
            const int nd = plus ? (icd + 1 == ncd ? 0 : icd + 1) : (icd == 0 ? ncd - 1 : icd - 1);
            const int nb0 = dir == 0 ? nd : ic0, nb1 = dir == 1 ? nd : ic1, nb2 = dir == 2 ? nd : ic2;
            const int nc = (nb2 * P.nc[1] + nb1) * P.nc[0] + nb0;
            const double* ot = trace + ((size_t)nc * 6 + (f ^ 1)) * TR;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                qn[v] = ot[v * n2 + m];
                fn[v] = ot[(5 + v) * n2 + m];
            }
            sn = ot[25 * n2 + m];
        }
        if constexpr (MX) {
            const double* qL = plus ? qo : qn;
            const double* qR = plus ? qn : qo;
            const double* fL = plus ? fo : fn;
            const double* fR = plus ? fn : fo;
            const float hs = 0.5f * fmaxf(f64_to_f32(so), f64_to_f32(sn));
#pragma unroll
            for (int v = 0; v < 5; ++v)
                Fst[cl][f][v][m] = 0.5f * (f64_to_f32(fL[v]) + f64_to_f32(fR[v])) -
                                   hs * f64_to_f32(__dsub_rn(qR[v], qL[v]));
        } else {
            double out[5];
            if (plus) rusanov5(qo, fo, so, qn, fn, sn, out);
            else rusanov5(qn, fn, sn, qo, fo, so, out);
#pragma unroll
            for (int v = 0; v < 5; ++v) Fst[cl][f][v][m] = out[v];
        }
    }
    __syncthreads();
    if (!active) return;
    double* uc = u + (size_t)cell * SL;
    const double* rc = rvol + (size_t)cell * SL;
    FT l1[3], l0[3], ih[3];
    {
        const int id[3] = {i, j, l};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if constexpr (MX) {
                l1[c] = f64_to_f32(B.lift1[id[c]]);
                l0[c] = f64_to_f32(B.lift0[id[c]]);
                ih[c] = f64_to_f32(P.inv_h[c]);
            } else {
                l1[c] = B.lift1[id[c]];
                l0[c] = B.lift0[id[c]];
                ih[c] = P.inv_h[c];
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        const FT face = (l1[0] * Fst[cl][0][v][l * n + j] - l0[0] * Fst[cl][1][v][l * n + j]) * ih[0] +
                        (l1[1] * Fst[cl][2][v][l * n + i] - l0[1] * Fst[cl][3][v][l * n + i]) * ih[1] +
                        (l1[2] * Fst[cl][4][v][j * n + i] - l0[2] * Fst[cl][5][v][j * n + i]) * ih[2];
        double fd;
        if constexpr (MX) fd = f32_to_f64(face);
        else fd = face;
        uc[v * n3 + node] += dt * (rc[v * n3 + node] - fd);
    }
}

// ---------------------------------------------------------------------------
// Mixed precision predictor: the same Picard iteration in FP32 on
// perturbation variables q' = (rho - rhobar, rho u, rho v, rho w, rhoE - Ebar)
// (the split in FP64 at load), total gradients = perturbation gradient +
// the FP64-formed derivative of the interpolated background.  With
// p' = (gamma-1)(E' - |m|^2/(2 rho) - g z rho') exact algebra, no FP32 value
// carries the background pressure through a difference.  Outputs keep the
// FP64 formats of the FP64 predictor: rvol converted, traces rebuilt as the
// FP64 base (the nodal background on x- and y-faces, its FP64 extrapolation
// on z-faces) plus the FP32 perturbation, the Rusanov speed in FP64 -- so
// the FP64 corrector runs unchanged.
template <int N>
struct Cfg3m {
    static constexpr size_t smem = (size_t)Cfg3<N>::cpb * Cfg3<N>::slots * 5 * Cfg3<N>::n3 * sizeof(float);
    // resident blocks asked of the register allocator: measured on the 25^3
    // bubble, degree 2 runs 12% faster at 4 blocks (72 registers, some
    // spills) than at the unconstrained 111 registers; degree 3 gains 1% at
    // 3 and loses at 4; degree 1 is indifferent
    static constexpr int minb = N == 2 ? 4 : N == 3 ? 3 : 1;
};

template <int N>
__global__ void __launch_bounds__(Cfg3<N>::threads, Cfg3m<N>::minb)
k3_predictor_mixed(const double* __restrict__ u, double* __restrict__ rvol, double* __restrict__ trace, int cells,
                   float dt, const BasisF B, const Phys3f P, const Phys3 P64, const Bg3m bg) {
    using C = Cfg3<N>;
    constexpr int n = C::n, n2 = C::n2, n3 = C::n3, SL = 5 * n3;
    extern __shared__ float smf[];
    const int cl = threadIdx.x / n3;
    const int node = threadIdx.x - cl * n3;
    const int l = node / n2, j = (node / n) % n, i = node % n;
    const int cell_raw = blockIdx.x * C::cpb + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const int iz = cell / (P64.nc[0] * P64.nc[1]);
    float* Q = smf + (size_t)cl * C::slots * SL;
    float* Fs = Q + n * SL;
    const int nb = iz * n + l;
    const float rb = bg.rbf[nb], pb = bg.pbf[nb], Hb = bg.Hbf[nb], dzr = bg.dzr[nb], dzE = bg.dzE[nb];
    const float gz = (float)(P64.g * bg.zn[nb]);

    float uu[5];
    {
        const double* uc = u + (size_t)cell * SL;
        uu[0] = f64_to_f32(__dsub_rn(uc[node], bg.rb[nb]));
        uu[1] = f64_to_f32(uc[n3 + node]);
        uu[2] = f64_to_f32(uc[2 * n3 + node]);
        uu[3] = f64_to_f32(uc[3 * n3 + node]);
        uu[4] = f64_to_f32(__dsub_rn(uc[4 * n3 + node], bg.Eb[nb]));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Q[v * n3 + node] = uu[v];
    __syncthreads();

    auto eval = [&](const float* Qk, float q[5], float g[3][5], float f[3][5], float& src) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float* Qv = Qk + v * n3;
            q[v] = Qv[node];
            float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx = fmaf(B.D[i][p], Qv[(l * n + j) * n + p], sx);
                sy = fmaf(B.D[j][p], Qv[(l * n + p) * n + i], sy);
                sz = fmaf(B.D[l][p], Qv[(p * n + j) * n + i], sz);
            }
            g[0][v] = sx * P.inv_h[0];
            g[1][v] = sy * P.inv_h[1];
            g[2][v] = sz * P.inv_h[2];
        }
        g[2][0] += dzr;
        g[2][4] += dzE;
        ns_flux3f(q, g, gz, rb, pb, Hb, P, f, src);
    };
    auto store = [&](const float f[3][5]) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int v = 0; v < 5; ++v) Fs[(b * 5 + v) * n3 + node] = f[b][v];
    };
    auto divergence = [&](int v) {
        const float* Fv = Fs + v * n3;
        const float* Gv = Fs + (5 + v) * n3;
        const float* Hv = Fs + (10 + v) * n3;
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sx = fmaf(B.D[i][p], Fv[(l * n + j) * n + p], sx);
            sy = fmaf(B.D[j][p], Gv[(l * n + p) * n + i], sy);
            sz = fmaf(B.D[l][p], Hv[(p * n + j) * n + i], sz);
        }
        return -(sx * P.inv_h[0] + sy * P.inv_h[1] + sz * P.inv_h[2]);
    };

    {
        float q[5], g[3][5], f[3][5], src;
        eval(Q, q, g, f, src);
        store(f);
        __syncthreads();
        float R0[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) R0[v] = (v == 3 ? src : 0.0f) + divergence(v);
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < 5; ++v) Q[k * SL + v * n3 + node] = uu[v] + dt * (B.Kw1[k] * R0[v]);
        __syncthreads();
    }
    // Sweeps 2..n.  Degrees <= 2 walk the time slices with a rolled loop
    // and accumulate the time contraction slice by slice (the same order as
    // a row-by-row sum; no register array indexed at run time): one inlined
    // flux evaluation instead of n.  Measured on the 25^3 bubble: degree 2
    // runs 4% faster this way (the unrolled kernel stalled on instruction
    // fetch), degrees 3 and 4 3% and 16% slower, so they keep the unrolled
    // form with the residuals of all slices in registers.
    constexpr int kSliceUnroll = N <= 2 ? 1 : n;
#pragma unroll 1
    for (int r = 1; r < n; ++r) {
        if constexpr (N <= 2) {
            float acc[n][5];
#pragma unroll
            for (int k = 0; k < n; ++k)
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[k][v] = 0.0f;
#pragma unroll 1
            for (int m = 0; m < n; ++m) {
                float q[5], g[3][5], f[3][5], src;
                eval(Q + m * SL, q, g, f, src);
                __syncthreads();
                store(f);
                __syncthreads();
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const float Rm = (v == 3 ? src : 0.0f) + divergence(v);
#pragma unroll
                    for (int k = 0; k < n; ++k) acc[k][v] = fmaf(B.Kw[k][m], Rm, acc[k][v]);
                }
            }
#pragma unroll
            for (int k = 0; k < n; ++k)
#pragma unroll
                for (int v = 0; v < 5; ++v) Q[k * SL + v * n3 + node] = uu[v] + dt * acc[k][v];
        } else {
            float R[n][5];
#pragma unroll
            for (int k = 0; k < n; ++k) {
                float q[5], g[3][5], f[3][5], src;
                eval(Q + k * SL, q, g, f, src);
                __syncthreads();
                store(f);
                __syncthreads();
#pragma unroll
                for (int v = 0; v < 5; ++v) R[k][v] = (v == 3 ? src : 0.0f) + divergence(v);
            }
#pragma unroll
            for (int k = 0; k < n; ++k)
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    float acc = 0.0f;
#pragma unroll
                    for (int m = 0; m < n; ++m) acc = fmaf(B.Kw[k][m], R[m][v], acc);
                    Q[k * SL + v * n3 + node] = uu[v] + dt * acc;
                }
        }
        __syncthreads();
    }

    float qb[5], fb[3][5], gb[3][5], sb = 0.0f;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        qb[v] = 0.0f;
#pragma unroll
        for (int b = 0; b < 3; ++b) fb[b][v] = gb[b][v] = 0.0f;
    }
#pragma unroll kSliceUnroll
    for (int k = 0; k < n; ++k) {
        float q[5], g[3][5], f[3][5], src;
        eval(Q + k * SL, q, g, f, src);
        const float wk = B.w[k];
        sb = fmaf(wk, src, sb);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            qb[v] = fmaf(wk, q[v], qb[v]);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                fb[b][v] = fmaf(wk, f[b][v], fb[b][v]);
                gb[b][v] = fmaf(wk, g[b][v], gb[b][v]);
            }
        }
    }
    __syncthreads();
    float* A = Q;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        A[v * n3 + node] = qb[v];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            A[(1 + b) * SL + v * n3 + node] = fb[b][v];
            A[(4 + b) * SL + v * n3 + node] = gb[b][v];
        }
    }
    __syncthreads();
    if (active) {
        double* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float* Fv = A + 1 * SL + v * n3;
            const float* Gv = A + 2 * SL + v * n3;
            const float* Hv = A + 3 * SL + v * n3;
            float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx = fmaf(B.Vx[p][i], Fv[(l * n + j) * n + p], sx);
                sy = fmaf(B.Vx[p][j], Gv[(l * n + p) * n + i], sy);
                sz = fmaf(B.Vx[p][l], Hv[(p * n + j) * n + i], sz);
            }
            rc[v * n3 + node] = f32_to_f64(sx * P.inv_h[0] + sy * P.inv_h[1] + sz * P.inv_h[2] + (v == 3 ? sb : 0.0f));
        }
    }
    const int ic0 = cell % P64.nc[0], ic1 = (cell / P64.nc[0]) % P64.nc[1];
    for (int idx = node; idx < 6 * n2; idx += n3) {
        const int f = idx / n2, m = idx - f * n2;
        const int a = m / n, b = m - a * n;
        const int dir = f >> 1;
        const float* phi = (f & 1) ? B.phi0 : B.phi1;
        // the gradient components are read only by slip-wall ghosts: written
        // for wall faces alone
        const int icd = dir == 0 ? ic0 : dir == 1 ? ic1 : iz;
        const int ncd = dir == 0 ? P64.nc[0] : dir == 1 ? P64.nc[1] : P64.nc[2];
        const int bcd = dir == 0 ? P64.bc[0] : dir == 1 ? P64.bc[1] : P64.bc[2];
        const bool wallface = bcd == ADG_BC_WALL && ((f & 1) ? icd == 0 : icd == ncd - 1);
        double rec[kTr3];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            if (c >= 2 && !wallface) {
#pragma unroll
                for (int v = 0; v < 5; ++v) rec[c * 5 + v] = 0.0;
                continue;
            }
            const int slot = c == 0 ? 0 : c == 1 ? 1 + dir : 2 + c;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float* S = A + slot * SL + v * n3;
                float s = 0.0f;
#pragma unroll
                for (int p = 0; p < n; ++p) {
                    const int at = dir == 0 ? (a * n + b) * n + p : dir == 1 ? (a * n + p) * n + b : (p * n + a) * n + b;
                    s = fmaf(phi[p], S[at], s);
                }
                rec[c * 5 + v] = f32_to_f64(s);
            }
        }
        // FP64 base of the face node: the nodal background at the node's height
        // on x- and y-faces, its extrapolation on z-faces
        double brho, bE;
        if (dir < 2) {
            brho = bg.rb[iz * n + a];
            bE = bg.Eb[iz * n + a];
        } else {
            const double* e = bg.ext + ((size_t)iz * 2 + (f & 1)) * 2;
            brho = e[0];
            bE = e[1];
        }
        // Rusanov speed in FP32 from the perturbation face state over its base
        {
            float rbf, pbf, zf;
            if (dir < 2) {
                rbf = bg.rbf[iz * n + a];
                pbf = bg.pbf[iz * n + a];
                zf = (float)bg.zn[iz * n + a];
            } else {
                const float* e = bg.zext + ((size_t)iz * 2 + (f & 1)) * 2;
                rbf = e[0];
                pbf = e[1];
                zf = (float)(P64.org[2] + (iz + ((f & 1) ? 0 : 1)) * P64.h[2]);
            }
            const float qp0 = (float)rec[0], qp4 = (float)rec[4];
            const float m0 = (float)rec[1], m1 = (float)rec[2], m2 = (float)rec[3];
            const float rho = rbf + qp0;
            const float rinv = __frcp_rn(rho);
            const float pp = P.gm1 * (qp4 - 0.5f * (m0 * m0 + m1 * m1 + m2 * m2) * rinv - P.g * zf * qp0);
            const float mn = dir == 0 ? m0 : dir == 1 ? m1 : m2;
            const float sp = fabsf(mn) * rinv + sqrtf(P.gamma * (pbf + pp) * rinv) +
                             2.0f * P.eta[dir] * P.lamv * rinv;
            rec[25] = f32_to_f64(sp);
        }
        rec[0] += brho;
        rec[4] += bE;
        if (active) {
            double* tr = trace + ((size_t)cell * 6 + f) * kTr3 * n2;
#pragma unroll
            for (int c = 0; c < kTr3; ++c)
                if (c < 10 || c == 25 || wallface) tr[c * n2 + m] = rec[c];
        }
    }    pdl_trigger();
}

// nodal values of a scenario: the 3D cosine bubble or the background
// (theta' at the background pressure, at rest), or the ABC field at time t
__global__ void k3_init(double* __restrict__ u, int cells, int n, int kind, double A, double a, double xc, double zc,
                        double t, const Basis B, const Phys3 P) {
    const int n3 = n * n * n;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)cells * n3) return;
    const int cell = (int)(gid / n3), node = (int)(gid % n3);
    const int l = node / (n * n), j = (node / n) % n, i = node % n;
    const int ix = cell % P.nc[0], iy = (cell / P.nc[0]) % P.nc[1], iz = cell / (P.nc[0] * P.nc[1]);
    const double x = P.org[0] + (ix + B.xi[i]) * P.h[0];
    const double y = P.org[1] + (iy + B.xi[j]) * P.h[1];
    const double z = P.org[2] + (iz + B.xi[l]) * P.h[2];
    double q[5];
    if (kind == ADG_SCEN_ABC) {
        double g[3][5];
        abc_field(x, y, z, t, P, q, g);
    } else {
        double th = 0.0;
        if (kind == ADG_SCEN_COSINE) {
            const double r = sqrt((x - xc) * (x - xc) + (y - xc) * (y - xc) + (z - zc) * (z - zc));
            th = r <= a ? 0.5 * A * (1.0 + cos(3.14159265358979323846 * r / a)) : 0.0;
        }
        const double ex = 1.0 - P.g * z / (P.cp * P.theta0);
        const double pb = P.p0 * pow(ex, P.cp / P.R);
        const double rho = pb / (P.R * (P.theta0 + th) * ex);
        q[0] = rho;
        q[1] = q[2] = q[3] = 0.0;
        q[4] = pb / P.gm1 + rho * P.g * z;
    }
    double* uc = u + (size_t)cell * 5 * n3;
    for (int v = 0; v < 5; ++v) uc[v * n3 + node] = q[v];
}

// per-block maxima of |v| + c + 2 eta lambda_v / rho over the nodes
__global__ void __launch_bounds__(256) k3_speed(const double* __restrict__ u, int cells, int n, double eta,
                                                double* __restrict__ part, const Basis B, const Phys3 P) {
    __shared__ double red[256];
    const int n3 = n * n * n;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (gid < (long long)cells * n3) {
        const int cell = (int)(gid / n3), node = (int)(gid % n3);
        const int l = node / (n * n);
        const int iz = cell / (P.nc[0] * P.nc[1]);
        const double z = P.org[2] + (iz + B.xi[l]) * P.h[2];
        const double* uc = u + (size_t)cell * 5 * n3;
        double q[5];
        for (int v = 0; v < 5; ++v) q[v] = uc[v * n3 + node];
        const double rinv = 1.0 / q[0];
        const double gg = P.gravity ? P.g : 0.0;
        const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        const double p = P.gm1 * (q[4] - 0.5 * m2 * rinv - q[0] * gg * z);
        s = sqrt(m2) * rinv + sqrt(P.gamma * p * rinv) + 2.0 * eta * P.lamv * rinv;
        if (!(s == s)) s = INFINITY;  // NaN state: reported as a non-finite speed
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <int N>
int launch3(bool pred, double* u, double* rvol, double* trace, int cells, double dt, double t, const Basis& B,
            const Phys3& P, const Bg3& bg, cudaStream_t s, bool mixed, const Phys3f& Pf) {
    using C = Cfg3<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    if (pred) {
        cudaError_t e = cudaFuncSetAttribute(k3_predictor<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (e != cudaSuccess) return (int)e;
        k3_predictor<N><<<blocks, C::threads, C::smem, s>>>(u, rvol, trace, cells, dt, B, P, bg);
    } else {
        // programmatic launch: scheduled while the predictor drains
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(C::threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = mixed ? cudaLaunchKernelEx(&cfg, k3_corrector<N, true>, u, rvol, trace, cells, dt, t, B, P, bg, Pf)
                                    : cudaLaunchKernelEx(&cfg, k3_corrector<N, false>, u, rvol, trace, cells, dt, t, B, P, bg, Pf);
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaGetLastError();
}

template <int N>
int launch3m(const double* u, double* rvol, double* trace, int cells, float dt, const BasisF& B, const Phys3f& P,
             const Phys3& P64, const Bg3m& bg, cudaStream_t s) {
    using C = Cfg3<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    cudaError_t e = cudaFuncSetAttribute(k3_predictor_mixed<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg3m<N>::smem);
    if (e != cudaSuccess) return (int)e;
    k3_predictor_mixed<N><<<blocks, C::threads, Cfg3m<N>::smem, s>>>(u, rvol, trace, cells, dt, B, P, P64, bg);
    return (int)cudaGetLastError();
}

int launch3m_any(int N, const double* u, double* rvol, double* trace, int cells, float dt, const BasisF& B,
                 const Phys3f& P, const Phys3& P64, const Bg3m& bg, cudaStream_t s) {
    switch (N) {
        case 1: return launch3m<1>(u, rvol, trace, cells, dt, B, P, P64, bg, s);
        case 2: return launch3m<2>(u, rvol, trace, cells, dt, B, P, P64, bg, s);
        case 3: return launch3m<3>(u, rvol, trace, cells, dt, B, P, P64, bg, s);
        case 4: return launch3m<4>(u, rvol, trace, cells, dt, B, P, P64, bg, s);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch3_any(int N, bool pred, double* u, double* rvol, double* trace, int cells, double dt, double t,
                const Basis& B, const Phys3& P, const Bg3& bg, cudaStream_t s, bool mixed, const Phys3f& Pf) {
    switch (N) {
        case 1: return launch3<1>(pred, u, rvol, trace, cells, dt, t, B, P, bg, s, mixed, Pf);
        case 2: return launch3<2>(pred, u, rvol, trace, cells, dt, t, B, P, bg, s, mixed, Pf);
        case 3: return launch3<3>(pred, u, rvol, trace, cells, dt, t, B, P, bg, s, mixed, Pf);
        case 4: return launch3<4>(pred, u, rvol, trace, cells, dt, t, B, P, bg, s, mixed, Pf);
        default: return (int)cudaErrorInvalidValue;
    }
}
}  // namespace
}  // namespace adg

struct adg_mesh3 {
    adg_mesh_desc d;
    int N = 0, n = 0, nz = 0, bc_z = 0, cells = 0;
    double z0 = 0, Lz = 0, t = 0;
    adg::Basis B;
    adg::Phys3 P;
    double* u = nullptr;      // [cells][5][n^3]
    double* rvol = nullptr;   // [cells][5][n^3]
    double* trace = nullptr;  // [cells][6][kTr3][n^2]
    double* bg = nullptr;     // pbar, rhobar at nodes [nz n] each, then at faces [nz + 1] each
    double* part = nullptr;   // stable-dt block maxima
    int part_blocks = 0;
    // mixed precision: FP32 basis and constants, background tables
    adg::BasisF Bf;
    adg::Phys3f Pf;
    double* mbg = nullptr;    // rhobar, Ebar, node height [nz n] each, then extrapolated z-face base [nz][2][2]
    float* mbgf = nullptr;    // rhobar, pbar, Ebar + pbar, d rhobar/dz, d Ebar/dz [nz n] each
};

using adg::cuda_fail;
using adg::fail;

namespace {

int dev3(const adg_mesh3* m) {
    const cudaError_t e = cudaSetDevice(m->d.device);
    return e == cudaSuccess ? ADG_OK : cuda_fail(e, "mesh3: cudaSetDevice");
}

void free3(adg_mesh3* m) {
    if (!m) return;
    cudaSetDevice(m->d.device);
    cudaFree(m->u);
    cudaFree(m->rvol);
    cudaFree(m->trace);
    cudaFree(m->bg);
    cudaFree(m->part);
    cudaFree(m->mbg);
    cudaFree(m->mbgf);
    delete m;
}

adg::Bg3 bg3(const adg_mesh3* m) {
    const int nn = m->nz * m->n;
    return adg::Bg3{m->bg, m->bg + nn, m->bg + 2 * nn, m->bg + 2 * nn + (m->nz + 1)};
}

adg::Bg3m bg3m(const adg_mesh3* m) {
    const size_t nn = (size_t)m->nz * m->n;
    adg::Bg3m b;
    b.rb = m->mbg;
    b.Eb = m->mbg + nn;
    b.zn = m->mbg + 2 * nn;
    b.ext = m->mbg + 3 * nn;
    b.rbf = m->mbgf;
    b.pbf = m->mbgf + nn;
    b.Hbf = m->mbgf + 2 * nn;
    b.dzr = m->mbgf + 3 * nn;
    b.dzE = m->mbgf + 4 * nn;
    b.zext = m->mbgf + 5 * nn;
    return b;
}

// FP32 basis and constants and the background tables of the mixed predictor
int build_mixed3(adg_mesh3* m) {
    const int n = m->n, nz = m->nz;
    const adg::Basis& B = m->B;
    adg::BasisF& b = m->Bf;
    std::memset(&b, 0, sizeof(b));
    for (int a = 0; a < n; ++a) {
        b.xi[a] = (float)B.xi[a];
        b.w[a] = (float)B.w[a];
        b.phi0[a] = (float)B.phi0[a];
        b.phi1[a] = (float)B.phi1[a];
        b.Kw1[a] = (float)B.Kw1[a];
        b.lift0[a] = (float)B.lift0[a];
        b.lift1[a] = (float)B.lift1[a];
        for (int c = 0; c < n; ++c) {
            b.D[a][c] = (float)B.D[a][c];
            b.Kw[a][c] = (float)B.Kw[a][c];
            b.Vx[a][c] = (float)B.Vx[a][c];
        }
    }
    const adg::Phys3& P = m->P;
    adg::Phys3f& f = m->Pf;
    std::memset(&f, 0, sizeof(f));
    f.gamma = (float)P.gamma;
    f.gm1 = (float)P.gm1;
    f.R = (float)P.R;
    f.invR = (float)P.invR;
    f.mu = (float)P.mu;
    f.kappa = (float)P.kappa;
    f.g = (float)P.g;
    f.lamv = (float)P.lamv;
    f.dTdz = (float)P.dTdz;
    for (int c = 0; c < 3; ++c) {
        f.inv_h[c] = (float)P.inv_h[c];
        f.eta[c] = (float)P.eta[c];
    }
    f.gravity = P.gravity;
    const size_t nn = (size_t)nz * n;
    std::vector<double> hd(3 * nn + 4 * (size_t)nz, 0.0);
    std::vector<float> hf(5 * nn + 4 * (size_t)nz, 0.0f);
    std::vector<double> rb(nn, 0.0), Eb(nn, 0.0), pb(nn, 0.0);
    for (int iz = 0; iz < nz; ++iz)
        for (int l = 0; l < n; ++l) {
            const size_t k = (size_t)iz * n + l;
            const double z = P.org[2] + (iz + B.xi[l]) * P.h[2];
            hd[2 * nn + k] = z;
            if (P.gravity) {
                const double ex = 1.0 - P.g * z / (P.cp * P.theta0);
                pb[k] = P.p0 * std::pow(ex, P.cp / P.R);
                rb[k] = pb[k] / (P.R * P.theta0 * ex);
                Eb[k] = pb[k] / P.gm1 + rb[k] * P.g * z;
            }
        }
    for (int iz = 0; iz < nz; ++iz) {
        for (int l = 0; l < n; ++l) {
            const size_t k = (size_t)iz * n + l;
            double dr = 0.0, dE = 0.0;
            for (int p = 0; p < n; ++p) {
                dr += B.D[l][p] * rb[(size_t)iz * n + p];
                dE += B.D[l][p] * Eb[(size_t)iz * n + p];
            }
            hd[k] = rb[k];
            hd[nn + k] = Eb[k];
            hf[k] = (float)rb[k];
            hf[nn + k] = (float)pb[k];
            hf[2 * nn + k] = (float)(Eb[k] + pb[k]);
            hf[3 * nn + k] = (float)(dr * P.inv_h[2]);
            hf[4 * nn + k] = (float)(dE * P.inv_h[2]);
        }
        for (int face = 0; face < 2; ++face) {  // 0: top (phi(1)), 1: bottom (phi(0))
            const double* phi = face == 0 ? B.phi1 : B.phi0;
            double er = 0.0, eE = 0.0;
            for (int p = 0; p < n; ++p) {
                er += phi[p] * rb[(size_t)iz * n + p];
                eE += phi[p] * Eb[(size_t)iz * n + p];
            }
            hd[3 * nn + ((size_t)iz * 2 + face) * 2] = er;
            hd[3 * nn + ((size_t)iz * 2 + face) * 2 + 1] = eE;
            const double zf = P.org[2] + (iz + (face == 0 ? 1 : 0)) * P.h[2];
            hf[5 * nn + ((size_t)iz * 2 + face) * 2] = (float)er;
            hf[5 * nn + ((size_t)iz * 2 + face) * 2 + 1] = (float)(P.gm1 * (eE - er * P.g * zf));
        }
    }
    if (cudaMalloc(&m->mbg, hd.size() * 8) != cudaSuccess || cudaMalloc(&m->mbgf, hf.size() * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "adg3_create: mixed-precision tables");
    }
    ADG_CK(cudaMemcpy(m->mbg, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice), "adg3_create: mixed tables");
    ADG_CK(cudaMemcpy(m->mbgf, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice), "adg3_create: mixed tables");
    return ADG_OK;
}

bool bc3_ok(int bc) { return bc == ADG_BC_PERIODIC || bc == ADG_BC_WALL || bc == ADG_BC_ANALYTIC; }

}  // namespace

extern "C" int adg3_create(const adg_mesh_desc* d, int nz, double z0, double Lz, int bc_z, adg_mesh3** out) {
    if (!d || !out) return fail(ADG_EINVAL, "adg3_create: NULL argument");
    *out = nullptr;
    if (d->degree < 1 || d->degree > ADG_MAX_DEGREE_3D) return fail(ADG_EINVAL, "adg3_create: degree out of range");
    if (d->nx < 1 || d->ny < 1 || nz < 1 || (long long)d->nx * d->ny * nz > (1LL << 24))
        return fail(ADG_EINVAL, "adg3_create: bad mesh size");
    if (!(d->Lx > 0.0) || !(d->Ly > 0.0) || !(Lz > 0.0) || !std::isfinite(z0))
        return fail(ADG_EINVAL, "adg3_create: Lx, Ly, Lz must be > 0");
    if (!bc3_ok(d->bc_x) || !bc3_ok(d->bc_y) || !bc3_ok(bc_z))
        return fail(ADG_EINVAL, "adg3_create: boundaries are periodic, ADG_BC_WALL or ADG_BC_ANALYTIC");
    if (!(d->gamma > 1.0) || !(d->R > 0.0) || !(d->Pr > 0.0) || !(d->mu >= 0.0))
        return fail(ADG_EINVAL, "adg3_create: invalid gas constants");
    if ((d->precision != ADG_PREC_FP64 && d->precision != ADG_PREC_MIXED) || d->source != ADG_SRC_NONE ||
        d->max_levels != 0)
        return fail(ADG_EUNSUPPORTED, "adg3_create: FP64 or mixed, no manufactured source, uniform mesh only");
    const bool analytic = d->bc_x == ADG_BC_ANALYTIC || d->bc_y == ADG_BC_ANALYTIC || bc_z == ADG_BC_ANALYTIC;
    if (analytic && (d->bc_field != ADG_FIELD_ABC || d->gravity))
        return fail(ADG_EINVAL, "adg3_create: analytic boundaries take bc_field ADG_FIELD_ABC without gravity");
    if (d->gravity && !(d->theta0 > 0.0 && d->p0 > 0.0 && d->g > 0.0))
        return fail(ADG_EINVAL, "adg3_create: gravity needs g, theta0, p0 > 0");
    int ndev = 0;
    ADG_CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (d->device < 0 || d->device >= ndev) return fail(ADG_EINVAL, "adg3_create: bad device ordinal");
    adg_mesh3* m = new adg_mesh3();
    m->d = *d;
    m->N = d->degree;
    m->n = d->degree + 1;
    m->nz = nz;
    m->z0 = z0;
    m->Lz = Lz;
    m->bc_z = bc_z;
    m->cells = d->nx * d->ny * nz;
    if (!adg::build_basis(m->N, m->B)) {
        delete m;
        return fail(ADG_EINVAL, "adg3_create: singular time-stiffness matrix");
    }
    adg::Phys3& P = m->P;
    std::memset(&P, 0, sizeof(P));
    std::memset(&m->Pf, 0, sizeof(m->Pf));
    P.gamma = d->gamma;
    P.gm1 = d->gamma - 1.0;
    P.R = d->R;
    P.invR = 1.0 / d->R;
    P.mu = d->mu;
    P.cp = d->gamma * d->R / (d->gamma - 1.0);
    P.kappa = d->mu * P.cp / d->Pr;
    P.gravity = d->gravity ? 1 : 0;
    P.g = d->gravity ? d->g : 0.0;
    P.p0 = d->p0;
    P.theta0 = d->theta0;
    P.lamv = std::max(4.0 / 3.0, d->gamma / d->Pr) * d->mu;
    P.dTdz = d->gravity ? -d->g / P.cp : 0.0;
    const double L[3] = {d->Lx, d->Ly, Lz}, o[3] = {d->x0, d->y0, z0};
    const int nc[3] = {d->nx, d->ny, nz}, bc[3] = {d->bc_x, d->bc_y, bc_z};
    for (int c = 0; c < 3; ++c) {
        P.h[c] = L[c] / nc[c];
        P.inv_h[c] = 1.0 / P.h[c];
        P.org[c] = o[c];
        P.nc[c] = nc[c];
        P.bc[c] = bc[c];
        P.eta[c] = (2 * m->N + 1) / (P.h[c] * std::sqrt(M_PI / 2.0));
    }
    P.field = d->bc_field;
    if (int rc = dev3(m)) {
        delete m;
        return rc;
    }
    const int n = m->n, n3 = n * n * n;
    const size_t st = (size_t)m->cells * 5 * n3;
    m->part_blocks = (int)(((long long)m->cells * n3 + 255) / 256);
    const size_t nbg = 2 * (size_t)nz * n + 2 * (size_t)(nz + 1);
    if (cudaMalloc(&m->u, st * 8) != cudaSuccess || cudaMalloc(&m->rvol, st * 8) != cudaSuccess ||
        cudaMalloc(&m->trace, (size_t)m->cells * 6 * adg::kTr3 * n * n * 8) != cudaSuccess ||
        cudaMalloc(&m->bg, nbg * 8) != cudaSuccess || cudaMalloc(&m->part, (size_t)m->part_blocks * 8) != cudaSuccess) {
        cudaGetLastError();
        free3(m);
        return fail(ADG_ENOMEM, "adg3_create: device allocation failed");
    }
    // isentropic background (Eq. 6) at node heights and at horizontal faces
    std::vector<double> h(nbg, 0.0);
    if (d->gravity) {
        auto bgp = [&](double z, double& p, double& r) {
            const double ex = 1.0 - d->g * z / (P.cp * d->theta0);
            p = d->p0 * std::pow(ex, P.cp / d->R);
            r = p / (d->R * d->theta0 * ex);
        };
        const int nn = nz * n;
        for (int iz = 0; iz < nz; ++iz)
            for (int l = 0; l < n; ++l) bgp(z0 + (iz + m->B.xi[l]) * P.h[2], h[iz * n + l], h[nn + iz * n + l]);
        for (int k = 0; k <= nz; ++k) bgp(z0 + k * P.h[2], h[2 * nn + k], h[2 * nn + (nz + 1) + k]);
    }
    if (cudaMemcpy(m->bg, h.data(), nbg * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->u, 0, st * 8) != cudaSuccess) {
        cudaGetLastError();
        free3(m);
        return fail(ADG_ECUDA, "adg3_create: initialisation failed");
    }
    if (d->precision == ADG_PREC_MIXED) {
        if (int rc = build_mixed3(m)) {
            free3(m);
            return rc;
        }
    }
    *out = m;
    return ADG_OK;
}

extern "C" void adg3_destroy(adg_mesh3* m) { free3(m); }

extern "C" size_t adg3_state_count(const adg_mesh3* m) {
    return m ? (size_t)m->cells * 5 * m->n * m->n * m->n : 0;
}

extern "C" int adg3_set_state(adg_mesh3* m, const double* u, size_t count, int on_device, void* stream) {
    if (!m || !u) return fail(ADG_EINVAL, "adg3_set_state: NULL argument");
    if (count != adg3_state_count(m)) return fail(ADG_EINVAL, "adg3_set_state: count mismatch");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "bad on_device");
    if (int rc = dev3(m)) return rc;
    ADG_CK(cudaMemcpyAsync(m->u, u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           (cudaStream_t)stream),
           "adg3_set_state");
    if (on_device == 0) ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "adg3_set_state sync");
    return ADG_OK;
}

extern "C" int adg3_get_state(adg_mesh3* m, double* u, size_t count, int on_device, void* stream) {
    if (!m || !u) return fail(ADG_EINVAL, "adg3_get_state: NULL argument");
    if (count != adg3_state_count(m)) return fail(ADG_EINVAL, "adg3_get_state: count mismatch");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "bad on_device");
    if (int rc = dev3(m)) return rc;
    ADG_CK(cudaMemcpyAsync(u, m->u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           (cudaStream_t)stream),
           "adg3_get_state");
    if (on_device == 0) ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "adg3_get_state sync");
    return ADG_OK;
}

extern "C" int adg3_set_time(adg_mesh3* m, double t) {
    if (!m || !std::isfinite(t)) return fail(ADG_EINVAL, "adg3_set_time: bad argument");
    m->t = t;
    return ADG_OK;
}

extern "C" double adg3_get_time(const adg_mesh3* m) { return m ? m->t : 0.0; }

extern "C" int adg3_init_scenario(adg_mesh3* m, const adg_scenario* s, void* stream) {
    if (!m || !s) return fail(ADG_EINVAL, "adg3_init_scenario: NULL argument");
    if (s->kind == ADG_SCEN_COSINE || s->kind == ADG_SCEN_BACKGROUND) {
        if (!m->d.gravity) return fail(ADG_EINVAL, "adg3_init_scenario: bubble scenarios need gravity");
        if (s->kind == ADG_SCEN_COSINE && !(s->a > 0.0)) return fail(ADG_EINVAL, "adg3_init_scenario: radius must be > 0");
    } else if (s->kind != ADG_SCEN_ABC) {
        return fail(ADG_EINVAL, "adg3_init_scenario: cosine bubble, background or ABC field");
    }
    if (int rc = dev3(m)) return rc;
    const long long total = (long long)m->cells * m->n * m->n * m->n;
    adg::k3_init<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        m->u, m->cells, m->n, s->kind, s->A, s->a, s->xc, s->zc, m->t, m->B, m->P);
    ADG_CK(cudaGetLastError(), "adg3_init_scenario launch");
    return ADG_OK;
}

extern "C" int adg3_step(adg_mesh3* m, double dt, int nsteps, void* stream) {
    if (!m) return fail(ADG_EINVAL, "adg3_step: NULL argument");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 1) return fail(ADG_EINVAL, "adg3_step: dt > 0, nsteps >= 1");
    if (int rc = dev3(m)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const adg::Bg3 bg = bg3(m);
    for (int k = 0; k < nsteps; ++k) {
        int e = m->d.precision == ADG_PREC_MIXED
                    ? adg::launch3m_any(m->N, m->u, m->rvol, m->trace, m->cells, (float)dt, m->Bf, m->Pf, m->P,
                                        bg3m(m), s)
                    : adg::launch3_any(m->N, true, m->u, m->rvol, m->trace, m->cells, dt, m->t, m->B, m->P, bg, s,
                                       false, m->Pf);
        if (e) return cuda_fail((cudaError_t)e, "adg3_step predictor");
        e = adg::launch3_any(m->N, false, m->u, m->rvol, m->trace, m->cells, dt, m->t, m->B, m->P, bg, s,
                             m->d.precision == ADG_PREC_MIXED, m->Pf);
        if (e) return cuda_fail((cudaError_t)e, "adg3_step corrector");
        m->t += dt;
    }
    return ADG_OK;
}

extern "C" int adg3_stable_dt(adg_mesh3* m, double cfl, double* dt, void* stream) {
    if (!m || !dt) return fail(ADG_EINVAL, "adg3_stable_dt: NULL argument");
    if (!(cfl > 0.0)) return fail(ADG_EINVAL, "adg3_stable_dt: cfl must be > 0");
    if (int rc = dev3(m)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const double h = std::min(m->P.h[0], std::min(m->P.h[1], m->P.h[2]));
    const double eta = (2 * m->N + 1) / (h * std::sqrt(M_PI / 2.0));
    adg::k3_speed<<<m->part_blocks, 256, 0, s>>>(m->u, m->cells, m->n, eta, m->part, m->B, m->P);
    ADG_CK(cudaGetLastError(), "adg3_stable_dt launch");
    std::vector<double> hp(m->part_blocks);
    ADG_CK(cudaMemcpyAsync(hp.data(), m->part, hp.size() * 8, cudaMemcpyDeviceToHost, s), "adg3_stable_dt copy");
    ADG_CK(cudaStreamSynchronize(s), "adg3_stable_dt sync");
    double lam = 0.0;
    for (double v : hp) lam = std::max(lam, v);
    if (!(lam > 0.0) || !std::isfinite(lam)) return fail(ADG_ENONFINITE, "adg3_stable_dt: non-finite or zero wave speed");
    *dt = cfl * h / (3.0 * (2 * m->N + 1) * lam);
    return ADG_OK;
}
