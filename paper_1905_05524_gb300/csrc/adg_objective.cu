// Potential-temperature maps of the warm-bubble sensitivity problem, on the
// device and with their adjoints, so that a differentiable rollout moves only
// device arrays through the C ABI:
//
//  * theta' -> state: the bubble initialisation of Sec. 4.2 (reading I1):
//    pressure at the isentropic background pbar(z) = p0 pi^(cp/R),
//    temperature (theta0 + theta') pi with the Exner function
//    pi = 1 - g z/(cp theta0), the fluid at rest, rhoE = pbar/(gamma-1) + rho g z;
//  * state -> theta' = T (p0/p)^(R/cp) - theta0 (Sec. 4.2, the indicator
//    variable of the TV criterion);
//  * the probe objective J = sum_p (theta'(x_p) - target_p)^2 with theta'
//    interpolated in the probe's cell by the nodal Lagrange basis, and dJ/du.
//
// All FP64, uniform meshes.  Reductions run in a fixed order (one block for
// J; each node's gradient sums the probes in index order), so results are
// bitwise reproducible.
#include <cuda_runtime.h>

#include "adg_mesh.h"
#include "adg_tv_cell.cuh"

namespace adg {
namespace {

constexpr int kObjThreads = 256;

__device__ __forceinline__ double node_height(int iy, int j, const Basis& B, const Phys& P) {
    return P.y0 + (iy + B.xi[j]) * P.hy;
}

// d theta / d (rho, rho u, rho v, rho E) at one node
__device__ __forceinline__ void theta_gradient(const double q[4], double z, const Phys& P, double th,
                                               double dth[4]) {
    const double rinv = 1.0 / q[0];
    const double gz = P.gravity ? P.g * z : 0.0;
    const double ke = 0.5 * (q[1] * q[1] + q[2] * q[2]) * rinv;
    const double p = P.gm1 * (q[3] - ke - q[0] * gz);
    const double dth_dp = th * (1.0 - P.Rcp) / p;  // theta ~ p^(1 - R/cp) / rho
    dth[0] = dth_dp * P.gm1 * (ke * rinv - gz) - th * rinv;
    dth[1] = -dth_dp * P.gm1 * q[1] * rinv;
    dth[2] = -dth_dp * P.gm1 * q[2] * rinv;
    dth[3] = dth_dp * P.gm1;
}

// probe p: its cell (clamped to the mesh) and local coordinates in [0, 1]
__device__ __forceinline__ int probe_cell(const double* xy, int p, const Phys& P, double& sx, double& sy) {
    const double fx = (xy[2 * p] - P.x0) / P.hx, fy = (xy[2 * p + 1] - P.y0) / P.hy;
    const int ix = min(max((int)floor(fx), 0), P.nx - 1);
    const int iy = min(max((int)floor(fy), 0), P.ny - 1);
    sx = fx - ix;
    sy = fy - iy;
    return iy * P.nx + ix;
}

// Lagrange basis function a of the nodes B.xi at s
__device__ __forceinline__ double lagrange(const Basis& B, int n, int a, double s) {
    double l = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != a) l *= (s - B.xi[m]) / (B.xi[a] - B.xi[m]);
    return l;
}

__global__ void k_theta_to_state(const double* __restrict__ th, double* __restrict__ u, int cells, int n,
                                 const Basis B, const Phys P) {
    const int n2 = n * n;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2, j = node / n;
    const double z = node_height(cell / P.nx, j, B, P);
    const double ex = 1.0 - P.g * z / (P.cp * P.theta0);
    const double pb = P.p0 * pow(ex, 1.0 / P.Rcp);
    const double rho = pb / (P.R * ((P.theta0 + th[gid]) * ex));
    double* uc = u + (size_t)cell * 4 * n2;
    uc[node] = rho;
    uc[n2 + node] = 0.0;
    uc[2 * n2 + node] = 0.0;
    uc[3 * n2 + node] = pb / P.gm1 + rho * P.g * z;
}

__global__ void k_theta_to_state_adj(const double* __restrict__ th, const double* __restrict__ lam_u,
                                     double* __restrict__ lam_th, int cells, int n, const Basis B, const Phys P) {
    const int n2 = n * n;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2, j = node / n;
    const double z = node_height(cell / P.nx, j, B, P);
    const double ex = 1.0 - P.g * z / (P.cp * P.theta0);
    const double pb = P.p0 * pow(ex, 1.0 / P.Rcp);
    const double T0 = P.theta0 + th[gid];
    const double rho = pb / (P.R * (T0 * ex));
    const double drho = -rho / T0;  // d rho / d theta'; d rhoE / d theta' = g z d rho / d theta'
    const double* lc = lam_u + (size_t)cell * 4 * n2;
    lam_th[gid] = drho * (lc[node] + P.g * z * lc[3 * n2 + node]);
}

__global__ void k_state_to_theta(const double* __restrict__ u, double* __restrict__ th, int cells, int n,
                                 const Basis B, const Phys P) {
    const int n2 = n * n;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2, j = node / n;
    const double* uc = u + (size_t)cell * 4 * n2;
    const double q[4] = {uc[node], uc[n2 + node], uc[2 * n2 + node], uc[3 * n2 + node]};
    th[gid] = theta_of(q, node_height(cell / P.nx, j, B, P), P) - P.theta0;
}

// one block: residuals r_p = theta'(x_p) - target_p and J = sum r_p^2 (fixed order)
__global__ void __launch_bounds__(kObjThreads)
k_probe_values(const double* __restrict__ u, int n, const double* __restrict__ xy,
               const double* __restrict__ target, int np, double* __restrict__ resid, double* __restrict__ J,
               const Basis B, const Phys P) {
    __shared__ double red[kObjThreads];
    const int n2 = n * n;
    double acc = 0.0;
    for (int p = threadIdx.x; p < np; p += kObjThreads) {
        double sx, sy;
        const int cell = probe_cell(xy, p, P, sx, sy);
        const int iy = cell / P.nx;
        const double* uc = u + (size_t)cell * 4 * n2;
        double v = 0.0;
        for (int j = 0; j < n; ++j) {
            const double ly = lagrange(B, n, j, sy);
            const double z = node_height(iy, j, B, P);
            for (int i = 0; i < n; ++i) {
                const int node = j * n + i;
                const double q[4] = {uc[node], uc[n2 + node], uc[2 * n2 + node], uc[3 * n2 + node]};
                v += ly * lagrange(B, n, i, sx) * (theta_of(q, z, P) - P.theta0);
            }
        }
        const double r = v - target[p];
        resid[p] = r;
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kObjThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = red[0];
}

// dJ/du at every node: 2 sum_p r_p l_j(y_p) l_i(x_p) d theta/du over the
// probes in the node's cell, in probe order
__global__ void k_probe_gradient(const double* __restrict__ u, int cells, int n, const double* __restrict__ xy,
                                 const double* __restrict__ resid, int np, double* __restrict__ g,
                                 const Basis B, const Phys P) {
    const int n2 = n * n;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2, j = node / n, i = node - j * n;
    double acc = 0.0;
    for (int p = 0; p < np; ++p) {
        double sx, sy;
        if (probe_cell(xy, p, P, sx, sy) != cell) continue;
        acc += 2.0 * resid[p] * lagrange(B, n, j, sy) * lagrange(B, n, i, sx);
    }
    const double* uc = u + (size_t)cell * 4 * n2;
    double* gc = g + (size_t)cell * 4 * n2;
    if (acc == 0.0) {
        for (int v = 0; v < 4; ++v) gc[v * n2 + node] = 0.0;
        return;
    }
    const double q[4] = {uc[node], uc[n2 + node], uc[2 * n2 + node], uc[3 * n2 + node]};
    const double z = node_height(cell / P.nx, j, B, P);
    double dth[4];
    theta_gradient(q, z, P, theta_of(q, z, P), dth);
    for (int v = 0; v < 4; ++v) gc[v * n2 + node] = acc * dth[v];
}

int check_uniform(const adg_mesh* m, const char* what) {
    if (!m) return fail(ADG_EINVAL, std::string(what) + ": NULL mesh");
    if (m->amr) return fail(ADG_EUNSUPPORTED, std::string(what) + ": uniform meshes only");
    return ADG_OK;
}

}  // namespace
}  // namespace adg

using adg::fail;

extern "C" {

int adg_theta_to_state(adg_mesh* m, const double* theta_p, double* u, void* stream) {
    if (int rc = adg::check_uniform(m, "theta_to_state")) return rc;
    if (!theta_p || !u) return fail(ADG_EINVAL, "theta_to_state: NULL array");
    if (!m->d.gravity) return fail(ADG_EINVAL, "theta_to_state: needs the background atmosphere (gravity)");
    if (int rc = adg::set_device(m)) return rc;
    const int total = m->cells * m->n * m->n;
    adg::k_theta_to_state<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta_p, u, m->cells, m->n, m->B,
                                                                                   m->P);
    ADG_CK(cudaGetLastError(), "theta_to_state launch");
    return ADG_OK;
}

int adg_theta_to_state_adjoint(adg_mesh* m, const double* theta_p, const double* lam_u, double* lam_theta,
                               void* stream) {
    if (int rc = adg::check_uniform(m, "theta_to_state_adjoint")) return rc;
    if (!theta_p || !lam_u || !lam_theta) return fail(ADG_EINVAL, "theta_to_state_adjoint: NULL array");
    if (!m->d.gravity) return fail(ADG_EINVAL, "theta_to_state_adjoint: needs the background atmosphere (gravity)");
    if (int rc = adg::set_device(m)) return rc;
    const int total = m->cells * m->n * m->n;
    adg::k_theta_to_state_adj<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta_p, lam_u, lam_theta,
                                                                                       m->cells, m->n, m->B, m->P);
    ADG_CK(cudaGetLastError(), "theta_to_state_adjoint launch");
    return ADG_OK;
}

int adg_state_to_theta(adg_mesh* m, const double* u, double* theta_p, void* stream) {
    if (int rc = adg::check_uniform(m, "state_to_theta")) return rc;
    if (!u || !theta_p) return fail(ADG_EINVAL, "state_to_theta: NULL array");
    if (int rc = adg::set_device(m)) return rc;
    const int total = m->cells * m->n * m->n;
    adg::k_state_to_theta<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(u, theta_p, m->cells, m->n, m->B,
                                                                                   m->P);
    ADG_CK(cudaGetLastError(), "state_to_theta launch");
    return ADG_OK;
}

int adg_probe_objective(adg_mesh* m, const double* u, int nprobes, const double* probes_xy, const double* target,
                        double* residual, double* J, double* dJ_du, void* stream) {
    if (int rc = adg::check_uniform(m, "probe_objective")) return rc;
    if (!u || !probes_xy || !target || !residual || !J) return fail(ADG_EINVAL, "probe_objective: NULL array");
    if (nprobes < 1) return fail(ADG_EINVAL, "probe_objective: nprobes must be >= 1");
    if (int rc = adg::set_device(m)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    adg::k_probe_values<<<1, adg::kObjThreads, 0, s>>>(u, m->n, probes_xy, target, nprobes, residual, J, m->B,
                                                        m->P);
    ADG_CK(cudaGetLastError(), "probe_objective launch");
    if (dJ_du) {
        const int total = m->cells * m->n * m->n;
        adg::k_probe_gradient<<<(total + 255) / 256, 256, 0, s>>>(u, m->cells, m->n, probes_xy, residual, nprobes,
                                                                  dJ_du, m->B, m->P);
        ADG_CK(cudaGetLastError(), "probe_objective gradient launch");
    }
    return ADG_OK;
}

}  // extern "C"
