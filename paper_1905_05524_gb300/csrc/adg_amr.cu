// Adaptive 3:1 tree mesh: FP64 step on leaves of different levels, TV
// indicator per leaf, and the refine/coarsen transfer (Sec. 3 refinement
// criterion; Sec. 4.2 runs on two refinement levels of a 3:1 tree).
//
// Mesh operations (the paper gives the criterion, not the operations):
//  * refinement: a leaf becomes 3 x 3 children whose nodal values are the
//    parent polynomial at the children's nodes (exact);
//  * coarsening: 9 sibling leaves, all flagged -1, become their parent, whose
//    nodal values are the L2 projection of the children by Gauss-Legendre
//    quadrature on each child (exact, conservative);
//  * 2-level balance: neighbouring leaves differ by at most one level and
//    refinement wins;
//  * hanging faces: the fine side evaluates the coarse trace on its third of
//    the face; the coarse side computes the same three fine numerical fluxes
//    (identical operands and order, so the values are bitwise equal) and
//    receives their L2 restriction onto its face basis -- conservative
//    because the restriction preserves the face integral; the Rusanov
//    penalty uses the fine cell size on both sides;
//  * leaves are ordered by (level, iy, ix).
// All leaves of all levels are advanced by one predictor launch and one
// corrector launch per step.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "adg_convert.cuh"
#include "adg_fp64_body.cuh"
#include "adg_internal.h"
#include "adg_mesh.h"
#include "adg_mixed_body.cuh"
#include "adg_mixed_x2.cuh"
#include "adg_mixed_point.cuh"
#include "adg_physics.cuh"
#include "adg_tv_cell.cuh"

namespace adg {

constexpr int kNbrInts = 5;  // type, id0, id1, id2, sub-face
enum { NB_CONF = 0, NB_COARSE = 1, NB_FINE = 2, NB_WALL = 3 };

// 1D prolongation Pro[a][m][q] = phi_q((a + xi_m)/3) and the face
// restriction weights Rw[a][m][q] = Pro[a][m][q] w_m / (3 w_q).
struct AmrOps {
    double Pro[3][kMaxN][kMaxN];
    double Rw[3][kMaxN][kMaxN];
};

// ------------------------------------------------------------------ host tree
struct AmrTree {
    int nx0 = 0, ny0 = 0, maxl = 0;
    bool per_x = false, per_y = false;
    std::vector<std::array<int, 3>> leaves;  // level, ix, iy
    // leaf index of every (level, ix, iy) cell, one dense grid per level
    // (-1: not a leaf); index() resets only the previous leaves' entries
    std::vector<std::vector<int>> grid;
    std::vector<std::array<int, 3>> indexed;
    // per (level, iy) row: the background tables of upload_tables (they depend
    // on the height only), computed once
    std::unordered_map<long long, std::vector<double>> rows;
    AmrOps ops;

    static long long key(int l, int ix, int iy) { return ((long long)l << 50) | ((long long)ix << 25) | iy; }
    void index() {
        std::sort(leaves.begin(), leaves.end(), [](const std::array<int, 3>& a, const std::array<int, 3>& b) {
            if (a[0] != b[0]) return a[0] < b[0];
            if (a[2] != b[2]) return a[2] < b[2];
            return a[1] < b[1];
        });
        if ((int)grid.size() < maxl + 1) grid.resize(maxl + 1);
        for (const auto& c : indexed) grid[c[0]][(size_t)c[2] * (nx0 * ipow3(c[0])) + c[1]] = -1;
        for (int k = 0; k < (int)leaves.size(); ++k) {
            const auto& c = leaves[k];
            std::vector<int>& g = grid[c[0]];
            const size_t NX = (size_t)nx0 * ipow3(c[0]), NY = (size_t)ny0 * ipow3(c[0]);
            if (g.empty()) g.assign(NX * NY, -1);
            g[(size_t)c[2] * NX + c[1]] = k;
        }
        indexed = leaves;
    }
    int find(int l, int ix, int iy) const {
        if (l < 0 || l >= (int)grid.size() || grid[l].empty()) return -1;
        const int NX = nx0 * ipow3(l), NY = ny0 * ipow3(l);
        if (ix < 0 || ix >= NX || iy < 0 || iy >= NY) return -1;
        return grid[l][(size_t)iy * NX + ix];
    }
    // face 0 E, 1 W, 2 N, 3 S; out[5] = type, id0, id1, id2, sub
    bool neighbour(int k, int f, int out[kNbrInts]) const {
        const int l = leaves[k][0], ix = leaves[k][1], iy = leaves[k][2];
        const int NX = nx0 * ipow3(l), NY = ny0 * ipow3(l);
        int jx = ix + (f == 0 ? 1 : f == 1 ? -1 : 0), jy = iy + (f == 2 ? 1 : f == 3 ? -1 : 0);
        out[1] = out[2] = out[3] = -1;
        out[4] = 0;
        if (jx < 0 || jx >= NX) {
            if (!per_x) { out[0] = NB_WALL; return true; }
            jx = (jx + NX) % NX;
        }
        if (jy < 0 || jy >= NY) {
            if (!per_y) { out[0] = NB_WALL; return true; }
            jy = (jy + NY) % NY;
        }
        int o = find(l, jx, jy);
        if (o >= 0) { out[0] = NB_CONF; out[1] = o; return true; }
        if (l > 0 && (o = find(l - 1, jx / 3, jy / 3)) >= 0) {
            out[0] = NB_COARSE;
            out[1] = o;
            out[4] = f < 2 ? iy % 3 : ix % 3;
            return true;
        }
        out[0] = NB_FINE;
        for (int s = 0; s < 3; ++s) {
            int cx, cy;
            if (f == 0) { cx = 3 * jx; cy = 3 * iy + s; }
            else if (f == 1) { cx = 3 * jx + 2; cy = 3 * iy + s; }
            else if (f == 2) { cx = 3 * ix + s; cy = 3 * jy; }
            else { cx = 3 * ix + s; cy = 3 * jy + 2; }
            out[1 + s] = find(l + 1, cx, cy);
            if (out[1 + s] < 0) return false;  // unbalanced tree
        }
        return true;
    }
    static int ipow3(int l) {
        int r = 1;
        while (l-- > 0) r *= 3;
        return r;
    }
};

static AmrTree* tree_of(adg_mesh* m) { return (AmrTree*)m->tree; }

// Upload geometry, neighbour and background tables of the current leaves.
// The background depends on the height only, so each (level, iy) row's
// values are computed once and cached in the tree.  Row layout (doubles):
// [n][2] node (pbar, rhobar); [4] faces (pbar, rhobar) north, south; for the
// mixed predictor [n][2] node (rhobar, Ebar), [2][2] (rhobar, Ebar) of the
// nodal background extrapolated to the north, south faces, [n][3] node
// (pbar, d rhobar/dz, d Ebar/dz), [2][2] extrapolated (rhobar, (gamma-1)
// (Ebar - rhobar g z_face)).
static int upload_tables(adg_mesh* m) {
    AmrTree* T = tree_of(m);
    const int L = (int)T->leaves.size(), n = m->n;
    const adg_mesh_desc* d = &m->d;
    const bool mixed = d->precision == ADG_PREC_MIXED;
    std::vector<double> geo((size_t)L * 4), bgl((size_t)L * n * 2 + (size_t)L * 4, 0.0);
    std::vector<int> nbr((size_t)L * 4 * kNbrInts);
    std::vector<double> h64(mixed ? (size_t)L * n * 2 + (size_t)L * 4 : 0, 0.0);
    std::vector<float> h32(mixed ? (size_t)L * n * 3 + (size_t)L * 4 : 0, 0.0f);
    const double cp = m->P.cp, g = d->gravity ? d->g : 0.0, gm1 = d->gamma - 1.0;
    auto bgp = [&](double z, double& pb, double& rb) {
        pb = rb = 0.0;
        if (!d->gravity) return;
        const double ex = 1.0 - d->g * z / (cp * d->theta0);
        pb = d->p0 * std::pow(ex, cp / d->R);
        rb = pb / (d->R * d->theta0 * ex);
    };
    const size_t o_face = (size_t)n * 2, o_m64 = o_face + 4, o_ext = o_m64 + (size_t)n * 2, o_m32 = o_ext + 4,
                 o_ext32 = o_m32 + (size_t)n * 3, row_len = o_ext32 + 4;
    auto row_of = [&](int l, int iy, double hy) -> const std::vector<double>& {
        std::vector<double>& r = T->rows[AmrTree::key(l, 0, iy)];
        if (!r.empty()) return r;
        r.assign(row_len, 0.0);
        std::vector<double> rb(n), Eb(n), pb(n);
        for (int j = 0; j < n; ++j) {
            const double z = d->y0 + (iy + m->B.xi[j]) * hy;
            bgp(z, r[(size_t)j * 2], r[(size_t)j * 2 + 1]);
            // the mixed predictor's base at the same node height (its own
            // formula for the height, as the leaf's origin plus xi hy)
            const double zm = (d->y0 + iy * hy) + m->B.xi[j] * hy;
            bgp(zm, pb[j], rb[j]);
            Eb[j] = pb[j] / gm1 + rb[j] * g * zm;
        }
        bgp(d->y0 + (iy + 1) * hy, r[o_face], r[o_face + 1]);  // north face
        bgp(d->y0 + iy * hy, r[o_face + 2], r[o_face + 3]);    // south face
        for (int j = 0; j < n; ++j) {
            double dr = 0.0, dE = 0.0;
            for (int p = 0; p < n; ++p) {
                dr += m->B.D[j][p] * rb[p];
                dE += m->B.D[j][p] * Eb[p];
            }
            r[o_m64 + (size_t)j * 2] = rb[j];
            r[o_m64 + (size_t)j * 2 + 1] = Eb[j];
            r[o_m32 + (size_t)j * 3] = pb[j];
            r[o_m32 + (size_t)j * 3 + 1] = dr / hy;
            r[o_m32 + (size_t)j * 3 + 2] = dE / hy;
        }
        for (int side = 0; side < 2; ++side) {  // 0: north (phi(1)), 1: south (phi(0))
            const double* phi = side == 0 ? m->B.phi1 : m->B.phi0;
            double er = 0.0, eE = 0.0;
            for (int p = 0; p < n; ++p) {
                er += phi[p] * rb[p];
                eE += phi[p] * Eb[p];
            }
            const double zf = (d->y0 + iy * hy) + (side == 0 ? hy : 0.0);
            r[o_ext + side * 2] = er;
            r[o_ext + side * 2 + 1] = eE;
            r[o_ext32 + side * 2] = er;
            r[o_ext32 + side * 2 + 1] = gm1 * (eE - er * g * zf);
        }
        return r;
    };
    double hmin = 1e300;
    for (int k = 0; k < L; ++k) {
        const int l = T->leaves[k][0], ix = T->leaves[k][1], iy = T->leaves[k][2];
        const double hx = d->Lx / (d->nx * AmrTree::ipow3(l)), hy = d->Ly / (d->ny * AmrTree::ipow3(l));
        hmin = std::fmin(hmin, std::fmin(hx, hy));
        geo[k * 4 + 0] = d->x0 + ix * hx;
        geo[k * 4 + 1] = d->y0 + iy * hy;
        geo[k * 4 + 2] = hx;
        geo[k * 4 + 3] = hy;
        const std::vector<double>& r = row_of(l, iy, hy);
        for (int j = 0; j < n; ++j) {
            bgl[((size_t)k * n + j) * 2] = r[(size_t)j * 2];
            bgl[((size_t)k * n + j) * 2 + 1] = r[(size_t)j * 2 + 1];
        }
        double* fb = bgl.data() + (size_t)L * n * 2 + (size_t)k * 4;
        for (int q = 0; q < 4; ++q) fb[q] = r[o_face + q];
        if (mixed) {
            for (int j = 0; j < n; ++j) {
                const size_t rr = (size_t)k * n + j;
                h64[rr * 2] = r[o_m64 + (size_t)j * 2];
                h64[rr * 2 + 1] = r[o_m64 + (size_t)j * 2 + 1];
                for (int q = 0; q < 3; ++q) h32[rr * 3 + q] = (float)r[o_m32 + (size_t)j * 3 + q];
            }
            for (int q = 0; q < 4; ++q) {
                h64[(size_t)L * n * 2 + (size_t)k * 4 + q] = r[o_ext + q];
                h32[(size_t)L * n * 3 + (size_t)k * 4 + q] = (float)r[o_ext32 + q];
            }
        }
        for (int f = 0; f < 4; ++f)
            if (!T->neighbour(k, f, &nbr[((size_t)k * 4 + f) * kNbrInts]))
                return fail(ADG_EINVAL, "adaptive mesh: level difference above one across a face");
    }
    m->hmin = hmin;
    // the tables live in buffers sized for leaf_cap leaves (grow-only, see
    // ensure_capacity); the layouts are those of the current L leaves
    const size_t C = (size_t)m->leaf_cap;
    if (!m->geo) {
        if (cudaMalloc(&m->geo, C * 4 * 8) != cudaSuccess || cudaMalloc(&m->nbr, C * 4 * kNbrInts * 4) != cudaSuccess ||
            cudaMalloc(&m->bgl, (C * n * 2 + C * 4) * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(ADG_ENOMEM, "adaptive mesh: tables");
        }
    }
    ADG_CK(cudaMemcpy(m->geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice), "amr tables");
    ADG_CK(cudaMemcpy(m->nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice), "amr tables");
    ADG_CK(cudaMemcpy(m->bgl, bgl.data(), bgl.size() * 8, cudaMemcpyHostToDevice), "amr tables");
    if (mixed) {
        if (!m->mbl64) {
            if (cudaMalloc(&m->mbl64, (C * n * 2 + C * 4) * 8) != cudaSuccess ||
                cudaMalloc(&m->mblf, (C * n * 3 + C * 4) * 4) != cudaSuccess) {
                cudaGetLastError();
                return fail(ADG_ENOMEM, "adaptive mesh: mixed tables");
            }
        }
        ADG_CK(cudaMemcpy(m->mbl64, h64.data(), h64.size() * 8, cudaMemcpyHostToDevice), "amr mixed tables");
        ADG_CK(cudaMemcpy(m->mblf, h32.data(), h32.size() * 4, cudaMemcpyHostToDevice), "amr mixed tables");
    }
    return ADG_OK;
}

// Grow the per-leaf buffers and tables to hold at least L leaves (with a
// quarter of headroom); they are never shrunk, so the adaptations of a run
// reallocate only while the leaf count reaches new highs (cudaFree
// synchronises the device).  The state m->u keeps its contents; every other
// per-leaf buffer is rewritten before it is read.  Sets *grew.
static int ensure_capacity(adg_mesh* m, int L, bool* grew) {
    *grew = false;
    if (L <= m->leaf_cap) return ADG_OK;
    const int cap = L + L / 4 + 16, n = m->n;
    const size_t C = (size_t)cap, cnt = C * n * n * 4, tr = C * 4 * kTraceComps * n;
    double* keep_u = m->u;
    cudaFree(m->rvol);
    cudaFree(m->trace);
    cudaFree(m->trace_bar);
    cudaFree(m->tv);
    cudaFree(m->part);
    cudaFree(m->u_spare);
    cudaFree(m->dtrans);
    cudaFree(m->geo);
    cudaFree(m->nbr);
    cudaFree(m->bgl);
    cudaFree(m->mbl64);
    cudaFree(m->mblf);
    m->rvol = m->trace = m->trace_bar = m->tv = m->part = m->u_spare = m->geo = m->bgl = m->mbl64 = nullptr;
    m->nbr = m->dtrans = nullptr;
    m->mblf = nullptr;
    m->u = keep_u;
    m->leaf_cap = cap;
    m->tv_prep_cells = -1;
    if (cudaMalloc(&m->rvol, cnt * 8) != cudaSuccess || cudaMalloc(&m->trace, tr * 8) != cudaSuccess ||
        cudaMalloc(&m->tv, C * 8) != cudaSuccess ||
        cudaMalloc(&m->part, 8 * tv_stats_scratch_doubles(m->N, cap)) != cudaSuccess ||
        cudaMalloc(&m->u_spare, cnt * 8) != cudaSuccess || cudaMalloc(&m->dtrans, C * 12 * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "adaptive mesh: buffers");
    }
    *grew = true;
    return ADG_OK;  // the tables are allocated by the next upload_tables
}

int amr_setup(adg_mesh* m) {
    AmrTree* T = new AmrTree();
    T->nx0 = m->d.nx;
    T->ny0 = m->d.ny;
    T->maxl = m->d.max_levels;
    T->per_x = m->d.bc_x == ADG_BC_PERIODIC;
    T->per_y = m->d.bc_y == ADG_BC_PERIODIC;
    for (int iy = 0; iy < T->ny0; ++iy)
        for (int ix = 0; ix < T->nx0; ++ix) T->leaves.push_back({0, ix, iy});
    T->index();
    std::memset(&T->ops, 0, sizeof(T->ops));
    const int n = m->n;
    for (int a = 0; a < 3; ++a)
        for (int mm = 0; mm < n; ++mm) {
            const double x = (a + m->B.xi[mm]) / 3.0;
            for (int q = 0; q < n; ++q) {
                double v = 1.0;
                for (int r = 0; r < n; ++r)
                    if (r != q) v *= (x - m->B.xi[r]) / (m->B.xi[q] - m->B.xi[r]);
                T->ops.Pro[a][mm][q] = v;
                T->ops.Rw[a][mm][q] = v * m->B.w[mm] / (3.0 * m->B.w[q]);
            }
        }
    m->tree = T;
    m->amr = 1;
    // the base mesh's buffers (u, rvol, trace, tv, part) were sized by
    // create_mesh for nx * ny leaves
    m->leaf_cap = (int)T->leaves.size();
    const size_t cnt = (size_t)m->leaf_cap * n * n * 4;
    if (cudaMalloc(&m->u_spare, cnt * 8) != cudaSuccess ||
        cudaMalloc(&m->dtrans, (size_t)m->leaf_cap * 12 * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "adaptive mesh: buffers");
    }
    return upload_tables(m);
}

void amr_free(adg_mesh* m) {
    delete tree_of(m);
    m->tree = nullptr;
    cudaFree(m->lts_ttrace);
    cudaFree(m->lts_acc);
    m->lts_ttrace = m->lts_acc = nullptr;
    m->lts_cap = 0;
    cudaFree(m->geo);
    cudaFree(m->nbr);
    cudaFree(m->bgl);
    cudaFree(m->mbl64);
    cudaFree(m->mblf);
    cudaFree(m->u_spare);
    cudaFree(m->dtrans);
    m->mbl64 = nullptr;
    m->mblf = nullptr;
    m->u_spare = nullptr;
    m->dtrans = nullptr;
}

// per-leaf constants: P with the leaf's cell sizes
__device__ __forceinline__ Phys leaf_phys(const Phys& P0, const double* geo, int cell, int N) {
    Phys P = P0;
    P.hx = geo[cell * 4 + 2];
    P.hy = geo[cell * 4 + 3];
    P.inv_hx = 1.0 / P.hx;
    P.inv_hy = 1.0 / P.hy;
    P.eta_x = (2.0 * N + 1.0) / (P.hx * 1.2533141373155002);  // sqrt(pi/2)
    P.eta_y = (2.0 * N + 1.0) / (P.hy * 1.2533141373155002);
    return P;
}

// ------------------------------------------------------------------ kernels
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_amr(const double* __restrict__ u, double* __restrict__ rvol, double* __restrict__ trace, int cells,
                double dt, const Basis B, const Phys P0, const double* __restrict__ geo,
                const double* __restrict__ bgl) {
    constexpr int n = N + 1, n2 = n * n;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int j = (threadIdx.x - cl * n2) / n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const Phys P = leaf_phys(P0, geo, cell, N);
    predictor_fp64_body<N, CPB>(u, rvol, trace, cell, active, dt, B, P, geo[cell * 4], geo[cell * 4 + 1],
                                bgl[((size_t)cell * n + j) * 2], bgl[((size_t)cell * n + j) * 2 + 1], sm);
}

// Local time stepping: the FP64 predictor on the leaf range [first, end) (one
// level) with dt of that level; REC adds the per-time-node face traces.
template <int N, int CPB, bool REC>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_amr_lts(const double* __restrict__ u, double* __restrict__ rvol, double* __restrict__ trace, int first,
                    int end, double dt, const Basis B, const Phys P0, const double* __restrict__ geo,
                    const double* __restrict__ bgl, double* __restrict__ ttrace) {
    constexpr int n = N + 1, n2 = n * n;
    extern __shared__ double sm[];
    const int cl = threadIdx.x / n2;
    const int j = (threadIdx.x - cl * n2) / n;
    const int cell_raw = first + blockIdx.x * CPB + cl;
    const bool active = cell_raw < end;
    const int cell = active ? cell_raw : end - 1;
    const Phys P = leaf_phys(P0, geo, cell, N);
    predictor_fp64_body<N, CPB, false, REC>(u, rvol, trace, cell, active, dt, B, P, geo[cell * 4], geo[cell * 4 + 1],
                                            bgl[((size_t)cell * n + j) * 2], bgl[((size_t)cell * n + j) * 2 + 1],
                                            sm, 0.0, ttrace);
}

// Mixed-precision predictor of the adaptive mesh: the Picard iteration of
// k_predictor_amr in FP32 on perturbation variables (the split against the
// leaf's nodal background in FP64 at load; gradients plus the FP64-formed
// derivative of the interpolated background), writing the FP64 formats of
// the FP64 predictor -- the volume residual converted, the traces rebuilt as
// an FP64 base plus the FP32 perturbation (x-faces: the nodal background of
// the node's row, which does not vary along x; y-faces: the FP64
// extrapolation of the leaf's nodal background) with the Rusanov speed in
// FP32 -- so the FP64 corrector with its hanging faces runs unchanged.
// Shared memory of the mixed adaptive predictor per leaf: q', F and G as
// float2 pairs of time slices, padded to a bank offset of 16 (mod 32 floats)
// between neighbouring leaves.
template <int N>
struct AmrMixCfg {
    static constexpr int n = N + 1;
    static constexpr int npair = (n + 1) / 2;
    static constexpr int raw = 3 * npair * 4 * n * n * 2;
    static constexpr int stride = raw + ((16 - raw % 32) + 32) % 32;
};

// Per-leaf tables: mb64 [leaves][n][2] (rhobar, Ebar) then [leaves][2 N, S][2]
// extrapolated (rhobar, Ebar); mbf [leaves][n][3] (pbar, d rhobar/dz,
// d Ebar/dz) then [leaves][2 N, S][2] (extrapolated rhobar, (gamma-1)(Ebar -
// rhobar g z_face)).
// Body of the tile of CPB leaves starting at leaf c0; shared by the per-mesh
// kernel and the batched persistent kernels.
template <int N, int CPB>
__device__ __forceinline__ void predictor_amr_mixed_body(const double* __restrict__ u, double* __restrict__ rvol,
                                                         double* __restrict__ trace, int cells, int c0, float dt,
                                                         const BasisF& B, const PhysF& P,
                                                         const double* __restrict__ geo,
                                                         const double* __restrict__ mb64,
                                                         const float* __restrict__ mbf, float* smf) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    constexpr int NPAIR = AmrMixCfg<N>::npair, PS = 4 * n2;  // slice pairs, pair stride (float2)
    float2* Q2 = reinterpret_cast<float2*>(smf + (size_t)cl * AmrMixCfg<N>::stride);  // [h][v][j][i]
    float2* F2 = Q2 + NPAIR * PS;                                                      // [h][v][j][i]
    float2* G2 = F2 + NPAIR * PS;                                                      // [h][v][j][i]
    const double hx = geo[cell * 4 + 2], hy = geo[cell * 4 + 3], yorg = geo[cell * 4 + 1];
    const float inv_hx = (float)(1.0 / hx), inv_hy = (float)(1.0 / hy);
    const float z = (float)(yorg + (double)B.xi[j] * hy);
    const size_t rowj = (size_t)cell * n + j;
    const double rb64 = mb64[rowj * 2], Eb64 = mb64[rowj * 2 + 1];
    const float rb = f64_to_f32(rb64), Eb = f64_to_f32(Eb64);
    const float pb = mbf[rowj * 3], dzr = mbf[rowj * 3 + 1], dzE = mbf[rowj * 3 + 2];

    float up[4];
    {
        const double* uc = u + (size_t)cell * SL;
        up[0] = f64_to_f32(__dsub_rn(uc[node], rb64));
        up[1] = f64_to_f32(uc[n2 + node]);
        up[2] = f64_to_f32(uc[2 * n2 + node]);
        up[3] = f64_to_f32(__dsub_rn(uc[3 * n2 + node], Eb64));
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Q2[v * n2 + node] = make_float2(up[v], up[v]);
    __syncthreads();

    // the uniform mixed predictor's slice-pair scheme (adg_mixed.cu) with this
    // leaf's spacing and background
    float dI[n], dJ[n];
#pragma unroll
    for (int p = 0; p < n; ++p) {
        dI[p] = B.D[i][p] * inv_hx;
        dJ[p] = B.D[j][p] * inv_hy;
    }
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
    // the x-contraction with this node's own value taken from the row load at p = i
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
    auto divergence = [&](int h, int v) { return add2(xdot(F2 + h * PS + v * n2), ydot(G2 + h * PS + v * n2)); };
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
        for (int v = 0; v < 4; ++v) R0[v] = (v == 2 ? f.S2.x : 0.f) - divergence(0, v).x;
#pragma unroll
        for (int g = 0; g < NPAIR; ++g) {
            const int l1 = 2 * g + 1 < n ? 2 * g + 1 : 2 * g;
#pragma unroll
            for (int v = 0; v < 4; ++v)
                store_q_pair(g, v, fmaf(dt, B.Kw1[2 * g] * R0[v], up[v]), fmaf(dt, B.Kw1[l1] * R0[v], up[v]));
        }
        __syncthreads();
    }
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
            for (int h = 0; h < NPAIR; ++h) R2[h] = fma2(bc2(-1.f), divergence(h, v), v == 2 ? S2h[h] : bc2(0.f));
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
    for (int v = 0; v < 4; ++v) Sb[v] = 0.f;
    Sb[2] = Sz;
    __syncthreads();
    float* A = reinterpret_cast<float*>(Q2);  // slots 0..4: qbar', Fbar, Gbar, qxbar, qybar
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        A[0 * SL + v * n2 + node] = qb[v];
        A[1 * SL + v * n2 + node] = Fb[v];
        A[2 * SL + v * n2 + node] = Gb[v];
        A[3 * SL + v * n2 + node] = qxb[v];
        A[4 * SL + v * n2 + node] = qyb[v];
    }
    __syncthreads();
    if (active) {
        double* rc = rvol + (size_t)cell * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int p = 0; p < n; ++p) {
                sx = fmaf(B.Vx[p][i], A[1 * SL + v * n2 + j * n + p], sx);
                sy = fmaf(B.Vx[p][j], A[2 * SL + v * n2 + p * n + i], sy);
            }
            rc[v * n2 + node] = f32_to_f64(sx * inv_hx + sy * inv_hy + Sb[v]);
        }
    }
    const float eta_x = (2.f * N + 1.f) / ((float)hx * 1.2533141f), eta_y = (2.f * N + 1.f) / ((float)hy * 1.2533141f);
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
                const float* S = A + slot * SL + v * n2;
                float s = 0.f;
#pragma unroll
                for (int p = 0; p < n; ++p) s = fmaf(phi[p], xface ? S[m * n + p] : S[p * n + m], s);
                rec[c * 4 + v] = s;
            }
        }
        // FP64 base and FP32 speed base of the face node
        double brho, bE;
        float rbf, pbf, zf;
        if (xface) {
            const size_t rm = (size_t)cell * n + m;
            brho = mb64[rm * 2];
            bE = mb64[rm * 2 + 1];
            rbf = f64_to_f32(brho);
            pbf = mbf[rm * 3];
            zf = (float)(yorg + (double)B.xi[m] * hy);
        } else {
            const size_t side = (size_t)cell * 2 + (f == 2 ? 0 : 1);
            const size_t o64 = (size_t)cells * n * 2 + side * 2, o32 = (size_t)cells * n * 3 + side * 2;
            brho = mb64[o64];
            bE = mb64[o64 + 1];
            rbf = mbf[o32];
            pbf = mbf[o32 + 1];
            zf = (float)(yorg + (f == 2 ? hy : 0.0));
        }
        const float rho = rbf + rec[0];
        const float rinv = __frcp_rn(rho);
        const float pp = P.gm1 * (rec[3] - 0.5f * (rec[1] * rec[1] + rec[2] * rec[2]) * rinv - P.g * zf * rec[0]);
        const float sp = fabsf((xface ? rec[1] : rec[2]) * rinv) + sqrtf(P.gamma * (pbf + pp) * rinv) +
                         2.f * (xface ? eta_x : eta_y) * P.lamv * rinv;
        if (active) {
            double* tr = trace + ((size_t)cell * 4 + f) * kTraceComps * n;
#pragma unroll
            for (int c = 0; c < 16; ++c) tr[c * n + m] = f32_to_f64(rec[c]);
            tr[0 * n + m] = brho + f32_to_f64(rec[0]);
            tr[3 * n + m] = bE + f32_to_f64(rec[3]);
            tr[16 * n + m] = f32_to_f64(sp);
        }
    }
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_predictor_amr_mixed(const double* __restrict__ u, double* __restrict__ rvol, double* __restrict__ trace, int cells,
                      float dt, const BasisF B, const PhysF P, const double* __restrict__ geo,
                      const double* __restrict__ mb64, const float* __restrict__ mbf) {
    extern __shared__ float smf[];
    predictor_amr_mixed_body<N, CPB>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P, geo, mb64, mbf, smf);
}

// face data (q-bar and normal flux) of record `rec` of a coarse face evaluated
// on its third `s` at fine node m
__device__ __forceinline__ void prolong_rec(const double* rec, int n, const AmrOps& O, int s, int m, double q[4],
                                            double f[4]) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        double a = 0.0, b = 0.0;
        for (int p = 0; p < n; ++p) {
            a += O.Pro[s][m][p] * rec[v * n + p];
            b += O.Pro[s][m][p] * rec[(4 + v) * n + p];
        }
        q[v] = a;
        f[v] = b;
    }
}

// Local-time-stepping arguments of a corrector launch on one level: W, the
// weights of the time average over the part of a coarser neighbour's step
// that this level's step covers (third kstep); ttrace, the per-time-node
// traces of the coarser level; acc[leaf][face][third][v][n], per spatial
// third of a coarse face, the time average of the fine numerical fluxes of
// the coarse leaf's sub-steps (the fine leaves add theirs; the coarse leaf
// reads them instead of computing fine fluxes).
struct LtsArgs {
    double W[kMaxN];
    const double* ttrace;
    double* acc;
    int total;  // leaves of the mesh (the background table's face part follows all leaves' node part)
};

template <int N, int CPB, bool LTS = false>
__device__ __forceinline__ void corrector_amr_body(double* __restrict__ u, const double* __restrict__ rvol,
                                                   const double* __restrict__ trace, int cells, int c0, double dt,
                                                   const Basis& B, const Phys& P0, const AmrOps& O,
                                                   const double* __restrict__ geo, const int* __restrict__ nbr,
                                                   const double* __restrict__ bgl, const LtsArgs* lts = nullptr) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2, TR = kTraceComps * n;
    __shared__ double Fsub[CPB][4][3][4][n];
    __shared__ double Fst[CPB][4][4][n];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = c0 + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const Phys P = leaf_phys(P0, geo, cell, N);
    const double yorg = geo[cell * 4 + 1];

    for (int idx = node; idx < 4 * 3 * n; idx += n2) {
        const int f = idx / (3 * n), rem = idx - f * 3 * n, s = rem / n, m = rem - s * n;
        const int* nb = nbr + ((size_t)cell * 4 + f) * kNbrInts;
        const int type = nb[0];
        if (type != NB_FINE && s > 0) continue;
        const bool xface = f < 2;
        const int of = f ^ 1;  // opposite face: E<->W, N<->S
        const bool own_minus = (f == 0 || f == 2);
        const double* own = trace + ((size_t)cell * 4 + f) * TR;
        double qo[4], fo[4], so;
        double qn[4], fn[4], sn;
        if (LTS && type == NB_FINE) {
            // coarse side under local time stepping: the fine leaves' fluxes, averaged over their sub-steps
            const double* a = lts->acc + ((((size_t)cell * 4 + f) * 3 + s) * 4) * n;
#pragma unroll
            for (int v = 0; v < 4; ++v) Fsub[cl][f][s][v][m] = a[v * n + m];
            continue;
        }
        if (type == NB_FINE) {
            // coarse side of a hanging face: own trace on third s vs fine neighbour s
            const int o = nb[1 + s];
            const Phys Pf = leaf_phys(P0, geo, o, N);
            // heights of the fine neighbour's face nodes (the same expression it uses itself)
            const double z = geo[o * 4 + 1] + (xface ? B.xi[m] * Pf.hy : (f == 2 ? 0.0 : Pf.hy));
            prolong_rec(own, n, O, s, m, qo, fo);
            so = wave_speed(qo, z, xface, Pf);
            const double* ot = trace + ((size_t)o * 4 + of) * TR;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qn[v] = ot[v * n + m];
                fn[v] = ot[(4 + v) * n + m];
            }
            sn = ot[16 * n + m];
        } else {
            double rec[kTraceComps];
#pragma unroll
            for (int c = 0; c < kTraceComps; ++c) rec[c] = own[c * n + m];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                qo[v] = rec[v];
                fo[v] = rec[4 + v];
            }
            so = rec[16];
            const double z = xface ? yorg + B.xi[m] * P.hy : yorg + (f == 2 ? P.hy : 0.0);
            if (type == NB_WALL) {
                double pb, rb;
                if (xface) {
                    pb = bgl[((size_t)cell * n + m) * 2];
                    rb = bgl[((size_t)cell * n + m) * 2 + 1];
                } else {
                    const double* fb = bgl + (size_t)(LTS ? lts->total : cells) * n * 2 + (size_t)cell * 4 +
                                       (f == 2 ? 0 : 2);
                    pb = fb[0];
                    rb = fb[1];
                }
                const double nx = f == 0 ? 1.0 : f == 1 ? -1.0 : 0.0;
                const double ny = f == 2 ? 1.0 : f == 3 ? -1.0 : 0.0;
                const double mn = rec[1] * nx + rec[2] * ny;
                qn[1] = rec[1] - 2.0 * mn * nx;
                qn[2] = rec[2] - 2.0 * mn * ny;
                qn[0] = P.gravity ? rb : rec[0];
                qn[3] = P.gravity ? pb / P.gm1 + rb * P.g * z : rec[3];
                Flux4 fl;
                ns_flux(qn, rec + 8, rec + 12, z, pb, rb, P, fl, true, 0.0, P.gravity ? -P.g / P.cp : 0.0);
#pragma unroll
                for (int v = 0; v < 4; ++v) fn[v] = xface ? fl.F[v] : fl.G[v];
                sn = wave_speed(qn, z, xface, P);
            } else if (type == NB_CONF) {
                const double* ot = trace + ((size_t)nb[1] * 4 + of) * TR;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    qn[v] = ot[v * n + m];
                    fn[v] = ot[(4 + v) * n + m];
                }
                sn = ot[16 * n + m];
            } else if (LTS) {  // NB_COARSE under local time stepping: the coarse trace averaged over this step
                double rec[8 * n];
                for (int c = 0; c < 8 * n; ++c) rec[c] = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double* tk = lts->ttrace + ((((size_t)nb[1] * n + k) * 4 + of) * 16) * n;
                    for (int c = 0; c < 8 * n; ++c) rec[c] += lts->W[k] * tk[c];
                }
                prolong_rec(rec, n, O, nb[4], m, qn, fn);
                sn = wave_speed(qn, z, xface, P);
            } else {  // NB_COARSE: the coarse trace on this cell's third of the face
                const double* ot = trace + ((size_t)nb[1] * 4 + of) * TR;
                prolong_rec(ot, n, O, nb[4], m, qn, fn);
                sn = wave_speed(qn, z, xface, P);
            }
        }
        double out[4];
        if (own_minus) rusanov(qo, fo, so, qn, fn, sn, out);
        else rusanov(qn, fn, sn, qo, fo, so, out);
        if (LTS && type == NB_COARSE && active) {  // this sub-step's share of the coarse leaf's face flux
            double* a = lts->acc + ((((size_t)nb[1] * 4 + of) * 3 + nb[4]) * 4) * n;
#pragma unroll
            for (int v = 0; v < 4; ++v) a[v * n + m] += out[v] * (1.0 / 3.0);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) Fsub[cl][f][s][v][m] = out[v];
    }
    __syncthreads();
    for (int idx = node; idx < 4 * n; idx += n2) {
        const int f = idx / n, q = idx - f * n;
        const bool fine = nbr[((size_t)cell * 4 + f) * kNbrInts] == NB_FINE;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double a;
            if (fine) {
                a = 0.0;
                for (int s = 0; s < 3; ++s)
                    for (int mm = 0; mm < n; ++mm) a += O.Rw[s][mm][q] * Fsub[cl][f][s][v][mm];
            } else {
                a = Fsub[cl][f][0][v][q];
            }
            Fst[cl][f][v][q] = a;
        }
    }
    __syncthreads();
    if (!active) return;
    double* uc = u + (size_t)cell * SL;
    const double* rc = rvol + (size_t)cell * SL;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double face = (B.lift1[i] * Fst[cl][0][v][j] - B.lift0[i] * Fst[cl][1][v][j]) * P.inv_hx +
                            (B.lift1[j] * Fst[cl][2][v][i] - B.lift0[j] * Fst[cl][3][v][i]) * P.inv_hy;
        uc[v * n2 + node] += dt * (rc[v * n2 + node] - face);
    }
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_amr(double* __restrict__ u, const double* __restrict__ rvol, const double* __restrict__ trace,
                int cells, double dt, const Basis B, const Phys P0, const AmrOps O, const double* __restrict__ geo,
                const int* __restrict__ nbr, const double* __restrict__ bgl) {
    corrector_amr_body<N, CPB>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P0, O, geo, nbr, bgl);
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_amr_lts(double* __restrict__ u, const double* __restrict__ rvol, const double* __restrict__ trace,
                    int first, int end, double dt, const Basis B, const Phys P0, const AmrOps O,
                    const double* __restrict__ geo, const int* __restrict__ nbr, const double* __restrict__ bgl,
                    const LtsArgs L) {
    corrector_amr_body<N, CPB, true>(u, rvol, trace, end, first + blockIdx.x * CPB, dt, B, P0, O, geo, nbr, bgl, &L);
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_tv_cells_amr(const double* __restrict__ u, double* __restrict__ tv, double* __restrict__ part, int cells,
               int var, const Basis B, const Phys P0, const double* __restrict__ geo) {
    static_assert(CPB == tv_cpb(N), "the TV statistics combine blocks of tv_cpb(N) cells");
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    __shared__ double fs[CPB][n2];
    __shared__ double red[CPB][n2];
    const int cl = threadIdx.x / n2;
    const int node = threadIdx.x - cl * n2;
    const int j = node / n, i = node - j * n;
    const int cell_raw = blockIdx.x * CPB + cl;
    const bool active = cell_raw < cells;
    const int cell = active ? cell_raw : cells - 1;
    const Phys P = leaf_phys(P0, geo, cell, N);
    const double* uc = u + (size_t)cell * SL;
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = uc[v * n2 + node];
    const double z = geo[cell * 4 + 1] + B.xi[j] * P.hy;
    const double f = var == ADG_TV_THETA ? theta_of(q, z, P) : q[0];
    const double r = tv_cell<N, double>(f, 0.0, node, i, j, B, P.inv_hx, P.inv_hy, fs[cl], red[cl], active,
                                        tv + cell);
    tv_block_triple<CPB>(r, node == 0, cl, min(CPB, cells - (int)blockIdx.x * CPB), part);
}

template <int N>
__global__ void k_init_amr(double* __restrict__ u, int cells, int kind, double A, double a, double xc, double zc,
                           const Basis B, const Phys P, const double* __restrict__ geo) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= cells * n2) return;
    const int cell = gid / n2, node = gid - cell * n2;
    const int j = node / n, i = node - j * n;
    const double x = geo[cell * 4] + B.xi[i] * geo[cell * 4 + 2];
    const double z = geo[cell * 4 + 1] + B.xi[j] * geo[cell * 4 + 3];
    double q[4];
    if (kind == ADG_SCEN_STEADY) {
        const double k = 2.0 * 3.14159265358979323846 / P.sL;
        const double rho = 1.0 + P.sa * sin(k * (x + z));
        q[0] = rho;
        q[1] = rho * P.sU;
        q[2] = rho * P.sU;
        q[3] = P.sp / P.gm1 + 0.5 * rho * (2.0 * P.sU * P.sU);
    } else {
        double th = 0.0;
        if (kind == ADG_SCEN_COSINE) {
            const double r = sqrt((x - xc) * (x - xc) + (z - zc) * (z - zc));
            th = r <= a ? 0.5 * A * (1.0 + cos(3.14159265358979323846 * r / a)) : 0.0;
        } else if (kind == ADG_SCEN_TWO_BUBBLES) {
            const double r1 = sqrt((x - 500.0) * (x - 500.0) + (z - 300.0) * (z - 300.0));
            const double r2 = sqrt((x - 560.0) * (x - 560.0) + (z - 640.0) * (z - 640.0));
            th = (r1 <= 150.0 ? 0.5 : 0.5 * exp(-((r1 - 150.0) * (r1 - 150.0)) / 2500.0)) +
                 (r2 <= 0.0 ? -0.15 : -0.15 * exp(-(r2 * r2) / 2500.0));
        }
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

template <int N>
__global__ void k_max_speed_amr(const double* __restrict__ u, double* __restrict__ partial, int cells,
                                const Basis B, const Phys P, const double* __restrict__ geo, double eta) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    __shared__ double red[256];
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (gid < cells * n2) {
        const int cell = gid / n2, node = gid - cell * n2;
        const int j = node / n;
        const double z = geo[cell * 4 + 1] + B.xi[j] * geo[cell * 4 + 3];
        const double* uc = u + (size_t)cell * SL;
        const double rho = uc[node], mx = uc[n2 + node], my = uc[2 * n2 + node], E = uc[3 * n2 + node];
        const double p = P.gm1 * (E - 0.5 * (mx * mx + my * my) / rho - rho * (P.gravity ? P.g * z : 0.0));
        s = sqrt(mx * mx + my * my) / rho + sqrt(P.gamma * p / rho) + 2.0 * eta * P.lamv / rho;
        if (!(s == s)) s = 1e300;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// transfer of the state to a new leaf set: per new leaf, copy (t = 0),
// prolongation from a parent at child position (a, b) (t = 1) or restriction
// of 9 children ordered b * 3 + a (t = 2).  trans[leaf] = t, a, b, src[9].
template <int N>
__global__ void k_amr_transfer(const double* __restrict__ uold, double* __restrict__ unew, int leaves,
                               const int* __restrict__ trans, const Basis B, const AmrOps O) {
    constexpr int n = N + 1, n2 = n * n, SL = 4 * n2;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= leaves * n2) return;
    const int leaf = gid / n2, node = gid - leaf * n2;
    const int j = node / n, i = node - j * n;
    const int* t = trans + (size_t)leaf * 12;
    double* out = unew + (size_t)leaf * SL;
    if (t[0] == 0) {
        const double* src = uold + (size_t)t[3] * SL;
#pragma unroll
        for (int v = 0; v < 4; ++v) out[v * n2 + node] = src[v * n2 + node];
    } else if (t[0] == 1) {
        const double* src = uold + (size_t)t[3] * SL;
        const int a = t[1], b = t[2];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r) {
                double row = 0.0;
                for (int q = 0; q < n; ++q) row += O.Pro[a][i][q] * src[v * n2 + r * n + q];
                acc += O.Pro[b][j][r] * row;
            }
            out[v * n2 + node] = acc;
        }
    } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    const double* src = uold + (size_t)t[3 + b * 3 + a] * SL;
                    for (int l = 0; l < n; ++l)
                        for (int mm = 0; mm < n; ++mm)
                            acc += O.Pro[b][l][j] * O.Pro[a][mm][i] * B.w[l] * B.w[mm] * src[v * n2 + l * n + mm];
                }
            out[v * n2 + node] = acc / (9.0 * B.w[j] * B.w[i]);
        }
    }
}

// ------------------------------------------------------------------ launchers
template <int N>
struct AmrCfg {
    static constexpr int n = N + 1;
    static constexpr int cpb = tv_cpb(N);
    static constexpr int threads = cpb * n * n;
    static constexpr size_t smem_pred = (size_t)cpb * 3 * n * 4 * n * n * sizeof(double);
};

#define AMR_DISPATCH(FN, ...)                     \
    switch (m->N) {                               \
        case 1: return FN<1>(__VA_ARGS__);        \
        case 2: return FN<2>(__VA_ARGS__);        \
        case 3: return FN<3>(__VA_ARGS__);        \
        case 4: return FN<4>(__VA_ARGS__);        \
        case 5: return FN<5>(__VA_ARGS__);        \
        case 6: return FN<6>(__VA_ARGS__);        \
        case 7: return FN<7>(__VA_ARGS__);        \
    }                                             \
    return fail(ADG_EINVAL, "bad degree");

// Leaves per block of the per-mesh mixed adaptive predictor (the TV
// statistics of adaptive meshes come from their own kernel, so this need not
// be tv_cpb).  Measured at N = 5 on the two-bubble tree (1065 leaves, under
// half a wave): 4 leaves 2.61e9, 2 leaves 2.60e9, 1 leaf 2.43e9 DOF-updates/s.
template <int N>
constexpr int amr_mixed_cpb() {
    return AmrCfg<N>::cpb;
}

template <int N>
static int pred_n(adg_mesh* m, double dt, cudaStream_t s) {
    using C = AmrCfg<N>;
    if (m->d.precision == ADG_PREC_MIXED) {
        constexpr int CM = amr_mixed_cpb<N>();
        auto km = k_predictor_amr_mixed<N, CM>;
        const size_t smem = (size_t)CM * AmrMixCfg<N>::stride * sizeof(float);
        ADG_CK(cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "amr pred mixed");
        km<<<(m->cells + CM - 1) / CM, CM * (N + 1) * (N + 1), smem, s>>>(m->u, m->rvol, m->trace, m->cells,
                                                                          (float)dt, m->Bf, m->Pf, m->geo, m->mbl64,
                                                                          m->mblf);
        ADG_CK(cudaGetLastError(), "amr mixed predictor launch");
        return ADG_OK;
    }
    auto kern = k_predictor_amr<N, C::cpb>;
    ADG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_pred), "amr pred");
    kern<<<(m->cells + C::cpb - 1) / C::cpb, C::threads, C::smem_pred, s>>>(m->u, m->rvol, m->trace, m->cells, dt,
                                                                             m->B, m->P, m->geo, m->bgl);
    ADG_CK(cudaGetLastError(), "amr predictor launch");
    return ADG_OK;
}
int amr_predictor(adg_mesh* m, double dt, void* stream) { AMR_DISPATCH(pred_n, m, dt, (cudaStream_t)stream) }

template <int N>
static int corr_n(adg_mesh* m, double dt, cudaStream_t s) {
    using C = AmrCfg<N>;
    k_corrector_amr<N, C::cpb><<<(m->cells + C::cpb - 1) / C::cpb, C::threads, 0, s>>>(
        m->u, m->rvol, m->trace, m->cells, dt, m->B, m->P, tree_of(m)->ops, m->geo, m->nbr, m->bgl);
    ADG_CK(cudaGetLastError(), "amr corrector launch");
    return ADG_OK;
}
int amr_corrector(adg_mesh* m, double dt, void* stream) { AMR_DISPATCH(corr_n, m, dt, (cudaStream_t)stream) }

template <int N>
static int tv_n(adg_mesh* m, int var, double* tv, double* part, cudaStream_t s) {
    using C = AmrCfg<N>;
    k_tv_cells_amr<N, C::cpb><<<(m->cells + C::cpb - 1) / C::cpb, C::threads, 0, s>>>(m->u, tv, part, m->cells,
                                                                                        var, m->B, m->P, m->geo);
    ADG_CK(cudaGetLastError(), "amr tv launch");
    return ADG_OK;
}
int amr_tv_cells(adg_mesh* m, int var, double* tv, double* part, void* stream) {
    AMR_DISPATCH(tv_n, m, var, tv, part, (cudaStream_t)stream)
}

template <int N>
static int init_amr_n(adg_mesh* m, const adg_scenario* sc, cudaStream_t s) {
    const int total = m->cells * (N + 1) * (N + 1);
    k_init_amr<N><<<(total + 255) / 256, 256, 0, s>>>(m->u, m->cells, sc->kind, sc->A, sc->a, sc->xc, sc->zc, m->B,
                                                      m->P, m->geo);
    ADG_CK(cudaGetLastError(), "amr init launch");
    return ADG_OK;
}
int amr_init_scenario(adg_mesh* m, const adg_scenario* sc, void* stream) {
    AMR_DISPATCH(init_amr_n, m, sc, (cudaStream_t)stream)
}

template <int N>
static int speed_amr_n(adg_mesh* m, double* lam, cudaStream_t s) {
    const int total = m->cells * (N + 1) * (N + 1);
    const int blocks = (total + 255) / 256;
    double* part = nullptr;
    if (cudaMalloc(&part, (size_t)blocks * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "amr stable_dt");
    }
    const double eta = (2.0 * N + 1.0) / (m->hmin * 1.2533141373155002);
    k_max_speed_amr<N><<<blocks, 256, 0, s>>>(m->u, part, m->cells, m->B, m->P, m->geo, eta);
    std::vector<double> h(blocks);
    cudaError_t e = cudaMemcpyAsync(h.data(), part, (size_t)blocks * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    if (e != cudaSuccess) return cuda_fail(e, "amr stable_dt");
    double mx = 0.0;
    for (double v : h) mx = std::fmax(mx, v);
    *lam = mx;
    return ADG_OK;
}
int amr_max_speed(adg_mesh* m, double* lam, void* stream) { AMR_DISPATCH(speed_amr_n, m, lam, (cudaStream_t)stream) }

// ------------------------------------------------------------ local time stepping
// One cycle (reading L1): level l steps with dt 3^(L-l); a level's step is its
// predictor (with per-time-node traces when a finer level exists), three
// steps of the next finer level, then its corrector.  Leaves are ordered by
// level, so a level is a contiguous range of leaves.
struct LtsRun {
    adg_mesh* m;
    cudaStream_t s;
    int L;
    std::vector<int> off;  // off[l] .. off[l + 1]: leaves of level l
    double dt;             // step of the finest level
    double W[3][kMaxN];    // time-average weights of the thirds of a step
};

template <int N>
static int lts_level_n(LtsRun& R, int l, double t, int kstep) {
    using C = AmrCfg<N>;
    adg_mesh* m = R.m;
    const int first = R.off[l], end = R.off[l + 1];
    const double dtl = R.dt * std::pow(3.0, R.L - l);
    const bool finer = l < R.L;
    (void)t;
    if (end > first) {
        const int blocks = (end - first + C::cpb - 1) / C::cpb;
        if (finer) {
            auto k = k_predictor_amr_lts<N, C::cpb, true>;
            ADG_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_pred), "lts pred");
            k<<<blocks, C::threads, C::smem_pred, R.s>>>(m->u, m->rvol, m->trace, first, end, dtl, m->B, m->P, m->geo,
                                                          m->bgl, m->lts_ttrace);
        } else {
            auto k = k_predictor_amr_lts<N, C::cpb, false>;
            ADG_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_pred), "lts pred");
            k<<<blocks, C::threads, C::smem_pred, R.s>>>(m->u, m->rvol, m->trace, first, end, dtl, m->B, m->P, m->geo,
                                                          m->bgl, nullptr);
        }
        ADG_CK(cudaGetLastError(), "lts predictor launch");
    }
    if (finer) {
        const size_t per_leaf = (size_t)4 * 3 * 4 * m->n;
        if (end > first)
            ADG_CK(cudaMemsetAsync(m->lts_acc + (size_t)first * per_leaf, 0, (size_t)(end - first) * per_leaf * 8, R.s),
                   "lts: clear flux sums");
        for (int ks = 0; ks < 3; ++ks)
            if (int rc = lts_level_n<N>(R, l + 1, t + ks * dtl / 3.0, ks)) return rc;
    }
    if (end > first) {
        LtsArgs A;
        std::memset(&A, 0, sizeof(A));
        for (int k = 0; k < m->n; ++k) A.W[k] = R.W[kstep][k];
        A.ttrace = m->lts_ttrace;
        A.acc = m->lts_acc;
        A.total = m->cells;
        const int blocks = (end - first + C::cpb - 1) / C::cpb;
        k_corrector_amr_lts<N, C::cpb><<<blocks, C::threads, 0, R.s>>>(m->u, m->rvol, m->trace, first, end, dtl, m->B,
                                                                        m->P, tree_of(m)->ops, m->geo, m->nbr, m->bgl, A);
        ADG_CK(cudaGetLastError(), "lts corrector launch");
    }
    return ADG_OK;
}

template <int N>
static int lts_cycle_n(LtsRun& R, int l0, double t) {
    if constexpr (N < 2) {
        (void)R;
        (void)l0;
        (void)t;
        return fail(ADG_EUNSUPPORTED, "step_lts: degree >= 2");
    } else {
        return lts_level_n<N>(R, l0, t, 0);
    }
}

int amr_step_lts(adg_mesh* m, double dt, double* cycle, void* stream) {
    AmrTree* T = tree_of(m);
    LtsRun R;
    R.m = m;
    R.s = (cudaStream_t)stream;
    R.dt = dt;
    int l0 = 1 << 30, L = 0;
    for (const auto& c : T->leaves) {
        l0 = std::min(l0, c[0]);
        L = std::max(L, c[0]);
    }
    R.L = L;
    R.off.assign(L + 2, 0);
    for (const auto& c : T->leaves) R.off[c[0] + 1]++;
    for (int l = 0; l <= L; ++l) R.off[l + 1] += R.off[l];
    // W[s][k] = sum_q w_q phi_k((s + xi_q)/3): the average over the third s of the step
    const int n = m->n;
    for (int s3 = 0; s3 < 3; ++s3)
        for (int k = 0; k < n; ++k) {
            double a = 0.0;
            for (int q = 0; q < n; ++q) {
                const double x = (s3 + m->B.xi[q]) / 3.0;
                double phi = 1.0;
                for (int r = 0; r < n; ++r)
                    if (r != k) phi *= (x - m->B.xi[r]) / (m->B.xi[k] - m->B.xi[r]);
                a += m->B.w[q] * phi;
            }
            R.W[s3][k] = a;
        }
    // per-time-node traces and flux sums, grow-only with the leaf capacity
    if (m->lts_cap < m->leaf_cap) {
        cudaFree(m->lts_ttrace);
        cudaFree(m->lts_acc);
        m->lts_ttrace = m->lts_acc = nullptr;
        const size_t C = (size_t)m->leaf_cap;
        if (cudaMalloc(&m->lts_ttrace, C * n * 4 * 16 * n * 8) != cudaSuccess ||
            cudaMalloc(&m->lts_acc, C * 4 * 3 * 4 * n * 8) != cudaSuccess) {
            cudaGetLastError();
            m->lts_cap = 0;
            return fail(ADG_ENOMEM, "step_lts: buffers");
        }
        m->lts_cap = m->leaf_cap;
    }
    if (cycle) *cycle = dt * std::pow(3.0, L - l0);
    switch (m->N) {
        case 1: return lts_cycle_n<1>(R, l0, m->t);
        case 2: return lts_cycle_n<2>(R, l0, m->t);
        case 3: return lts_cycle_n<3>(R, l0, m->t);
        case 4: return lts_cycle_n<4>(R, l0, m->t);
        case 5: return lts_cycle_n<5>(R, l0, m->t);
        case 6: return lts_cycle_n<6>(R, l0, m->t);
        case 7: return lts_cycle_n<7>(R, l0, m->t);
    }
    return fail(ADG_EINVAL, "bad degree");
}

template <int N>
static int transfer_n(adg_mesh* m, const double* uold, double* unew, int leaves, const int* trans, cudaStream_t s) {
    const int total = leaves * (N + 1) * (N + 1);
    k_amr_transfer<N><<<(total + 127) / 128, 128, 0, s>>>(uold, unew, leaves, trans, m->B, tree_of(m)->ops);
    ADG_CK(cudaGetLastError(), "amr transfer launch");
    return ADG_OK;
}
static int amr_transfer(adg_mesh* m, const double* uold, double* unew, int leaves, const int* trans,
                        cudaStream_t s) {
    AMR_DISPATCH(transfer_n, m, uold, unew, leaves, trans, s)
}


// ------------------------------------------------------------------ batches
// Batched persistent kernels: a fixed grid walks a list of tiles of many
// independent meshes -- uniform instances (tile.inst >= 0, the mixed
// predictor and corrector bodies of adg_mixed_body.cuh) and adaptive ones
// (tile.inst < 0, the leaves of every level: the mixed leaf predictor and the
// FP64 corrector with its hanging faces).  Tile t goes to block t mod grid,
// so the schedule is static and the results do not depend on timing.  Both
// kinds run CPB cells (leaves) per block with one thread per node.
template <int N, int CPB>
struct BatchSmem {
    static constexpr size_t uni = MixCfg<N, CPB>::smem_pred;
    static constexpr size_t amr = (size_t)CPB * AmrMixCfg<N>::stride * sizeof(float);
    static constexpr size_t bytes = uni > amr ? uni : amr;
};

template <int N, int CPB, bool AMR>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1), (AMR ? 1 : MixCfg<N, CPB>::minb))
k_predictor_batch(const MixedInst* __restrict__ insts, const AmrInst* __restrict__ ainsts,
                  const BatchTile* __restrict__ tiles, int ntiles, const BasisF B) {
    extern __shared__ float smf[];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (!AMR || tl.inst >= 0) {
            const MixedInst& I = insts[tl.inst];
            const PhysF P = I.P;
            const MixedBg bg = I.bg;
            predictor_mixed_body<N, CPB>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dtf, B, P, bg, smf);
        } else {
            const AmrInst& I = ainsts[-tl.inst - 1];
            const PhysF P = I.Pf;
            predictor_amr_mixed_body<N, CPB>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dtf, B, P, I.geo, I.mb64,
                                             I.mbf, smf);
        }
        __syncthreads();
    }
}

template <int N, int CPB, bool AMR>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_batch(const MixedInst* __restrict__ insts, const AmrInst* __restrict__ ainsts,
                  const BatchTile* __restrict__ tiles, int ntiles, const BasisF Bf, const Basis B, const AmrOps O) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (!AMR || tl.inst >= 0) {
            const MixedInst& I = insts[tl.inst];
            const PhysF P = I.P;
            const MixedBg bg = I.bg;
            corrector_mixed_body<N, CPB>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dt, Bf, P, bg);
        } else {
            const AmrInst& I = ainsts[-tl.inst - 1];
            const Phys P = I.P;
            corrector_amr_body<N, CPB>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dt, B, P, O, I.geo, I.nbr, I.bgl);
        }
        __syncthreads();
    }
}

// Node-pair predictor over the tiles of uniform instances (candidate 3 of a
// batch without adaptive instances at N = 3, 5): the per-mesh node-pair body,
// two nodes per thread, MixCfg2's cells per tile.
template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1) / 2, (MixCfg2<N, CPB>::minb))
k_predictor_batch_x2(const MixedInst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                     const BasisF B) {
    extern __shared__ float smf[];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        const MixedInst& I = insts[tl.inst];
        const PhysF P = I.P;
        const MixedBg bg = I.bg;
        predictor_mixed_body_x2<N, CPB>(I.u, I.rvol, I.trace, I.cells, tl.c0, I.dtf, B, P, bg, smf);
        __syncthreads();
    }
}

template <int N>
static int batch_x2(const MixedInst* insts, const BatchTile* tiles, int ntiles, const BasisF& Bf, int* cpb_out,
                    int* blocks_io, cudaStream_t s) {
    using C = MixCfg2<N>;
    auto kern = k_predictor_batch_x2<N, C::cpb>;
    if (cpb_out) *cpb_out = C::cpb;
    if (!tiles) {  // query: set the smem limit and size the persistent grid (not during capture)
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_pred);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::threads, C::smem_pred);
        if (e != cudaSuccess) return (int)e;
        if (blocks_io) *blocks_io = per_sm > 0 ? per_sm * sms : sms;
        return 0;
    }
    kern<<<*blocks_io, C::threads, C::smem_pred, s>>>(insts, tiles, ntiles, Bf);
    return (int)cudaGetLastError();
}

// Tile-size candidates per degree: half, default and double the default cells
// per block (kept within 1024 threads and the shared-memory limit).
template <int N, int K>
struct BatchCand {
    static constexpr int base = MixCfg<N>::cpb_default;
    static constexpr int raw = K == 0 ? base / 2 : K == 1 ? base : base * 2;
    static constexpr int cpb = raw < 1 ? 1 : ((raw * (N + 1) * (N + 1) > 1024) ? base : raw);
};

template <int N, int K, bool AMR>
static int batch_nka(int phase, const MixedInst* insts, const AmrInst* ainsts, const BatchTile* tiles, int ntiles,
                     const BasisF& Bf, const Basis& B, const AmrOps* O, int* cpb_out, int* blocks_io,
                     cudaStream_t s) {
    constexpr int CPB = BatchCand<N, K>::cpb;
    constexpr int threads = CPB * (N + 1) * (N + 1);
    constexpr size_t smem = AMR ? BatchSmem<N, CPB>::bytes : MixCfg<N, CPB>::smem_pred;
    if (cpb_out) *cpb_out = CPB;
    if (!tiles) {  // query: set the smem limit and size the persistent grid (not during capture)
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e;
        if (phase == 0) {
            e = cudaFuncSetAttribute(k_predictor_batch<N, CPB, AMR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_predictor_batch<N, CPB, AMR>, threads,
                                                                  smem);
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_corrector_batch<N, CPB, AMR>, threads, 0);
        }
        if (e != cudaSuccess) return (int)e;
        if (blocks_io) *blocks_io = per_sm > 0 ? per_sm * sms : sms;
        return 0;
    }
    const int blocks = *blocks_io;
    if (phase == 0) {
        k_predictor_batch<N, CPB, AMR><<<blocks, threads, smem, s>>>(insts, ainsts, tiles, ntiles, Bf);
    } else {
        AmrOps none;
        if (!O) std::memset(&none, 0, sizeof(none));
        k_corrector_batch<N, CPB, AMR><<<blocks, threads, 0, s>>>(insts, ainsts, tiles, ntiles, Bf, B, O ? *O : none);
    }
    return (int)cudaGetLastError();
}

template <int N>
static int batch_n(int cand, int phase, const MixedInst* insts, const AmrInst* ainsts, const BatchTile* tiles,
                   int ntiles, const BasisF& Bf, const Basis& B, const AmrOps* O, int* cpb_out, int* blocks_out,
                   cudaStream_t s) {
    const bool amr = ainsts != nullptr;
#define ADG_BATCH_CASE(K)                                                                                    \
    case K:                                                                                                  \
        return amr ? batch_nka<N, K, true>(phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s) \
                   : batch_nka<N, K, false>(phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
    switch (cand) {
        ADG_BATCH_CASE(0)
        ADG_BATCH_CASE(1)
        ADG_BATCH_CASE(2)
        case 3:  // the node-pair predictor where it exists, else candidate 1
            if constexpr (N == 3 || N == 5)
                if (!amr && phase == 0) return batch_x2<N>(insts, tiles, ntiles, Bf, cpb_out, blocks_out, s);
            return amr ? batch_nka<N, 1, true>(phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s)
                       : batch_nka<N, 1, false>(phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
    }
#undef ADG_BATCH_CASE
    return (int)cudaErrorInvalidValue;
}

int launch_batch_mixed(int N, int cand, int phase, const MixedInst* insts, const AmrInst* ainsts,
                       const BatchTile* tiles, int ntiles, const BasisF& Bf, const Basis& B, const void* ops,
                       int* cpb_out, int* blocks_out, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const AmrOps* O = (const AmrOps*)ops;
    switch (N) {
        case 1: return batch_n<1>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 2: return batch_n<2>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 3: return batch_n<3>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 4: return batch_n<4>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 5: return batch_n<5>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 6: return batch_n<6>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
        case 7: return batch_n<7>(cand, phase, insts, ainsts, tiles, ntiles, Bf, B, O, cpb_out, blocks_out, s);
    }
    return (int)cudaErrorInvalidValue;
}

// the prolongation/restriction operators of an adaptive mesh (for batches)
const void* amr_ops(const adg_mesh* m) { return m->tree ? &((const AmrTree*)m->tree)->ops : nullptr; }

}  // namespace adg

// ------------------------------------------------------------------ C ABI
using adg::AmrTree;

extern "C" size_t adg_leaf_count(const adg_mesh* m) {
    return m ? (size_t)m->cells : 0;
}

extern "C" int adg_leaf_info(const adg_mesh* m, int* out, size_t count) {
    if (!m || !out) return adg::fail(ADG_EINVAL, "leaf_info: NULL argument");
    if (count != 3 * (size_t)m->cells) return adg::fail(ADG_EINVAL, "leaf_info: count != 3 * leaves");
    if (!m->amr) {
        for (int c = 0; c < m->cells; ++c) {
            out[3 * c] = 0;
            out[3 * c + 1] = c % m->d.nx;
            out[3 * c + 2] = c / m->d.nx;
        }
        return ADG_OK;
    }
    const AmrTree* T = (const AmrTree*)m->tree;
    for (int c = 0; c < m->cells; ++c)
        for (int a = 0; a < 3; ++a) out[3 * c + a] = T->leaves[c][a];
    return ADG_OK;
}

extern "C" int adg_adapt(adg_mesh* m, const int8_t* flags_dev, int* leaves_out, void* stream) {
    using namespace adg;
    if (!m || !flags_dev) return fail(ADG_EINVAL, "adapt: NULL argument");
    if (!m->amr) return fail(ADG_EINVAL, "adapt: mesh was created with max_levels = 0");
    if (int rc = set_device(m)) return rc;
    AmrTree* T = (AmrTree*)m->tree;
    const int L = m->cells;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int8_t> fl(L);
    ADG_CK(cudaMemcpyAsync(fl.data(), flags_dev, L, cudaMemcpyDeviceToHost, s), "adapt: flags");
    ADG_CK(cudaStreamSynchronize(s), "adapt: sync");
    // refinement set with 2-level balance (refinement wins)
    std::vector<char> refine(L, 0);
    for (int k = 0; k < L; ++k) refine[k] = fl[k] > 0 && T->leaves[k][0] < T->maxl;
    int nb[kNbrInts];
    for (bool changed = true; changed;) {
        changed = false;
        for (int k = 0; k < L; ++k) {
            if (!refine[k]) continue;
            for (int f = 0; f < 4; ++f) {
                T->neighbour(k, f, nb);
                if (nb[0] == NB_COARSE && !refine[nb[1]]) {
                    refine[nb[1]] = 1;
                    changed = true;
                }
            }
        }
    }
    // coarsening: complete sibling groups all flagged -1, none refined, parent balanced
    std::unordered_map<long long, std::vector<int>> groups;
    for (int k = 0; k < L; ++k)
        if (T->leaves[k][0] > 0)
            groups[AmrTree::key(T->leaves[k][0] - 1, T->leaves[k][1] / 3, T->leaves[k][2] / 3)].push_back(k);
    std::vector<char> coarse_member(L, 0);
    std::vector<std::pair<std::array<int, 3>, std::vector<int>>> coarsen;
    for (auto& g : groups) {
        const std::vector<int>& ks = g.second;
        if (ks.size() != 9) continue;
        bool ok = true;
        for (int k : ks)
            if (fl[k] >= 0 || refine[k]) ok = false;
        const int plv = T->leaves[ks[0]][0] - 1;
        for (int k : ks) {
            if (!ok) break;
            for (int f = 0; f < 4; ++f) {
                T->neighbour(k, f, nb);
                if (nb[0] == NB_FINE) ok = false;
                if (nb[0] == NB_CONF && std::find(ks.begin(), ks.end(), nb[1]) == ks.end() &&
                    T->leaves[nb[1]][0] + (refine[nb[1]] ? 1 : 0) > plv + 1)
                    ok = false;
            }
        }
        if (!ok) continue;
        for (int k : ks) coarse_member[k] = 1;
        coarsen.push_back({{plv, T->leaves[ks[0]][1] / 3, T->leaves[ks[0]][2] / 3}, ks});
    }
    // new leaf list with its transfer rule
    struct NewLeaf {
        std::array<int, 3> c;
        int t, a, b;
        int src[9];
    };
    std::vector<NewLeaf> nl;
    for (int k = 0; k < L; ++k) {
        if (coarse_member[k]) continue;
        const auto& c = T->leaves[k];
        if (refine[k]) {
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    NewLeaf x{{c[0] + 1, 3 * c[1] + a, 3 * c[2] + b}, 1, a, b, {k}};
                    nl.push_back(x);
                }
        } else {
            NewLeaf x{c, 0, 0, 0, {k}};
            nl.push_back(x);
        }
    }
    for (auto& g : coarsen) {
        NewLeaf x{g.first, 2, 0, 0, {0}};
        for (int k : g.second) x.src[(T->leaves[k][2] % 3) * 3 + (T->leaves[k][1] % 3)] = k;
        nl.push_back(x);
    }
    std::sort(nl.begin(), nl.end(), [](const NewLeaf& x, const NewLeaf& y) {
        if (x.c[0] != y.c[0]) return x.c[0] < y.c[0];
        if (x.c[2] != y.c[2]) return x.c[2] < y.c[2];
        return x.c[1] < y.c[1];
    });
    const int L2 = (int)nl.size();
    std::vector<int> trans((size_t)L2 * 12, 0);
    for (int k = 0; k < L2; ++k) {
        trans[k * 12 + 0] = nl[k].t;
        trans[k * 12 + 1] = nl[k].a;
        trans[k * 12 + 2] = nl[k].b;
        for (int q = 0; q < 9; ++q) trans[k * 12 + 3 + q] = nl[k].src[q];
    }
    bool grew = false;
    if (int rc0 = ensure_capacity(m, L2, &grew)) return rc0;
    ADG_CK(cudaMemcpyAsync(m->dtrans, trans.data(), trans.size() * 4, cudaMemcpyHostToDevice, s), "adapt: upload");
    int rc = amr_transfer(m, m->u, m->u_spare, L2, m->dtrans, s);
    if (rc) return rc;
    ADG_CK(cudaStreamSynchronize(s), "adapt: transfer sync");
    std::swap(m->u, m->u_spare);
    ++m->epoch;  // the state (and, if grown, every per-leaf buffer) moved: batches rebuild their tables
    if (grew) {  // the spare (the old state) still has the old capacity
        cudaFree(m->u_spare);
        m->u_spare = nullptr;
        if (cudaMalloc(&m->u_spare, (size_t)m->leaf_cap * m->n * m->n * 4 * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(ADG_ENOMEM, "adapt: spare state");
        }
    }
    T->leaves.clear();
    for (auto& x : nl) T->leaves.push_back(x.c);
    T->index();
    m->cells = L2;
    m->tv_prep_cells = -1;  // the statistics' combine weights depend on the leaf count
    rc = upload_tables(m);
    if (rc) return rc;
    m->predicted = false;
    if (leaves_out) *leaves_out = L2;
    return ADG_OK;
}
