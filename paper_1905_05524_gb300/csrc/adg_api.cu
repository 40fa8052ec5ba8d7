// C ABI of the GB300 ADER-DG library: mesh lifetime, basis construction,
// state transfer and the host side of every entry point in include/aderdg.h.
#include <cuda_runtime.h>

#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "adg_internal.h"
#include "adg_mesh.h"

namespace {
thread_local std::string g_err;
}  // namespace

namespace adg {
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return ADG_ECUDA;
}
}  // namespace adg
using adg::cuda_fail;
using adg::fail;

namespace {

// ---------------------------------------------------------------- basis
// Gauss-Legendre nodes on [-1, 1] by Newton's method on the three-term
// recurrence of the Legendre polynomials, mapped to [0, 1].
void gauss_legendre01(int n, double* xi, double* w) {
    for (int r = 0; r < n; ++r) {
        double x = std::cos(M_PI * (r + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, p = x;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2.0 * k - 1.0) * x * p - (k - 1.0) * pm) / k;
                pm = p;
                p = pk;
            }
            if (n == 1) { p = x; pm = 1.0; }
            dp = n * (x * p - pm) / (x * x - 1.0);
            const double dx = p / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double pm = 1.0, p = x;
        for (int k = 2; k <= n; ++k) {
            const double pk = ((2.0 * k - 1.0) * x * p - (k - 1.0) * pm) / k;
            pm = p;
            p = pk;
        }
        if (n == 1) { p = x; pm = 1.0; }
        dp = n * (x * p - pm) / (x * x - 1.0);
        // roots come out in descending x; store ascending
        xi[n - 1 - r] = 0.5 * (x + 1.0);
        w[n - 1 - r] = 1.0 / ((1.0 - x * x) * dp * dp);  // = (2/((1-x^2) P'^2)) / 2
    }
}

double lagrange(const double* xi, int n, int j, double x) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != j) v *= (x - xi[m]) / (xi[j] - xi[m]);
    return v;
}

bool invert(int n, const double* A, double* Ainv) {  // Gauss-Jordan, partial pivoting
    double M[adg::kMaxN][2 * adg::kMaxN];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) M[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
        if (std::fabs(M[piv][c]) < 1e-300) return false;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) std::swap(M[c][k], M[piv][k]);
        const double d = M[c][c];
        for (int k = 0; k < 2 * n; ++k) M[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[r][c];
            for (int k = 0; k < 2 * n; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r][n + c];
    return true;
}

}  // namespace

bool adg::build_basis(int N, adg::Basis& B) {
    std::memset(&B, 0, sizeof(B));
    const int n = N + 1;
    B.n = n;
    gauss_legendre01(n, B.xi, B.w);
    double lam[adg::kMaxN];
    for (int j = 0; j < n; ++j) {
        lam[j] = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != j) lam[j] /= (B.xi[j] - B.xi[m]);
    }
    for (int i = 0; i < n; ++i) {
        double diag = 0.0;
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            B.D[i][j] = (lam[j] / lam[i]) / (B.xi[i] - B.xi[j]);
            diag -= B.D[i][j];
        }
        B.D[i][i] = diag;
    }
    for (int j = 0; j < n; ++j) {
        B.phi0[j] = lagrange(B.xi, n, j, 0.0);
        B.phi1[j] = lagrange(B.xi, n, j, 1.0);
        B.lift0[j] = B.phi0[j] / B.w[j];
        B.lift1[j] = B.phi1[j] / B.w[j];
    }
    // K1[l][k] = phi_l(1) phi_k(1) - w_k D[k][l]
    double K1[adg::kMaxN * adg::kMaxN], K1i[adg::kMaxN * adg::kMaxN];
    for (int l = 0; l < n; ++l)
        for (int k = 0; k < n; ++k) K1[l * n + k] = B.phi1[l] * B.phi1[k] - B.w[k] * B.D[k][l];
    if (!invert(n, K1, K1i)) return false;
    for (int l = 0; l < n; ++l) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            B.Kw[l][k] = K1i[l * n + k] * B.w[k];
            s += B.Kw[l][k];
        }
        B.Kw1[l] = s;
    }
    for (int p = 0; p < n; ++p)
        for (int i = 0; i < n; ++i) B.Vx[p][i] = B.w[p] * B.D[p][i] / B.w[i];
    return true;
}

using adg::build_basis;

namespace {

void free_mesh(adg_mesh* m) {
    if (!m) return;
    cudaFree(m->u);
    cudaFree(m->rvol);
    cudaFree(m->trace);
    cudaFree(m->trace_bar);
    cudaFree(m->tv);
    cudaFree(m->stats);
    cudaFree(m->part);
    cudaFree(m->speed);
    cudaFree(m->flag);
    cudaFree(m->bgbuf);
    cudaFree(m->mixbuf);
    cudaFree(m->halo);
    if (m->amr) adg::amr_free(m);
    delete m;
}

// FP32 copies of basis/constants and the FP64/FP32 background tables of the
// mixed-precision path.
int build_mixed(adg_mesh* m) {
    const adg_mesh_desc* d = &m->d;
    const int n = m->n, ny = d->ny;
    adg::BasisF& b = m->Bf;
    std::memset(&b, 0, sizeof(b));
    for (int a = 0; a < n; ++a) {
        b.xi[a] = (float)m->B.xi[a];
        b.w[a] = (float)m->B.w[a];
        b.phi0[a] = (float)m->B.phi0[a];
        b.phi1[a] = (float)m->B.phi1[a];
        b.Kw1[a] = (float)m->B.Kw1[a];
        b.lift0[a] = (float)m->B.lift0[a];
        b.lift1[a] = (float)m->B.lift1[a];
        for (int c = 0; c < n; ++c) {
            b.D[a][c] = (float)m->B.D[a][c];
            b.Kw[a][c] = (float)m->B.Kw[a][c];
            b.Vx[a][c] = (float)m->B.Vx[a][c];
        }
    }
    const adg::Phys& P = m->P;
    adg::PhysF& f = m->Pf;
    std::memset(&f, 0, sizeof(f));
    f.gamma = (float)P.gamma; f.gm1 = (float)P.gm1; f.R = (float)P.R; f.invR = (float)P.invR;
    f.mu = (float)P.mu; f.kappa = (float)P.kappa; f.g = d->gravity ? (float)P.g : 0.f;
    f.cp = (float)P.cp; f.lamv = (float)P.lamv; f.eta_x = (float)P.eta_x; f.eta_y = (float)P.eta_y;
    f.hx = (float)P.hx; f.hy = (float)P.hy; f.inv_hx = (float)P.inv_hx; f.inv_hy = (float)P.inv_hy;
    f.x0 = (float)P.x0; f.y0 = (float)P.y0;
    f.sa = (float)P.sa; f.sL = (float)P.sL; f.sU = (float)P.sU; f.sp = (float)P.sp;
    f.gravity = P.gravity; f.source = P.source; f.nx = P.nx; f.ny = P.ny; f.bc_x = P.bc_x; f.bc_y = P.bc_y;
    // tables
    const size_t nn = (size_t)ny * n;
    std::vector<double> rb(nn, 0.0), Eb(nn, 0.0);
    std::vector<float> pb(nn, 0.f), dzr(nn, 0.f), dzE(nn, 0.f), face((size_t)ny * 2 * adg::kFaceBg, 0.f);
    if (d->gravity) {
        for (int iy = 0; iy < ny; ++iy) {
            double zn[adg::kMaxN], pn[adg::kMaxN];
            for (int j = 0; j < n; ++j) {
                const double z = d->y0 + (iy + m->B.xi[j]) * P.hy;
                const double ex = 1.0 - d->g * z / (P.cp * d->theta0);
                const double p = d->p0 * std::pow(ex, P.cp / d->R);
                const double r = p / (d->R * d->theta0 * ex);
                zn[j] = z;
                pn[j] = p;
                rb[iy * n + j] = r;
                Eb[iy * n + j] = p / P.gm1 + r * d->g * z;
                pb[iy * n + j] = (float)p;
            }
            for (int j = 0; j < n; ++j) {
                double sr = 0.0, sE = 0.0;
                for (int p = 0; p < n; ++p) {
                    sr += m->B.D[j][p] * rb[iy * n + p];
                    sE += m->B.D[j][p] * Eb[iy * n + p];
                }
                dzr[iy * n + j] = (float)(sr * P.inv_hy);
                dzE[iy * n + j] = (float)(sE * P.inv_hy);
            }
            for (int side = 0; side < 2; ++side) {  // 0: north (phi(1)), 1: south (phi(0))
                const double* phi = side == 0 ? m->B.phi1 : m->B.phi0;
                double r = 0.0, E = 0.0;
                for (int j = 0; j < n; ++j) {
                    r += phi[j] * rb[iy * n + j];
                    E += phi[j] * Eb[iy * n + j];
                }
                const double zf = d->y0 + (iy + (side == 0 ? 1 : 0)) * P.hy;
                const double exf = 1.0 - d->g * zf / (P.cp * d->theta0);
                const double pfx = d->p0 * std::pow(exf, P.cp / d->R);
                const double rfx = pfx / (d->R * d->theta0 * exf);
                const double Efx = pfx / P.gm1 + rfx * d->g * zf;
                float* fb = face.data() + ((size_t)iy * 2 + side) * adg::kFaceBg;
                fb[0] = (float)r;
                fb[1] = (float)E;
                fb[2] = (float)(P.gm1 * (E - r * d->g * zf));
                fb[3] = (float)rfx;
                fb[4] = (float)Efx;
                fb[5] = (float)pfx;
                fb[6] = (float)(rfx - r);  // wall faces keep these; interior ones are overwritten below
                fb[7] = (float)(Efx - E);
            }
            (void)zn;
            (void)pn;
        }
        // faces between rows (and the wrap face of a periodic y): the upper
        // row's extrapolated background minus the lower row's, in FP64, the
        // same FP32 value on both sides of the face
        auto extrap = [&](int iy, int side, double& r, double& E) {
            const double* phi = side == 0 ? m->B.phi1 : m->B.phi0;
            r = E = 0.0;
            for (int j = 0; j < n; ++j) {
                r += phi[j] * rb[iy * n + j];
                E += phi[j] * Eb[iy * n + j];
            }
        };
        const bool wall_y = d->bc_y == ADG_BC_WALL;
        for (int iy = 0; iy < ny; ++iy) {
            const int up = iy + 1 < ny ? iy + 1 : 0;
            if (wall_y && iy + 1 == ny) continue;
            double rl, El, ru, Eu;
            extrap(iy, 0, rl, El);   // lower row, north face
            extrap(up, 1, ru, Eu);   // upper row, south face
            const float dr = (float)(ru - rl), dE = (float)(Eu - El);
            float* fn = face.data() + ((size_t)iy * 2 + 0) * adg::kFaceBg;
            float* fs = face.data() + ((size_t)up * 2 + 1) * adg::kFaceBg;
            fn[6] = fs[6] = dr;
            fn[7] = fs[7] = dE;
        }
    }
    const size_t bytes = nn * 8 * 2 + nn * 4 * 3 + face.size() * 4;
    if (cudaMalloc(&m->mixbuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "create_mesh: mixed tables");
    }
    char* p = (char*)m->mixbuf;
    auto put = [&](const void* src, size_t nb) {
        void* dst = p;
        cudaMemcpy(dst, src, nb, cudaMemcpyHostToDevice);
        p += nb;
        return dst;
    };
    m->mbg.rb = (const double*)put(rb.data(), nn * 8);
    m->mbg.Eb = (const double*)put(Eb.data(), nn * 8);
    m->mbg.pb = (const float*)put(pb.data(), nn * 4);
    m->mbg.dzr = (const float*)put(dzr.data(), nn * 4);
    m->mbg.dzE = (const float*)put(dzE.data(), nn * 4);
    m->mbg.face = (const float*)put(face.data(), face.size() * 4);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "create_mesh: mixed tables upload");
    return ADG_OK;
}

}  // namespace

int adg::set_device(const adg_mesh* m) {
    ADG_CK(cudaSetDevice(m->d.device), "cudaSetDevice");
    return ADG_OK;
}
using adg::set_device;

extern "C" {

const char* adg_last_error(void) { return g_err.c_str(); }

int adg_create_mesh(const adg_mesh_desc* d, adg_mesh** out) {
    if (!d || !out) return fail(ADG_EINVAL, "create_mesh: NULL argument");
    *out = nullptr;
    if (d->degree < 1 || d->degree > ADG_MAX_DEGREE)
        return fail(ADG_EINVAL, "create_mesh: degree must be in [1, 7]");
    if (d->nx < 1 || d->ny < 1) return fail(ADG_EINVAL, "create_mesh: nx, ny must be >= 1");
    if ((long long)d->nx * d->ny > (1LL << 26)) return fail(ADG_EINVAL, "create_mesh: too many cells");
    if (!(d->Lx > 0.0) || !(d->Ly > 0.0)) return fail(ADG_EINVAL, "create_mesh: Lx, Ly must be > 0");
    auto known_x = [](int b) { return b == ADG_BC_PERIODIC || b == ADG_BC_WALL || b == ADG_BC_NOSLIP ||
                                      b == ADG_BC_ANALYTIC; };
    if (!known_x(d->bc_x) || d->bc_y < 0 || d->bc_y > ADG_BC_ANALYTIC)
        return fail(ADG_EINVAL, "create_mesh: unknown boundary condition");
    const bool cfd_bc = d->bc_x >= ADG_BC_NOSLIP || d->bc_y >= ADG_BC_NOSLIP;
    if (cfd_bc && (d->precision != ADG_PREC_FP64 || d->max_levels != 0 || d->gravity))
        return fail(ADG_EUNSUPPORTED, "create_mesh: no-slip and analytic boundaries are built for uniform FP64 "
                                      "meshes without gravity");
    if ((d->bc_x == ADG_BC_ANALYTIC || d->bc_y == ADG_BC_ANALYTIC) && d->bc_field != ADG_FIELD_TAYLOR_GREEN)
        return fail(ADG_EINVAL, "create_mesh: analytic boundaries need bc_field = ADG_FIELD_TAYLOR_GREEN");
    if (!std::isfinite(d->lid_u)) return fail(ADG_EINVAL, "create_mesh: lid_u must be finite");
    const bool exch = d->bc_y >= ADG_BC_EXCHANGE && d->bc_y <= ADG_BC_EXCHANGE_WALL;
    if (exch && (d->precision != ADG_PREC_FP64 || d->max_levels != 0))
        return fail(ADG_EUNSUPPORTED, "create_mesh: strip exchange is built for uniform FP64 meshes");
    if (!(d->gamma > 1.0) || !(d->R > 0.0) || !(d->Pr > 0.0) || !(d->mu >= 0.0))
        return fail(ADG_EINVAL, "create_mesh: invalid gas constants");
    if (d->source != ADG_SRC_NONE && d->source != ADG_SRC_STEADY && d->source != ADG_SRC_PAPER)
        return fail(ADG_EINVAL, "create_mesh: unknown source");
    if (d->source != ADG_SRC_NONE && !(d->src_L > 0.0))
        return fail(ADG_EINVAL, "create_mesh: a manufactured source needs src_L > 0");
    if (d->source == ADG_SRC_PAPER && (d->precision != ADG_PREC_FP64 || d->max_levels != 0 || d->gravity))
        return fail(ADG_EUNSUPPORTED, "create_mesh: the time-dependent source is built for uniform FP64 meshes "
                                      "without gravity");
    if (d->precision != ADG_PREC_FP64 && d->precision != ADG_PREC_MIXED && d->precision != ADG_PREC_MIXED_TF32 &&
        d->precision != ADG_PREC_MIXED_BF16X3)
        return fail(ADG_EINVAL, "create_mesh: unknown precision");
    if ((d->precision == ADG_PREC_MIXED_TF32 || d->precision == ADG_PREC_MIXED_BF16X3) &&
        (d->max_levels != 0 || !adg::tc_degree_supported(d->degree)))
        return fail(ADG_EUNSUPPORTED, "create_mesh: the tensor-core precisions are built for uniform meshes of "
                                      "degree 3, 5, 7");
    if (d->gravity && !(d->theta0 > 0.0 && d->p0 > 0.0))
        return fail(ADG_EINVAL, "create_mesh: gravity needs theta0 > 0 and p0 > 0");
    if (d->max_levels < 0 || d->max_levels > 4) return fail(ADG_EINVAL, "create_mesh: max_levels must be in [0, 4]");
    int ndev = 0;
    ADG_CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (d->device < 0 || d->device >= ndev) return fail(ADG_EINVAL, "create_mesh: bad device ordinal");

    adg_mesh* m = new adg_mesh();
    m->d = *d;
    m->N = d->degree;
    m->n = d->degree + 1;
    m->cells = d->nx * d->ny;
    if (!build_basis(m->N, m->B)) {
        delete m;
        return fail(ADG_EINVAL, "create_mesh: singular time-stiffness matrix");
    }
    adg::Phys& P = m->P;
    std::memset(&P, 0, sizeof(P));
    P.gamma = d->gamma;
    P.gm1 = d->gamma - 1.0;
    P.R = d->R;
    P.invR = 1.0 / d->R;
    P.mu = d->mu;
    P.cp = d->gamma * d->R / (d->gamma - 1.0);
    P.kappa = d->mu * P.cp / d->Pr;
    P.g = d->g;
    P.p0 = d->p0;
    P.theta0 = d->theta0;
    P.Rcp = d->R / P.cp;
    P.lamv = std::fmax(4.0 / 3.0, d->gamma / d->Pr) * d->mu;
    P.hx = d->Lx / d->nx;
    P.hy = d->Ly / d->ny;
    P.inv_hx = 1.0 / P.hx;
    P.inv_hy = 1.0 / P.hy;
    P.x0 = d->x0;
    P.y0 = d->y0;
    P.eta_x = (2.0 * m->N + 1.0) / (P.hx * std::sqrt(M_PI / 2.0));
    P.eta_y = (2.0 * m->N + 1.0) / (P.hy * std::sqrt(M_PI / 2.0));
    P.gravity = d->gravity ? 1 : 0;
    P.source = d->source;
    P.sa = d->src_a;
    P.sL = d->src_L;
    P.sU = d->src_U;
    P.sp = d->src_p;
    P.nx = d->nx;
    P.ny = d->ny;
    P.bc_x = d->bc_x;
    P.bc_y = d->bc_y;
    P.lid_u = d->lid_u;
    P.bc_field = d->bc_field;

    int rc = set_device(m);
    if (rc) { delete m; return rc; }
    const size_t cnt = (size_t)m->cells * m->n * m->n * 4;
    const size_t tr = (size_t)m->cells * 4 * adg::kTraceComps * m->n;
    int nb = 0;
    adg::launch_max_speed(m->N, nullptr, nullptr, m->cells, m->B, m->P, &nb, nullptr);
    m->speed_blocks = nb;
    const size_t nbg = 2 * (size_t)d->ny * m->n + 2 * (size_t)(d->ny + 1);
    if (cudaMalloc(&m->u, cnt * 8) != cudaSuccess || cudaMalloc(&m->rvol, cnt * 8) != cudaSuccess ||
        cudaMalloc(&m->trace, tr * 8) != cudaSuccess || cudaMalloc(&m->tv, (size_t)m->cells * 8) != cudaSuccess ||
        cudaMalloc(&m->stats, 4 * 8) != cudaSuccess || cudaMalloc(&m->speed, (size_t)nb * 8) != cudaSuccess ||
        cudaMalloc(&m->part, 8 * adg::tv_stats_scratch_doubles(m->N, m->cells)) != cudaSuccess ||
        cudaMalloc(&m->flag, sizeof(int)) != cudaSuccess || cudaMalloc(&m->bgbuf, nbg * 8) != cudaSuccess) {
        cudaGetLastError();
        free_mesh(m);
        return fail(ADG_ENOMEM, "create_mesh: device allocation failed");
    }
    if (cudaMemset(m->stats, 0, 4 * 8) != cudaSuccess) {  // mean, sigma and the given pair
        cudaGetLastError();
        free_mesh(m);
        return fail(ADG_ECUDA, "create_mesh: workspace initialisation failed");
    }
    // hydrostatic background tables (Eq. 6, isentropic reading): zero without gravity
    std::vector<double> h(nbg, 0.0);
    double* pn = h.data();
    double* rn = pn + (size_t)d->ny * m->n;
    double* pf = rn + (size_t)d->ny * m->n;
    double* rf = pf + (d->ny + 1);
    if (d->gravity) {
        auto bgp = [&](double z, double& pb, double& rb) {
            const double ex = 1.0 - d->g * z / (P.cp * d->theta0);
            pb = d->p0 * std::pow(ex, P.cp / d->R);
            rb = pb / (d->R * d->theta0 * ex);
        };
        for (int iy = 0; iy < d->ny; ++iy)
            for (int j = 0; j < m->n; ++j)
                bgp(d->y0 + (iy + m->B.xi[j]) * P.hy, pn[iy * m->n + j], rn[iy * m->n + j]);
        for (int f = 0; f <= d->ny; ++f) bgp(d->y0 + f * P.hy, pf[f], rf[f]);
    }
    if (cudaMemcpy(m->bgbuf, h.data(), nbg * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->u, 0, cnt * 8) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        free_mesh(m);
        return cuda_fail(e, "create_mesh: upload");
    }
    if (d->precision != ADG_PREC_FP64) {
        int rc2 = build_mixed(m);
        if (rc2) {
            free_mesh(m);
            return rc2;
        }
    }
    if (d->max_levels > 0) {
        int rc3 = adg::amr_setup(m);
        if (rc3) {
            free_mesh(m);
            return rc3;
        }
    }
    if (d->bc_y >= ADG_BC_EXCHANGE && d->bc_y <= ADG_BC_EXCHANGE_WALL) {
        const size_t hb = 2 * (size_t)d->nx * adg::kTraceComps * m->n * 8;
        if (cudaMalloc(&m->halo, hb) != cudaSuccess || cudaMemset(m->halo, 0, hb) != cudaSuccess) {
            cudaGetLastError();
            free_mesh(m);
            return fail(ADG_ENOMEM, "create_mesh: halo buffers");
        }
        m->bg.halo_s = m->halo;
        m->bg.halo_n = m->halo + (size_t)d->nx * adg::kTraceComps * m->n;
    }
    m->bg.pbar_node = m->bgbuf;
    m->bg.rhobar_node = m->bgbuf + (size_t)d->ny * m->n;
    m->bg.pbar_face = m->bgbuf + 2 * (size_t)d->ny * m->n;
    m->bg.rhobar_face = m->bg.pbar_face + (d->ny + 1);
    *out = m;
    return ADG_OK;
}

void adg_destroy_mesh(adg_mesh* m) {
    if (!m) return;
    cudaSetDevice(m->d.device);
    cudaDeviceSynchronize();
    free_mesh(m);
}

size_t adg_state_count(const adg_mesh* m) {
    return m ? (size_t)m->cells * m->n * m->n * 4 : 0;
}

int adg_set_state(adg_mesh* m, const double* u, size_t count, int on_device, void* stream) {
    if (!m || !u) return fail(ADG_EINVAL, "set_state: NULL argument");
    if (count != adg_state_count(m)) return fail(ADG_EINVAL, "set_state: count != cells*(N+1)^2*4");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "set_state: bad on_device");
    if (int rc = set_device(m)) return rc;
    ADG_CK(cudaMemcpyAsync(m->u, u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           (cudaStream_t)stream), "set_state");
    m->predicted = false;
    return ADG_OK;
}

int adg_get_state(adg_mesh* m, double* u, size_t count, int on_device, void* stream) {
    if (!m || !u) return fail(ADG_EINVAL, "get_state: NULL argument");
    if (count != adg_state_count(m)) return fail(ADG_EINVAL, "get_state: count != cells*(N+1)^2*4");
    if (on_device < 0 || on_device > ADG_COPY_HOST_ASYNC) return fail(ADG_EINVAL, "get_state: bad on_device");
    if (int rc = set_device(m)) return rc;
    ADG_CK(cudaMemcpyAsync(u, m->u, count * 8, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           (cudaStream_t)stream), "get_state");
    if (on_device == 0) ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "get_state sync");
    return ADG_OK;
}

double* adg_state_ptr(adg_mesh* m) { return m ? m->u : nullptr; }

int adg_set_time(adg_mesh* m, double t) {
    if (!m) return fail(ADG_EINVAL, "set_time: NULL mesh");
    m->t = t;
    return ADG_OK;
}

double adg_get_time(const adg_mesh* m) { return m ? m->t : 0.0; }

int adg_init_scenario(adg_mesh* m, const adg_scenario* s, void* stream) {
    if (!m || !s) return fail(ADG_EINVAL, "init_scenario: NULL argument");
    if (s->kind < ADG_SCEN_STEADY || s->kind > ADG_SCEN_CAVITY)
        return fail(ADG_EINVAL, "init_scenario: unknown scenario");
    const bool no_gravity = s->kind == ADG_SCEN_STEADY || s->kind == ADG_SCEN_PAPER ||
                              s->kind == ADG_SCEN_TAYLOR_GREEN || s->kind == ADG_SCEN_CAVITY;
    if ((s->kind == ADG_SCEN_TAYLOR_GREEN || s->kind == ADG_SCEN_CAVITY) && m->d.gravity)
        return fail(ADG_EINVAL, "init_scenario: the CFD scenarios run without gravity");
    if (!no_gravity && !m->d.gravity)
        return fail(ADG_EINVAL, "init_scenario: bubble scenarios need gravity");
    if (s->kind == ADG_SCEN_STEADY && m->d.source != ADG_SRC_STEADY)
        return fail(ADG_EINVAL, "init_scenario: steady field needs the steady source");
    if (s->kind == ADG_SCEN_PAPER && m->d.source != ADG_SRC_PAPER)
        return fail(ADG_EINVAL, "init_scenario: the Eq. 8 field needs the time-dependent source");
    if (s->kind == ADG_SCEN_COSINE && !(s->a > 0.0))
        return fail(ADG_EINVAL, "init_scenario: cosine bubble radius must be > 0");
    if (int rc = set_device(m)) return rc;
    if (m->amr) {
        if (int rc = adg::amr_init_scenario(m, s, stream)) return rc;
    } else {
        int e = adg::launch_init_scenario(m->N, m->u, m->cells, s->kind, s->A, s->a, s->xc, s->zc, m->B, m->P, stream);
        if (e) return cuda_fail((cudaError_t)e, "init_scenario");
    }
    m->predicted = false;
    m->t = 0.0;
    return ADG_OK;
}

int adg_step_lts(adg_mesh* m, double dt, double* cycle, void* stream) {
    if (!m) return fail(ADG_EINVAL, "step_lts: NULL mesh");
    if (!m->amr) return fail(ADG_EINVAL, "step_lts: adaptive meshes only (max_levels > 0)");
    if (m->d.precision != ADG_PREC_FP64) return fail(ADG_EUNSUPPORTED, "step_lts: FP64 meshes only");
    if (m->N < 2) return fail(ADG_EUNSUPPORTED, "step_lts: degree >= 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADG_EINVAL, "step_lts: dt must be finite and > 0");
    if (int rc = set_device(m)) return rc;
    double c = 0.0;
    if (int rc = adg::amr_step_lts(m, dt, &c, stream)) return rc;
    m->t += c;
    m->predicted = false;
    if (cycle) *cycle = c;
    return ADG_OK;
}

int adg_predictor(adg_mesh* m, double dt, void* stream) {
    if (!m) return fail(ADG_EINVAL, "predictor: NULL mesh");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADG_EINVAL, "predictor: dt must be finite and > 0");
    if (int rc = set_device(m)) return rc;
    if (m->amr) {
        if (int rc = adg::amr_predictor(m, dt, stream)) return rc;
        m->predicted = true;
        m->pred_dt = dt;
        return ADG_OK;
    }
    int e;
    if (m->d.precision == ADG_PREC_FP64)
        e = adg::launch_predictor_fp64(m->N, m->u, m->rvol, m->trace, m->cells, dt, m->t, m->B, m->P, m->bg, stream);
    else if (m->d.precision == ADG_PREC_MIXED_TF32 || m->d.precision == ADG_PREC_MIXED_BF16X3)
        e = adg::launch_predictor_mixed_tc(m->N, m->u, (float*)m->rvol, (float*)m->trace, m->cells, dt, m->Bf,
                                           m->Pf, m->mbg, m->d.precision == ADG_PREC_MIXED_BF16X3, stream);
    else
        e = adg::launch_predictor_mixed(m->N, m->u, (float*)m->rvol, (float*)m->trace, m->cells, dt, m->Bf,
                                        m->Pf, m->mbg, stream);
    if (e) return cuda_fail((cudaError_t)e, "predictor launch");
    m->predicted = true;
    m->pred_dt = dt;
    return ADG_OK;
}

// corrector of a uniform or adaptive mesh; epi (uniform meshes only): the TV
// indicator of the updated state in the same kernel
static int corrector_impl(adg_mesh* m, double dt, void* stream, const adg::TvEpilogue* epi) {
    if (!m) return fail(ADG_EINVAL, "corrector: NULL mesh");
    if (!m->predicted || m->pred_dt != dt)
        return fail(ADG_ESTATE, "corrector: needs a preceding predictor with the same dt");
    if (int rc = set_device(m)) return rc;
    if (m->amr) {
        if (epi) return fail(ADG_EUNSUPPORTED, "corrector: no TV epilogue on adaptive meshes");
        if (int rc = adg::amr_corrector(m, dt, stream)) return rc;
        m->predicted = false;
        return ADG_OK;
    }
    int e = m->d.precision == ADG_PREC_FP64
                ? adg::launch_corrector_fp64(m->N, m->u, m->rvol, m->trace, m->cells, dt, m->B, m->P, m->bg, stream,
                                             epi, m->t)
                : adg::launch_corrector_mixed(m->N, m->u, (const float*)m->rvol, (const float*)m->trace, m->cells,
                                              dt, m->Bf, m->Pf, m->mbg, stream, epi);
    if (e) return cuda_fail((cudaError_t)e, "corrector launch");
    m->predicted = false;
    return ADG_OK;
}

int adg_corrector(adg_mesh* m, double dt, void* stream) { return corrector_impl(m, dt, stream, nullptr); }

int adg_step(adg_mesh* m, double dt, void* stream) {
    int rc = adg_predictor(m, dt, stream);
    if (rc) return rc;
    rc = adg_corrector(m, dt, stream);
    if (rc) return rc;
    m->t += dt;
    return ADG_OK;
}

int adg_stable_dt(adg_mesh* m, double cfl, double* dt, void* stream) {
    if (!m || !dt) return fail(ADG_EINVAL, "stable_dt: NULL argument");
    if (!(cfl > 0.0)) return fail(ADG_EINVAL, "stable_dt: cfl must be > 0");
    if (int rc = set_device(m)) return rc;
    if (m->amr) {
        double lam = 0.0;
        if (int rc = adg::amr_max_speed(m, &lam, stream)) return rc;
        if (!(lam > 0.0) || !std::isfinite(lam) || lam >= 1e300)
            return fail(ADG_ENONFINITE, "stable_dt: non-finite or non-positive wave speed");
        *dt = cfl * m->hmin / (2.0 * (2.0 * m->N + 1.0) * lam);
        return ADG_OK;
    }
    int nb = 0;
    int e = adg::launch_max_speed(m->N, m->u, m->speed, m->cells, m->B, m->P, &nb, stream);
    if (e) return cuda_fail((cudaError_t)e, "stable_dt launch");
    std::vector<double> h(nb);
    ADG_CK(cudaMemcpyAsync(h.data(), m->speed, nb * 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "stable_dt copy");
    ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "stable_dt sync");
    double lam = 0.0;
    for (double v : h) lam = std::fmax(lam, v);
    if (!(lam > 0.0) || !std::isfinite(lam) || lam >= 1e300)
        return fail(ADG_ENONFINITE, "stable_dt: non-finite or non-positive wave speed");
    const double hmin = std::fmin(m->P.hx, m->P.hy);
    *dt = cfl * hmin / (2.0 * (2.0 * m->N + 1.0) * lam);
    return ADG_OK;
}

static int tv_check(const adg_mesh* m, int var, double T_r, double T_c) {
    if (var != ADG_TV_RHO && var != ADG_TV_THETA) return fail(ADG_EINVAL, "tv_indicator: unknown variable");
    if (var == ADG_TV_THETA && !m->d.gravity)
        return fail(ADG_EINVAL, "tv_indicator: theta needs the atmosphere constants (gravity on)");
    if (!(T_r > T_c)) return fail(ADG_EINVAL, "tv_indicator: needs T_r > T_c");
    return ADG_OK;
}

// combine weights of the statistics ready for the current cell count
static int tv_prepare(adg_mesh* m, void* stream) {
    if (m->tv_prep_cells != m->cells) {
        int e = adg::tv_stats_prepare(m->N, m->cells, m->part, stream);
        if (e) return cuda_fail((cudaError_t)e, "tv_indicator: statistics weights");
        m->tv_prep_cells = m->cells;
    }
    return ADG_OK;
}

// statistics from the block triples in m->part, flags, optional host copy of (mean, sigma)
static int tv_finish(adg_mesh* m, const double* tvbuf, double T_r, double T_c, int8_t* flags, double* stats,
                     void* stream) {
    const adg::TvStatsArgs st = adg::tv_stats_args(m->N, m->cells, m->part);
    int e = adg::launch_tv_stats_flags(tvbuf, st, T_r, T_c, m->stats, flags, stream);
    if (e) return cuda_fail((cudaError_t)e, "tv_indicator statistics");
    if (stats) {
        ADG_CK(cudaMemcpyAsync(stats, m->stats, 16, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "tv stats copy");
        ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "tv stats sync");
    }
    return ADG_OK;
}

int adg_tv_indicator(adg_mesh* m, int var, double T_r, double T_c, double* tv, int8_t* flags,
                     double* stats, void* stream) {
    if (!m) return fail(ADG_EINVAL, "tv_indicator: NULL mesh");
    if (int rc = tv_check(m, var, T_r, T_c)) return rc;
    if (int rc = set_device(m)) return rc;
    if (int rc = tv_prepare(m, stream)) return rc;
    double* tvbuf = tv ? tv : m->tv;
    if (m->amr) {
        if (int rc = adg::amr_tv_cells(m, var, tvbuf, m->part, stream)) return rc;
    } else {
        int e = m->d.precision == ADG_PREC_FP64
                    ? adg::launch_tv_cells(m->N, m->u, tvbuf, m->part, m->cells, var, m->B, m->P, stream)
                    : adg::launch_tv_cells_mixed(m->N, m->u, tvbuf, m->part, m->cells, var, m->Bf, m->Pf, m->mbg,
                                                 m->d.theta0, m->P.Rcp, stream);
        if (e) return cuda_fail((cudaError_t)e, "tv_indicator cells");
    }
    return tv_finish(m, tvbuf, T_r, T_c, flags, stats, stream);
}

int adg_step_tv(adg_mesh* m, double dt, int var, double T_r, double T_c, double* tv, int8_t* flags,
                double* stats, void* stream) {
    if (!m) return fail(ADG_EINVAL, "step_tv: NULL mesh");
    if (int rc = tv_check(m, var, T_r, T_c)) return rc;
    if (m->amr) {  // adaptive meshes: the two calls in turn
        if (int rc = adg_step(m, dt, stream)) return rc;
        return adg_tv_indicator(m, var, T_r, T_c, tv, flags, stats, stream);
    }
    if (int rc = set_device(m)) return rc;
    if (int rc = tv_prepare(m, stream)) return rc;
    if (int rc = adg_predictor(m, dt, stream)) return rc;
    adg::TvEpilogue epi;
    epi.tv = tv ? tv : m->tv;
    epi.part = m->part;
    epi.var = var;
    epi.theta0 = m->d.theta0;
    epi.Rcp = m->P.Rcp;
    if (int rc = corrector_impl(m, dt, stream, &epi)) return rc;
    m->t += dt;
    return tv_finish(m, epi.tv, T_r, T_c, flags, stats, stream);
}

int adg_step_adjoint(adg_mesh* m, double dt, const double* u_n, const double* lam_np1, double* lam_n,
                     void* stream) {
    if (!m || !u_n || !lam_np1 || !lam_n) return fail(ADG_EINVAL, "step_adjoint: NULL argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADG_EINVAL, "step_adjoint: dt must be finite and > 0");
    if (m->d.precision != ADG_PREC_FP64) return fail(ADG_EUNSUPPORTED, "step_adjoint: FP64 meshes only");
    if (m->N > 5) return fail(ADG_EUNSUPPORTED, "step_adjoint: built for degree <= 5");
    if (m->amr) return fail(ADG_EUNSUPPORTED, "step_adjoint: uniform meshes only");
    if (m->d.bc_y >= ADG_BC_EXCHANGE || m->d.bc_x >= ADG_BC_NOSLIP)
        return fail(ADG_EUNSUPPORTED, "step_adjoint: built for periodic and slip-wall boundaries");
    if (m->d.source == ADG_SRC_PAPER)
        return fail(ADG_EUNSUPPORTED, "step_adjoint: time-dependent source not supported");
    if (lam_n == lam_np1 || lam_n == u_n) return fail(ADG_EINVAL, "step_adjoint: lam_n must not alias the inputs");
    if (int rc = set_device(m)) return rc;
    const size_t tr = (size_t)m->cells * 4 * adg::kTraceComps * m->n;
    if (!m->trace_bar && cudaMalloc(&m->trace_bar, tr * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "step_adjoint: trace adjoint buffer");
    }
    // forward traces at u_n (workspace), then the two adjoint kernels
    int e = adg::launch_predictor_fp64(m->N, u_n, m->rvol, m->trace, m->cells, dt, m->t, m->B, m->P, m->bg, stream);
    if (e) return cuda_fail((cudaError_t)e, "step_adjoint: forward predictor");
    m->predicted = false;
    e = adg::launch_step_adjoint_fp64(m->N, u_n, lam_np1, lam_n, m->trace, m->trace_bar, m->cells, dt, m->B, m->P,
                                      m->bg, stream);
    if (e) return cuda_fail((cudaError_t)e, "step_adjoint: adjoint kernels");
    return ADG_OK;
}

int adg_get_boundary_traces(adg_mesh* m, double* south, double* north, void* stream) {
    if (!m) return fail(ADG_EINVAL, "get_boundary_traces: NULL mesh");
    if (m->d.bc_y < ADG_BC_EXCHANGE || m->d.bc_y > ADG_BC_EXCHANGE_WALL)
        return fail(ADG_EINVAL, "get_boundary_traces: bc_y has no exchange side");
    if (!m->predicted) return fail(ADG_ESTATE, "get_boundary_traces: call adg_predictor first");
    if (int rc = set_device(m)) return rc;
    const size_t TR = (size_t)adg::kTraceComps * m->n, nx = m->d.nx;
    cudaStream_t s = (cudaStream_t)stream;
    // record of face f of cell c starts at (c * 4 + f) * TR: strided gather of one row
    if (south)
        ADG_CK(cudaMemcpy2DAsync(south, TR * 8, m->trace + 3 * TR, 4 * TR * 8, TR * 8, nx, cudaMemcpyDeviceToDevice, s),
               "get_boundary_traces: south");
    if (north)
        ADG_CK(cudaMemcpy2DAsync(north, TR * 8, m->trace + ((size_t)(m->d.ny - 1) * nx * 4 + 2) * TR, 4 * TR * 8,
                                 TR * 8, nx, cudaMemcpyDeviceToDevice, s),
               "get_boundary_traces: north");
    return ADG_OK;
}

int adg_set_halo_traces(adg_mesh* m, const double* south, const double* north, void* stream) {
    if (!m) return fail(ADG_EINVAL, "set_halo_traces: NULL mesh");
    if (m->d.bc_y < ADG_BC_EXCHANGE || m->d.bc_y > ADG_BC_EXCHANGE_WALL)
        return fail(ADG_EINVAL, "set_halo_traces: bc_y has no exchange side");
    if (int rc = set_device(m)) return rc;
    const size_t bytes = (size_t)m->d.nx * adg::kTraceComps * m->n * 8;
    cudaStream_t s = (cudaStream_t)stream;
    if (south) ADG_CK(cudaMemcpyAsync(m->halo, south, bytes, cudaMemcpyDeviceToDevice, s), "set_halo_traces: south");
    if (north)
        ADG_CK(cudaMemcpyAsync(m->halo + bytes / 8, north, bytes, cudaMemcpyDeviceToDevice, s), "set_halo_traces: north");
    return ADG_OK;
}

int adg_tv_flags(adg_mesh* m, const double* tv, double count, double mean, double M2, double T_r, double T_c,
                 int8_t* flags, void* stream) {
    if (!m || !tv || !flags) return fail(ADG_EINVAL, "tv_flags: NULL argument");
    if (!(count > 0.0) || !(M2 >= 0.0) || !(T_r > T_c)) return fail(ADG_EINVAL, "tv_flags: bad statistics");
    if (int rc = set_device(m)) return rc;
    const double ms[2] = {mean, std::sqrt(M2 / count)};  // population sigma, as the device forms it
    double* given = m->stats + 2;  // the two spare slots of the statistics buffer
    ADG_CK(cudaMemcpyAsync(given, ms, sizeof(ms), cudaMemcpyHostToDevice, (cudaStream_t)stream), "tv_flags");
    int e = adg::launch_tv_flags_given(tv, m->cells, given, T_r, T_c, flags, stream);
    if (e) return cuda_fail((cudaError_t)e, "tv_flags launch");
    // the host pair must outlive the copy
    ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "tv_flags sync");
    return ADG_OK;
}

int adg_check_finite(adg_mesh* m, void* stream) {
    if (!m) return fail(ADG_EINVAL, "check_finite: NULL mesh");
    if (int rc = set_device(m)) return rc;
    ADG_CK(cudaMemsetAsync(m->flag, 0, sizeof(int), (cudaStream_t)stream), "check_finite memset");
    int e = adg::launch_check_finite(m->u, adg_state_count(m), m->flag, stream);
    if (e) return cuda_fail((cudaError_t)e, "check_finite launch");
    int h = 0;
    ADG_CK(cudaMemcpyAsync(&h, m->flag, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "check_finite copy");
    ADG_CK(cudaStreamSynchronize((cudaStream_t)stream), "check_finite sync");
    return h ? fail(ADG_ENONFINITE, "state contains NaN or Inf") : ADG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// adg_step_noalloc: one FP64 step on a caller-owned state without any device
// allocation.  It serves callers that must not call cudaMalloc: an
// application whose own pool allocator has reserved the device memory, a
// latency-critical loop that cannot afford cudaMalloc's implicit device-wide
// synchronisation, or a plug-in whose host forbids allocator calls after
// start-up.  The scratch the predictor/corrector pair needs (background
// tables, volume residual, face traces) lives in one file-scope device array
// of fixed size; every GPU that loads this library holds it until exit.
// Every call outside stream capture looks the array's device address up again
// (cudaGetSymbolAddress, no synchronisation), so a device reset that reloads
// the module cannot leave a stale address behind; a call on a capturing
// stream uses the address of the last uncaptured call on that device, so the
// first call on a device must come before any stream capture.  All calls
// share the array: calls whose work overlaps on the GPU race.
namespace {

constexpr size_t kNoallocBytes = (size_t)32 << 20;  // ADG_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};
std::mutex g_noalloc_mu;

// isentropic background at node heights and face heights (Eq. 6, reading R7)
__global__ void k_noalloc_background(double* pn, double* rn, double* pf, double* rf, int ny, int n,
                                     adg::Basis B, double y0, double hy, double g, double cp,
                                     double R, double p0, double theta0, int gravity) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int nodes = ny * n;
    if (a < nodes + ny + 1) {
        const double z = a < nodes ? y0 + (a / n + B.xi[a % n]) * hy : y0 + (a - nodes) * hy;
        double p = 0.0, r = 0.0;
        if (gravity) {
            const double ex = 1.0 - g * z / (cp * theta0);
            p = p0 * pow(ex, cp / R);
            r = p / (R * theta0 * ex);
        }
        if (a < nodes) {
            pn[a] = p;
            rn[a] = r;
        } else {
            pf[a - nodes] = p;
            rf[a - nodes] = r;
        }
    }
}

}  // namespace

extern "C" int adg_step_noalloc(const adg_mesh_desc* d, double* u, size_t count, double dt, void* stream) {
    if (!d || !u) return fail(ADG_EINVAL, "step_noalloc: NULL argument");
    if (d->degree < 1 || d->degree > ADG_MAX_DEGREE)
        return fail(ADG_EINVAL, "step_noalloc: degree must be in [1, 7]");
    if (d->nx < 1 || d->ny < 1 || !(d->Lx > 0.0) || !(d->Ly > 0.0))
        return fail(ADG_EINVAL, "step_noalloc: bad mesh size");
    if (d->bc_x < 0 || d->bc_x > 1 || d->bc_y < 0 || d->bc_y > 1)
        return fail(ADG_EINVAL, "step_noalloc: unknown boundary condition");
    if (!(d->gamma > 1.0) || !(d->R > 0.0) || !(d->Pr > 0.0) || !(d->mu >= 0.0))
        return fail(ADG_EINVAL, "step_noalloc: invalid gas constants");
    if (d->source != ADG_SRC_NONE && !(d->source == ADG_SRC_STEADY && d->src_L > 0.0))
        return fail(ADG_EINVAL, "step_noalloc: unknown source");
    if (d->gravity && !(d->theta0 > 0.0 && d->p0 > 0.0))
        return fail(ADG_EINVAL, "step_noalloc: gravity needs theta0 > 0 and p0 > 0");
    if (d->precision != ADG_PREC_FP64) return fail(ADG_EUNSUPPORTED, "step_noalloc: FP64 precision only");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADG_EINVAL, "step_noalloc: dt must be finite and > 0");
    if (d->device < 0 || d->device >= kNoallocMaxDevices) return fail(ADG_EINVAL, "step_noalloc: bad device ordinal");
    if (d->max_levels != 0) return fail(ADG_EUNSUPPORTED, "step_noalloc: uniform meshes only (max_levels must be 0)");
    if ((long long)d->nx * d->ny > (1LL << 26)) return fail(ADG_EINVAL, "step_noalloc: more than 2^26 cells");

    const int N = d->degree, n = N + 1;
    const size_t cells = (size_t)d->nx * d->ny;
    const size_t nbg = 2 * (size_t)d->ny * n + 2 * (size_t)(d->ny + 1);
    const size_t cnt = cells * n * n * 4;
    if (count != cnt) return fail(ADG_EINVAL, "step_noalloc: count != nx*ny*(N+1)^2*4");
    const size_t ntr = cells * 4 * adg::kTraceComps * n;
    auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t need = up256(nbg * 8) + up256(cnt * 8) + up256(ntr * 8);
    if (need > kNoallocBytes) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "step_noalloc: mesh needs %zu bytes of scratch, the static limit is %zu bytes "
                      "(ADG_NOALLOC_SCRATCH_BYTES)", need, kNoallocBytes);
        return fail(ADG_EINVAL, msg);
    }

    // the caller's current device is restored on every return
    int prev_dev = 0;
    ADG_CK(cudaGetDevice(&prev_dev), "step_noalloc: cudaGetDevice");
    struct DeviceRestore {
        int dev;
        ~DeviceRestore() { cudaSetDevice(dev); }
    } restore{prev_dev};
    ADG_CK(cudaSetDevice(d->device), "step_noalloc: cudaSetDevice");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ADG_CK(cudaStreamIsCapturing((cudaStream_t)stream, &cap), "step_noalloc: cudaStreamIsCapturing");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (cap == cudaStreamCaptureStatusNone) {  // look the address up (again): valid after a device reset
            void* p = nullptr;
            ADG_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch), "step_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[d->device] = p;
        } else if (!g_noalloc_ptr[d->device]) {
            return fail(ADG_ESTATE, "step_noalloc: the first call on a device must come before stream capture");
        }
        base = g_noalloc_ptr[d->device];
    }

    adg::Basis B;
    if (!build_basis(N, B)) return fail(ADG_EINVAL, "step_noalloc: singular time-stiffness matrix");
    adg::Phys P;
    std::memset(&P, 0, sizeof(P));
    P.gamma = d->gamma;
    P.gm1 = d->gamma - 1.0;
    P.R = d->R;
    P.invR = 1.0 / d->R;
    P.mu = d->mu;
    P.cp = d->gamma * d->R / (d->gamma - 1.0);
    P.kappa = d->mu * P.cp / d->Pr;
    P.g = d->g;
    P.p0 = d->p0;
    P.theta0 = d->theta0;
    P.Rcp = d->R / P.cp;
    P.lamv = std::fmax(4.0 / 3.0, d->gamma / d->Pr) * d->mu;
    P.hx = d->Lx / d->nx;
    P.hy = d->Ly / d->ny;
    P.inv_hx = 1.0 / P.hx;
    P.inv_hy = 1.0 / P.hy;
    P.x0 = d->x0;
    P.y0 = d->y0;
    P.eta_x = (2.0 * N + 1.0) / (P.hx * std::sqrt(M_PI / 2.0));
    P.eta_y = (2.0 * N + 1.0) / (P.hy * std::sqrt(M_PI / 2.0));
    P.gravity = d->gravity ? 1 : 0;
    P.source = d->source;
    P.sa = d->src_a;
    P.sL = d->src_L;
    P.sU = d->src_U;
    P.sp = d->src_p;
    P.nx = d->nx;
    P.ny = d->ny;
    P.bc_x = d->bc_x;
    P.bc_y = d->bc_y;

    // scratch layout: background tables | rvol | trace (every entry is written
    // before it is read, so nothing needs clearing between calls)
    unsigned char* s = (unsigned char*)base;
    double* pn = (double*)s;
    double* rn = pn + (size_t)d->ny * n;
    double* pf = rn + (size_t)d->ny * n;
    double* rf = pf + (d->ny + 1);
    double* rvol = (double*)(s + up256(nbg * 8));
    double* trace = (double*)(s + up256(nbg * 8) + up256(cnt * 8));
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((nbg / 2 + 255) / 256);
    k_noalloc_background<<<nb, 256, 0, st>>>(pn, rn, pf, rf, d->ny, n, B, d->y0, P.hy, d->g, P.cp, d->R,
                                             d->p0, d->theta0, P.gravity);
    ADG_CK(cudaGetLastError(), "step_noalloc: background launch");
    adg::Background bg{pn, rn, pf, rf};
    int e = adg::launch_predictor_fp64(N, u, rvol, trace, (int)cells, dt, 0.0, B, P, bg, stream);
    if (e) return cuda_fail((cudaError_t)e, "step_noalloc: predictor launch");
    e = adg::launch_corrector_fp64(N, u, rvol, trace, (int)cells, dt, B, P, bg, stream);
    if (e) return cuda_fail((cudaError_t)e, "step_noalloc: corrector launch");
    return ADG_OK;
}

// ---------------------------------------------------------------------------
// Batched persistent step: many independent mixed-precision meshes --
// uniform instances of different sizes and adaptive ones with leaves of every
// level -- advanced by one predictor and one corrector launch per step, each a
// persistent grid walking a static tile list; nsteps steps are captured once
// into a CUDA graph and replayed.  The tile size (cells per block) of the
// predictor is chosen by timing the candidates on the batch itself, and the
// choice is kept in a JSON cache keyed by degree, precision and SM count.
struct adg_batch {
    int device = 0, N = 0, k = 0;
    int precision = ADG_PREC_MIXED;         // of every member
    std::vector<adg_mesh*> meshes;
    std::vector<int> slot;                  // mesh -> index in its kind's table (uniform or adaptive)
    std::vector<unsigned> epoch;            // mesh epochs the tables were built for
    std::vector<adg::MixedInst> host_insts;
    std::vector<adg::AmrInst> host_ainsts;
    std::vector<adg::Fp64Inst> host_finsts;
    adg::MixedInst* insts = nullptr;
    adg::Fp64Inst* finsts = nullptr;
    adg::AmrInst* ainsts = nullptr;
    const void* ops = nullptr;              // prolongation/restriction of the adaptive instances
    adg::BatchTile* tiles_pred = nullptr;
    adg::BatchTile* tiles_corr = nullptr;
    int ntiles_pred = 0, ntiles_corr = 0;
    int cand_pred = 1, cand_corr = 1;
    int cpb_pred = 0, cpb_corr = 0, blocks_pred = 0, blocks_corr = 0;
    long long cells = 0;
    std::vector<double> last_dt;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int graph_steps = 0;
    double tune_ms[adg::kBatchCandidates] = {0, 0, 0, 0};
    int tune_source = 0;                    // 0: timed now, 1: in-process cache, 2: JSON cache file
};

namespace {

std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune_cache;  // key -> candidate
bool g_tune_file_read = false;

// The JSON tuner cache: $ADG_TUNE_CACHE if set (an empty value disables the
// file), else tune_cache.json beside libaderdg.so.  One entry per line,
//   {"key": "<degree, precision, SM count, problem-size bucket>", "candidate": c},
// inside a JSON array; a missing or unreadable file is an empty cache.
std::string tune_cache_path() {
    if (const char* env = std::getenv("ADG_TUNE_CACHE")) return env;
    Dl_info info;
    if (dladdr((void*)&tune_cache_path, &info) && info.dli_fname) {
        std::string f(info.dli_fname);
        const size_t slash = f.rfind('/');
        return (slash == std::string::npos ? std::string(".") : f.substr(0, slash)) + "/tune_cache.json";
    }
    return "";
}

void read_tune_file() {  // caller holds g_tune_mu
    g_tune_file_read = true;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        const char* k = std::strstr(line, "\"key\": \"");
        const char* c = std::strstr(line, "\"candidate\": ");
        if (!k || !c) continue;
        k += 8;
        const char* e = std::strchr(k, '"');
        int cand = -1;
        if (!e || std::sscanf(c + 13, "%d", &cand) != 1 || cand < 0 || cand >= adg::kBatchCandidates) continue;
        const std::string key(k, e - k);
        bool have = false;
        for (auto& kv : g_tune_cache) have = have || kv.first == key;
        if (!have) g_tune_cache.push_back({key, cand});
    }
    std::fclose(f);
}

void write_tune_file() {  // caller holds g_tune_mu; best effort (a read-only location keeps the cache in memory)
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "[\n");
    for (size_t i = 0; i < g_tune_cache.size(); ++i)
        std::fprintf(f, "  {\"key\": \"%s\", \"candidate\": %d}%s\n", g_tune_cache[i].first.c_str(),
                     g_tune_cache[i].second, i + 1 < g_tune_cache.size() ? "," : "");
    std::fprintf(f, "]\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

std::vector<adg::BatchTile> make_tiles(const adg_batch* b, int cpb) {
    std::vector<adg::BatchTile> t;
    for (int a = 0; a < b->k; ++a) {
        const adg_mesh* m = b->meshes[a];
        const int id = m->amr ? -b->slot[a] - 1 : b->slot[a];
        for (int c = 0; c < m->cells; c += cpb) t.push_back({id, c});
    }
    return t;
}

void drop_graph(adg_batch* b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_steps = 0;
}

void free_batch(adg_batch* b) {
    if (!b) return;
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->insts);
    cudaFree(b->ainsts);
    cudaFree(b->finsts);
    cudaFree(b->tiles_pred);
    cudaFree(b->tiles_corr);
    delete b;
}

int launch_phase(adg_batch* b, int cand, int phase, const adg::BatchTile* tiles, int ntiles, int* cpb, int* blocks,
                 cudaStream_t s) {
    if (b->precision == ADG_PREC_FP64)
        return adg::launch_batch_fp64(b->N, phase, b->finsts, tiles, ntiles, b->meshes[0]->B, cpb, blocks, s);
    return adg::launch_batch_mixed(b->N, cand, phase, b->insts, b->host_ainsts.empty() ? nullptr : b->ainsts, tiles,
                                   ntiles, b->meshes[0]->Bf, b->meshes[0]->B, b->ops, cpb, blocks, s);
}

int upload_tiles(adg_batch* b, int cand, int phase, adg::BatchTile** dst, int* ntiles, int* cpb, int* blocks) {
    int c = 0, bl = 0;
    int e = launch_phase(b, cand, phase, nullptr, 0, &c, &bl, nullptr);
    if (e) return cuda_fail((cudaError_t)e, "batch: query");
    std::vector<adg::BatchTile> t = make_tiles(b, c);
    cudaFree(*dst);
    *dst = nullptr;
    if (cudaMalloc(dst, t.size() * sizeof(adg::BatchTile)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "batch: tile list");
    }
    ADG_CK(cudaMemcpy(*dst, t.data(), t.size() * sizeof(adg::BatchTile), cudaMemcpyHostToDevice), "batch: tiles");
    *ntiles = (int)t.size();
    *cpb = c;
    *blocks = bl;
    return ADG_OK;
}

// (Re)build the instance tables from the meshes' current buffers and leaf
// counts (after an adaptation of a member the state moved and the leaf count
// changed); dt values are kept.
int build_instances(adg_batch* b) {
    b->host_insts.clear();
    b->host_ainsts.clear();
    b->host_finsts.clear();
    b->cells = 0;
    for (int a = 0; a < b->k; ++a) {
        adg_mesh* m = b->meshes[a];
        const double dt = b->last_dt[a] > 0.0 ? b->last_dt[a] : 0.0;
        if (b->precision == ADG_PREC_FP64) {
            adg::Fp64Inst I;
            I.u = m->u;
            I.rvol = m->rvol;
            I.trace = m->trace;
            I.cells = m->cells;
            I.dt = dt;
            I.P = m->P;
            I.bg = m->bg;
            b->slot[a] = (int)b->host_finsts.size();
            b->host_finsts.push_back(I);
        } else if (m->amr) {
            adg::AmrInst I;
            I.u = m->u;
            I.rvol = m->rvol;
            I.trace = m->trace;
            I.cells = m->cells;
            I.dt = dt;
            I.dtf = (float)dt;
            I.Pf = m->Pf;
            I.P = m->P;
            I.geo = m->geo;
            I.nbr = m->nbr;
            I.bgl = m->bgl;
            I.mb64 = m->mbl64;
            I.mbf = m->mblf;
            b->slot[a] = (int)b->host_ainsts.size();
            b->host_ainsts.push_back(I);
            b->ops = adg::amr_ops(m);
        } else {
            adg::MixedInst I;
            I.u = m->u;
            I.rvol = (float*)m->rvol;
            I.trace = (float*)m->trace;
            I.cells = m->cells;
            I.dt = dt;
            I.dtf = (float)dt;
            I.P = m->Pf;
            I.bg = m->mbg;
            b->slot[a] = (int)b->host_insts.size();
            b->host_insts.push_back(I);
        }
        b->epoch[a] = m->epoch;
        b->cells += m->cells;
    }
    cudaFree(b->insts);
    cudaFree(b->ainsts);
    cudaFree(b->finsts);
    b->insts = nullptr;
    b->ainsts = nullptr;
    b->finsts = nullptr;
    const size_t nu = std::max<size_t>(1, b->host_insts.size()), na = std::max<size_t>(1, b->host_ainsts.size());
    const size_t nf = std::max<size_t>(1, b->host_finsts.size());
    if (cudaMalloc(&b->insts, nu * sizeof(adg::MixedInst)) != cudaSuccess ||
        cudaMalloc(&b->ainsts, na * sizeof(adg::AmrInst)) != cudaSuccess ||
        cudaMalloc(&b->finsts, nf * sizeof(adg::Fp64Inst)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ADG_ENOMEM, "batch: instance tables");
    }
    if (!b->host_insts.empty())
        ADG_CK(cudaMemcpy(b->insts, b->host_insts.data(), b->host_insts.size() * sizeof(adg::MixedInst),
                          cudaMemcpyHostToDevice), "batch: instance table");
    if (!b->host_ainsts.empty())
        ADG_CK(cudaMemcpy(b->ainsts, b->host_ainsts.data(), b->host_ainsts.size() * sizeof(adg::AmrInst),
                          cudaMemcpyHostToDevice), "batch: adaptive instance table");
    if (!b->host_finsts.empty())
        ADG_CK(cudaMemcpy(b->finsts, b->host_finsts.data(), b->host_finsts.size() * sizeof(adg::Fp64Inst),
                          cudaMemcpyHostToDevice), "batch: FP64 instance table");
    return ADG_OK;
}

}  // namespace

extern "C" int adg_batch_create(adg_mesh* const* meshes, int k, adg_batch** out) {
    if (!meshes || !out || k < 1) return fail(ADG_EINVAL, "batch_create: need k >= 1 meshes");
    *out = nullptr;
    for (int a = 0; a < k; ++a) {
        if (!meshes[a]) return fail(ADG_EINVAL, "batch_create: NULL mesh");
        if (meshes[a]->N != meshes[0]->N || meshes[a]->d.device != meshes[0]->d.device)
            return fail(ADG_EINVAL, "batch_create: meshes must share degree and device");
        const adg_mesh* m = meshes[a];
        if (m->d.precision != meshes[0]->d.precision)
            return fail(ADG_EINVAL, "batch_create: meshes must share the precision");
        if (m->d.precision == ADG_PREC_FP64) {
            // uniform FP64 members: the graph replays fixed arguments, so no
            // time-dependent source or boundary data, and no strip exchange
            if (m->amr) return fail(ADG_EUNSUPPORTED, "batch_create: FP64 members must be uniform meshes");
            if (m->d.source == ADG_SRC_PAPER || m->d.bc_x == ADG_BC_ANALYTIC || m->d.bc_y == ADG_BC_ANALYTIC)
                return fail(ADG_EUNSUPPORTED, "batch_create: no time-dependent source or boundary in a batch");
            if (m->bg.halo_s || m->bg.halo_n)
                return fail(ADG_EUNSUPPORTED, "batch_create: strip-exchange meshes cannot be batched");
        } else if (m->d.precision != ADG_PREC_MIXED) {
            return fail(ADG_EUNSUPPORTED, "batch_create: batched launch is built for ADG_PREC_MIXED and FP64 meshes");
        }
        for (int c = 0; c < a; ++c)
            if (meshes[c] == meshes[a]) return fail(ADG_EINVAL, "batch_create: a mesh appears twice");
    }
    adg_batch* b = new adg_batch();
    b->device = meshes[0]->d.device;
    b->precision = meshes[0]->d.precision;
    b->N = meshes[0]->N;
    b->k = k;
    b->meshes.assign(meshes, meshes + k);
    b->last_dt.assign(k, -1.0);
    b->slot.assign(k, 0);
    b->epoch.assign(k, 0);
    if (int rc = set_device(meshes[0])) { delete b; return rc; }
    if (int rc = build_instances(b)) { free_batch(b); return rc; }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        free_batch(b);
        return cuda_fail(e, "batch_create: setup");
    }
    if (b->precision == ADG_PREC_FP64) {  // one tile size (the per-mesh cells per block)
        b->cand_pred = b->cand_corr = 0;
        int rc = upload_tiles(b, 0, 0, &b->tiles_pred, &b->ntiles_pred, &b->cpb_pred, &b->blocks_pred);
        if (!rc) rc = upload_tiles(b, 0, 1, &b->tiles_corr, &b->ntiles_corr, &b->cpb_corr, &b->blocks_corr);
        if (rc) { free_batch(b); return rc; }
        *out = b;
        return ADG_OK;
    }
    // autotune the predictor tile size (the predictor only reads the state)
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    int bucket = 0;
    for (long long c = b->cells; c > 1; c >>= 1) ++bucket;
    char keybuf[128];
    std::snprintf(keybuf, sizeof(keybuf), "degree=%d precision=mixed sms=%d cells~2^%d candidates=%d%s", b->N, sms,
                  bucket, adg::kBatchCandidates,
                  b->host_ainsts.empty() ? "" : " adaptive");
    const std::string key(keybuf);
    int best = -1;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (!g_tune_file_read) read_tune_file();
        for (auto& kv : g_tune_cache)
            if (kv.first == key) best = kv.second;
    }
    b->tune_source = best >= 0 ? 2 : 0;
    if (best < 0) {
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int c = 0; c < adg::kBatchCandidates; ++c) {
            int rc = upload_tiles(b, c, 0, &b->tiles_pred, &b->ntiles_pred, &b->cpb_pred, &b->blocks_pred);
            if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); free_batch(b); return rc; }
            int e = launch_phase(b, c, 0, b->tiles_pred, b->ntiles_pred, nullptr, &b->blocks_pred, b->cap);  // warm-up
            cudaEventRecord(e0, b->cap);
            for (int r = 0; r < 3 && !e; ++r)
                e = launch_phase(b, c, 0, b->tiles_pred, b->ntiles_pred, nullptr, &b->blocks_pred, b->cap);
            cudaEventRecord(e1, b->cap);
            if (e || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                free_batch(b);
                return cuda_fail(e ? (cudaError_t)e : cudaGetLastError(), "batch_create: autotune");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            b->tune_ms[c] = ms / 3.0;
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        bool have = false;
        for (auto& kv : g_tune_cache) have = have || kv.first == key;
        if (!have) {
            g_tune_cache.push_back({key, best});
            write_tune_file();
        }
    }
    b->cand_pred = best;
    int rc = upload_tiles(b, b->cand_pred, 0, &b->tiles_pred, &b->ntiles_pred, &b->cpb_pred, &b->blocks_pred);
    if (!rc) rc = upload_tiles(b, b->cand_corr, 1, &b->tiles_corr, &b->ntiles_corr, &b->cpb_corr, &b->blocks_corr);
    if (rc) { free_batch(b); return rc; }
    *out = b;
    return ADG_OK;
}

extern "C" int adg_batch_info(const adg_batch* b, int* info, int n) {
    if (!b || !info || n < 1) return fail(ADG_EINVAL, "batch_info: NULL argument");
    const int v[13] = {b->ntiles_pred, b->cpb_pred, b->blocks_pred, b->ntiles_corr, b->cpb_corr, b->blocks_corr,
                       (int)(b->tune_ms[0] * 1e6), (int)(b->tune_ms[1] * 1e6), (int)(b->tune_ms[2] * 1e6),
                       b->cand_pred, b->tune_source, (int)b->host_ainsts.size(), (int)(b->tune_ms[3] * 1e6)};
    for (int a = 0; a < n && a < 13; ++a) info[a] = v[a];
    return ADG_OK;
}

extern "C" int adg_batch_set_candidate(adg_batch* b, int cand) {
    if (!b) return fail(ADG_EINVAL, "batch_set_candidate: NULL batch");
    if (cand < 0 || cand >= adg::kBatchCandidates) return fail(ADG_EINVAL, "batch_set_candidate: candidate not in 0..3");
    if (b->precision == ADG_PREC_FP64)
        return fail(ADG_EUNSUPPORTED, "batch_set_candidate: FP64 batches have one tile size");
    ADG_CK(cudaSetDevice(b->device), "batch_set_candidate: cudaSetDevice");
    ADG_CK(cudaDeviceSynchronize(), "batch_set_candidate: synchronise");
    drop_graph(b);
    b->cand_pred = cand;
    return upload_tiles(b, cand, 0, &b->tiles_pred, &b->ntiles_pred, &b->cpb_pred, &b->blocks_pred);
}

extern "C" int adg_batch_step(adg_batch* b, const double* dt, int nsteps, void* stream) {
    if (!b || !dt) return fail(ADG_EINVAL, "batch_step: NULL argument");
    if (nsteps < 1) return fail(ADG_EINVAL, "batch_step: nsteps must be >= 1");
    for (int a = 0; a < b->k; ++a)
        if (!(dt[a] > 0.0) || !std::isfinite(dt[a])) return fail(ADG_EINVAL, "batch_step: dt must be finite and > 0");
    ADG_CK(cudaSetDevice(b->device), "batch_step: cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    bool moved = false;
    for (int a = 0; a < b->k; ++a) moved = moved || b->epoch[a] != b->meshes[a]->epoch;
    if (moved) {
        // a member adapted: its state moved and its leaf count changed; rebuild the
        // tables and tile lists and capture the graph again (the previous graph may
        // still be running on another stream: wait for the device first)
        ADG_CK(cudaDeviceSynchronize(), "batch_step: synchronise before rebuild");
        drop_graph(b);
        if (int rc = build_instances(b)) return rc;
        int rc = upload_tiles(b, b->cand_pred, 0, &b->tiles_pred, &b->ntiles_pred, &b->cpb_pred, &b->blocks_pred);
        if (!rc) rc = upload_tiles(b, b->cand_corr, 1, &b->tiles_corr, &b->ntiles_corr, &b->cpb_corr, &b->blocks_corr);
        if (rc) return rc;
    }
    bool changed = false;
    for (int a = 0; a < b->k; ++a)
        if (dt[a] != b->last_dt[a]) {
            changed = true;
            b->last_dt[a] = dt[a];
            if (b->precision == ADG_PREC_FP64) {
                b->host_finsts[b->slot[a]].dt = dt[a];
            } else if (b->meshes[a]->amr) {
                b->host_ainsts[b->slot[a]].dt = dt[a];
                b->host_ainsts[b->slot[a]].dtf = (float)dt[a];
            } else {
                b->host_insts[b->slot[a]].dt = dt[a];
                b->host_insts[b->slot[a]].dtf = (float)dt[a];
            }
        }
    if (changed) {
        if (!b->host_insts.empty())
            ADG_CK(cudaMemcpyAsync(b->insts, b->host_insts.data(), b->host_insts.size() * sizeof(adg::MixedInst),
                                   cudaMemcpyHostToDevice, s), "batch_step: dt upload");
        if (!b->host_ainsts.empty())
            ADG_CK(cudaMemcpyAsync(b->ainsts, b->host_ainsts.data(), b->host_ainsts.size() * sizeof(adg::AmrInst),
                                   cudaMemcpyHostToDevice, s), "batch_step: dt upload");
        if (!b->host_finsts.empty())
            ADG_CK(cudaMemcpyAsync(b->finsts, b->host_finsts.data(), b->host_finsts.size() * sizeof(adg::Fp64Inst),
                                   cudaMemcpyHostToDevice, s), "batch_step: dt upload");
        // the staging vectors must stay valid until the copies have run
        ADG_CK(cudaStreamSynchronize(s), "batch_step: dt upload sync");
    }
    if (!b->exec || b->graph_steps != nsteps) {
        drop_graph(b);
        ADG_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batch_step: begin capture");
        int e = 0;
        for (int st = 0; st < nsteps && !e; ++st) {
            e = launch_phase(b, b->cand_pred, 0, b->tiles_pred, b->ntiles_pred, nullptr, &b->blocks_pred, b->cap);
            if (!e) e = launch_phase(b, b->cand_corr, 1, b->tiles_corr, b->ntiles_corr, nullptr, &b->blocks_corr, b->cap);
        }
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
        if (e) { if (g) cudaGraphDestroy(g); return cuda_fail((cudaError_t)e, "batch_step: capture launch"); }
        if (ce != cudaSuccess) return cuda_fail(ce, "batch_step: end capture");
        b->graph = g;
        ADG_CK(cudaGraphInstantiate(&b->exec, g, 0), "batch_step: instantiate");
        b->graph_steps = nsteps;
    }
    ADG_CK(cudaGraphLaunch(b->exec, s), "batch_step: graph launch");
    for (int a = 0; a < b->k; ++a) {
        b->meshes[a]->t += nsteps * dt[a];
        b->meshes[a]->predicted = false;
    }
    return ADG_OK;
}

extern "C" void adg_batch_destroy(adg_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
}
