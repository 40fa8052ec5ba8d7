// Point-wise FP64 physics of the 2D compressible Navier-Stokes system with
// gravity (Sec. 2 of Krenz, Rannabauer, Bader):
//   Eq. 1  F = F^h(Q) + F^v(Q, grad Q), Q = (rho, rho u, rho v, rho E)
//   Eq. 2  p = (gamma-1)(rhoE - 1/2 |rho v|^2 / rho - rho g z)
//   Eq. 3  T = p / (rho R)
//   Eq. 4  sigma = mu ((2/3) div v I - (grad v + grad v^T))
//   Eq. 5  kappa = mu c_p / Pr
//   Eq. 7  momentum flux with p' = p - pbar(z), source -g rho' in the z row
// Gradients of v, p, T follow from grad Q by the chain rule.
#pragma once
#include "adg_internal.h"

namespace adg {

struct Flux4 {
    double F[4], G[4], S[4];
};

// F, G and the physical source S at one point.  heat: if use_heat, (Tx, Ty)
// replaces grad T in the heat flux (slip-wall ghost, Eq. 10).
__device__ __forceinline__ void ns_flux(const double q[4], const double qx[4], const double qy[4],
                                        double z, double pbar, double rhobar, const Phys& P,
                                        Flux4& o, bool use_heat = false, double hTx = 0.0,
                                        double hTy = 0.0) {
    const double rho = q[0], mx = q[1], my = q[2], E = q[3];
    const double rinv = 1.0 / rho;
    const double u = mx * rinv, v = my * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (E - 0.5 * (mx * u + my * v) - rho * gz);
    const double pp = p - pbar;
    const double T = p * rinv * P.invR;
    const double ux = (qx[1] - u * qx[0]) * rinv;
    const double uy = (qy[1] - u * qy[0]) * rinv;
    const double vx = (qx[2] - v * qx[0]) * rinv;
    const double vy = (qy[2] - v * qy[0]) * rinv;
    const double kin = 0.5 * (u * u + v * v);
    const double rg = P.gravity ? rho * P.g : 0.0;
    double Tx, Ty;
    if (use_heat) {
        Tx = hTx;
        Ty = hTy;
    } else {
        const double px = P.gm1 * (qx[3] - (u * qx[1] + v * qx[2]) + kin * qx[0] - gz * qx[0]);
        const double py = P.gm1 * (qy[3] - (u * qy[1] + v * qy[2]) + kin * qy[0] - gz * qy[0] - rg);
        Tx = (px - P.R * T * qx[0]) * rinv * P.invR;
        Ty = (py - P.R * T * qy[0]) * rinv * P.invR;
    }
    const double div = ux + vy;
    const double sxx = P.mu * ((2.0 / 3.0) * div - 2.0 * ux);
    const double syy = P.mu * ((2.0 / 3.0) * div - 2.0 * vy);
    const double sxy = -P.mu * (uy + vx);
    const double Ep = E + p;
    o.F[0] = mx;
    o.F[1] = mx * u + pp + sxx;
    o.F[2] = my * u + sxy;
    o.F[3] = u * Ep + u * sxx + v * sxy - P.kappa * Tx;
    o.G[0] = my;
    o.G[1] = mx * v + sxy;
    o.G[2] = my * v + pp + syy;
    o.G[3] = v * Ep + u * sxy + v * syy - P.kappa * Ty;
    o.S[0] = 0.0;
    o.S[1] = 0.0;
    o.S[2] = P.gravity ? -P.g * (rho - rhobar) : 0.0;
    o.S[3] = 0.0;
}

// Steady manufactured source: rho = 1 + a sin(k s), s = x + y, k = 2 pi / L,
// u = v = U, p = const.  Closed form of dF/dx + dG/dy for that field
// (convective part 2 U a k cos(k s) (1, U, U, U^2) and the heat-conduction
// term -kappa Laplace(T) with T = p / (rho R)).
__device__ __forceinline__ void steady_source(double x, double y, const Phys& P, double S[4]) {
    const double k = 2.0 * 3.14159265358979323846 / P.sL;
    double sn, cs;
    sincos(k * (x + y), &sn, &cs);
    const double a = P.sa, U = P.sU;
    const double rho = 1.0 + a * sn;
    const double c = 2.0 * U * a * k * cs;
    const double lapT = (2.0 * P.sp * P.invR) * (a * k * k * sn / (rho * rho) +
                                                 2.0 * a * a * k * k * cs * cs / (rho * rho * rho));
    S[0] = c;
    S[1] = c * U;
    S[2] = c * U;
    S[3] = c * U * U - P.kappa * lapT;
}

// Rusanov speed |v.n| + c + 2 eta lambda_v of a face state (normal along x
// if xdir, else along y), lambda_v = max(4/3, gamma/Pr) mu / rho.
__device__ __forceinline__ double wave_speed(const double q[4], double z, bool xdir, const Phys& P) {
    const double rinv = 1.0 / q[0];
    const double u = q[1] * rinv, v = q[2] * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v) - q[0] * gz);
    const double c = sqrt(P.gamma * p * rinv);
    const double vn = xdir ? fabs(u) : fabs(v);
    const double eta = xdir ? P.eta_x : P.eta_y;
    return vn + c + 2.0 * eta * P.lamv * rinv;
}

// Numerical flux (F_L + F_R)/2 - max(s_L, s_R) (q_R - q_L)/2, written with
// explicit round-to-nearest intrinsics so that both cells sharing a face
// obtain the bitwise-identical value (exact conservation).
__device__ __forceinline__ void rusanov(const double qL[4], const double fL[4], double sL,
                                        const double qR[4], const double fR[4], double sR,
                                        double out[4]) {
    const double s = fmax(sL, sR);
    const double hs = __dmul_rn(-0.5, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double avg = __dmul_rn(0.5, __dadd_rn(fL[v], fR[v]));
        out[v] = __fma_rn(hs, __dsub_rn(qR[v], qL[v]), avg);
    }
}

}  // namespace adg

namespace adg {

// Reverse (adjoint) of ns_flux: given the adjoints Fb, Gb, Sb of its outputs
// at the point (q, qx, qy), accumulate the adjoints of q, qx, qy.  With
// use_heat the heat-flux gradient is a constant (wall ghost) and carries no
// adjoint to qx, qy.  Written line by line against ns_flux above.
__device__ __forceinline__ void ns_flux_adj(const double q[4], const double qx[4], const double qy[4],
                                            double z, const Phys& P, const double Fb[4], const double Gb[4],
                                            const double Sb[4], double qb[4], double qxb[4], double qyb[4],
                                            bool use_heat = false) {
    // ---- forward recompute
    const double rho = q[0], mx = q[1], my = q[2], E = q[3];
    const double rinv = 1.0 / rho;
    const double u = mx * rinv, v = my * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (E - 0.5 * (mx * u + my * v) - rho * gz);
    const double T = p * rinv * P.invR;
    const double ux = (qx[1] - u * qx[0]) * rinv;
    const double uy = (qy[1] - u * qy[0]) * rinv;
    const double vx = (qx[2] - v * qx[0]) * rinv;
    const double vy = (qy[2] - v * qy[0]) * rinv;
    const double kin = 0.5 * (u * u + v * v);
    double px = 0.0, py = 0.0;
    if (!use_heat) {
        px = P.gm1 * (qx[3] - (u * qx[1] + v * qx[2]) + kin * qx[0] - gz * qx[0]);
        py = P.gm1 * (qy[3] - (u * qy[1] + v * qy[2]) + kin * qy[0] - gz * qy[0] - (P.gravity ? rho * P.g : 0.0));
    }
    const double div = ux + vy;
    const double sxx = P.mu * ((2.0 / 3.0) * div - 2.0 * ux);
    const double syy = P.mu * ((2.0 / 3.0) * div - 2.0 * vy);
    const double sxy = -P.mu * (uy + vx);
    const double Ep = E + p;
    // ---- reverse
    double mx_b = Fb[0] + Fb[1] * u + Gb[1] * v;
    double my_b = Gb[0] + Fb[2] * u + Gb[2] * v;
    double u_b = Fb[1] * mx + Fb[2] * my + Fb[3] * (Ep + sxx) + Gb[3] * sxy;
    double v_b = Fb[3] * sxy + Gb[1] * mx + Gb[2] * my + Gb[3] * (Ep + syy);
    double pp_b = Fb[1] + Gb[2];
    double sxx_b = Fb[1] + Fb[3] * u;
    double syy_b = Gb[2] + Gb[3] * v;
    double sxy_b = Fb[2] + Fb[3] * v + Gb[1] + Gb[3] * u;
    const double Ep_b = Fb[3] * u + Gb[3] * v;
    const double Tx_b = -P.kappa * Fb[3];
    const double Ty_b = -P.kappa * Gb[3];
    double rho_b = P.gravity ? -P.g * Sb[2] : 0.0;
    double E_b = Ep_b;
    double p_b = Ep_b + pp_b;
    double rinv_b = 0.0, T_b = 0.0, kin_b = 0.0;
    // stresses
    const double uy_b = -P.mu * sxy_b;
    const double vx_b = -P.mu * sxy_b;
    const double div_b = P.mu * (2.0 / 3.0) * (sxx_b + syy_b);
    const double ux_b = -2.0 * P.mu * sxx_b + div_b;
    const double vy_b = -2.0 * P.mu * syy_b + div_b;
    // heat flux
    if (!use_heat) {
        const double a = rinv * P.invR;
        const double px_b = Tx_b * a, py_b = Ty_b * a;
        T_b += -P.R * a * (qx[0] * Tx_b + qy[0] * Ty_b);
        qxb[0] += -P.R * T * a * Tx_b;
        qyb[0] += -P.R * T * a * Ty_b;
        rinv_b += P.invR * ((px - P.R * T * qx[0]) * Tx_b + (py - P.R * T * qy[0]) * Ty_b);
        // px, py
        qxb[3] += P.gm1 * px_b;
        qyb[3] += P.gm1 * py_b;
        u_b += -P.gm1 * (qx[1] * px_b + qy[1] * py_b);
        v_b += -P.gm1 * (qx[2] * px_b + qy[2] * py_b);
        qxb[1] += -P.gm1 * u * px_b;
        qyb[1] += -P.gm1 * u * py_b;
        qxb[2] += -P.gm1 * v * px_b;
        qyb[2] += -P.gm1 * v * py_b;
        kin_b += P.gm1 * (qx[0] * px_b + qy[0] * py_b);
        qxb[0] += P.gm1 * (kin - gz) * px_b;
        qyb[0] += P.gm1 * (kin - gz) * py_b;
        if (P.gravity) rho_b += -P.gm1 * P.g * py_b;
    }
    u_b += u * kin_b;
    v_b += v * kin_b;
    // velocity gradients
    qxb[1] += rinv * ux_b;
    u_b += -qx[0] * rinv * ux_b;
    qxb[0] += -u * rinv * ux_b;
    rinv_b += (qx[1] - u * qx[0]) * ux_b;
    qyb[1] += rinv * uy_b;
    u_b += -qy[0] * rinv * uy_b;
    qyb[0] += -u * rinv * uy_b;
    rinv_b += (qy[1] - u * qy[0]) * uy_b;
    qxb[2] += rinv * vx_b;
    v_b += -qx[0] * rinv * vx_b;
    qxb[0] += -v * rinv * vx_b;
    rinv_b += (qx[2] - v * qx[0]) * vx_b;
    qyb[2] += rinv * vy_b;
    v_b += -qy[0] * rinv * vy_b;
    qyb[0] += -v * rinv * vy_b;
    rinv_b += (qy[2] - v * qy[0]) * vy_b;
    // T = p rinv / R
    p_b += rinv * P.invR * T_b;
    rinv_b += p * P.invR * T_b;
    // p = gm1 (E - (mx u + my v)/2 - rho gz)
    E_b += P.gm1 * p_b;
    const double kem_b = -0.5 * P.gm1 * p_b;
    rho_b += -P.gm1 * gz * p_b;
    mx_b += u * kem_b;
    u_b += mx * kem_b;
    my_b += v * kem_b;
    v_b += my * kem_b;
    // u = mx rinv, v = my rinv
    mx_b += rinv * u_b;
    rinv_b += mx * u_b;
    my_b += rinv * v_b;
    rinv_b += my * v_b;
    rho_b += -rinv * rinv * rinv_b;
    qb[0] += rho_b;
    qb[1] += mx_b;
    qb[2] += my_b;
    qb[3] += E_b;
}

// Reverse of wave_speed: accumulate d s / d q * sb into qb.  |v.n| takes the
// sign of v.n (0 at exactly 0).
__device__ __forceinline__ void wave_speed_adj(const double q[4], double z, bool xdir, const Phys& P,
                                               double sb, double qb[4]) {
    const double rinv = 1.0 / q[0];
    const double u = q[1] * rinv, v = q[2] * rinv;
    const double gz = P.gravity ? P.g * z : 0.0;
    const double p = P.gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v) - q[0] * gz);
    const double c = sqrt(P.gamma * p * rinv);
    const double eta = xdir ? P.eta_x : P.eta_y;
    const double vn = xdir ? u : v;
    const double sgn = vn > 0.0 ? 1.0 : (vn < 0.0 ? -1.0 : 0.0);
    double u_b = xdir ? sgn * sb : 0.0;
    double v_b = xdir ? 0.0 : sgn * sb;
    const double c_b = sb;
    double rinv_b = 2.0 * eta * P.lamv * sb;
    const double p_b = P.gamma * rinv / (2.0 * c) * c_b;
    rinv_b += P.gamma * p / (2.0 * c) * c_b;
    qb[3] += P.gm1 * p_b;
    const double kem_b = -0.5 * P.gm1 * p_b;
    qb[0] += -P.gm1 * gz * p_b;
    qb[1] += u * kem_b;
    u_b += q[1] * kem_b;
    qb[2] += v * kem_b;
    v_b += q[2] * kem_b;
    qb[1] += rinv * u_b;
    rinv_b += q[1] * u_b;
    qb[2] += rinv * v_b;
    rinv_b += q[2] * v_b;
    qb[0] += -rinv * rinv * rinv_b;
}

}  // namespace adg

namespace adg {

// ---------------------------------------------------------------------------
// The paper's manufactured solution (Sec. 4.1, Eq. 8) as a source term:
// p = cos(phi)/10 + 1/gamma, rho = sin(phi)/2 + 1, v = (1,1) sin(phi)/4 with
// phi = k (x + y) - 2 pi t, k = 2 pi / L (pi/5 on the paper's [0,10]^2).  All
// fields depend on phi only, so dF/dx = k dF/dphi, dQ/dt = -2 pi dQ/dphi, and
// S = dQ/dt + dF/dx + dG/dy is evaluated exactly by running the point-wise
// flux on first-order dual numbers (value, d/dphi) -- forward-mode
// differentiation of the same flux formula (gravity off).
struct Dd {
    double v, d;
};
__device__ __forceinline__ Dd operator+(Dd a, Dd b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dd operator-(Dd a, Dd b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dd operator-(Dd a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dd operator*(Dd a, Dd b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dd operator*(double s, Dd a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dd operator/(Dd a, Dd b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }

__device__ __forceinline__ void ns_flux_dual(const Dd q[4], const Dd qx[4], const Dd qy[4], const Phys& P, Dd F[4],
                                             Dd G[4]) {
    const Dd rho = q[0], mx = q[1], my = q[2], E = q[3];
    const Dd u = mx / rho, v = my / rho;
    const Dd p = P.gm1 * (E - 0.5 * (mx * u + my * v));
    const Dd T = p / (P.R * rho);
    const Dd ux = (qx[1] - u * qx[0]) / rho, uy = (qy[1] - u * qy[0]) / rho;
    const Dd vx = (qx[2] - v * qx[0]) / rho, vy = (qy[2] - v * qy[0]) / rho;
    const Dd kin = 0.5 * (u * u + v * v);
    const Dd px = P.gm1 * (qx[3] - (u * qx[1] + v * qx[2]) + kin * qx[0]);
    const Dd py = P.gm1 * (qy[3] - (u * qy[1] + v * qy[2]) + kin * qy[0]);
    const Dd Tx = (px - P.R * (T * qx[0])) / (P.R * rho);
    const Dd Ty = (py - P.R * (T * qy[0])) / (P.R * rho);
    const Dd div = ux + vy;
    const Dd sxx = P.mu * ((2.0 / 3.0) * div - 2.0 * ux);
    const Dd syy = P.mu * ((2.0 / 3.0) * div - 2.0 * vy);
    const Dd sxy = -P.mu * (uy + vx);
    const Dd Ep = E + p;
    F[0] = mx;
    F[1] = mx * u + p + sxx;
    F[2] = my * u + sxy;
    F[3] = u * Ep + u * sxx + v * sxy - P.kappa * Tx;
    G[0] = my;
    G[1] = mx * v + sxy;
    G[2] = my * v + p + syy;
    G[3] = v * Ep + u * sxy + v * syy - P.kappa * Ty;
}

// Q(phi) and its first two phi-derivatives for the manufactured field
__device__ __forceinline__ void paper_field(double phi, const Phys& P, double Q[4], double Q1[4], double Q2[4]) {
    double s, c;
    sincos(phi, &s, &c);
    const double r = 1.0 + 0.5 * s, r1 = 0.5 * c, r2 = -0.5 * s;
    const double u = 0.25 * s, u1 = 0.25 * c, u2 = -0.25 * s;  // v = u
    const double p = 0.1 * c + 1.0 / P.gamma, p1 = -0.1 * s, p2 = -0.1 * c;
    const double m = r * u, m1 = r1 * u + r * u1, m2 = r2 * u + 2.0 * r1 * u1 + r * u2;
    const double E = p / P.gm1 + r * u * u;
    const double E1 = p1 / P.gm1 + r1 * u * u + 2.0 * r * u * u1;
    const double E2 = p2 / P.gm1 + r2 * u * u + 4.0 * r1 * u * u1 + 2.0 * r * (u1 * u1 + u * u2);
    Q[0] = r; Q[1] = m; Q[2] = m; Q[3] = E;
    Q1[0] = r1; Q1[1] = m1; Q1[2] = m1; Q1[3] = E1;
    Q2[0] = r2; Q2[1] = m2; Q2[2] = m2; Q2[3] = E2;
}

__device__ __forceinline__ void paper_source(double x, double y, double t, const Phys& P, double S[4]) {
    const double k = 2.0 * 3.14159265358979323846 / P.sL;
    const double phi = k * (x + y) - 2.0 * 3.14159265358979323846 * t;
    double Q[4], Q1[4], Q2[4];
    paper_field(phi, P, Q, Q1, Q2);
    Dd q[4], g[4], F[4], G[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        q[v] = {Q[v], Q1[v]};
        g[v] = {k * Q1[v], k * Q2[v]};
    }
    ns_flux_dual(q, g, g, P, F, G);
#pragma unroll
    for (int v = 0; v < 4; ++v) S[v] = -2.0 * 3.14159265358979323846 * Q1[v] + k * (F[v].d + G[v].d);
}

}  // namespace adg
