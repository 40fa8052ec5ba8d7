// FP32 point-wise physics on perturbation variables, shared by the mixed-
// precision predictors of uniform meshes (adg_mixed.cu) and adaptive meshes
// (adg_amr.cu): the flux of Sec. 2 (Eqs. 1-7) from q' = (rho - rhobar, rho u,
// rho v, rhoE - Ebar) with p' = (gamma-1)(rhoE' - |rho v|^2/(2 rho) - g z rho')
// formed by exact algebra, and the Rusanov speed.
#pragma once
#include "adg_internal.h"

namespace adg {

struct FluxF {
    float F[4], G[4], S[4];
};

// Point-wise flux from perturbation variables qp (rho', m, m, E'), full
// gradients (gx, gy), background (rb, Eb, pb) at height z.
__device__ __forceinline__ void ns_flux_pert(const float qp[4], const float gx[4], const float gy[4],
                                             float z, float rb, float Eb, float pb, const PhysF& P,
                                             FluxF& o, bool use_heat = false, float hTy = 0.f) {
    const float rho = rb + qp[0];
    const float mx = qp[1], my = qp[2];
    const float rinv = __frcp_rn(rho);
    const float u = mx * rinv, v = my * rinv;
    const float gz = P.g * z;
    const float pp = P.gm1 * (qp[3] - 0.5f * (mx * u + my * v) - gz * qp[0]);
    const float p = pb + pp;
    const float E = Eb + qp[3];
    const float T = p * rinv * P.invR;
    const float ux = (gx[1] - u * gx[0]) * rinv;
    const float uy = (gy[1] - u * gy[0]) * rinv;
    const float vx = (gx[2] - v * gx[0]) * rinv;
    const float vy = (gy[2] - v * gy[0]) * rinv;
    const float kin = 0.5f * (u * u + v * v);
    float Tx, Ty;
    if (use_heat) {
        Tx = 0.f;
        Ty = hTy;
    } else {
        const float px = P.gm1 * (gx[3] - (u * gx[1] + v * gx[2]) + kin * gx[0] - gz * gx[0]);
        const float py = P.gm1 * (gy[3] - (u * gy[1] + v * gy[2]) + kin * gy[0] - gz * gy[0] - rho * P.g);
        Tx = (px - P.R * T * gx[0]) * rinv * P.invR;
        Ty = (py - P.R * T * gy[0]) * rinv * P.invR;
    }
    const float div = ux + vy;
    const float sxx = P.mu * ((2.f / 3.f) * div - 2.f * ux);
    const float syy = P.mu * ((2.f / 3.f) * div - 2.f * vy);
    const float sxy = -P.mu * (uy + vx);
    const float Ep = E + p;
    o.F[0] = mx;
    o.F[1] = mx * u + pp + sxx;
    o.F[2] = my * u + sxy;
    o.F[3] = u * Ep + u * sxx + v * sxy - P.kappa * Tx;
    o.G[0] = my;
    o.G[1] = mx * v + sxy;
    o.G[2] = my * v + pp + syy;
    o.G[3] = v * Ep + u * sxy + v * syy - P.kappa * Ty;
    o.S[0] = 0.f;
    o.S[1] = 0.f;
    o.S[2] = -P.g * qp[0];
    o.S[3] = 0.f;
}

__device__ __forceinline__ float wave_speed_f(float rho, float mx, float my, float pp, float pb,
                                              bool xdir, const PhysF& P) {
    const float rinv = __frcp_rn(rho);
    const float c = sqrtf(P.gamma * (pb + pp) * rinv);
    const float vn = fabsf((xdir ? mx : my) * rinv);
    return vn + c + 2.f * (xdir ? P.eta_x : P.eta_y) * P.lamv * rinv;
}

}  // namespace adg
