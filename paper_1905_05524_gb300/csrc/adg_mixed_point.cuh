// FP32 point-wise physics on perturbation variables, shared by the mixed-
// precision predictors of uniform meshes (adg_mixed.cu) and adaptive meshes
// (adg_amr.cu): the flux of Sec. 2 (Eqs. 1-7) from q' = (rho - rhobar, rho u,
// rho v, rhoE - Ebar) with p' = (gamma-1)(rhoE' - |rho v|^2/(2 rho) - g z rho')
// formed by exact algebra (one node, or two time slices of one node in
// packed FP32x2), and the Rusanov speed.
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

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (sm_100 and later): one instruction works on two
// FP32 lanes, each rounded like its scalar counterpart.  The predictor runs
// the point-wise flux on two time slices at once and keeps the slices in
// pairs through its contractions.
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fnma2(float2 a, float2 b, float2 c) {  // c - a b
    return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}
// approximate reciprocal (hardware rcp, relative error ~2^-23); rho is O(1)
// and never subnormal, so flushing subnormals changes nothing
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct FluxF2 {
    float2 F[4], G[4], S2;  // S2: the only non-zero physical source, -g rho' (z-momentum)
};

// ns_flux_pert on a pair of time slices at one node (the interior form:
// gradients of T from the state, no wall heat flux).
__device__ __forceinline__ void ns_flux_pert2(const float2 qp[4], const float2 gx[4], const float2 gy[4],
                                              float z, float rb, float Eb, float pb, const PhysF& P,
                                              FluxF2& o) {
    const float2 rho = add2(bc2(rb), qp[0]);
    const float2 mx = qp[1], my = qp[2];
    const float2 rinv = make_float2(rcp_fast(rho.x), rcp_fast(rho.y));
    const float2 u = mul2(mx, rinv), v = mul2(my, rinv);
    const float gz = P.g * z;
    // p' = (gamma-1) (E' - (mx u + my v)/2 - g z rho')
    const float2 m2 = fma2(my, v, mul2(mx, u));
    const float2 pp = mul2(bc2(P.gm1), fma2(bc2(-gz), qp[0], fma2(bc2(-0.5f), m2, qp[3])));
    const float2 p = add2(bc2(pb), pp);
    const float2 E = add2(bc2(Eb), qp[3]);
    const float2 T = mul2(mul2(p, rinv), bc2(P.invR));
    const float2 ux = mul2(fnma2(u, gx[0], gx[1]), rinv);
    const float2 uy = mul2(fnma2(u, gy[0], gy[1]), rinv);
    const float2 vx = mul2(fnma2(v, gx[0], gx[2]), rinv);
    const float2 vy = mul2(fnma2(v, gy[0], gy[2]), rinv);
    // kin - g z, the common factor of the density gradient in grad p
    const float2 kg = fma2(bc2(0.5f), fma2(v, v, mul2(u, u)), bc2(-gz));
    const float2 px = mul2(bc2(P.gm1), fma2(kg, gx[0], fnma2(v, gx[2], fnma2(u, gx[1], gx[3]))));
    const float2 py = mul2(bc2(P.gm1),
                           fnma2(rho, bc2(P.g), fma2(kg, gy[0], fnma2(v, gy[2], fnma2(u, gy[1], gy[3])))));
    const float2 RT = mul2(bc2(P.R), T);
    const float2 ri = mul2(rinv, bc2(P.invR));
    const float2 Tx = mul2(fnma2(RT, gx[0], px), ri);
    const float2 Ty = mul2(fnma2(RT, gy[0], py), ri);
    const float2 div = add2(ux, vy);
    const float2 sxx = mul2(bc2(P.mu), fma2(bc2(2.f / 3.f), div, mul2(bc2(-2.f), ux)));
    const float2 syy = mul2(bc2(P.mu), fma2(bc2(2.f / 3.f), div, mul2(bc2(-2.f), vy)));
    const float2 sxy = mul2(bc2(-P.mu), add2(uy, vx));
    const float2 Ep = add2(E, p);
    o.F[0] = mx;
    o.F[1] = fma2(mx, u, add2(pp, sxx));
    o.F[2] = fma2(my, u, sxy);
    o.F[3] = fma2(bc2(-P.kappa), Tx, fma2(v, sxy, mul2(u, add2(Ep, sxx))));
    o.G[0] = my;
    o.G[1] = fma2(mx, v, sxy);
    o.G[2] = fma2(my, v, add2(pp, syy));
    o.G[3] = fma2(bc2(-P.kappa), Ty, fma2(u, sxy, mul2(v, add2(Ep, syy))));
    o.S2 = mul2(bc2(-P.g), qp[0]);
}

}  // namespace adg
