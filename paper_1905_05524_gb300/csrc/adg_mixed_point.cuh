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
// gradients (gx, gy), background (rb, Eb, pb) at height z.  Explicit rounding
// throughout: the slip-wall ghost that uses it is inlined into the per-mesh
// and the batched correctors, which must agree bitwise.
__device__ __forceinline__ void ns_flux_pert(const float qp[4], const float gx[4], const float gy[4],
                                             float z, float rb, float Eb, float pb, const PhysF& P,
                                             FluxF& o, bool use_heat = false, float hTy = 0.f) {
    const float rho = __fadd_rn(rb, qp[0]);
    const float mx = qp[1], my = qp[2];
    const float rinv = __frcp_rn(rho);
    const float u = __fmul_rn(mx, rinv), v = __fmul_rn(my, rinv);
    const float gz = __fmul_rn(P.g, z);
    const float m2 = __fmaf_rn(my, v, __fmul_rn(mx, u));
    const float pp = __fmul_rn(P.gm1, __fmaf_rn(-gz, qp[0], __fmaf_rn(-0.5f, m2, qp[3])));
    const float p = __fadd_rn(pb, pp);
    const float E = __fadd_rn(Eb, qp[3]);
    const float T = __fmul_rn(__fmul_rn(p, rinv), P.invR);
    const float ux = __fmul_rn(__fmaf_rn(-u, gx[0], gx[1]), rinv);
    const float uy = __fmul_rn(__fmaf_rn(-u, gy[0], gy[1]), rinv);
    const float vx = __fmul_rn(__fmaf_rn(-v, gx[0], gx[2]), rinv);
    const float vy = __fmul_rn(__fmaf_rn(-v, gy[0], gy[2]), rinv);
    const float kg = __fmaf_rn(0.5f, __fmaf_rn(v, v, __fmul_rn(u, u)), -gz);  // kinetic energy per mass - g z
    float Tx, Ty;
    if (use_heat) {
        Tx = 0.f;
        Ty = hTy;
    } else {
        const float px = __fmul_rn(P.gm1, __fmaf_rn(kg, gx[0], __fmaf_rn(-v, gx[2], __fmaf_rn(-u, gx[1], gx[3]))));
        const float py = __fmul_rn(P.gm1, __fmaf_rn(-rho, P.g, __fmaf_rn(kg, gy[0],
                                                  __fmaf_rn(-v, gy[2], __fmaf_rn(-u, gy[1], gy[3])))));
        const float RT = __fmul_rn(P.R, T), ri = __fmul_rn(rinv, P.invR);
        Tx = __fmul_rn(__fmaf_rn(-RT, gx[0], px), ri);
        Ty = __fmul_rn(__fmaf_rn(-RT, gy[0], py), ri);
    }
    const float div = __fadd_rn(ux, vy);
    const float sxx = __fmul_rn(P.mu, __fmaf_rn(2.f / 3.f, div, __fmul_rn(-2.f, ux)));
    const float syy = __fmul_rn(P.mu, __fmaf_rn(2.f / 3.f, div, __fmul_rn(-2.f, vy)));
    const float sxy = __fmul_rn(-P.mu, __fadd_rn(uy, vx));
    const float Ep = __fadd_rn(E, p);
    o.F[0] = mx;
    o.F[1] = __fmaf_rn(mx, u, __fadd_rn(pp, sxx));
    o.F[2] = __fmaf_rn(my, u, sxy);
    o.F[3] = __fmaf_rn(-P.kappa, Tx, __fmaf_rn(v, sxy, __fmul_rn(u, __fadd_rn(Ep, sxx))));
    o.G[0] = my;
    o.G[1] = __fmaf_rn(mx, v, sxy);
    o.G[2] = __fmaf_rn(my, v, __fadd_rn(pp, syy));
    o.G[3] = __fmaf_rn(-P.kappa, Ty, __fmaf_rn(u, sxy, __fmul_rn(v, __fadd_rn(Ep, syy))));
    o.S[0] = 0.f;
    o.S[1] = 0.f;
    o.S[2] = __fmul_rn(-P.g, qp[0]);
    o.S[3] = 0.f;
}

// The scalar expressions below round explicitly (no contraction left to the
// compiler): they are inlined into several kernels (the per-mesh and batched
// predictors, node-per-thread and node-pair forms), which must agree bitwise.
__device__ __forceinline__ float wave_speed_f(float rho, float mx, float my, float pp, float pb,
                                              bool xdir, const PhysF& P) {
    const float rinv = __frcp_rn(rho);
    const float c = sqrtf(__fmul_rn(__fmul_rn(P.gamma, __fadd_rn(pb, pp)), rinv));
    const float vn = fabsf(__fmul_rn(xdir ? mx : my, rinv));
    return __fmaf_rn(__fmul_rn(__fmul_rn(2.f, xdir ? P.eta_x : P.eta_y), P.lamv), rinv, __fadd_rn(vn, c));
}

// coordinate o + (cell index + node) h of a node (or face: node = 0 or 1)
__device__ __forceinline__ float node_coord_f(float o, int cell, float node, float h) {
    return __fmaf_rn(__fadd_rn((float)cell, node), h, o);
}

// pressure perturbation of a trace record (rho', m_x, m_y, E') at height z
__device__ __forceinline__ float trace_pp_f(const float* rec, float rinv, float z, const PhysF& P) {
    const float m2 = __fmaf_rn(rec[1], rec[1], __fmul_rn(rec[2], rec[2]));
    const float ke = __fmul_rn(__fmul_rn(0.5f, m2), rinv);
    return __fmul_rn(P.gm1, __fsub_rn(__fsub_rn(rec[3], ke), __fmul_rn(__fmul_rn(P.g, z), rec[0])));
}

// the steady manufactured field's source (Sec. 4.1 workload: rho = 1 + a sin k(x+z),
// u = v = U, p = const) at (x, z)
__device__ __forceinline__ void steady_source_f(float x, float z, const PhysF& P, float Sm[4]) {
    const float k = __fdiv_rn(6.283185307179586f, P.sL);
    float sn, cs;
    sincosf(__fmul_rn(k, __fadd_rn(x, z)), &sn, &cs);
    const float a = P.sa, U = P.sU;
    const float rho = __fmaf_rn(a, sn, 1.f);
    const float c = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(2.f, U), a), k), cs);
    const float r2 = __fmul_rn(rho, rho);
    const float t1 = __fdiv_rn(__fmul_rn(__fmul_rn(__fmul_rn(a, k), k), sn), r2);
    const float t2 = __fdiv_rn(__fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(2.f, a), a), k), k),
                                         __fmul_rn(cs, cs)),
                               __fmul_rn(r2, rho));
    const float lapT = __fmul_rn(__fmul_rn(__fmul_rn(2.f, P.sp), P.invR), __fadd_rn(t1, t2));
    Sm[0] = c;
    Sm[1] = __fmul_rn(c, U);
    Sm[2] = __fmul_rn(c, U);
    Sm[3] = __fsub_rn(__fmul_rn(__fmul_rn(c, U), U), __fmul_rn(P.kappa, lapT));
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
