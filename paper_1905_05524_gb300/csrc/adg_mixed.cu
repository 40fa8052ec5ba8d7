// Mixed-precision ADER-DG predictor and corrector for sm_103a.
//
// Same scheme as adg_fp64.cu (Sec. 3: Picard space-time predictor, Rusanov-
// type viscous corrector), with the arithmetic split by what it needs:
//
//  * FP64: the perturbation split against the hydrostatic background,
//    u' = u - ubar(z) (rho and rhoE: this is where rhoE cancels against the
//    background energy, Eqs. 2, 6, 7), and the corrector's accumulation
//    u^{n+1} = u^n + dt * du.
//  * FP32: everything between -- the Picard sweeps on the perturbation
//    q' = q - ubar, the contractions (gradients, flux divergence, time
//    update), the point-wise fluxes and the face traces/Riemann fluxes.
//    The pressure perturbation is formed directly from perturbations,
//        p' = (gamma-1) (rhoE' - |rho v|^2 / (2 rho) - g z rho'),
//    which is exact algebra (pbar = (gamma-1)(Ebar - rhobar g z)), so no FP32
//    quantity ever carries the large background values through a difference.
//  * Background gradients: the nodal derivative of the interpolated background
//    (rhobar, Ebar) is formed once in FP64 on the host and added in FP32.
//
// Without gravity the background is zero and q' is the full state.
#include <cuda_runtime.h>

#include "adg_convert.cuh"
#include "adg_internal.h"
#include "adg_mixed_body.cuh"
#include "adg_mixed_x2.cuh"
#include "adg_mixed_point.cuh"
#include "adg_tv_cell.cuh"

namespace adg {


template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1), (MixCfg<N, CPB>::minb))
k_predictor_mixed(const double* __restrict__ u, float* __restrict__ rvol, float* __restrict__ trace,
                  int cells, float dt, const BasisF B, const PhysF P, const MixedBg bg) {
    extern __shared__ float smf[];
    predictor_mixed_body<N, CPB>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P, bg, smf);
    pdl_trigger();  // the corrector (launched programmatically) may be scheduled
}

template <int N, int CPB>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1) / 2, (MixCfg2<N, CPB>::minb))
k_predictor_mixed_x2(const double* __restrict__ u, float* __restrict__ rvol, float* __restrict__ trace,
                     int cells, float dt, const BasisF B, const PhysF P, const MixedBg bg) {
    extern __shared__ float smf[];
    predictor_mixed_body_x2<N, CPB>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P, bg, smf);
    pdl_trigger();  // the corrector (launched programmatically) may be scheduled
}

template <int N, int CPB, bool TV>
__global__ void __launch_bounds__(CPB*(N + 1) * (N + 1))
k_corrector_mixed(double* __restrict__ u, const float* __restrict__ rvol,
                  const float* __restrict__ trace, int cells, double dt, const BasisF B,
                  const PhysF P, const MixedBg bg, const TvEpilogue epi) {
    pdl_wait();  // the predictor's residual and traces are complete and visible
    corrector_mixed_body<N, CPB, TV>(u, rvol, trace, cells, blockIdx.x * CPB, dt, B, P, bg, epi);
    pdl_trigger();
}

// Cells per block of the per-mesh node-per-thread predictor launch; the
// corrector and the TV statistics keep tv_cpb(N).  At N = 6 (49 threads a
// cell) two cells fill 98 threads, a fourth warp of two lanes that issues
// every instruction for them; five cells (245 threads in eight warps, two
// resident blocks at 128 registers) ran the 243x243 step in 2.38 against
// 2.53 ms (three cells: 2.61, ten: 2.55).
template <int N>
constexpr int pred_cpb() {
    return N == 6 ? 5 : MixCfg<N>::cpb_default;
}

template <int N>
static int launch_pred_mixed(const double* u, float* rvol, float* trace, int cells, float dt,
                             const BasisF& B, const PhysF& P, const MixedBg& bg, cudaStream_t s) {
    if constexpr (N == 3 || N == 5) {  // node pairs (measured slower at N = 7: 232 registers, 8 warps per SM)
        using C2 = MixCfg2<N>;
        auto kern = k_predictor_mixed_x2<N, C2::cpb>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C2::smem_pred);
        if (e != cudaSuccess) return (int)e;
        const int blocks = (cells + C2::cpb - 1) / C2::cpb;
        kern<<<blocks, C2::threads, C2::smem_pred, s>>>(u, rvol, trace, cells, dt, B, P, bg);
        return (int)cudaGetLastError();
    }
    using C = MixCfg<N, pred_cpb<N>()>;
    auto kern = k_predictor_mixed<N, C::cpb>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_pred);
    if (e != cudaSuccess) return (int)e;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    kern<<<blocks, C::threads, C::smem_pred, s>>>(u, rvol, trace, cells, dt, B, P, bg);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_corr_mixed(double* u, const float* rvol, const float* trace, int cells, double dt,
                             const BasisF& B, const PhysF& P, const MixedBg& bg, const TvEpilogue* epi,
                             cudaStream_t s) {
    using C = MixCfg<N>;
    const int blocks = (cells + C::cpb - 1) / C::cpb;
    // programmatic launch: scheduled while the predictor drains, waits for it
    // in pdl_wait() before reading its outputs
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
    cudaError_t e;
    if (epi)
        e = cudaLaunchKernelEx(&cfg, k_corrector_mixed<N, C::cpb, true>, u, rvol, trace, cells, dt, B, P, bg, *epi);
    else
        e = cudaLaunchKernelEx(&cfg, k_corrector_mixed<N, C::cpb, false>, u, rvol, trace, cells, dt, B, P, bg,
                               TvEpilogue{});
    return e != cudaSuccess ? (int)e : (int)cudaGetLastError();
}

int launch_predictor_mixed(int N, const double* u, float* rvol, float* trace, int cells, double dt,
                           const BasisF& B, const PhysF& P, const MixedBg& bg, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const float dtf = (float)dt;
    switch (N) {
        case 1: return launch_pred_mixed<1>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 2: return launch_pred_mixed<2>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 3: return launch_pred_mixed<3>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 4: return launch_pred_mixed<4>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 5: return launch_pred_mixed<5>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 6: return launch_pred_mixed<6>(u, rvol, trace, cells, dtf, B, P, bg, s);
        case 7: return launch_pred_mixed<7>(u, rvol, trace, cells, dtf, B, P, bg, s);
    }
    return (int)cudaErrorInvalidValue;
}

int launch_corrector_mixed(int N, double* u, const float* rvol, const float* trace, int cells,
                           double dt, const BasisF& B, const PhysF& P, const MixedBg& bg, void* stream,
                           const TvEpilogue* epi) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (N) {
        case 1: return launch_corr_mixed<1>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 2: return launch_corr_mixed<2>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 3: return launch_corr_mixed<3>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 4: return launch_corr_mixed<4>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 5: return launch_corr_mixed<5>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 6: return launch_corr_mixed<6>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
        case 7: return launch_corr_mixed<7>(u, rvol, trace, cells, dt, B, P, bg, epi, s);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace adg
