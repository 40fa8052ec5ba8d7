// Conversions between binary64 and binary32 by integer operations on the
// IEEE-754 encodings.  On this GPU the hardware conversion instructions run
// on the (narrow) FP64 pipe, which makes them the most expensive operations
// of the mixed-precision kernels; these versions use the integer pipes.
//  * f64_to_f32: round to nearest, ties to even; results below the binary32
//    normal range become +-0, above it +-inf (the solver's values are far from
//    both ends); +-inf stays +-inf and NaN stays NaN (a quiet NaN of the same
//    sign).
//  * f32_to_f64: exact for normal numbers; subnormal inputs become +-0.
#pragma once
#include <cuda_runtime.h>

namespace adg {

__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned int hi = (unsigned int)__double2hiint(d);
    const unsigned int lo = (unsigned int)__double2loint(d);
    const unsigned int sign = hi & 0x80000000u;
    const unsigned int ein = (hi >> 20) & 0x7FFu;
    const int e = (int)ein - 1023 + 127;
    const unsigned int m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 of the 52 mantissa bits
    const unsigned int rest = lo & 0x1FFFFFFFu;                      // the 29 bits dropped
    unsigned int r = sign | ((unsigned int)e << 23) | m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;  // carry may bump the exponent
    if (e <= 0) r = sign;
    if (e >= 255) r = sign | 0x7F800000u;
    if (ein == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u) r = sign | 0x7FC00000u;  // NaN input
    return __uint_as_float(r);
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int sign = b & 0x80000000u;
    const unsigned int e = (b >> 23) & 0xFFu;
    const unsigned int m = b & 0x7FFFFFu;
    unsigned int hi = sign | ((e + (1023u - 127u)) << 20) | (m >> 3);
    unsigned int lo = m << 29;
    if (e == 0u) { hi = sign; lo = 0u; }
    if (e == 255u) { hi = sign | 0x7FF00000u | (m ? 0x80000u : 0u); lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// the programmatic-serialization attribute may be scheduled while the
// previous kernel of its stream is still finishing; pdl_wait() blocks until
// that kernel has completed and its memory operations are visible, so every
// read of its outputs must follow it.  pdl_trigger() tells the scheduler that
// this block no longer needs to delay the dependent kernel.  Both are no-ops
// for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace adg
