// Peak arithmetic throughput of the plain (non-tensor) FP64 and FP32 FMA
// pipes on the current GPU.  The ADER-DG predictor is bound by these pipes
// (not by HBM), so its roofline denominator is measured here rather than
// taken from a datasheet.
//
// Build:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_peak fma_peak.cu
// Run:    ./fma_peak            -> one JSON line per precision
//
// Each thread runs ACC independent FMA chains (enough instruction-level
// parallelism to hide the pipe latency); the grid is a multiple of the SM
// count.  FLOPs counted as 2 per FMA.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return 1; } } while (0)

template <typename T, int ACC>
__global__ void fma_loop(T* out, int iters, T a, T b) {
    T acc[ACC];
#pragma unroll
    for (int c = 0; c < ACC; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < ACC; ++c) acc[c] = acc[c] * a + b;
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < ACC; ++c) s += acc[c];
    if (s == (T)-12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the loop alive
}

template <typename T>
static int run(const char* name, int sms, double clock_khz) {
    constexpr int ACC = 8;
    const int threads = 256, blocks = sms * 8;
    T* out = nullptr;
    CK(cudaMalloc(&out, sizeof(T) * threads * blocks));
    int iters = sizeof(T) == 8 ? 64 : 4096;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int rep = 0; rep < 7; ++rep) {
        CK(cudaEventRecord(e0));
        fma_loop<T, ACC><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep == 0) {  // calibrate once: aim at ~20 ms per launch, bounded
            double scale = 20.0 / (ms > 0.01f ? ms : 0.01f);
            if (scale > 1.0) iters = (int)(iters * (scale < 64.0 ? scale : 64.0));
        } else if (ms < best_ms) {
            best_ms = ms;
        }
    }
    double flops = 2.0 * ACC * 16.0 * (double)iters * threads * blocks;
    double tflops = flops / (best_ms * 1e-3) / 1e12;
    double per_sm_clk = flops / 2.0 / (best_ms * 1e-3) / sms / (clock_khz * 1e3);
    printf("{\"pipe\": \"%s_fma\", \"tflops\": %.4f, \"ms\": %.3f, \"fma_per_sm_per_clk_at_max_clock\": %.3f, "
           "\"sms\": %d, \"max_clock_mhz\": %.0f}\n", name, tflops, best_ms, per_sm_clk, sms, clock_khz / 1e3);
    CK(cudaFree(out));
    return 0;
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    CK(cudaSetDevice(dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    if (run<double>("fp64", sms, clk)) return 1;
    if (run<float>("fp32", sms, clk)) return 1;
    return 0;
}
