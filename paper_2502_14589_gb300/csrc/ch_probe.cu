// ch_probe.cu -- measured peak of the arithmetic that bounds the FP64 kernels.
//
// On GB300 an FP64 stencil or Gram-Schmidt pass has an arithmetic intensity far above the
// FP64 ridge point, so its roofline is the FP64 FMA issue rate, not HBM.  The rate is
// measured here rather than taken from a data sheet: every thread of a full grid (a multiple
// of the SM count, several resident blocks per SM) runs independent FMA chains from
// registers, with no memory traffic inside the timed loop, and CUDA events on the caller's
// stream time the launch.  The chains' results are stored so the compiler keeps the work.
#include <math.h>

#include "ch_internal.cuh"

namespace ch {
void set_error(const char *msg);
}

namespace {

constexpr int kProbeChains = 8;      // independent FMA chains per thread (covers the latency)
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads)
k_fp64_fma_probe(int iters, double a, double b, double *out) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

ch_status ch_probe_fp64_peak(void *cuda_stream, double *tflops) {
    if (!tflops) { ch::set_error("null argument"); return CH_EINVAL; }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_probe, kProbeThreads, 0);
    if (e != cudaSuccess) { ch::set_error(cudaGetErrorString(e)); return CH_ECUDA; }
    const int blocks = sms * (per_sm > 4 ? 4 : per_sm);
    const int iters = 4096;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc((void **)&out, sizeof(double) * (size_t)blocks * kProbeThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // first launch warms up
        cudaEventRecord(e0, s);
        k_fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-7, out);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) { ch::set_error(cudaGetErrorString(e)); return CH_ECUDA; }
    const double flops = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return CH_OK;
}

}  // extern "C"
