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

constexpr int kProbeMaxChains = 16;

// CH independent FMA chains per thread (CH a compile-time constant: the chains live in
// registers), iters rounds.
template <int CH>
__global__ void k_fp64_fma_probe(int iters, double a, double b, double *out) {
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best FMA rate over a few launch shapes (threads per block, resident blocks, chains): the
// FP64 units are fed only when enough independent FMAs are in flight per sub-partition.
cudaError_t probe_shape(const void *fn, int chains, int threads, int sms, cudaStream_t s, double *out,
                        cudaEvent_t e0, cudaEvent_t e1, double *best_tflops) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * per_sm;
    int iters = 2048;
    double a = 0.999999, b = 1e-7;
    void *args[] = {&iters, &a, &b, &out};
    for (int rep = 0; rep < 3; ++rep) {                  // the first launch warms up
        cudaEventRecord(e0, s);
        e = cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, 0, s);
        if (e != cudaSuccess) return e;
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return e;
        const double fl = 2.0 * chains * (double)iters * blocks * threads;
        if (rep > 0 && ms > 0.f && fl / (ms * 1e-3) / 1e12 > *best_tflops) *best_tflops = fl / (ms * 1e-3) / 1e12;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

ch_status ch_probe_fp64_peak(void *cuda_stream, double *tflops) {
    if (!tflops) { ch::set_error("null argument"); return CH_EINVAL; }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { ch::set_error(cudaGetErrorString(e)); return CH_ECUDA; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the largest grid: 2048 threads per SM
    e = cudaMalloc((void **)&out, sizeof(double) * (size_t)sms * 2048);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    const struct { const void *fn; int chains; } kernels[] = {
        {(const void *)k_fp64_fma_probe<4>, 4}, {(const void *)k_fp64_fma_probe<8>, 8},
        {(const void *)k_fp64_fma_probe<kProbeMaxChains>, kProbeMaxChains}};
    const int thread_counts[] = {256, 1024};
    for (const auto &k : kernels)
        for (int th : thread_counts)
            if (e == cudaSuccess) e = probe_shape(k.fn, k.chains, th, sms, s, out, e0, e1, &best);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) { ch::set_error(cudaGetErrorString(e)); return CH_ECUDA; }
    *tflops = best;
    return CH_OK;
}

}  // extern "C"
