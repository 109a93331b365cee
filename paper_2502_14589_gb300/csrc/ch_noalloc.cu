// ch_noalloc.cu -- ch_energy_mass_noalloc: the discrete energy and mass of a grid vector
// without a grid object and without any device allocation.
//
// Some callers cannot let a library allocate device memory: applications that hand all
// device memory out of their own pool (a caching allocator or a fixed arena sized at
// start-up) and must keep the library from taking memory behind their back, and callers
// that keep work running concurrently on several streams, because cudaMalloc / cudaFree
// may synchronise the device and stall that work.  ch_create_grid allocates workspace,
// so this entry point instead takes its reduction scratch from a fixed array in the
// library's device image.
//
// The scratch is g_noalloc_scratch below: one static __device__ array of 16 KiB + 256 B
// (per-block partial sums for at most kNoAllocBlocks = 1024 blocks, then an arrival
// counter).  Every GPU that loads the library holds it until the process exits.  All calls
// on a device share it and it keeps the last call's contents: the counter is cleared at the
// start of every call, and calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and must be serialised by the
// caller.  The first call on each device looks up the device address of the array with
// cudaGetSymbolAddress (the host-side name of a __device__ array is only a stand-in, not a
// device address), with that device current; that look-up is cached per device.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "ch_internal.cuh"

namespace ch {
void set_error(const char *msg);
}

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = 1024;
constexpr int kNoAllocMaxDevices = 64;

// partials: [0, 2*kNoAllocBlocks) doubles; counter: the unsigned int after them.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocBlocks + 32];

__device__ __forceinline__ unsigned nbp(unsigned i, unsigned c, unsigned n, unsigned st) {
    return (c + 1u == n) ? i - (n - 1u) * st : i + st;
}

// Energy sum F(y) + eps^2/2 sum_a ((y_{i+e_a} - y_i)/h_a)^2 and mass sum y over the grid;
// the last block to arrive adds the block partials in index order and writes
// out[0] = h^d * energy sum, out[1] = h^d * mass sum.
__global__ void __launch_bounds__(kNoAllocThreads)
k_energy_mass_noalloc(int dim, int n0, int n1, int n2, double eps2, double vol,
                      const double *__restrict__ y, double *__restrict__ out,
                      double *scratch) {
    const unsigned N = (unsigned)n0 * (unsigned)n1 * (unsigned)n2;
    double *partials = scratch;
    unsigned int *counter = (unsigned int *)(scratch + 2 * kNoAllocBlocks);
    double e = 0.0, m = 0.0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double yi = y[i];
        const double u = 1.0 - yi * yi;
        const unsigned c0 = i % (unsigned)n0, r = i / (unsigned)n0, c1 = r % (unsigned)n1;
        const double d0 = (y[nbp(i, c0, n0, 1u)] - yi) * (double)n0;
        const double d1 = (y[nbp(i, c1, n1, n0)] - yi) * (double)n1;
        double gs = d0 * d0 + d1 * d1;
        if (dim == 3) {
            const unsigned c2 = r / (unsigned)n1;
            const double d2 = (y[nbp(i, c2, n2, (unsigned)n0 * n1)] - yi) * (double)n2;
            gs += d2 * d2;
        }
        e += fma(0.5 * eps2, gs, 0.25 * u * u);
        m += yi;
    }
    __shared__ double se[kNoAllocThreads / 32], sm[kNoAllocThreads / 32];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        m += __shfl_down_sync(0xffffffffu, m, o);
    }
    if ((threadIdx.x & 31) == 0) { se[threadIdx.x >> 5] = e; sm[threadIdx.x >> 5] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += se[w]; b += sm[w]; }
        partials[blockIdx.x] = a;
        partials[kNoAllocBlocks + blockIdx.x] = b;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
        a += __ldcg(&partials[k]);
        b += __ldcg(&partials[kNoAllocBlocks + k]);
    }
    out[0] = vol * a;
    out[1] = vol * b;
    *counter = 0u;
}

std::mutex g_mu;
double *g_scratch_addr[kNoAllocMaxDevices] = {nullptr};

ch_status fail(ch_status st, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ch::set_error(buf);          // reported by ch_last_error()
    return st;
}

}  // namespace

extern "C" {

ch_status ch_energy_mass_noalloc(int dim, const int64_t n[3], double eps, const double *y,
                                 double *out, void *cuda_stream) {
    if (!n || !y || !out) return fail(CH_EINVAL, "null argument");
    if (dim != 2 && dim != 3) return fail(CH_EINVAL, "dim must be 2 or 3");
    if (!(eps > 0.0) || !isfinite(eps)) return fail(CH_EINVAL, "eps must be finite and > 0");
    int64_t N = 1;
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 1 || n[a] > (1 << 20)) return fail(CH_EINVAL, "n[%d] out of range", a);
        N *= n[a];
    }
    if (N >= ((int64_t)1 << 31))
        return fail(CH_EINVAL, "grid of %lld points exceeds the 2^31 - 1 points this entry point indexes",
                    (long long)N);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CH_EINVAL, "device index %d not supported", dev);
    // y and out must be memory of this device: a host pointer or another GPU's memory
    // would be dereferenced by a kernel running here.
    const struct { const void *p; const char *name; } bufs[2] = {{y, "y"}, {out, "out"}};
    for (const auto &b : bufs) {
        cudaPointerAttributes at;
        e = cudaPointerGetAttributes(&at, b.p);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CH_EINVAL, "%s is not a CUDA pointer: %s", b.name, cudaGetErrorString(e));
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return fail(CH_EINVAL, "%s must be device memory of the current device %d", b.name, dev);
    }
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(CH_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = (double *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    e = cudaMemsetAsync(scratch + 2 * kNoAllocBlocks, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return fail(CH_ECUDA, "clearing the counter: %s", cudaGetErrorString(e));
    const int n0 = (int)n[0], n1 = (int)n[1], n2 = dim == 3 ? (int)n[2] : 1;
    double vol = 1.0;
    for (int a = 0; a < dim; ++a) vol /= (double)n[a];
    const int blocks = (int)((N + kNoAllocThreads - 1) / kNoAllocThreads < kNoAllocBlocks
                                 ? (N + kNoAllocThreads - 1) / kNoAllocThreads
                                 : kNoAllocBlocks);
    k_energy_mass_noalloc<<<blocks, kNoAllocThreads, 0, stream>>>(dim, n0, n1, n2, eps * eps, vol,
                                                                  y, out, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CH_ECUDA, "launch: %s", cudaGetErrorString(e));
    return CH_OK;
}

}  // extern "C"
