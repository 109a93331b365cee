// ch_stencil.cu -- streaming kernels of the Cahn-Hilliard hot path, FP64.
//
// Every operator application is split into two elementwise stages with no redundant halo
// work (FP64 on GB300 runs at 2 FMA/clk/SM, so the kernels are bound by FP64 instruction
// issue, not HBM, and the minimum DP-instruction count per point is the design target):
//   stage 1 (7-point in 3D, 5-point in 2D):  t = D (.) x - sum_a kap_a (x_{+a} + x_{-a})
//   stage 2:                                 w = c0 t - sum_a c_a (t_{+a} + t_{-a})
// With D = 3 y^2 - 1 [+1 Eyre] + eps^2 sigma, kap_a = eps^2 s_a, c0 = sigma, c_a = s_a this
// is A_hat v = A (J + eps^2 A [+ I]) v of Eqs. (A_g), (A_g_cs); other coefficient choices
// give f(y) of Eq. (IVP), the LIM residual g_hat - A_hat y (Fig. 1) and the PC
// estimate of Eq. (LIMest).  Neighbour indices wrap periodically, or on a Neumann grid a
// neighbour beyond the boundary is the point itself (cell-centred mirror, Eq. CH), which
// the same formulas then treat correctly.  With a variable mobility (the Remark on Eq.
// CHmob) stage 2 is the flux form of A_M with the grid's face mobilities instead.
#include <math.h>

#include "ch_internal.cuh"

namespace ch {

// Neighbour of point i (coordinate c along an axis of n points and index stride st) on the
// plus / minus side: the periodic image past the boundary (bc = 0) or the point itself
// (bc = 1, the cell-centred Neumann mirror).
__device__ __forceinline__ unsigned nb_p(unsigned i, unsigned c, unsigned n, unsigned st, int bc) {
    return (c + 1u == n) ? (bc ? i : i - (n - 1u) * st) : i + st;
}
__device__ __forceinline__ unsigned nb_m(unsigned i, unsigned c, unsigned n, unsigned st, int bc) {
    return (c == 0u) ? (bc ? i : i + (n - 1u) * st) : i - st;
}

// Pair sums x_{+a} + x_{-a} of the neighbours of point i along every axis.
template <int DIM, typename T>
__device__ __forceinline__ void pair_sums(const Geom &g, const T *__restrict__ x, unsigned i,
                                          T (&ps)[3]) {
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned c0 = i % n0;
    const unsigned r = i / n0;
    const unsigned c1 = r % n1;
    ps[0] = x[nb_p(i, c0, n0, 1u, g.bc)] + x[nb_m(i, c0, n0, 1u, g.bc)];
    ps[1] = x[nb_p(i, c1, n1, n0, g.bc)] + x[nb_m(i, c1, n1, n0, g.bc)];
    if (DIM == 3) {
        const unsigned n2 = (unsigned)g.n[2], s2 = n0 * n1;
        const unsigned c2 = r / n1;
        ps[2] = x[nb_p(i, c2, n2, s2, g.bc)] + x[nb_m(i, c2, n2, s2, g.bc)];
    } else {
        ps[2] = T(0);
    }
}

// Differences (x_i - x_{i+a}) + (x_i - x_{i-a}) along every axis (the FP32 stages).
template <int DIM, typename T>
__device__ __forceinline__ void pair_diffs(const Geom &g, const T *__restrict__ x, unsigned i,
                                           T (&pd)[3]) {
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned c0 = i % n0;
    const unsigned r = i / n0;
    const unsigned c1 = r % n1;
    const T xi = x[i];
    pd[0] = (xi - x[nb_p(i, c0, n0, 1u, g.bc)]) + (xi - x[nb_m(i, c0, n0, 1u, g.bc)]);
    pd[1] = (xi - x[nb_p(i, c1, n1, n0, g.bc)]) + (xi - x[nb_m(i, c1, n1, n0, g.bc)]);
    if (DIM == 3) {
        const unsigned n2 = (unsigned)g.n[2], s2 = n0 * n1;
        const unsigned c2 = r / n1;
        pd[2] = (xi - x[nb_p(i, c2, n2, s2, g.bc)]) + (xi - x[nb_m(i, c2, n2, s2, g.bc)]);
    } else {
        pd[2] = T(0);
    }
}

// Face mobilities of axis a in precision T (FP64 or the FP32 copies of a mixed grid).
template <typename T> __device__ __forceinline__ const T *face_mob(const Geom &g, int a);
template <> __device__ __forceinline__ const double *face_mob<double>(const Geom &g, int a) { return g.mf[a]; }
template <> __device__ __forceinline__ const float *face_mob<float>(const Geom &g, int a) { return g.mff[a]; }

// Flux form of the outer operator with variable mobility (the Remark on Eq. CHmob) at i:
//   (A_M t)_i = sum_a [mf_a[i] (t_i - t_{i+e_a}) + mf_a[i-e_a] (t_i - t_{i-e_a})],
// the face on the minus side being the plus face of the minus neighbour (a Neumann mirror
// neighbour is the point itself, so that face's difference is zero).
template <int DIM, typename T>
__device__ __forceinline__ T flux_at(const Geom &g, const T *__restrict__ t, unsigned i) {
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned c0 = i % n0, r = i / n0, c1 = r % n1;
    const T ti = t[i];
    const T *m0 = face_mob<T>(g, 0), *m1 = face_mob<T>(g, 1);
    unsigned p = nb_p(i, c0, n0, 1u, g.bc), m = nb_m(i, c0, n0, 1u, g.bc);
    T acc = m0[i] * (ti - t[p]);
    acc = fma(m0[m], ti - t[m], acc);
    p = nb_p(i, c1, n1, n0, g.bc); m = nb_m(i, c1, n1, n0, g.bc);
    acc = fma(m1[i], ti - t[p], acc);
    acc = fma(m1[m], ti - t[m], acc);
    if (DIM == 3) {
        const unsigned n2 = (unsigned)g.n[2], s2 = n0 * n1, c2 = r / n1;
        const T *m2 = face_mob<T>(g, 2);
        p = nb_p(i, c2, n2, s2, g.bc); m = nb_m(i, c2, n2, s2, g.bc);
        acc = fma(m2[i], ti - t[p], acc);
        acc = fma(m2[m], ti - t[m], acc);
    }
    return acc;
}

// The two stages of A_hat v in the basis precision, at point i.
//   FP64: t = D x - sum_a kap_a (x_{+a} + x_{-a}),  D = J + eps^2 sigma  (fewest FP64 ops);
//         w = c0 t - sum_a c_a (t_{+a} + t_{-a}).
//   FP32: t = J x + sum_a kap_a ((x - x_{+a}) + (x - x_{-a})),  D holds J (+1 Eyre);
//         w = sum_a c_a ((t - t_{+a}) + (t - t_{-a})).
// The FP32 form is the same operator without the cancellation of the pair-sum form: there
// the eps^2 sigma x term (about 400 x at 1024^2, eps = 0.01) and the smooth part of the
// neighbour sums cancel in FP32 rounding, while neighbour differences of a smooth field are
// exact (Sterbenz) and only the small second differences are rounded.
template <int DIM, typename VT>
__device__ __forceinline__ VT stage1_at(const Geom &g, const VT *__restrict__ x,
                                        const VT *__restrict__ D, unsigned i, VT k0, VT k1, VT k2) {
    VT q[3];
    VT acc = D[i] * x[i];
    if constexpr (sizeof(VT) == 8) {
        pair_sums<DIM>(g, x, i, q);
        k0 = -k0; k1 = -k1; k2 = -k2;
    } else {
        pair_diffs<DIM>(g, x, i, q);
    }
    acc = fma(k0, q[0], acc);
    acc = fma(k1, q[1], acc);
    if (DIM == 3) acc = fma(k2, q[2], acc);
    return acc;
}
// gm: the scale the coefficients carry (gam_j, or 1); with a variable mobility stage 2 is
// gm (A_M t)_i by the flux form instead.
template <int DIM, typename VT>
__device__ __forceinline__ VT stage2_at(const Geom &g, const VT *__restrict__ t, unsigned i,
                                        VT c0, VT c1, VT c2, VT c3, VT gm) {
    if (g.mf[0]) return gm * flux_at<DIM, VT>(g, t, i);
    VT q[3];
    VT r;
    if constexpr (sizeof(VT) == 8) {
        pair_sums<DIM>(g, t, i, q);
        r = c0 * t[i];
        c1 = -c1; c2 = -c2; c3 = -c3;
        r = fma(c1, q[0], r);
    } else {
        pair_diffs<DIM>(g, t, i, q);
        r = c1 * q[0];
    }
    r = fma(c2, q[1], r);
    if (DIM == 3) r = fma(c3, q[2], r);
    return r;
}

// Dot-product accumulators.  FP64 vectors: plain FMA accumulation.  FP32 vectors (mixed
// precision): every product is split exactly into p + e (e = fma(a, b, -p)) and summed with
// a compensated two-sum in FP32 pairs, so the per-thread sum carries ~2^-44 relative error;
// the block and grid trees then add in FP64.
template <typename VT> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    // add a value (a short FP32 dot product) with the compensated two-sum only
    __device__ __forceinline__ void add_value(float p) {
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

#define GRID_LOOP(i, N) \
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < (unsigned)(N); i += gridDim.x * blockDim.x)

// Grid-stride loop that handles two elements (i, i + stride) per trip, so each thread has
// twice the loads in flight; per-thread accumulation order is the same as GRID_LOOP's.
#define GRID_LOOP2(N, ...)                                                                \
    {                                                                                     \
        const unsigned stride_ = gridDim.x * blockDim.x;                                  \
        unsigned i_ = blockIdx.x * blockDim.x + threadIdx.x;                              \
        for (; i_ + stride_ < (unsigned)(N); i_ += 2 * stride_) {                         \
            { const unsigned i = i_; __VA_ARGS__ }                                        \
            { const unsigned i = i_ + stride_; __VA_ARGS__ }                              \
        }                                                                                 \
        if (i_ < (unsigned)(N)) { const unsigned i = i_; __VA_ARGS__ }                    \
    }

// ---------------------------------------------------------------------------------------
// Per-step preparation from the linearisation point y^n:
//   D = 3 y^2 - 1 (+1 Eyre) + eps^2 sigma   (diagonal of J_n + eps^2 A [+I] before -kap sums)
//   G = 2 y^3 (+ y Eyre)                    (= J_n y - F'(y) [+ y], inner part of g_hat)
//   min / max of y^2                        (bound of Fig. 1: lambda_max from d_min, d_max)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_prep(Geom g, const double *__restrict__ y, double dconst, int eyre, double *__restrict__ D,
       double *__restrict__ G, int want_minmax, double *partials, unsigned int *ticket,
       Ctrl *ctrl) {
    double mn = INFINITY, mx = -INFINITY;
    GRID_LOOP(i, g.N) {
        const double yi = y[i];
        const double y2 = yi * yi;
        D[i] = fma(3.0, y2, dconst);
        if (G) G[i] = eyre ? fma(2.0 * y2, yi, yi) : 2.0 * y2 * yi;
        mn = fmin(mn, y2);
        mx = fmax(mx, y2);
    }
    if (!want_minmax) return;
    block_minmax(mn, mx);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = mn;
        partials[gridDim.x + blockIdx.x] = mx;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    mn = INFINITY; mx = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        mn = fmin(mn, __ldcg(&partials[b]));
        mx = fmax(mx, __ldcg(&partials[gridDim.x + b]));
    }
    block_minmax(mn, mx);
    if (threadIdx.x == 0) {
        ctrl->red[4] = mn;
        ctrl->red[5] = mx;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// Arnoldi product of Fig. 2 on the unnormalised basis vector x = W_j (v_j = gam_j W_j):
//   tstage: t = D (.) x - sum_a kap_a (x_{+a} + x_{-a})
//   wstage: w = gam_j (sigma t - sum_a s_a (t_{+a} + t_{-a}))  = A_hat v_j
//           and h_{1j} = w . v_1 = gam_1 (w . W_1)           (first Gram-Schmidt pass)
// ---------------------------------------------------------------------------------------
template <int DIM, typename VT>
__global__ void __launch_bounds__(kThreads)
k_tstage(Geom g, const VT *__restrict__ x, const VT *__restrict__ D, VT *__restrict__ t,
         const Ctrl *ctrl, int guarded) {
    if (guarded && !ctrl->active) return;
    const VT k0 = (VT)g.kap[0], k1 = (VT)g.kap[1], k2 = (VT)g.kap[2];
    GRID_LOOP2(g.N, {
        t[i] = stage1_at<DIM, VT>(g, x, D, i, k0, k1, k2);
    })
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kThreads)
k_wstage(Geom g, const VT *__restrict__ t, VT *__restrict__ w, const VT *__restrict__ v1,
         double *hout, int jm1, double *partials, unsigned int *ticket, Ctrl *ctrl, int guarded) {
    if (guarded && !ctrl->active) return;
    const double gam = guarded ? ctrl->gam[jm1] : 1.0;
    const VT c0 = (VT)(gam * g.sigma), c1 = (VT)(gam * g.s[0]), c2 = (VT)(gam * g.s[1]),
             c3 = (VT)(gam * g.s[2]);
    DotAcc<VT> acc;
    GRID_LOOP2(g.N, {
        const VT r = stage2_at<DIM, VT>(g, t, i, c0, c1, c2, c3, (VT)gam);
        w[i] = r;
        if (v1) acc.add(r, v1[i]);
    })
    if (!v1) return;
    double tot1[1] = {acc.value()};
    grid_sum<1>(tot1, partials, ticket, [&](double (&tot)[1]) { *hout = ctrl->gam[0] * tot[0]; });
}

// ---------------------------------------------------------------------------------------
// Modified Gram-Schmidt pass k of Fig. 2, fused with the next dot product:
//   w -= h_{kj} v_k  (= h_{kj} gam_k W_k),  then  h_{k+1,j} = w . v_{k+1}   (k < j)
//                                           or    ||w||^2 for h_{j+1,j}    (k = j)
// ---------------------------------------------------------------------------------------
// 16-byte vectors of the basis precision: double2 / float4.
template <typename VT> struct Vec16;
template <> struct Vec16<double> { typedef double2 T; static constexpr int W = 2; };
template <> struct Vec16<float> { typedef float4 T; static constexpr int W = 4; };

template <typename V> __device__ __forceinline__ auto &lane(V &v, int k);
__device__ __forceinline__ double &lane(double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float &lane(float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

template <typename VT>
__global__ void __launch_bounds__(kThreads)
k_mgs(int64_t N, VT *__restrict__ w, const VT *__restrict__ vk, const VT *__restrict__ vk1,
      double *hk, double *hout, int k, int last, int ldh_next, double *partials,
      unsigned int *ticket, Ctrl *ctrl) {
    if (!ctrl->active) return;
    typedef typename Vec16<VT>::T V;
    constexpr int WD = Vec16<VT>::W;
    const VT c = (VT)(*hk * ctrl->gam[k - 1]);
    DotAcc<VT> acc;
    // all vectors start on 256-byte boundaries; the N % WD tail is done element by element
    const unsigned nv = (unsigned)(N / WD);
    V *w4 = reinterpret_cast<V *>(w);
    const V *a4 = reinterpret_cast<const V *>(vk);
    const V *b4 = reinterpret_cast<const V *>(last ? vk : vk1);
    GRID_LOOP2(nv, {
        V x = w4[i];
        const V a = a4[i], b = b4[i];
        for (int q = 0; q < WD; ++q) {      // WD is a compile-time constant: fully unrolled
            const VT r = fma(-c, lane(const_cast<V &>(a), q), lane(x, q));
            lane(x, q) = r;
            acc.add(r, last ? r : lane(const_cast<V &>(b), q));
        }
        w4[i] = x;
    })
    for (int64_t i = (int64_t)nv * WD + blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const VT r = fma(-c, vk[i], w[i]);
        w[i] = r;
        acc.add(r, last ? r : vk1[i]);
    }
    double tot1[1] = {acc.value()};
    if (!last)
        grid_sum<1>(tot1, partials, ticket, [&](double (&tot)[1]) { *hout = ctrl->gam[k] * tot[0]; });
    else   // Fig. 2: h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
        grid_sum<1>(tot1, partials, ticket, [&](double (&tot)[1]) {
            ctrl->hnext2 = tot[0];
            const double h = sqrt(tot[0]);
            hk[ldh_next] = h;
            ctrl->gam[k] = 1.0 / h;
        });
}

// ---------------------------------------------------------------------------------------
// One whole Arnoldi iteration j (Fig. 2, with the scale of v_{j+1}) in one
// cooperative launch of one 1024-thread block per SM: t-stage, w-stage with h_{1j}, then
// the j modified Gram-Schmidt passes, separated by grid barriers.  After each barrier every
// block adds the per-block partials in block order itself (the same value in every block,
// no serialised tail); partial buffers alternate between rounds, so a fast block never
// overwrites sums a slow block is still reading.
//
// FP64 on GB300 is slow per instruction as well as in throughput: a warp-wide FP64 add
// holds its SM sub-partition for 64 cycles, and 32 warps issuing one FP64 instruction each
// cost ~600 cycles.  Scalar work between passes (h, the next coefficient) is therefore done
// by one thread and broadcast through shared memory, and the reduction trees use as few
// dependent FP64 adds as the fixed summation order allows.
// ---------------------------------------------------------------------------------------
constexpr int kArnThreads = 1024;
constexpr long long kBarrierSpinLimit = 1ll << 24;     // ~1 s of short sleeps

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier on a monotonic arrival counter.  The counter starts at 0 and every launch
// adds the grid size G once per barrier, so it is a multiple of G between launches.  A block
// reads it once at kernel start: fewer than G arrivals can precede that read (nobody passes
// the first barrier without this block), so rounding down to a multiple of G gives the
// launch's base and round r ends when the counter reaches base + (r + 1) G.  Arrival is a
// fire-and-forget release reduction; waiters poll with acquire loads.  Every wait is
// bounded: on timeout the block records CH_ETIMEOUT and goes on, so the kernel always ends
// and the host reports the failure (and clears the counter).
struct GridBarrier {
    unsigned long long *bar;
    int *status;
    unsigned long long next;   // counter value that ends the next round (thread 0)
    __device__ __forceinline__ GridBarrier(unsigned long long *b, int *st) : bar(b), status(st), next(0) {
        if (threadIdx.x == 0) {
            const unsigned long long G = gridDim.x;
            next = ld_acquire(bar) / G * G + G;
        }
    }
    // Thread 0 arrives and waits.  The release reduction orders the block's earlier writes
    // (made visible to thread 0 by a preceding __syncthreads) before the arrival.
    __device__ __forceinline__ void arrive_wait_t0() {
        red_release_add(bar, 1ull);
        long long spins = 0;
        while (ld_acquire(bar) < next) {
            if (++spins > kBarrierSpinLimit) { *status = CH_ETIMEOUT; break; }
            __nanosleep(32);
        }
        next += gridDim.x;
    }
    // Whole-block barrier across the grid.
    __device__ __forceinline__ void sync() {
        __syncthreads();
        if (threadIdx.x == 0) arrive_wait_t0();
        __syncthreads();
    }
    // Warp-0 barrier across the grid, for rounds where only thread 0 has written data other
    // blocks read (its partial sum): the rest of the block need not wait on it.
    __device__ __forceinline__ void sync_w0() {
        if (threadIdx.x == 0) arrive_wait_t0();
        __syncwarp();
    }
};

// Sum of one value per thread of a kArnThreads block, valid in thread 0 only: four warps
// (one per SM sub-partition) each add 256 values from shared memory (8 per lane as a
// pairwise tree) and finish with a shuffle tree; thread 0 adds the four pairwise.  Ten
// dependent FP64 adds in all.  sh holds kArnThreads + 8 doubles.
__device__ __forceinline__ double arn_block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid < 4) {
        const double *p = sh + wid * (kArnThreads / 4) + lane;
        double a = ((p[0] + p[32]) + (p[64] + p[96])) + ((p[128] + p[160]) + (p[192] + p[224]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[kArnThreads + wid] = a;
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) s = (sh[kArnThreads] + sh[kArnThreads + 1]) + (sh[kArnThreads + 2] + sh[kArnThreads + 3]);
    return s;
}

constexpr int kMaxArnBlocks = 32 * 5;   // grid of the iteration kernels: at most 5 partials per lane

// Sum of the per-block partials by warp 0 (lane l adds slots l + 32 s pairwise over s, then
// a shuffle tree); the value is valid in thread 0 only and identical in every block.  The
// loads are issued together, so the L2 round trip is paid once.  Call from warp 0.
__device__ __forceinline__ double arn_grid_sum_w0(const double *part) {
    const unsigned G = gridDim.x, lane = threadIdx.x;
    double v[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) v[s] = (lane + 32u * s < G) ? __ldcg(&part[lane + 32u * s]) : 0.0;
    double a = ((v[0] + v[1]) + (v[2] + v[3])) + v[4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    return a;
}

// Scalars shared by the block between passes.
template <typename VT>
struct ArnShared {
    double h;      // h_{k,j} of the coming pass
    VT c;          // its coefficient h_{k,j} gam_{k-1} in the basis precision
};

// End of round k + 1 (thread 0 has posted this block's partial): warp 0 waits at the grid
// barrier and sums the partials, and in thread 0
//   k < j:  h_{k+1,j} = gam_k sum (row k of H), next coefficient h_{k+1,j} gam_k;
//   k = j:  h_{j+1,j} = sqrt(sum) (Fig. 2), gam_j = 1 / h_{j+1,j};
// k = 0 is the w-stage round: h_{1j} = gam_0 sum.  Block 0 writes H and the control block.
template <typename VT>
__device__ __forceinline__ void arn_finish_round(GridBarrier &gb, const double *part, int k, int j,
                                                 double *H, int ldh, Ctrl *ctrl, ArnShared<VT> *sc) {
    if (threadIdx.x < 32) {
        gb.sync_w0();
        const double sum = arn_grid_sum_w0(part);
        if (threadIdx.x == 0) {
            if (k < j) {
                const double g = ctrl->gam[k];
                const double h = g * sum;
                sc->h = h;
                sc->c = (VT)(h * g);
                if (blockIdx.x == 0) H[k * ldh + (j - 1)] = h;
            } else if (blockIdx.x == 0) {
                const double hn = sqrt(sum);
                ctrl->hnext2 = sum;
                H[j * ldh + (j - 1)] = hn;
                ctrl->gam[j] = 1.0 / hn;
            }
        }
    }
    __syncthreads();
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kArnThreads, 1)
k_arnoldi(Geom g, VT *__restrict__ slot0, VT *__restrict__ V, int64_t ldv, const VT *__restrict__ D,
          VT *__restrict__ t, double *H, int ldh, int j, double *partials, Ctrl *ctrl) {
    if (!ctrl->active) return;                  // same value in every block
    __shared__ double sh[kArnThreads + 8];
    __shared__ ArnShared<VT> sc;
    auto W = [&](int c) -> VT * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    GridBarrier gb(&ctrl->bar, &ctrl->status);
    const unsigned N = (unsigned)g.N;
    const unsigned G = gridDim.x;
    const VT *x = W(j);
    VT *w = W(j + 1);
    const VT *v1 = W(1);
    // ---- stage 1: t = D (.) x - sum_a kap_a (x_{+a} + x_{-a})
    {
        const VT k0 = (VT)g.kap[0], k1 = (VT)g.kap[1], k2 = (VT)g.kap[2];
        GRID_LOOP2(N, {
            t[i] = stage1_at<DIM, VT>(g, x, D, i, k0, k1, k2);
        })
    }
    gb.sync();
    // ---- stage 2: w = gam_j (sigma t - sum_a s_a (t_{+a} + t_{-a})), partial w . W_1
    {
        const double gam = ctrl->gam[j - 1];
        const VT c0 = (VT)(gam * g.sigma), c1 = (VT)(gam * g.s[0]), c2 = (VT)(gam * g.s[1]),
                 c3 = (VT)(gam * g.s[2]);
        DotAcc<VT> acc;
        GRID_LOOP2(N, {
            const VT r = stage2_at<DIM, VT>(g, t, i, c0, c1, c2, c3, (VT)gam);
            w[i] = r;
            acc.add(r, v1[i]);
        })
        const double bsum = arn_block_sum(acc.value(), sh);
        if (threadIdx.x == 0) partials[G + blockIdx.x] = bsum;
    }
    arn_finish_round<VT>(gb, partials + G, 0, j, H, ldh, ctrl, &sc);     // h_{1j}
    // ---- modified Gram-Schmidt passes k = 1..j and the norm h_{j+1,j}
    for (int k = 1; k <= j; ++k) {
        const bool last = (k == j);
        const VT c = sc.c;
        const VT *vk = W(k), *vk1 = last ? W(k) : W(k + 1);
        double *part = partials + (size_t)((k + 1) & 1) * G;       // round k + 1
        DotAcc<VT> acc;
        GRID_LOOP2(N, {
            const VT r = fma(-c, vk[i], w[i]);
            w[i] = r;
            acc.add(r, last ? r : vk1[i]);
        })
        const double bsum = arn_block_sum(acc.value(), sh);
        if (threadIdx.x == 0) part[blockIdx.x] = bsum;
        arn_finish_round<VT>(gb, part, k, j, H, ldh, ctrl, &sc);
    }
}

// ---------------------------------------------------------------------------------------
// Shared-memory resident form of the same iteration for grids of at most R elements per
// thread (element r of a thread is i0 + r S, S = threads in the grid: the order of
// GRID_LOOP, so every sum and result is bit-identical to k_arnoldi).  Three buffers of
// R x 1024 values, in slots private to each thread: w from the w-stage to the last pass
// (stored as W_{j+1} there) and the two basis columns a pass needs.  Pass k updates with
// v_k, dots with v_{k+1}, then starts an asynchronous copy (cp.async) of v_{k+2} into the
// slots v_k has just left, so that load runs during the block reduction and the grid
// barrier instead of on the critical path of the next pass; v_1 and v_2 are requested at
// kernel start.  The passes then read only shared memory.
// ---------------------------------------------------------------------------------------
template <typename VT>
__device__ __forceinline__ void cp_async_elem(VT *dst, const VT *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(VT) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy this thread's elements of column v into its slots of buffer b (zeros past N).
template <typename VT>
__device__ __forceinline__ void prefetch_col(VT *b, const VT *v, unsigned i0, unsigned S,
                                             unsigned N, int R) {
#pragma unroll 4
    for (int r = 0; r < R; ++r) {
        const unsigned i = i0 + (unsigned)r * S;
        cp_async_elem(b + r * kArnThreads + threadIdx.x, v + (i < N ? i : 0u), i < N);
    }
}

constexpr int kArnResMaxBytes = 3 * 8 * kArnThreads * 8;   // 3 buffers of 8 FP64 per thread

template <int DIM, typename VT>
__global__ void __launch_bounds__(kArnThreads, 1)
k_arnoldi_res(Geom g, VT *__restrict__ slot0, VT *__restrict__ V, int64_t ldv,
              const VT *__restrict__ D, VT *__restrict__ t, double *H, int ldh, int j,
              double *partials, Ctrl *ctrl, int R) {
    if (!ctrl->active) return;                  // same value in every block
    __shared__ double sh[kArnThreads + 8];
    __shared__ ArnShared<VT> sc;
    extern __shared__ __align__(16) unsigned char dyn[];
    VT *bufW = reinterpret_cast<VT *>(dyn), *bufA = bufW + R * kArnThreads,
       *bufB = bufA + R * kArnThreads;
    auto W = [&](int c) -> VT * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    GridBarrier gb(&ctrl->bar, &ctrl->status);
    const unsigned N = (unsigned)g.N;
    const unsigned G = gridDim.x, S = G * kArnThreads;
    const unsigned i0 = blockIdx.x * kArnThreads + threadIdx.x;
    const int me = threadIdx.x;
    prefetch_col<VT>(bufA, W(1), i0, S, N, R);                   // v_1
    if (j >= 2) prefetch_col<VT>(bufB, W(2), i0, S, N, R);       // v_2
    // ---- stage 1: t = D (.) x - sum_a kap_a (x_{+a} + x_{-a})
    {
        const VT *x = W(j);
        const VT k0 = (VT)g.kap[0], k1 = (VT)g.kap[1], k2 = (VT)g.kap[2];
        GRID_LOOP2(N, {
            t[i] = stage1_at<DIM, VT>(g, x, D, i, k0, k1, k2);
        })
    }
    gb.sync();
    // ---- stage 2: w = gam_j (sigma t - sum_a s_a (t_{+a} + t_{-a})), partial w . W_1
    {
        const double gam = ctrl->gam[j - 1];
        const VT c0 = (VT)(gam * g.sigma), c1 = (VT)(gam * g.s[0]), c2 = (VT)(gam * g.s[1]),
                 c3 = (VT)(gam * g.s[2]);
        cp_async_wait_all();
        DotAcc<VT> acc;
        int slot = me;
        GRID_LOOP2(N, {
            const VT q = stage2_at<DIM, VT>(g, t, i, c0, c1, c2, c3, (VT)gam);
            bufW[slot] = q;
            acc.add(q, bufA[slot]);
            slot += kArnThreads;                // elements of this thread come in order
        })
        const double bsum = arn_block_sum(acc.value(), sh);
        if (threadIdx.x == 0) partials[G + blockIdx.x] = bsum;
    }
    arn_finish_round<VT>(gb, partials + G, 0, j, H, ldh, ctrl, &sc);     // h_{1j}
    VT *out = W(j + 1);
    // elements of this thread that exist (the rest of its slots hold zeros)
    const int Rn = i0 < N ? (int)min((unsigned)R, (N - i0 + S - 1) / S) : 0;
    // ---- modified Gram-Schmidt passes k = 1..j and the norm h_{j+1,j};
    //      odd passes update with buffer A and dot with B, even passes the other way round
    for (int k = 1; k <= j; ++k) {
        const bool last = (k == j);
        const VT c = sc.c;
        VT *U = (k & 1) ? bufA : bufB;
        const VT *Dt = (k & 1) ? bufB : bufA;
        const VT *pre = (k + 2 <= j) ? W(k + 2) : nullptr;
        double *part = partials + (size_t)((k + 1) & 1) * G;       // round k + 1
        cp_async_wait_all();                                       // v_{k+1} has landed
        DotAcc<VT> acc;
        if (!last) {
#pragma unroll 4
            for (int r = 0; r < Rn; ++r) {
                const int slot = r * kArnThreads + me;
                const VT x = fma(-c, U[slot], bufW[slot]);
                bufW[slot] = x;
                acc.add(x, Dt[slot]);
                if (pre) cp_async_elem(U + slot, pre + i0 + (unsigned)r * S, true);  // v_{k+2}
            }
        } else {
#pragma unroll 4
            for (int r = 0; r < Rn; ++r) {
                const int slot = r * kArnThreads + me;
                const VT x = fma(-c, U[slot], bufW[slot]);
                out[i0 + (unsigned)r * S] = x;
                acc.add(x, x);
            }
        }
        const double bsum = arn_block_sum(acc.value(), sh);
        if (threadIdx.x == 0) part[blockIdx.x] = bsum;
        arn_finish_round<VT>(gb, part, k, j, H, ldh, ctrl, &sc);
    }
}

// ---------------------------------------------------------------------------------------
// Arnoldi iteration j for an FP32 basis with Gram-corrected modified Gram-Schmidt.
//
// Fig. 2's modified Gram-Schmidt gives h_kj = v_k . w^(k-1) with w^(k-1) = w - sum_{i<k} h_ij v_i, i.e.
//     h_kj = c_k - sum_{i<k} G_ki h_ij,   c_k = v_k . w,   G_ki = v_k . v_i   (i < k),
// an identity for any computed basis, so these are the modified Gram-Schmidt coefficients
// (not classical Gram-Schmidt, which drops the G terms).  All c_k, and the Gram row of the
// newest vector v_j, come from one sweep over the basis and one grid-wide reduction; the
// update and the new norm from a second sweep.  An iteration needs 3 grid synchronisations
// instead of j + 2, which is what bounds the FP32 iteration (its arithmetic is cheap).  The
// rounding differs from the sequential passes (the FP64 path keeps them, for parity with
// the oracle).
//
//   stage 1, stage 2 (w = A_hat v_j, into the W_{j+1} slot)      | barrier after stage 1
//   round A: c_k = v_k . w (k = 1..j), G_ji = v_j . v_i (i < j)   | grid reduction
//   forward substitution for h_kj (warp 0 of every block, identical)
//   round B: w' = w - sum_k h_kj v_k and ||w'||^2                 | grid reduction
//   h_{j+1,j} = ||w'||, gam_j = 1 / h_{j+1,j}
//
// Per-thread dot products are compensated FP32 pairs (DotAcc<float>); block and grid sums
// add those pairs in double-float FP32 arithmetic in a fixed order (FP64 adds would cost 64
// cycles each on GB300), so results are deterministic.
// ---------------------------------------------------------------------------------------
constexpr int kGsChunk = 8;                          // values per block reduction
constexpr int kGsSmemBytes = kGsChunk * kArnThreads * (int)sizeof(float2)      // block sums
                             + 4 * kArnThreads * (int)sizeof(float4);             // w, v_j cache

// Block sums of nk <= kGsChunk per-thread pairs acc[q] (1024 threads), written as pairs
// to out[q] by the warps q.  red holds kGsChunk x 1024 pairs.
__device__ __forceinline__ void gs_block_sums(const DotAcc<float> (&acc)[kGsChunk], int nk,
                                              float2 *red, float2 *out) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < kGsChunk; ++q) red[q * kArnThreads + tid] = make_float2(acc[q].s, acc[q].c);
    __syncthreads();
    // level 1: value q = tid / 128; thread adds 8 consecutive pairs of its value
    const int q1 = tid >> 7, sg = tid & 127;
    float2 a = make_float2(0.f, 0.f);
    if (q1 < nk) {
        const float2 *p = red + q1 * kArnThreads + sg * 8;
        a = ff_add(ff_add(ff_add(p[0], p[1]), ff_add(p[2], p[3])), ff_add(ff_add(p[4], p[5]), ff_add(p[6], p[7])));
    }
    __syncthreads();
    if (q1 < nk) red[q1 * kArnThreads + sg] = a;
    __syncthreads();
    // level 2: warp q adds the 128 partials of value q (4 per lane, then a shuffle tree)
    const int wq = tid >> 5, lane = tid & 31;
    if (wq < nk) {
        const float2 *p = red + wq * kArnThreads + lane * 4;
        float2 b = ff_add(ff_add(p[0], p[1]), ff_add(p[2], p[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 c;
            c.x = __shfl_down_sync(0xffffffffu, b.x, o);
            c.y = __shfl_down_sync(0xffffffffu, b.y, o);
            b = ff_add(b, c);
        }
        if (lane == 0) out[wq] = b;
    }
    __syncthreads();
}

// Grid sum of value q over the G block pairs part[q * G + b], by warp q (pairs added in a
// fixed order), as a double in lane 0.
__device__ __forceinline__ double gs_grid_sum_warp(const float2 *part, int q) {
    const unsigned G = gridDim.x, lane = threadIdx.x & 31;
    float2 v[kMaxArnBlocks / 32];
#pragma unroll
    for (int s = 0; s < kMaxArnBlocks / 32; ++s) {
        const unsigned b = lane + 32u * s;
        v[s] = make_float2(0.f, 0.f);
        if (b < G) {
            const float2 x = __ldcg(reinterpret_cast<const float2 *>(part) + (size_t)q * G + b);
            v[s] = x;
        }
    }
    float2 a = v[0];
#pragma unroll
    for (int s = 1; s < kMaxArnBlocks / 32; ++s) a = ff_add(a, v[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 c;
        c.x = __shfl_down_sync(0xffffffffu, a.x, o);
        c.y = __shfl_down_sync(0xffffffffu, a.y, o);
        a = ff_add(a, c);
    }
    return (double)a.x + (double)a.y;
}

// Difference sums d_a = (x - x_{+a}) + (x - x_{-a}) of the four consecutive points 4q..4q+3
// (one row when n0 % 4 == 0), from 16-byte loads of the point's row and of the neighbouring
// rows (planes) plus two scalars across the row ends; the same operations per point as
// pair_diffs, so results are identical to the scalar stages.
template <int DIM>
__device__ __forceinline__ void group_diffs(const Geom &g, const float *__restrict__ x, unsigned q,
                                            float4 &xc, float4 (&d)[3]) {
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned i = 4u * q, c0 = i % n0, r = i / n0, c1 = r % n1;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const unsigned r4 = n0 / 4u;                                  // float4s per row
    xc = x4[q];
    const float xl = x[c0 == 0u ? i + n0 - 1u : i - 1u];
    const float xr = x[c0 + 4u == n0 ? i + 4u - n0 : i + 4u];
    d[0] = make_float4((xc.x - xc.y) + (xc.x - xl), (xc.y - xc.z) + (xc.y - xc.x),
                       (xc.z - xc.w) + (xc.z - xc.y), (xc.w - xr) + (xc.w - xc.z));
    const float4 yp = x4[c1 + 1u == n1 ? q - (n1 - 1u) * r4 : q + r4];
    const float4 ym = x4[c1 == 0u ? q + (n1 - 1u) * r4 : q - r4];
    d[1] = make_float4((xc.x - yp.x) + (xc.x - ym.x), (xc.y - yp.y) + (xc.y - ym.y),
                       (xc.z - yp.z) + (xc.z - ym.z), (xc.w - yp.w) + (xc.w - ym.w));
    if (DIM == 3) {
        const unsigned n2 = (unsigned)g.n[2], c2 = r / n1, p4 = r4 * n1;
        const float4 zp = x4[c2 + 1u == n2 ? q - (n2 - 1u) * p4 : q + p4];
        const float4 zm = x4[c2 == 0u ? q + (n2 - 1u) * p4 : q - p4];
        d[2] = make_float4((xc.x - zp.x) + (xc.x - zm.x), (xc.y - zp.y) + (xc.y - zm.y),
                           (xc.z - zp.z) + (xc.z - zm.z), (xc.w - zp.w) + (xc.w - zm.w));
    } else {
        d[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int DIM>
__global__ void __launch_bounds__(kArnThreads, 1)
k_arnoldi_gmgs(Geom g, float *__restrict__ slot0, float *__restrict__ V, int64_t ldv,
               const float *__restrict__ D, float *__restrict__ t, double *H, int ldh, int j,
               float2 *gpart, double *gram, int ldg, Ctrl *ctrl) {
    if (!ctrl->active) return;                  // same value in every block
    extern __shared__ __align__(16) unsigned char dyn[];
    float2 *red = reinterpret_cast<float2 *>(dyn);
    // at most two groups per thread (grids up to 8 points per thread): w and v_j stay in
    // shared memory between stage 2 and the end of the iteration
    float4 *wsm = reinterpret_cast<float4 *>(red + kGsChunk * kArnThreads);   // [2][1024]
    float4 *xsm = wsm + 2 * kArnThreads;                                       // [2][1024]
    __shared__ double gams[kGsMaxJ + 1];        // gam_0..gam_j
    __shared__ float hsm[32];                   // h of the substitution sweeps
    __shared__ float2 bout[kGsChunk];
    __shared__ double cs[kGsMaxJ + 1];          // grid sums of the round
    __shared__ float gs[kGsMaxJ][kGsMaxJ + 2];  // G_ki (k > i), 0-based; odd row stride: no bank conflicts
    __shared__ float as[kGsMaxJ];               // update coefficients h_kj gam_{k-1}
    auto W = [&](int c) -> float * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    GridBarrier gb(&ctrl->bar, &ctrl->status);
    const unsigned N = (unsigned)g.N;
    const unsigned G = gridDim.x;
    float *w = W(j + 1);
    float2 *pA = gpart, *pB = gpart + (size_t)2 * (kGsMaxJ + 1) * G;
    for (int e = threadIdx.x; e < j; e += blockDim.x) gams[e] = ctrl->gam[e];
    // Gram rows of v_2..v_{j-1} against the earlier vectors (from iterations 2..j-1); the
    // row of v_j comes from this iteration's round A
    for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
        const int k = e / j, i = e % j;
        gs[k][i] = (i < k && k < j - 1) ? (float)gram[(size_t)k * ldg + i] : 0.f;
    }
    // The stages and the sweeps visit the points in groups of four consecutive ones (group
    // q: points 4q..4q+3, groups strided over the grid's threads; the last group may be
    // partial), so every column is read with 16-byte loads and a thread keeps the same
    // points from stage 2 to the end of the iteration: w needs no barrier between them.
    // Rows of a multiple of four points take whole groups in the stencil stages too.
    const unsigned NG = (N + 3u) / 4u, S = G * kArnThreads;
    const unsigned q0 = blockIdx.x * kArnThreads + threadIdx.x;
    // (grouped stencils assume periodic rows and unit mobility; other grids take the scalar path)
    const bool rows4 = (g.n[0] & 3) == 0 && g.bc == 0 && g.mf[0] == nullptr;
    const bool res = NG <= 2u * S;
    // ---- stage 1: t = J x + sum_a kap_a ((x - x_{+a}) + (x - x_{-a}))
    {
        const float *x = W(j);
        const float k0 = (float)g.kap[0], k1 = (float)g.kap[1], k2 = (float)g.kap[2];
        if (rows4) {
            for (unsigned q = q0; q < NG; q += S) {
                float4 xc, d[3];
                group_diffs<DIM>(g, x, q, xc, d);
                const float4 dq = reinterpret_cast<const float4 *>(D)[q];
                float4 r;
                r.x = dq.x * xc.x; r.y = dq.y * xc.y; r.z = dq.z * xc.z; r.w = dq.w * xc.w;
                r.x = fmaf(k0, d[0].x, r.x); r.y = fmaf(k0, d[0].y, r.y);
                r.z = fmaf(k0, d[0].z, r.z); r.w = fmaf(k0, d[0].w, r.w);
                r.x = fmaf(k1, d[1].x, r.x); r.y = fmaf(k1, d[1].y, r.y);
                r.z = fmaf(k1, d[1].z, r.z); r.w = fmaf(k1, d[1].w, r.w);
                if (DIM == 3) {
                    r.x = fmaf(k2, d[2].x, r.x); r.y = fmaf(k2, d[2].y, r.y);
                    r.z = fmaf(k2, d[2].z, r.z); r.w = fmaf(k2, d[2].w, r.w);
                }
                reinterpret_cast<float4 *>(t)[q] = r;
            }
        } else {
            GRID_LOOP2(N, {
                t[i] = stage1_at<DIM, float>(g, x, D, i, k0, k1, k2);
            })
        }
    }
    gb.sync();
    auto ld4 = [&](const float *col, unsigned q, bool full) -> float4 {
        if (full) return reinterpret_cast<const float4 *>(col)[q];
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4u * q + 0u < N) r.x = col[4u * q + 0u];
        if (4u * q + 1u < N) r.y = col[4u * q + 1u];
        if (4u * q + 2u < N) r.z = col[4u * q + 2u];
        return r;                                   // a partial group has at most 3 points
    };
    // ---- stage 2: w = gam_j sum_a s_a ((t - t_{+a}) + (t - t_{-a})) = A_hat v_j, one group of
    //      four points (zeros past N)
    const double gam2 = ctrl->gam[j - 1];
    const float sc0 = (float)(gam2 * g.sigma), sc1 = (float)(gam2 * g.s[0]), sc2 = (float)(gam2 * g.s[1]),
                sc3 = (float)(gam2 * g.s[2]);
    auto stage2_group = [&](unsigned q) -> float4 {
        if (rows4) {
            float4 tc, d[3];
            group_diffs<DIM>(g, t, q, tc, d);
            float4 r;
            r.x = sc1 * d[0].x; r.y = sc1 * d[0].y; r.z = sc1 * d[0].z; r.w = sc1 * d[0].w;
            r.x = fmaf(sc2, d[1].x, r.x); r.y = fmaf(sc2, d[1].y, r.y);
            r.z = fmaf(sc2, d[1].z, r.z); r.w = fmaf(sc2, d[1].w, r.w);
            if (DIM == 3) {
                r.x = fmaf(sc3, d[2].x, r.x); r.y = fmaf(sc3, d[2].y, r.y);
                r.z = fmaf(sc3, d[2].z, r.z); r.w = fmaf(sc3, d[2].w, r.w);
            }
            return r;
        }
        float r[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (unsigned e = 0; e < 4u; ++e)
            if (4u * q + e < N) r[e] = stage2_at<DIM, float>(g, t, 4u * q + e, sc0, sc1, sc2, sc3, (float)gam2);
        return make_float4(r[0], r[1], r[2], r[3]);
    };
    auto st4 = [&](float *col, unsigned q, bool full, const float4 &v) {
        if (full) {
            reinterpret_cast<float4 *>(col)[q] = v;
        } else {
            if (4u * q + 0u < N) col[4u * q + 0u] = v.x;
            if (4u * q + 1u < N) col[4u * q + 1u] = v.y;
            if (4u * q + 2u < N) col[4u * q + 2u] = v.z;
        }
    };
    // the four products of a group are summed with plain FP32 FMAs (their rounding, random
    // over the grid, stays far below the basis rounding after the exact cross-thread sums);
    // only the running sums are compensated
    auto dot4 = [](const float4 &a, const float4 &b) {
        return __fmaf_rn(a.w, b.w, __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x))));
    };
    const bool down = (j & 1) != 0;
    const float *xj = W(j);
    const int ncA = (j + 3) / 4;
    // Round A: one sweep gives c_k = v_k . w (k = 1..j) and the Gram row of the newest basis
    // vector, G_ji = v_j . v_i (i < j): each column is read once for both, four columns per
    // pass over the points with their 16-byte loads issued together.  Consecutive sweeps
    // walk the basis in opposite directions, so each starts on the columns read last, the
    // likeliest to be still in L2.
    if (res) {
        // grids of at most 8 points per thread: w and v_j stay in shared memory from stage 2
        // to the end of the iteration
        for (unsigned q = q0, ri = 0; q < NG; q += S, ++ri) {
            wsm[ri * kArnThreads + threadIdx.x] = stage2_group(q);
            xsm[ri * kArnThreads + threadIdx.x] = ld4(xj, q, 4u * q + 3u < N);
        }
        for (int cA = 0; cA < ncA; ++cA) {
            const int k0 = 1 + (down ? ncA - 1 - cA : cA) * 4;
            const int nk = min(4, j - k0 + 1);
            DotAcc<float> acc[kGsChunk];                  // [u]: W_k . w, [4 + u]: W_k . W_j
            auto accum = [&](const float4 (&v)[4], const float4 &wv, const float4 &xv) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < nk) {
                        acc[u].add_value(dot4(wv, v[u]));
                        if (k0 + u < j) acc[4 + u].add_value(dot4(xv, v[u]));
                    }
            };
            // both groups of the thread: all eight loads in flight at once
            const unsigned qa = q0, qb = q0 + S;
            const bool ha = qa < NG, hb = qb < NG;
            const bool fa = 4u * qa + 3u < N, fb = 4u * qb + 3u < N;
            float4 va[4], vb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                va[u] = (ha && u < nk) ? ld4(W(k0 + u), qa, fa) : make_float4(0.f, 0.f, 0.f, 0.f);
                vb[u] = (hb && u < nk) ? ld4(W(k0 + u), qb, fb) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (ha) accum(va, wsm[threadIdx.x], xsm[threadIdx.x]);
            if (hb) accum(vb, wsm[kArnThreads + threadIdx.x], xsm[kArnThreads + threadIdx.x]);
            gs_block_sums(acc, kGsChunk, red, bout);
            const int u = threadIdx.x & 3;
            if (threadIdx.x < 4 && u < nk)
                pA[(size_t)(k0 - 1 + u) * G + blockIdx.x] = bout[u];
            else if (threadIdx.x >= 4 && threadIdx.x < 8 && u < nk && k0 + u < j)
                pA[(size_t)(kGsMaxJ + 1 + k0 - 1 + u) * G + blockIdx.x] = bout[4 + u];
        }
    } else {
        // Larger grids: stage 2 runs here, tile by tile (two groups per thread), and each
        // tile's w and v_j meet every basis column while still on chip, so w is written once
        // and neither it nor v_j is read again in round A (v_j serves as column j too).
        // Per-thread sums cover one tile and one column chunk; they are added across the
        // warp by a transposing shuffle tree and accumulated in the warp's 64 pair slots in
        // shared memory (slot k - 1: W_k . w, slot 32 + i - 1: W_i . W_j).
        float2 *accw = red + (threadIdx.x >> 5) * 64;
        const unsigned lane = threadIdx.x & 31u;
        accw[lane] = make_float2(0.f, 0.f);
        accw[32 + lane] = make_float2(0.f, 0.f);
        __syncwarp();
        // The tile loop runs the same number of trips in every thread of the block (the
        // shuffle tree needs whole warps); threads past the grid's last group add zeros.
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (unsigned base = blockIdx.x * kArnThreads; base < NG; base += 2u * S) {
            const unsigned qa = base + threadIdx.x, qb = qa + S;
            const bool ha = qa < NG, hb = qb < NG;
            const bool fa = ha && 4u * qa + 3u < N, fb = hb && 4u * qb + 3u < N;
            {
                const float4 wa = ha ? stage2_group(qa) : zero4;
                if (ha) st4(w, qa, fa, wa);
                wsm[threadIdx.x] = wa;
                xsm[threadIdx.x] = ha ? ld4(xj, qa, fa) : zero4;
                const float4 wb = hb ? stage2_group(qb) : zero4;
                if (hb) st4(w, qb, fb, wb);
                wsm[kArnThreads + threadIdx.x] = wb;
                xsm[kArnThreads + threadIdx.x] = hb ? ld4(xj, qb, fb) : zero4;
            }
            for (int cA = 0; cA < ncA; ++cA) {
                const int k0 = 1 + (down ? ncA - 1 - cA : cA) * 4;
                const int nk = min(4, j - k0 + 1);
                float4 va[4], vb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < nk && k0 + u < j) {
                        va[u] = ha ? ld4(W(k0 + u), qa, fa) : zero4;
                        vb[u] = hb ? ld4(W(k0 + u), qb, fb) : zero4;
                    } else if (u < nk) {                    // column j is v_j itself
                        va[u] = xsm[threadIdx.x];
                        vb[u] = xsm[kArnThreads + threadIdx.x];
                    } else {
                        va[u] = vb[u] = zero4;
                    }
                }
                DotAcc<float> acc[kGsChunk];                  // [u]: W_k . w, [4 + u]: W_k . W_j
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 wv = wsm[r * kArnThreads + threadIdx.x], xv = xsm[r * kArnThreads + threadIdx.x];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc[u].add_value(dot4(wv, r == 0 ? va[u] : vb[u]));
                        acc[4 + u].add_value(dot4(xv, r == 0 ? va[u] : vb[u]));
                    }
                }
                float2 p[kGsChunk];
#pragma unroll
                for (int u = 0; u < kGsChunk; ++u) p[u] = make_float2(acc[u].s, acc[u].c);
                // transposing shuffle tree: after the exchanges at distances 16, 8 and 4 a
                // lane holds value (lane >> 2) of its quad-group; distances 2 and 1 finish it
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool hi = (lane & 16u) != 0;
                    const float2 keep = hi ? p[i + 4] : p[i], send = hi ? p[i] : p[i + 4];
                    float2 r;
                    r.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
                    r.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
                    p[i] = ff_add(keep, r);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const bool hi = (lane & 8u) != 0;
                    const float2 keep = hi ? p[i + 2] : p[i], send = hi ? p[i] : p[i + 2];
                    float2 r;
                    r.x = __shfl_xor_sync(0xffffffffu, send.x, 8);
                    r.y = __shfl_xor_sync(0xffffffffu, send.y, 8);
                    p[i] = ff_add(keep, r);
                }
                float2 s;
                {
                    const bool hi = (lane & 4u) != 0;
                    const float2 keep = hi ? p[1] : p[0], send = hi ? p[0] : p[1];
                    float2 r;
                    r.x = __shfl_xor_sync(0xffffffffu, send.x, 4);
                    r.y = __shfl_xor_sync(0xffffffffu, send.y, 4);
                    s = ff_add(keep, r);
                }
#pragma unroll
                for (int o = 2; o > 0; o >>= 1) {
                    float2 r;
                    r.x = __shfl_xor_sync(0xffffffffu, s.x, o);
                    r.y = __shfl_xor_sync(0xffffffffu, s.y, o);
                    s = ff_add(s, r);
                }
                const int v = (int)(lane >> 2), u = v & 3;
                if ((lane & 3u) == 0 && u < nk && (v < 4 || k0 + u < j)) {
                    const int slot = (v < 4 ? 0 : 32) + k0 - 1 + u;
                    accw[slot] = ff_add(accw[slot], s);
                }
            }
        }
        __syncthreads();
        // block sums: warp q adds slot q (and slot 32 + q) over the 32 warps
        {
            const int wq = threadIdx.x >> 5;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int slot = wq + 32 * h;
                if (h == 0 ? wq < j : wq < j - 1) {
                    float2 b = red[lane * 64 + slot];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float2 c;
                        c.x = __shfl_down_sync(0xffffffffu, b.x, o);
                        c.y = __shfl_down_sync(0xffffffffu, b.y, o);
                        b = ff_add(b, c);
                    }
                    if (lane == 0) pA[(size_t)(h == 0 ? wq : kGsMaxJ + 1 + wq) * G + blockIdx.x] = b;
                }
            }
        }
    }
    gb.sync();
    {   // slot k-1: W_k . w;  slot 32 + i - 1: W_i . W_j
        const int wq = threadIdx.x >> 5;
        if (wq < j) {
            const double sum = gs_grid_sum_warp(pA, wq);
            if ((threadIdx.x & 31) == 0) cs[wq] = gams[wq] * sum;          // c_k = v_k . w
        }
        if (wq < j - 1) {
            const double sum = gs_grid_sum_warp(pA, kGsMaxJ + 1 + wq);
            if ((threadIdx.x & 31) == 0) {
                const double gji = gams[j - 1] * gams[wq] * sum;            // G_ji = v_j . v_i
                gs[j - 1][wq] = (float)gji;
                if (blockIdx.x == 0) gram[(size_t)(j - 1) * ldg + wq] = gji;
            }
        }
    }
    __syncthreads();
    // ---- forward substitution h_k = c_k - sum_{i<k} G_ki h_i (lane k-1 of warp 0).  The
    //      corrections are small next to c_k and are accumulated in FP32; h_k is FP64.
    //      G is strictly lower triangular, so the sweeps h <- c - G h reach the solution
    //      after at most j of them, and after a few when the basis is nearly orthogonal;
    //      each sweep is one independent FMA chain per lane instead of j dependent shuffle
    //      steps.  The sweeps stop once the FP32 corrections no longer change (the same
    //      decision in every block); otherwise the sequential substitution finishes.
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        const double r = l < j ? cs[l] : 0.0;
        const float rf = (float)r;
        float corr = 0.f;
        bool done = false;
        for (int sweep = 0; sweep < 4 && !done; ++sweep) {
            hsm[l] = __fsub_rn(rf, corr);
            __syncwarp();
            float c2 = 0.f;
            if (l < j)
                for (int i = 0; i < l; ++i) c2 = __fmaf_rn(gs[l][i], hsm[i], c2);
            __syncwarp();
            done = __all_sync(0xffffffffu, c2 == corr);
            corr = c2;
        }
        if (!done) {
            corr = 0.f;
            float gnext = l < j ? gs[l][0] : 0.f;   // the next G entry is read one step ahead
            for (int i = 0; i < j; ++i) {
                const float gcur = (l > i && l < j) ? gnext : 0.f;
                gnext = (i + 1 < j && l < j) ? gs[l][i + 1] : 0.f;
                const float hi = __shfl_sync(0xffffffffu, __fsub_rn(rf, corr), i);
                corr = __fmaf_rn(gcur, hi, corr);
            }
        }
        if (l < j) {
            const double h = r - (double)corr;
            as[l] = (float)(h * gams[l]);
            if (blockIdx.x == 0) H[l * ldh + (j - 1)] = h;
        }
    }
    __syncthreads();
    // ---- round B: w' = w - sum_k h_kj v_k (eight columns per batch) and ||w'||^2
    {
        const int ncU = (j + 7) / 8;
        DotAcc<float> acc[kGsChunk];
        for (unsigned q = q0, ri = 0; q < NG; q += S, ++ri) {
            const bool full = 4u * q + 3u < N;
            float4 x = res ? wsm[ri * kArnThreads + threadIdx.x] : ld4(w, q, full);
            for (int cB = 0; cB < ncU; ++cB) {
                const int k0 = 1 + (down ? cB : ncU - 1 - cB) * 8;
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = k0 + u <= j ? ld4(W(k0 + u), q, full) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (k0 + u <= j) {
                        const float a_ = -as[k0 + u - 1];
                        x.x = __fmaf_rn(a_, v[u].x, x.x);
                        x.y = __fmaf_rn(a_, v[u].y, x.y);
                        x.z = __fmaf_rn(a_, v[u].z, x.z);
                        x.w = __fmaf_rn(a_, v[u].w, x.w);
                    }
            }
            if (full) {
                reinterpret_cast<float4 *>(w)[q] = x;
            } else {
                if (4u * q + 0u < N) w[4u * q + 0u] = x.x;
                if (4u * q + 1u < N) w[4u * q + 1u] = x.y;
                if (4u * q + 2u < N) w[4u * q + 2u] = x.z;
            }
            // zero past N (partial groups hold zeros)
            acc[0].add_value(__fmaf_rn(x.w, x.w, __fmaf_rn(x.z, x.z, __fmaf_rn(x.y, x.y, __fmul_rn(x.x, x.x)))));
        }
        gs_block_sums(acc, 1, red, bout);
        if (threadIdx.x == 0) pB[blockIdx.x] = bout[0];
    }
    gb.sync();
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double nrm2 = gs_grid_sum_warp(pB, 0);
        if (threadIdx.x == 0) {
            const double hn = sqrt(nrm2);                         // h_{j+1,j} (Fig. 2)
            ctrl->hnext2 = nrm2;
            H[j * ldh + (j - 1)] = hn;
            ctrl->gam[j] = 1.0 / hn;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Arnoldi iteration j for an FP64 basis with the Gram-corrected coefficients (the identity
// h_kj = c_k - sum_{i<k} G_ki h_ij of k_arnoldi_gmgs, in FP64 throughout):
//   stage 1, stage 2 (w = A_hat v_j into the W_{j+1} slot)       | barrier after stage 1
//   round A: c_k = v_k . w (k = 1..j), G_ji = v_j . v_i (i < j)   | grid reduction
//   forward substitution for h_kj (warp 0 of every block, identical)
//   round B: w' = w - sum_k h_kj v_k and ||w'||^2                 | grid reduction
// Three grid synchronisations per iteration instead of j + 2, for 2j + 1 more FMAs per point
// than the sequential passes: the form for grids whose passes are bound by synchronisation
// rather than by FP64 issue or HBM (up to kG64MaxPoints points).  FP64 block and grid sums
// in a fixed order: deterministic.  gpart holds 2 (kGsMaxJ + 1) G partials, gram the Gram
// rows of the run (row k for vector k + 1, ldg = row stride).
// ---------------------------------------------------------------------------------------
constexpr int kG64Vals = 8;                  // values per block reduction (4 columns x 2)

// Block sums of nv <= 8 per-thread doubles acc[q] (1024 threads), in out[q] for all threads.
__device__ __forceinline__ void g64_block_sums(const double (&acc)[kG64Vals], int nv, double *red,
                                               double *out) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < kG64Vals; ++q) red[q * kArnThreads + tid] = acc[q];
    __syncthreads();
    const int wq = tid >> 5, lane = tid & 31;
    if (wq < nv) {      // warp q adds value q: 32 per lane in pairwise groups of 8, then shuffles
        const double *p = red + wq * kArnThreads + lane;
        double c[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            double v[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = p[32 * (8 * h + m)];
            c[h] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        }
        double a = (c[0] + c[1]) + (c[2] + c[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[wq] = a;
    }
    __syncthreads();
}

// Sum of the G per-block partials part[0..G) by one warp (any warp of the block), pairwise
// in a fixed order; valid in its lane 0 and identical in every block.
__device__ __forceinline__ double g64_grid_sum(const double *part) {
    const unsigned G = gridDim.x, lane = threadIdx.x & 31u;
    double v[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) v[s] = (lane + 32u * s < G) ? __ldcg(&part[lane + 32u * s]) : 0.0;
    double a = ((v[0] + v[1]) + (v[2] + v[3])) + v[4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    return a;
}

template <int DIM>
__global__ void __launch_bounds__(kArnThreads, 1)
k_arnoldi_g64(Geom g, double *__restrict__ slot0, double *__restrict__ V, int64_t ldv,
              const double *__restrict__ D, double *__restrict__ t, double *H, int ldh, int j,
              double *gpart, double *gram, int ldg, Ctrl *ctrl) {
    if (!ctrl->active) return;                  // same value in every block
    extern __shared__ __align__(16) unsigned char dyn[];
    double *red = reinterpret_cast<double *>(dyn);            // kG64Vals x 1024
    __shared__ double bout[kG64Vals];
    __shared__ double gams[kGsMaxJ + 1];
    __shared__ double cs[kGsMaxJ + 1];
    __shared__ double gs[kGsMaxJ][kGsMaxJ + 1];    // G_ki (k > i), 0-based
    __shared__ double as[kGsMaxJ];
    auto W = [&](int c) -> double * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    GridBarrier gb(&ctrl->bar, &ctrl->status);
    const unsigned N = (unsigned)g.N;
    const unsigned G = gridDim.x;
    double *w = W(j + 1);
    double *pA = gpart, *pB = gpart + (size_t)2 * (kGsMaxJ + 1) * G;
    for (int e = threadIdx.x; e < j; e += blockDim.x) gams[e] = ctrl->gam[e];
    for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
        const int k = e / j, i = e % j;
        gs[k][i] = (i < k && k < j - 1) ? gram[(size_t)k * ldg + i] : 0.0;
    }
    // ---- stage 1: t = D (.) x - sum_a kap_a (x_{+a} + x_{-a})
    {
        const double *x = W(j);
        GRID_LOOP2(N, {
            t[i] = stage1_at<DIM, double>(g, x, D, i, g.kap[0], g.kap[1], g.kap[2]);
        })
    }
    gb.sync();
    // ---- stage 2: w = gam_j (sigma t - sum_a s_a (t_{+a} + t_{-a}))
    {
        const double gam = gams[j - 1];
        const double c0 = gam * g.sigma, c1 = gam * g.s[0], c2 = gam * g.s[1], c3 = gam * g.s[2];
        GRID_LOOP2(N, {
            w[i] = stage2_at<DIM, double>(g, t, i, c0, c1, c2, c3, gam);
        })
    }
    // ---- round A: c_k = W_k . w and W_k . W_j, four columns per sweep over this thread's points
    const double *xj = W(j);
    for (int k0 = 1; k0 <= j; k0 += 4) {
        const int nk = min(4, j - k0 + 1);
        double acc[kG64Vals];
#pragma unroll
        for (int q = 0; q < kG64Vals; ++q) acc[q] = 0.0;
        const double *v0 = W(k0), *v1 = nk > 1 ? W(k0 + 1) : v0, *v2 = nk > 2 ? W(k0 + 2) : v0,
                     *v3 = nk > 3 ? W(k0 + 3) : v0;
        GRID_LOOP(i, N) {
            const double wv = w[i], xv = xj[i];
            const double a0 = v0[i], a1 = v1[i], a2 = v2[i], a3 = v3[i];
            acc[0] = fma(wv, a0, acc[0]); acc[4] = fma(xv, a0, acc[4]);
            acc[1] = fma(wv, a1, acc[1]); acc[5] = fma(xv, a1, acc[5]);
            acc[2] = fma(wv, a2, acc[2]); acc[6] = fma(xv, a2, acc[6]);
            acc[3] = fma(wv, a3, acc[3]); acc[7] = fma(xv, a3, acc[7]);
        }
        g64_block_sums(acc, kG64Vals, red, bout);
        if (threadIdx.x == 0)
            for (int u = 0; u < nk; ++u) {
                pA[(size_t)(k0 - 1 + u) * G + blockIdx.x] = bout[u];
                if (k0 + u < j) pA[(size_t)(kGsMaxJ + 1 + k0 - 1 + u) * G + blockIdx.x] = bout[4 + u];
            }
    }
    gb.sync();
    {   // slot k-1: W_k . w;  slot 32 + i - 1: W_i . W_j  (warp v sums value v over the blocks)
        const int wq = threadIdx.x >> 5;
        for (int v = wq; v < 2 * j - 1; v += 32) {
            const bool isc = v < j;
            const int k = isc ? v : v - j;
            const double sum = g64_grid_sum(pA + (size_t)(isc ? k : kGsMaxJ + 1 + k) * G);
            if ((threadIdx.x & 31) == 0) {
                if (isc) {
                    cs[k] = gams[k] * sum;                                    // c_k = v_k . w
                } else {
                    const double gji = gams[j - 1] * gams[k] * sum;           // G_jk = v_j . v_k
                    gs[j - 1][k] = gji;
                    if (blockIdx.x == 0) gram[(size_t)(j - 1) * ldg + k] = gji;
                }
            }
        }
    }
    __syncthreads();
    // ---- forward substitution h_k = c_k - sum_{i<k} G_ki h_i, sequential (lane k-1 of warp 0)
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        double corr = 0.0;
        for (int i = 0; i < j; ++i) {
            const double hi = __shfl_sync(0xffffffffu, (l < j ? cs[l] : 0.0) - corr, i);
            if (l > i && l < j) corr = fma(gs[l][i], hi, corr);
        }
        if (l < j) {
            const double h = cs[l] - corr;
            as[l] = h * gams[l];
            if (blockIdx.x == 0) H[l * ldh + (j - 1)] = h;
        }
    }
    __syncthreads();
    // ---- round B: w' = w - sum_k h_kj v_k (eight columns per batch) and ||w'||^2
    {
        double nrm = 0.0;
        GRID_LOOP(i, N) {
            double x = w[i];
            for (int k0 = 1; k0 <= j; k0 += 8) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = k0 + u <= j ? W(k0 + u)[i] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (k0 + u <= j) x = fma(-as[k0 + u - 1], v[u], x);
            }
            w[i] = x;
            nrm = fma(x, x, nrm);
        }
        double acc[kG64Vals] = {nrm, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        g64_block_sums(acc, 1, red, bout);
        if (threadIdx.x == 0) pB[blockIdx.x] = bout[0];
    }
    gb.sync();
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double nrm2 = g64_grid_sum(pB);
        if (threadIdx.x == 0) {
            const double hn = sqrt(nrm2);                         // h_{j+1,j} (Fig. 2)
            ctrl->hnext2 = nrm2;
            H[j * ldh + (j - 1)] = hn;
            ctrl->gam[j] = 1.0 / hn;
        }
    }
}

constexpr int kG64SmemBytes = kG64Vals * kArnThreads * (int)sizeof(double);

void launch_arnoldi_g64(const Launch &L, int blocks, const Geom &g, double *slot0, double *V,
                        int64_t ldv, const double *D, double *t, double *H, int ldh, int j,
                        double *gpart, double *gram, int ldg) {
    LaunchScope scope(L, CH_K_ARNOLDI);
    {   // algorithmic work of the iteration as the sequential passes count it (the Gram form
        // does 2j + 1 more FMAs per point, which are not counted as work)
        const double N = (double)g.N, d = g.dim;
        scope.work(((1.0 + 3.0 * d) + (3.0 + 3.0 * d) + 4.0 * j) * N, (5.0 + j) * 8.0 * N);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(kArnThreads, 1, 1);
    cfg.dynamicSmemBytes = kG64SmemBytes;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g.dim == 3)
        cudaLaunchKernelEx(&cfg, k_arnoldi_g64<3>, g, slot0, V, ldv, D, t, H, ldh, j, gpart, gram, ldg, L.ctrl);
    else
        cudaLaunchKernelEx(&cfg, k_arnoldi_g64<2>, g, slot0, V, ldv, D, t, H, ldh, j, gpart, gram, ldg, L.ctrl);
}

void launch_arnoldi_gmgs(const Launch &L, int blocks, const Geom &g, float *slot0, float *V,
                         int64_t ldv, const float *D, float *t, double *H, int ldh, int j,
                         float2 *gpart, double *gram, int ldg) {
    LaunchScope scope(L, CH_K_ARNOLDI);
    {   // stages as the MGS form; j + (j - 1) dots, j update fma and the norm (FP32)
        const double N = (double)g.N, d = g.dim;
        scope.work(((1.0 + 3.0 * d) + (1.0 + 3.0 * d) + 6.0 * j + 2.0) * N, (6.0 + 2.0 * j) * 4.0 * N);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(kArnThreads, 1, 1);
    cfg.dynamicSmemBytes = kGsSmemBytes;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g.dim == 3)
        cudaLaunchKernelEx(&cfg, k_arnoldi_gmgs<3>, g, slot0, V, ldv, D, t, H, ldh, j, gpart, gram, ldg, L.ctrl);
    else
        cudaLaunchKernelEx(&cfg, k_arnoldi_gmgs<2>, g, slot0, V, ldv, D, t, H, ldh, j, gpart, gram, ldg, L.ctrl);
}

template <typename VT>
int arnoldi_blocks(int dim, int64_t N) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dim == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<3, VT>, kArnThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<2, VT>, kArnThreads, 0);
    const int64_t want = (N + 2 * kArnThreads - 1) / (2 * kArnThreads);
    return (int)std::min<int64_t>(std::min<int64_t>(want, (int64_t)per_sm * sms), kMaxArnBlocks);
}
template int arnoldi_blocks<double>(int, int64_t);
template int arnoldi_blocks<float>(int, int64_t);

template <typename VT>
void launch_arnoldi(const Launch &L, int blocks, const Geom &g, VT *slot0, VT *V, int64_t ldv,
                    const VT *D, VT *t, double *H, int ldh, int j) {
    LaunchScope scope(L, CH_K_ARNOLDI);
    {   // stage 1: mul + d (add + fma); stage 2: the same + the dot fma; j passes of 2 fma.
        // Bytes: x, D, t written, t read, v_1..v_j read once, W_{j+1} written.
        const double N = (double)g.N, d = g.dim;
        scope.work(((1.0 + 3.0 * d) + (3.0 + 3.0 * d) + 4.0 * j) * N, (5.0 + j) * sizeof(VT) * N);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(kArnThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Ctrl *ctrl = L.ctrl;
    double *partials = L.partials;
    const int64_t per_thread = (g.N + (int64_t)blocks * kArnThreads - 1) / ((int64_t)blocks * kArnThreads);
    if (per_thread * 3 * kArnThreads * (int64_t)sizeof(VT) <= kArnResMaxBytes) {
        const int R = (int)per_thread;
        cfg.dynamicSmemBytes = (size_t)3 * R * kArnThreads * sizeof(VT);
        if (g.dim == 3)
            cudaLaunchKernelEx(&cfg, k_arnoldi_res<3, VT>, g, slot0, V, ldv, D, t, H, ldh, j, partials, ctrl, R);
        else
            cudaLaunchKernelEx(&cfg, k_arnoldi_res<2, VT>, g, slot0, V, ldv, D, t, H, ldh, j, partials, ctrl, R);
        return;
    }
    if (g.dim == 3)
        cudaLaunchKernelEx(&cfg, k_arnoldi<3, VT>, g, slot0, V, ldv, D, t, H, ldh, j, partials, ctrl);
    else
        cudaLaunchKernelEx(&cfg, k_arnoldi<2, VT>, g, slot0, V, ldv, D, t, H, ldh, j, partials, ctrl);
}

// Allow the resident kernels their dynamic shared memory (a function attribute, not a stream
// operation: set at grid creation, outside any graph capture).
int arnoldi_setup() {
    const void *fns[] = {(const void *)k_arnoldi_res<2, double>, (const void *)k_arnoldi_res<3, double>,
                         (const void *)k_arnoldi_res<2, float>, (const void *)k_arnoldi_res<3, float>};
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kArnResMaxBytes);
        if (e != cudaSuccess) return (int)e;
    }
    const void *gfns[] = {(const void *)k_arnoldi_gmgs<2>, (const void *)k_arnoldi_gmgs<3>};
    for (const void *f : gfns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGsSmemBytes);
        if (e != cudaSuccess) return (int)e;
    }
    const void *g64fns[] = {(const void *)k_arnoldi_g64<2>, (const void *)k_arnoldi_g64<3>};
    for (const void *f : g64fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kG64SmemBytes);
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}
template void launch_arnoldi<double>(const Launch &, int, const Geom &, double *, double *, int64_t,
                                     const double *, double *, double *, int, int);
template void launch_arnoldi<float>(const Launch &, int, const Geom &, float *, float *, int64_t,
                                    const float *, float *, double *, int, int);

// ---------------------------------------------------------------------------------------
// Krylov combine of Fig. 2: y_next = y0 + V_j (beta u) = y0 + sum_c coef_c W_c, coef_c = beta gam_c u_c.
// Column 0 is `v0`, columns 1.. start at V with stride ldv.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_combine(int64_t N, const double *__restrict__ y0, const double *__restrict__ v0,
          const double *__restrict__ V, int64_t ldv, double *__restrict__ ynext,
          const Ctrl *ctrl) {
    const int j = ctrl->jexit;
    __shared__ double coef[130];
    for (int c = threadIdx.x; c < j; c += blockDim.x) coef[c] = ctrl->coef[c];
    __syncthreads();
    GRID_LOOP2(N, {
        double acc = 0.0;
        if (j > 0) acc = coef[0] * v0[i];
        for (int c = 1; c < j; ++c) acc = fma(coef[c], V[(c - 1) * ldv + i], acc);
        ynext[i] = y0[i] + acc;
    })
}

// Mixed precision, pass 1: increment d = sum_c coef_c W_c in FP32 and its sum (mass) in
// compensated FP32 -> FP64 (red[6]).
__global__ void __launch_bounds__(kThreads)
k_combine32a(int64_t N, const float *__restrict__ v0, const float *__restrict__ V, int64_t ldv,
             float *__restrict__ d, double *partials, unsigned int *ticket, Ctrl *ctrl) {
    const int j = ctrl->jexit;
    __shared__ float coef[130];
    for (int c = threadIdx.x; c < j; c += blockDim.x) coef[c] = (float)ctrl->coef[c];
    __syncthreads();
    DotAcc<float> acc;
    GRID_LOOP(i, N) {
        float a = 0.f;
        if (j > 0) a = coef[0] * v0[i];
        for (int c = 1; c < j; ++c) a = fmaf(coef[c], V[(c - 1) * ldv + i], a);
        d[i] = a;
        acc.add(a, 1.0f);
    }
    double tot1[1] = {acc.value()};
    grid_sum<1>(tot1, partials, ticket, [&](double (&tot)[1]) { ctrl->red[6] = tot[0]; });
}

// Mixed precision, pass 2: y_next = y0 + (d - mean(d)); the increment of every Krylov step
// has zero mean in exact arithmetic (columns of A sum to zero, Eq. m), so removing the mean
// the FP32 rounding left keeps the mass to FP64 rounding.
__global__ void __launch_bounds__(kThreads)
k_combine32b(int64_t N, const double *__restrict__ y0, const float *__restrict__ d,
             double *__restrict__ ynext, const Ctrl *ctrl) {
    const double mean = ctrl->jexit > 0 ? ctrl->red[6] / (double)N : 0.0;
    GRID_LOOP(i, N) ynext[i] = y0[i] + ((double)d[i] - mean);
}

// FP64 -> FP32 copy y = x + shift (the start vector of a mixed-precision Krylov run with
// shift 0; the FP32 stage coefficient J = D - eps^2 sigma with shift -eps^2 sigma).
__global__ void __launch_bounds__(kThreads)
k_to32(int64_t N, const double *__restrict__ x, double shift, float *__restrict__ y) {
    GRID_LOOP(i, N) y[i] = (float)(x[i] + shift);
}

// ---------------------------------------------------------------------------------------
// Right-hand side of Eq. (IVP), f = -A mu with mu = F'(y) + eps^2 A y, and the pieces the
// schemes need from the same pass:
//   rhs1: mu = (y^2 + eps^2 sigma - 1) y - sum_a kap_a (y_{+a} + y_{-a}); q = 2y^3 [+ y]
//   rhs2: f = -(sigma mu - sum_a s_a (mu_{+a} + mu_{-a}));  g_hat = A q   (Eq. A_g)
//         mode bit 0: ||f||^2 -> red[0];  bit 1: ||g_hat||^2 -> red[1];
//         bit 2: Eq. (LIMest) sums with y_PC = y0 + tau/2 (f0 + f(y1)):
//                ||y1 - y_PC||^2 -> red[2], ||y_PC||^2 -> red[3]
//         bit 3: tau of the estimate is the step the Krylov run took (ctrl->tau)
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_rhs1(Geom g, const double *__restrict__ y, int eyre, double *__restrict__ mu,
       double *__restrict__ q) {
    const double cshift = g.eps2 * g.sigma - 1.0;
    GRID_LOOP2(g.N, {
        double ps[3];
        pair_sums<DIM>(g, y, i, ps);
        const double yi = y[i];
        const double y2 = yi * yi;
        double m = (y2 + cshift) * yi;
        m = fma(-g.kap[0], ps[0], m);
        m = fma(-g.kap[1], ps[1], m);
        if (DIM == 3) m = fma(-g.kap[2], ps[2], m);
        mu[i] = m;
        if (q) q[i] = eyre ? fma(2.0 * y2, yi, yi) : 2.0 * y2 * yi;
    })
}

template <int DIM, int K>
__global__ void __launch_bounds__(kThreads)
k_rhs2(Geom g, const double *__restrict__ mu, const double *__restrict__ q,
       double *__restrict__ f, const double *__restrict__ y0, const double *__restrict__ f0,
       const double *__restrict__ y1, double half_tau, int mode, double *partials,
       unsigned int *ticket, Ctrl *ctrl) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (mode & 8) half_tau = 0.5 * ctrl->tau;
    const bool mob = g.mf[0] != nullptr;
    GRID_LOOP2(g.N, {
        double r;
        if (mob) {
            r = -flux_at<DIM, double>(g, mu, i);
        } else {
            double ps[3];
            pair_sums<DIM>(g, mu, i, ps);
            r = -g.sigma * mu[i];
            r = fma(g.s[0], ps[0], r);
            r = fma(g.s[1], ps[1], r);
            if (DIM == 3) r = fma(g.s[2], ps[2], r);
        }
        f[i] = r;
        if (mode & 1) acc[0] = fma(r, r, acc[0]);
        if (mode & 2) {
            double gh;
            if (mob) {
                gh = flux_at<DIM, double>(g, q, i);
            } else {
                double qs[3];
                pair_sums<DIM>(g, q, i, qs);
                gh = g.sigma * q[i];
                gh = fma(-g.s[0], qs[0], gh);
                gh = fma(-g.s[1], qs[1], gh);
                if (DIM == 3) gh = fma(-g.s[2], qs[2], gh);
            }
            acc[1] = fma(gh, gh, acc[1]);
        }
        if (mode & 4) {
            const double ypc = fma(half_tau, f0[i] + r, y0[i]);
            const double d = y1[i] - ypc;
            acc[2] = fma(d, d, acc[2]);
            acc[3] = fma(ypc, ypc, acc[3]);
        }
    })
    if constexpr (K > 0) {
        double red[K];
#pragma unroll
        for (int k = 0; k < K; ++k) red[k] = acc[k];
        grid_sum<K>(red, partials, ticket, [&](double (&tot)[K]) {
            for (int k = 0; k < 4; ++k) ctrl->red[k] = k < K ? tot[k] : 0.0;
        });
    }
}

// ---------------------------------------------------------------------------------------
// Residual of the linearised implicit Euler system, r = g_hat - A_hat x  (the LIM update of Fig. 1,
// and the start vector of Fig. 2 for a restart from x = y_cur):
//   resid1: t = G - D (.) x + sum_a kap_a (x_{+a} + x_{-a})
//   resid2: r = sigma t - sum_a s_a (t_{+a} + t_{-a}),  ||r||^2 -> red[0]
//   lim2:   y_next = (y^n + tau a_m y_prev + tau r) / (1 + tau a_m)
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_resid1(Geom g, const double *__restrict__ x, const double *__restrict__ D,
         const double *__restrict__ G, double *__restrict__ t) {
    GRID_LOOP2(g.N, {
        double ps[3];
        pair_sums<DIM>(g, x, i, ps);
        double acc = fma(-D[i], x[i], G[i]);
        acc = fma(g.kap[0], ps[0], acc);
        acc = fma(g.kap[1], ps[1], acc);
        if (DIM == 3) acc = fma(g.kap[2], ps[2], acc);
        t[i] = acc;
    })
}

template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_resid2(Geom g, const double *__restrict__ t, double *__restrict__ out, double *partials,
         unsigned int *ticket, Ctrl *ctrl) {
    double acc[1] = {0.0};
    const bool mob = g.mf[0] != nullptr;
    GRID_LOOP2(g.N, {
        double r;
        if (mob) {
            r = flux_at<DIM, double>(g, t, i);
        } else {
            double ps[3];
            pair_sums<DIM>(g, t, i, ps);
            r = g.sigma * t[i];
            r = fma(-g.s[0], ps[0], r);
            r = fma(-g.s[1], ps[1], r);
            if (DIM == 3) r = fma(-g.s[2], ps[2], r);
        }
        out[i] = r;
        acc[0] = fma(r, r, acc[0]);
    })
    grid_sum<1>(acc, partials, ticket, [&](double (&tot)[1]) { ctrl->red[0] = tot[0]; });
}

// y_next = alpha (y^n + tau a y_prev + tau r) with alpha = 1/(1 + tau a) and r = A t; alpha tau
// is folded into the stage-2 coefficients: y_next = fma(alpha tau a, y_prev, fma(alpha, y^n, r'')).
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_lim2(Geom g, const double *__restrict__ t, const double *__restrict__ yn,
       const double *__restrict__ yprev, double *__restrict__ ynext, double tau_a, double tau,
       double alpha) {
    const double at = alpha * tau;
    const double c0 = at * g.sigma, c1 = at * g.s[0], c2 = at * g.s[1], c3 = at * g.s[2];
    const double ca = alpha * tau_a;
    const bool mob = g.mf[0] != nullptr;
    GRID_LOOP2(g.N, {
        double r;
        if (mob) {
            r = at * flux_at<DIM, double>(g, t, i);
        } else {
            double ps[3];
            pair_sums<DIM>(g, t, i, ps);
            r = c0 * t[i];
            r = fma(-c1, ps[0], r);
            r = fma(-c2, ps[1], r);
            if (DIM == 3) r = fma(-c3, ps[2], r);
        }
        ynext[i] = fma(ca, yprev[i], fma(alpha, yn[i], r));
    })
}

// ---------------------------------------------------------------------------------------
// LIM iteration of Fig. 1 in increment form for mixed-precision grids.  With
// y_prev = y^n + d and the identity g_hat - A_hat y^n = f(y^n) (Eq. A_g), the update reads
//     d_next = alpha (tau a_m d + tau (f^n - A_hat d)),   y^{n+1} = y^n + d_final,
// the same iterate as Fig. 1's, with rounding relative to the increment d, not to y.  Stage 1
// is k_tstage<float> on d (FP32 difference form with J); lim32: A t in FP32 and the update,
// f^n read in FP64.  d_prev == nullptr is the first iteration (d = 0, a_1 = 0).
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_lim32(Geom g, const float *__restrict__ t, const double *__restrict__ fn,
        const float *__restrict__ dprev, float *__restrict__ dnext, float ta, float atau) {
    const float c1 = (float)g.s[0], c2 = (float)g.s[1], c3 = (float)g.s[2];
    GRID_LOOP2(g.N, {
        float ad = 0.f;
        if (dprev) ad = stage2_at<DIM, float>(g, t, i, 0.f, c1, c2, c3, 1.f);      // A_hat d
        const float r = (float)fn[i] - ad;
        dnext[i] = dprev ? fmaf(ta, dprev[i], atau * r) : atau * r;
    })
}

// Sum of an FP32 increment (compensated, into red[6]) and y_next = y0 + (d - mean(d)): the
// increment of a LIM step has zero sum in exact arithmetic (columns of A sum to zero, Eq. m),
// so the FP32 rounding's share of the mass is removed.
__global__ void __launch_bounds__(kThreads)
k_sum32(int64_t N, const float *__restrict__ d, double *partials, unsigned int *ticket, Ctrl *ctrl) {
    DotAcc<float> acc;
    GRID_LOOP(i, N) acc.add_value(d[i]);
    double tot1[1] = {acc.value()};
    grid_sum<1>(tot1, partials, ticket, [&](double (&tot)[1]) { ctrl->red[6] = tot[0]; });
}

__global__ void __launch_bounds__(kThreads)
k_add_increment(int64_t N, const double *__restrict__ y0, const float *__restrict__ d,
                double *__restrict__ ynext, const Ctrl *ctrl) {
    const double mean = ctrl->red[6] / (double)N;
    GRID_LOOP(i, N) ynext[i] = y0[i] + ((double)d[i] - mean);
}

// Energy of Eq. (Ediscr) (periodic forward differences) and mass: red[6], red[7] (unscaled
// sums; the host multiplies by h^d).
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_energy(Geom g, const double *__restrict__ y, double *partials, unsigned int *ticket,
         Ctrl *ctrl) {
    double acc[2] = {0.0, 0.0};
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    GRID_LOOP(i, g.N) {
        const double yi = y[i];
        const double u = 1.0 - yi * yi;
        double e = 0.25 * u * u;
        const unsigned c0 = i % n0, r = i / n0, c1 = r % n1;
        double d0 = (y[nb_p(i, c0, n0, 1u, g.bc)] - yi) * (double)g.n[0];
        double d1 = (y[nb_p(i, c1, n1, n0, g.bc)] - yi) * (double)g.n[1];
        double gs = d0 * d0 + d1 * d1;
        if (DIM == 3) {
            const unsigned c2 = r / n1;
            double d2 = (y[nb_p(i, c2, (unsigned)g.n[2], n0 * n1, g.bc)] - yi) * (double)g.n[2];
            gs += d2 * d2;
        }
        acc[0] += fma(0.5 * g.eps2, gs, e);
        acc[1] += yi;
    }
    grid_sum<2>(acc, partials, ticket, [&](double (&tot)[2]) {
        ctrl->red[6] = tot[0];
        ctrl->red[7] = tot[1];
    });
}

// ---------------------------------------------------------------------------------------
// Face mobilities of a variable-mobility grid from nodal values M (the Remark on Eq.
// CHmob): mf_a[i] = s_a (M_i + M_{i+e_a}) / 2, with FP32 copies when mff is given.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_face_mob(Geom g, const double *__restrict__ M, double *mf0, double *mf1, double *mf2,
           float *mff0, float *mff1, float *mff2) {
    const unsigned n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1], n2 = (unsigned)g.n[2];
    double *mf[3] = {mf0, mf1, mf2};
    float *mff[3] = {mff0, mff1, mff2};
    GRID_LOOP(i, g.N) {
        const unsigned c0 = i % n0, r = i / n0, c1 = r % n1, c2 = r / n1;
        const unsigned nb[3] = {nb_p(i, c0, n0, 1u, g.bc), nb_p(i, c1, n1, n0, g.bc),
                                nb_p(i, c2, n2, n0 * n1, g.bc)};
        for (int a = 0; a < g.dim; ++a) {
            const double v = g.s[a] * (0.5 * (M[i] + M[nb[a]]));
            mf[a][i] = v;
            if (mff[a]) mff[a][i] = (float)v;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Spectral bound of Fig. 1 by explicit columns, for grids where the closed form of the
// periodic constant-mobility operator does not hold (Neumann boundaries, variable
// mobility): column j of A_hat is A_M (d_j e_j + eps^2 A e_j), d_j = 3 y_j^2 - 1 (+1
// Eyre), formed entry by entry (entries falling on one point are added), and its absolute
// sum taken; the maximum over all columns goes to red[4].
// ---------------------------------------------------------------------------------------
constexpr int kColMax = 32;     // distinct entries of a column: at most 25 (3D), 13 (2D)

__device__ __forceinline__ int col_add(unsigned (&idx)[kColMax], double (&val)[kColMax], int cnt,
                                       unsigned k, double v) {
    for (int e = 0; e < cnt; ++e)
        if (idx[e] == k) { val[e] += v; return cnt; }
    idx[cnt] = k; val[cnt] = v;
    return cnt + 1;
}

__global__ void __launch_bounds__(kThreads)
k_colmax(Geom g, const double *__restrict__ y, double dshift, double *partials,
         unsigned int *ticket, Ctrl *ctrl) {
    const unsigned n[3] = {(unsigned)g.n[0], (unsigned)g.n[1], (unsigned)g.n[2]};
    const unsigned st[3] = {1u, n[0], n[0] * n[1]};
    double mn = INFINITY, mx = -INFINITY;
    GRID_LOOP(j, g.N) {
        // t = d_j e_j + eps^2 A e_j
        unsigned ti[1 + 2 * 3];
        double tv[1 + 2 * 3];
        int nt = 1;
        ti[0] = j; tv[0] = fma(3.0, y[j] * y[j], dshift);
        for (int a = 0; a < g.dim; ++a) {
            const unsigned c = (j / st[a]) % n[a];
            const unsigned pj = nb_p(j, c, n[a], st[a], g.bc), mj = nb_m(j, c, n[a], st[a], g.bc);
            const double k = g.eps2 * g.s[a];
            // 2 s_a e_j - s_a e_{j+a} - s_a e_{j-a}, a mirror neighbour being j itself
            tv[0] += 2.0 * k;
            const unsigned nbs[2] = {pj, mj};
            for (int q = 0; q < 2; ++q) {
                int e = 0;
                while (e < nt && ti[e] != nbs[q]) ++e;
                if (e == nt) { ti[nt] = nbs[q]; tv[nt] = 0.0; ++nt; }
                tv[e] -= k;
            }
        }
        // column = A_M t: every entry k of t spreads over its faces, face by face
        unsigned idx[kColMax];
        double val[kColMax];
        int cnt = 0;
        for (int e = 0; e < nt; ++e) {
            const unsigned k = ti[e];
            const double v = tv[e];
            for (int a = 0; a < g.dim; ++a) {
                const unsigned c = (k / st[a]) % n[a];
                const unsigned pk = nb_p(k, c, n[a], st[a], g.bc), mk = nb_m(k, c, n[a], st[a], g.bc);
                const double fp = g.mf[a] ? g.mf[a][k] : g.s[a];     // face k | k + e_a
                const double fm = g.mf[a] ? g.mf[a][mk] : g.s[a];    // face k - e_a | k
                cnt = col_add(idx, val, cnt, k, fp * v);
                cnt = col_add(idx, val, cnt, pk, -fp * v);
                cnt = col_add(idx, val, cnt, k, fm * v);
                cnt = col_add(idx, val, cnt, mk, -fm * v);
            }
        }
        double sum = 0.0;
        for (int e = 0; e < cnt; ++e) sum += fabs(val[e]);
        mx = fmax(mx, sum);
    }
    block_minmax(mn, mx);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[gridDim.x + blockIdx.x] = mx;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    mx = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) mx = fmax(mx, __ldcg(&partials[gridDim.x + b]));
    block_minmax(mn, mx);
    if (threadIdx.x == 0) {
        ctrl->red[4] = mx;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// Krylov start (the start vector of Fig. 2) from the norms left in red[] by rhs2 / resid2:
// beta = ||W_1||, gam_1 = 1/beta; tol_phi by Eq. (tol_phi) unless fixed (> 0).
// beta == 0 (stationary linear IVP) leaves the run inactive with jexit = 0, y_next = y0.
// ---------------------------------------------------------------------------------------
__global__ void k_krylov_arm(Ctrl *ctrl, double tau0, double tol_phi_fixed, double tol,
                             int use_ghat) {
    const double beta = sqrt(ctrl->red[0]);
    ctrl->beta = beta;
    ctrl->tau0 = tau0;
    ctrl->tau = tau0;
    ctrl->jexit = 0;
    ctrl->converged = 0;
    ctrl->shrunk = 0;
    ctrl->phi_evals = 0;
    ctrl->hnext2 = 0.0;
    ctrl->resnorm = 0.0;
    double tp = tol_phi_fixed;
    if (!(tp > 0.0)) {
        const double ng = use_ghat ? sqrt(ctrl->red[1]) : 0.0;
        double a = ng / (10.0 * beta);
        double m = a < 0.1 ? a : 0.1;
        if (10.0 * tol < m) m = 10.0 * tol;
        tp = m > 1e-7 ? m : 1e-7;
    }
    ctrl->tol_phi = tp;
    if (!isfinite(beta)) {
        ctrl->status = CH_ENONFINITE;
        ctrl->active = 0;
        return;
    }
    ctrl->active = beta > 0.0 ? 1 : 0;
    ctrl->gam[0] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// ---------------------------------------------------------------------------------------
// Host launchers.  All reductions use ticket 0: kernels of one grid are serialised on its
// stream, and the last block of each kernel resets the ticket before the kernel ends.
// ---------------------------------------------------------------------------------------
#define DISPATCH_DIM(CLS, g, KERNEL, ...)                                              \
    do {                                                                               \
        LaunchScope scope_(L, CLS);                                                    \
        if ((g).dim == 3) KERNEL<3><<<L.blocks, kThreads, 0, L.stream>>>(__VA_ARGS__); \
        else KERNEL<2><<<L.blocks, kThreads, 0, L.stream>>>(__VA_ARGS__);              \
    } while (0)

void launch_prep(const Launch &L, const Geom &g, const double *y, int eyre, double *D,
                 double *G, int want_minmax) {
    const double dconst = -1.0 + (eyre ? 1.0 : 0.0) + g.eps2 * g.sigma;
    LaunchScope scope(L, CH_K_PREP);
    k_prep<<<L.blocks, kThreads, 0, L.stream>>>(g, y, dconst, eyre, D, G, want_minmax,
                                                 L.partials, &L.ctrl->ticket[0], L.ctrl);
}

#define DISPATCH_DIM_T(CLS, g, KERNEL, VT, ...)                                            \
    do {                                                                                   \
        LaunchScope scope_(L, CLS);                                                        \
        if ((g).dim == 3) KERNEL<3, VT><<<L.blocks, kThreads, 0, L.stream>>>(__VA_ARGS__); \
        else KERNEL<2, VT><<<L.blocks, kThreads, 0, L.stream>>>(__VA_ARGS__);              \
    } while (0)

template <typename VT>
void launch_tstage(const Launch &L, const Geom &g, const VT *x, const VT *D, VT *t, int guarded) {
    DISPATCH_DIM_T(CH_K_TSTAGE, g, k_tstage, VT, g, x, D, t, L.ctrl, guarded);
}

template <typename VT>
void launch_wstage(const Launch &L, const Geom &g, const VT *t, VT *w, const VT *v1,
                   double *hout, int jm1, int guarded) {
    DISPATCH_DIM_T(CH_K_WSTAGE, g, k_wstage, VT, g, t, w, v1, hout, jm1, L.partials,
                   &L.ctrl->ticket[0], L.ctrl, guarded);
}

// hk points at H[k-1][j-1]; with `last` (k == j) the pass also stores h_{j+1,j} at
// hk + ldh_next (= H[j][j-1], ldh_next = ldh) and gam[j] = 1/h_{j+1,j}.
template <typename VT>
void launch_mgs(const Launch &L, int64_t N, VT *w, const VT *vk, const VT *vk1, double *hk,
                double *hout, int k, int last, int ldh_next) {
    LaunchScope scope(L, CH_K_MGS);
    k_mgs<VT><<<L.blocks, kThreads, 0, L.stream>>>(N, w, vk, vk1, hk, hout, k, last, ldh_next,
                                                    L.partials, &L.ctrl->ticket[0], L.ctrl);
}

template void launch_tstage<double>(const Launch &, const Geom &, const double *, const double *, double *, int);
template void launch_tstage<float>(const Launch &, const Geom &, const float *, const float *, float *, int);
template void launch_wstage<double>(const Launch &, const Geom &, const double *, double *, const double *, double *, int, int);
template void launch_wstage<float>(const Launch &, const Geom &, const float *, float *, const float *, double *, int, int);
template void launch_mgs<double>(const Launch &, int64_t, double *, const double *, const double *, double *, double *, int, int, int);
template void launch_mgs<float>(const Launch &, int64_t, float *, const float *, const float *, double *, double *, int, int, int);

void launch_combine32(const Launch &L, int64_t N, const double *y0, const float *v0,
                      const float *V, int64_t ldv, float *d, double *ynext) {
    {
        LaunchScope scope(L, CH_K_COMBINE);
        k_combine32a<<<L.blocks, kThreads, 0, L.stream>>>(N, v0, V, ldv, d, L.partials,
                                                          &L.ctrl->ticket[0], L.ctrl);
    }
    LaunchScope scope(L, CH_K_COMBINE);
    k_combine32b<<<L.blocks, kThreads, 0, L.stream>>>(N, y0, d, ynext, L.ctrl);
}

void launch_to32(const Launch &L, int64_t N, const double *x, float *y, double shift) {
    LaunchScope scope(L, CH_K_PREP);
    k_to32<<<L.blocks, kThreads, 0, L.stream>>>(N, x, shift, y);
}

void launch_combine(const Launch &L, int64_t N, const double *y0, const double *v0,
                    const double *V, int64_t ldv, double *ynext) {
    LaunchScope scope(L, CH_K_COMBINE);
    k_combine<<<L.blocks, kThreads, 0, L.stream>>>(N, y0, v0, V, ldv, ynext, L.ctrl);
}

void launch_rhs1(const Launch &L, const Geom &g, const double *y, int eyre, double *mu,
                 double *q) {
    DISPATCH_DIM(CH_K_RHS1, g, k_rhs1, g, y, eyre, mu, q);
}

void launch_rhs2(const Launch &L, const Geom &g, const double *mu, const double *q,
                 double *f, const double *y0, const double *f0, const double *y1,
                 double half_tau, int mode) {
    // number of reduced values: the highest of ||f||^2, ||g_hat||^2, est sums requested
    const int K = (mode & 4) ? 4 : (mode & 2) ? 2 : (mode & 1) ? 1 : 0;
    LaunchScope scope_(L, CH_K_RHS2);
#define RHS2_ARGS g, mu, q, f, y0, f0, y1, half_tau, mode, L.partials, &L.ctrl->ticket[0], L.ctrl
    if (g.dim == 3) {
        if (K == 4) k_rhs2<3, 4><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else if (K == 2) k_rhs2<3, 2><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else if (K == 1) k_rhs2<3, 1><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else k_rhs2<3, 0><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
    } else {
        if (K == 4) k_rhs2<2, 4><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else if (K == 2) k_rhs2<2, 2><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else if (K == 1) k_rhs2<2, 1><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
        else k_rhs2<2, 0><<<L.blocks, kThreads, 0, L.stream>>>(RHS2_ARGS);
    }
#undef RHS2_ARGS
}

void launch_resid1(const Launch &L, const Geom &g, const double *x, const double *D,
                   const double *G, double *t) {
    LaunchScope scope(L, CH_K_RESID1);
    scope.work((2.0 + 3.0 * g.dim) * g.N, 32.0 * g.N);      // fma + d (add + fma); x, D, G, t
    if (g.dim == 3) k_resid1<3><<<L.blocks, kThreads, 0, L.stream>>>(g, x, D, G, t);
    else k_resid1<2><<<L.blocks, kThreads, 0, L.stream>>>(g, x, D, G, t);
}

void launch_resid2(const Launch &L, const Geom &g, const double *t, double *out) {
    DISPATCH_DIM(CH_K_RESID2, g, k_resid2, g, t, out, L.partials, &L.ctrl->ticket[0], L.ctrl);
}

void launch_lim2(const Launch &L, const Geom &g, const double *t, const double *yn,
                 const double *yprev, double *ynext, double tau_a, double tau, double alpha) {
    LaunchScope scope(L, CH_K_LIM2);
    scope.work((5.0 + 3.0 * g.dim) * g.N, 32.0 * g.N);      // stage 2 + update; t, yn, yprev, ynext
    if (g.dim == 3) k_lim2<3><<<L.blocks, kThreads, 0, L.stream>>>(g, t, yn, yprev, ynext, tau_a, tau, alpha);
    else k_lim2<2><<<L.blocks, kThreads, 0, L.stream>>>(g, t, yn, yprev, ynext, tau_a, tau, alpha);
}

void launch_lim32(const Launch &L, const Geom &g, const float *t, const double *fn,
                  const float *dprev, float *dnext, double ta, double atau) {
    LaunchScope scope(L, CH_K_LIM2);
    scope.work((4.0 + 3.0 * g.dim) * g.N, 24.0 * g.N);     // stage 2 + update; t, f, d_prev, d_next
    if (g.dim == 3) k_lim32<3><<<L.blocks, kThreads, 0, L.stream>>>(g, t, fn, dprev, dnext, (float)ta, (float)atau);
    else k_lim32<2><<<L.blocks, kThreads, 0, L.stream>>>(g, t, fn, dprev, dnext, (float)ta, (float)atau);
}

void launch_add_increment(const Launch &L, int64_t N, const double *y0, const float *d, double *ynext) {
    {
        LaunchScope scope(L, CH_K_COMBINE);
        k_sum32<<<L.blocks, kThreads, 0, L.stream>>>(N, d, L.partials, &L.ctrl->ticket[0], L.ctrl);
    }
    LaunchScope scope(L, CH_K_COMBINE);
    k_add_increment<<<L.blocks, kThreads, 0, L.stream>>>(N, y0, d, ynext, L.ctrl);
}

void launch_energy(const Launch &L, const Geom &g, const double *y) {
    DISPATCH_DIM(CH_K_ENERGY, g, k_energy, g, y, L.partials, &L.ctrl->ticket[0], L.ctrl);
}

void launch_face_mob(const Launch &L, const Geom &g, const double *M, double *const mf[3],
                     float *const mff[3]) {
    LaunchScope scope(L, CH_K_PREP);
    k_face_mob<<<L.blocks, kThreads, 0, L.stream>>>(g, M, mf[0], mf[1], mf[2], mff[0], mff[1], mff[2]);
}

void launch_colmax(const Launch &L, const Geom &g, const double *y, int eyre) {
    LaunchScope scope(L, CH_K_PREP);
    k_colmax<<<L.blocks, kThreads, 0, L.stream>>>(g, y, -1.0 + (eyre ? 1.0 : 0.0), L.partials,
                                                   &L.ctrl->ticket[0], L.ctrl);
}

void launch_krylov_arm(const Launch &L, double tau0, double tol_phi_fixed, double tol,
                       int use_ghat) {
    LaunchScope scope(L, CH_K_ARM);
    k_krylov_arm<<<1, 1, 0, L.stream>>>(L.ctrl, tau0, tol_phi_fixed, tol, use_ghat);
}

}  // namespace ch
