// ch_internal.cuh -- internal types and device helpers of the GB300 Cahn-Hilliard library.
//
// Layout in HBM: every grid vector is N contiguous values, x fastest
// (index = i0 + n0 (i1 + n1 i2)); the Krylov basis is (mmax_capacity + 1) such vectors,
// each starting on a 256-byte boundary.  All kernels are grid-stride loops over a fixed
// number of blocks per grid object, so every reduction is summed in the same order on
// every run (bit-reproducible): per-thread partial sums, a fixed warp-shuffle/shared-memory
// tree per block, then the last block to finish (atomic ticket, no waiting) sums the
// per-block partials in index order.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "ch.h"

namespace ch {

constexpr int kThreads = 256;          // threads per block of the streaming kernels
constexpr int kBlocksPerSM = 4;        // grid of the streaming kernels: 4 x 256 threads per SM
constexpr int kMaxRed = 4;             // values reduced by one kernel at most

// NVTX range over a host scope: the phases of the method (integration, Krylov run, LIM
// iterations) appear as named ranges in profilers; without a profiler attached the
// push/pop calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Grid geometry, passed by value.  -A = discrete Laplacian, h_a = 1/n_a:
//   (A v)_i = sum_a s_a (2 v_i - v_{i+e_a} - v_{i-e_a}),   s_a = 1/h_a^2 = n_a^2,
// with the neighbour beyond the boundary either the periodic image (bc = 0) or, for the
// homogeneous Neumann conditions of Eq. (CH) on cell-centred nodes (bc = 1), the mirror
// image of the point inside, which is the point itself.  With a variable mobility (the
// Remark on Eq. CHmob) the outer operator is the flux form
//   (A_M t)_i = sum_a [mf_a[i] (t_i - t_{i+e_a}) + mf_a[i-e_a] (t_i - t_{i-e_a})],
// mf_a[i] = s_a (M_i + M_{i+e_a}) / 2 the scaled mobility of the face between i and i+e_a
// (a face to a mirror neighbour carries no flux: its difference is zero).
struct Geom {
    int dim;
    int n[3];
    int64_t N;
    int64_t st[3];      // index stride of each axis: 1, n0, n0 n1
    double s[3];        // s_a
    double kap[3];      // eps^2 s_a
    double sigma;       // 2 sum_a s_a  (diagonal of A away from a Neumann boundary)
    double eps2;        // eps^2
    int bc;             // 0: periodic; 1: homogeneous Neumann, cell-centred
    const double *mf[3];  // face mobilities (FP64); nullptr: unit mobility
    const float *mff[3];  // FP32 copies for the mixed-precision stages (mixed grids)
};

// Device-resident control block of one grid: scalars produced by one kernel and consumed
// by later kernels or by the host (copied to pinned memory).  Kernels of a Krylov run
// return immediately once `active` is 0, so the host may queue iterations ahead.
struct Ctrl {
    int active;         // 1 while the Arnoldi loop of Fig. 2 runs
    int jexit;          // Krylov dimension j at exit
    int status;         // ch_status of the last device-side failure (0 = none)
    int converged;      // 1: resnorm(tau0) <= tol_phi (the residual test of Fig. 2)
    int shrunk;         // 1: the step trace of Fig. 2 cut the step
    int phi_evals;      // projected-phi evaluations of this run
    int pad[2];
    double tau0;        // tentative step of this run
    double tol_phi;
    double tau;         // step taken by this run
    double beta;        // ||v_1|| (the start vector of Fig. 2)
    double rinv;        // 1/beta, then 1/h_{j+1,j}: scale of the next basis vector
    double hnext2;      // ||w||^2 of the last Arnoldi iteration
    double resnorm;
    double red[8];      // generic reduced scalars (norms, est sums, min/max)
    double gam[130];    // v_c = gam[c-1] W_c: scale of each stored (unnormalised) basis vector
    double coef[130];   // beta gam_c u_c: coefficients of the Krylov combine (Fig. 2)
    double upd[130];    // batch Gram-corrected iteration: update coefficients h_kj gam_{k-1}
    double resj[130];   // resnorm(tau0) of Krylov dimension j (block-parallel phi)
    unsigned int ticket[8];
    alignas(128) unsigned long long bar;   // grid-barrier arrivals (own cache line)
};

// ---------------------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void warp_sum(double (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
}

// Block-wide sum of K values; result valid in thread 0.  Fixed order => deterministic.
// FP64 adds issue at 2 lanes/clk/SM on GB300, so a shuffle tree in every warp is costly:
// the per-thread values go to shared memory and one warp adds them (a strided pass, then
// a 5-level shuffle tree), about a quarter of the FP64 warp instructions of a per-warp tree.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
    __shared__ double sh[K][kThreads];
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = 0.0;
            for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) a += sh[k][i];
            v[k] = a;
        }
        warp_sum<K>(v);
    }
    __syncthreads();
}

// Each block contributes K partial sums; the last block to arrive sums all partials in
// block-index order and calls `fin(totals)` on thread 0.  `partials` holds K x gridDim.x
// doubles, `ticket` is a counter that starts (and is left) at 0.
template <int K, typename Fin>
__device__ __forceinline__ void grid_sum(double (&v)[K], double *partials, unsigned int *ticket,
                                         Fin fin) {
    __shared__ bool last;
    block_sum<K>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            acc[k] += __ldcg(&partials[k * gridDim.x + b]);
    }
    block_sum<K>(acc);          // same code and order in whichever block is last
    if (threadIdx.x == 0) {
        fin(acc);
        *ticket = 0u;
    }
}

// Double-float (FP32 pair hi + lo) addition with a two-sum of the high parts: the sums of
// the FP32 reductions of the mixed-precision path, in a fixed order (FP64 adds issue at a
// small fraction of the FP32 rate on GB300).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// Min / max variant (for lambda_max): partial pairs reduced with fmin / fmax.
__device__ __forceinline__ void block_minmax(double &mn, double &mx) {
    __shared__ double smn[kThreads / 32], smx[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { smn[wid] = mn; smx[wid] = mx; }
    __syncthreads();
    if (wid == 0) {
        mn = (lane < (int)(blockDim.x >> 5)) ? smn[lane] : INFINITY;
        mx = (lane < (int)(blockDim.x >> 5)) ? smx[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Host-side launch interface (defined in the .cu files, called by ch_api.cu)
// ---------------------------------------------------------------------------------------
// Per-class launch counts, and optional CUDA-event timing of every launch of one class
// (events recorded on the grid's stream right before and after each such launch).
// Arnoldi iterations are queued ahead of the host's convergence check, so a launch may find
// its Krylov run already ended and return at once: for that class the control block's
// `active` flag is copied to pinned memory before each timed launch, and launches that found
// it 0 count neither time nor work.
struct Timing {
    int cls = -1;                       // class being timed, -1 = none
    std::vector<cudaEvent_t> ev;        // 2 events per timed launch (slot)
    std::vector<double> wflops, wbytes; // algorithmic work of each slot
    int *active = nullptr;              // pinned: `active` at each slot's launch (Arnoldi class)
    size_t used = 0;                    // slots in use
    double total_ms = 0.0;
    int64_t timed = 0;                  // timed launches that did work
    int64_t counts[CH_K_COUNT] = {0};
    double flops = 0.0, bytes = 0.0;    // algorithmic work of the timed launches that did work
    void harvest();                     // defined in ch_api.cu
};

struct Launch {
    int blocks;                 // fixed per grid object
    cudaStream_t stream;
    double *partials;           // kMaxRed x blocks
    Ctrl *ctrl;                 // device control block
    int64_t *launches;          // host counter of kernel launches
    Timing *timing;
};

// RAII bracket around one kernel launch: counts it and, when its class is being timed,
// records the start/stop events.
struct LaunchScope {
    const Launch &L;
    int cls;
    bool timed;
    LaunchScope(const Launch &l, int c) : L(l), cls(c), timed(false) {
        ++*L.launches;
        if (!L.timing) return;
        ++L.timing->counts[c];
        if (L.timing->cls == c) {
            Timing &T = *L.timing;
            if (2 * (T.used + 1) > T.ev.size()) T.harvest();
            if (2 * (T.used + 1) <= T.ev.size()) {
                T.wflops[T.used] = T.wbytes[T.used] = 0.0;
                if (c == CH_K_ARNOLDI && T.active)
                    cudaMemcpyAsync(&T.active[T.used], &L.ctrl->active, sizeof(int), cudaMemcpyDeviceToHost,
                                    L.stream);
                cudaEventRecord(T.ev[2 * T.used], L.stream);
                timed = true;
            }
        }
    }
    // Algorithmic work of this launch (floating-point operations, an FMA counting 2, and the
    // bytes the method must move), accumulated when the launch is timed.
    void work(double flops, double bytes) const {
        if (!timed) return;
        L.timing->wflops[L.timing->used] = flops;
        L.timing->wbytes[L.timing->used] = bytes;
    }
    ~LaunchScope() {
        if (!timed) return;
        cudaEventRecord(L.timing->ev[2 * L.timing->used + 1], L.stream);
        ++L.timing->used;
    }
};

// Stencil and streaming kernels, FP64 (ch_stencil.cu)
void launch_prep(const Launch &L, const Geom &g, const double *y, int eyre, double *D,
                 double *G, int want_minmax);
template <typename VT>
void launch_tstage(const Launch &L, const Geom &g, const VT *x, const VT *D, VT *t, int guarded);
template <typename VT>
void launch_wstage(const Launch &L, const Geom &g, const VT *t, VT *w, const VT *v1,
                   double *hout, int jm1, int guarded);
template <typename VT>
void launch_mgs(const Launch &L, int64_t N, VT *w, const VT *vk, const VT *vk1, double *hk,
                double *hout, int k, int last, int ldh_next);
// Whole Arnoldi iteration j in one cooperative launch of `blocks` blocks (grid barriers
// between passes; L.partials must hold 2 x blocks doubles).  arnoldi_blocks gives the grid
// for N points: at most the number of blocks that can be resident at once, 0 if none.
template <typename VT>
void launch_arnoldi(const Launch &L, int blocks, const Geom &g, VT *slot0, VT *V, int64_t ldv,
                    const VT *D, VT *t, double *H, int ldh, int j);
template <typename VT>
int arnoldi_blocks(int dim, int64_t N);
// FP32-basis Arnoldi iteration j <= kGsMaxJ with Gram-corrected modified Gram-Schmidt
// (3 grid synchronisations).  gpart: 3 x (kGsMaxJ + 1) x blocks float2 of scratch; gram:
// the Gram matrix of the normalised basis, row k (vector k + 1) at gram + k ldg, rows
// 1..j-2 written by the earlier iterations of the same Krylov run, row j - 1 by this one.
constexpr int kGsMaxJ = 31;
void launch_arnoldi_gmgs(const Launch &L, int blocks, const Geom &g, float *slot0, float *V,
                         int64_t ldv, const float *D, float *t, double *H, int ldh, int j,
                         float2 *gpart, double *gram, int ldg);
// FP64-basis Arnoldi iteration j <= kGsMaxJ with the Gram-corrected coefficients (three grid
// synchronisations); gpart: 3 x (kGsMaxJ + 1) x blocks doubles, gram as above.
void launch_arnoldi_g64(const Launch &L, int blocks, const Geom &g, double *slot0, double *V,
                        int64_t ldv, const double *D, double *t, double *H, int ldh, int j,
                        double *gpart, double *gram, int ldg);
int arnoldi_setup();   // cudaError_t of setting the kernels' shared-memory limits
void launch_combine32(const Launch &L, int64_t N, const double *y0, const float *v0,
                      const float *V, int64_t ldv, float *d, double *ynext);
void launch_to32(const Launch &L, int64_t N, const double *x, float *y, double shift = 0.0);
void launch_combine(const Launch &L, int64_t N, const double *y0, const double *v0,
                    const double *V, int64_t ldv, double *ynext);
void launch_rhs1(const Launch &L, const Geom &g, const double *y, int eyre, double *mu,
                 double *q);
void launch_rhs2(const Launch &L, const Geom &g, const double *mu, const double *q,
                 double *f, const double *y0, const double *f0, const double *y1,
                 double half_tau, int mode);
void launch_resid1(const Launch &L, const Geom &g, const double *x, const double *D,
                   const double *G, double *t);
void launch_resid2(const Launch &L, const Geom &g, const double *t, double *out);
void launch_lim2(const Launch &L, const Geom &g, const double *t, const double *yn,
                 const double *yprev, double *ynext, double tau_a, double tau, double alpha);
void launch_energy(const Launch &L, const Geom &g, const double *y);
// LIM iteration of Fig. 1 on the FP32 increment d = y_prev - y^n (mixed grids): t from
// launch_tstage<float>(d, J); d_next = ta d_prev + atau (f^n - A t), ta = alpha tau a_m,
// atau = alpha tau (dprev == nullptr: the first iteration from d = 0); then
// y_next = y0 + d - mean(d).
void launch_lim32(const Launch &L, const Geom &g, const float *t, const double *fn,
                  const float *dprev, float *dnext, double ta, double atau);
void launch_add_increment(const Launch &L, int64_t N, const double *y0, const float *d, double *ynext);
// Face mobilities mf_a = s_a (M_i + M_{i+e_a}) / 2 (and FP32 copies when mff[a] != nullptr)
// from nodal values M; ||A_hat||_1 by explicit columns into red[4] (Neumann or variable-
// mobility grids, where the periodic closed form does not hold).
void launch_face_mob(const Launch &L, const Geom &g, const double *M, double *const mf[3],
                     float *const mff[3]);
void launch_colmax(const Launch &L, const Geom &g, const double *y, int eyre);
void launch_krylov_arm(const Launch &L, double tau0, double tol_phi_fixed, double tol,
                       int use_ghat);

// Projected phi, residual test and step trace of Fig. 2 (ch_phi.cu)
int phi_setup();
void launch_phi(const Launch &L, double *H, int ldh, int j, int mmax, double *u,
                double *scratch);
// Block-parallel projected phi for Krylov dimensions j0..j1 (Fig. 2, projected phi and residual test for each j
// from the same H), then the decision: the first j whose residual test passes ends the run;
// with none and j1 == mmax the step trace of Fig. 2 runs at mmax.
void launch_phi_block(const Launch &L, double *H, int ldh, int j0, int j1, int mmax, double *u,
                      double *ub, int ldu);
// Batched projected phi: one 8-CTA cluster per instance, j + 1 <= 64.
void launch_phi_batch(const Launch &L, Ctrl *ctrls, double *Hs, int64_t hstride, double *us,
                      int64_t ustride, int ldh, int j, int mmax, int count);

}  // namespace ch
