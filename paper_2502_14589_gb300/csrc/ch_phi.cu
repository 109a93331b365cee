// ch_phi.cu -- projected phi evaluation, residual test and residual-time step choice of the
// Krylov method of Fig. 2, in FP64 on one thread block.
//
// u = s phi(-s H_j) e_1 (Eqs. phi, yt_m) is the last column of exp([[-s H_j, s e_1], [0, 0]]).
// The exponential uses the diagonal Pade approximant of degree 13 with scaling and squaring
// (N.J. Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005); the scaling exponent is the least
// integer sq >= 0 with ||M||_1 / 2^sq <= theta_13, found by exact halving.  The Pade
// denominator system is solved by Gauss-Jordan elimination with partial pivoting.
// All matrices (n = j+1 <= 129) live in shared memory when n <= 64, else in global scratch.
#include <cooperative_groups.h>
#include <math.h>

#include "ch_internal.cuh"

namespace cg = cooperative_groups;

namespace ch {

constexpr int kPhiThreads = 512;
constexpr int kPhiCluster = 8;     // CTAs of the cluster that shares the matrix products
constexpr int kPhiSmemMaxN = 64;
constexpr int kMaxHalvings = 60;   // fixed rule for the step trace of Fig. 2
constexpr int kBisections = 12;

constexpr int kTraceSlots = kBisections + 1;   // exp(M(lo0 / 2^b)), b = 0..12
constexpr int kTraceMaxN = 32;                  // trace by products when n <= 32

struct PhiWork {
    double *b[6];       // six n x n buffers (row-major, ld = n)
    double *fcol;       // n
    double *colsum;     // n
    double *slot[kTraceSlots];  // trace matrices (nullptr when the trace uses fresh evaluations)
    double *cur, *tmp;  // trace: exp(M(lo)) and scratch
    double c[14];       // Pade coefficients
    double chain[64];   // (j-1, j) entry of exp(M(s / 2^m)), m = 0..sq, from the squarings
    int sq;
    int piv;
    double pinv;
    double norm1;
    double res;
    double entry;
};

// C = A B on one thread block.
struct MatmulBlock {
    __device__ __forceinline__ void operator()(int n, const double *A, const double *B,
                                               double *C, bool pre = false) const {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int r = e / n, c = e - r * n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(A[r * n + k], B[k * n + c], acc);
            C[e] = acc;
        }
        __syncthreads();
    }
};

// C = A B on a cluster: every CTA holds the same copies of A and B in its shared memory,
// computes a slice of rows of C and stores it into the C of every CTA of the cluster
// (distributed shared memory).  A cluster barrier after the product (all slices arrived);
// with `pre` also one before it, for the products whose C another CTA may still be reading
// in the preceding local phase (the first product of an exponential and its first squaring).
struct MatmulCluster {
    __device__ __forceinline__ void operator()(int n, const double *A, const double *B,
                                               double *C, bool pre = false) const {
        cg::cluster_group cl = cg::this_cluster();
        const int rank = (int)cl.block_rank(), nr = (int)cl.num_blocks();
        const int r0 = rank * n / nr, r1 = (rank + 1) * n / nr;
        double *dst[kPhiCluster];
        for (int q = 0; q < nr; ++q) dst[q] = cl.map_shared_rank(C, q);
        if (pre) cl.sync();
        for (int e = threadIdx.x; e < (r1 - r0) * n; e += blockDim.x) {
            const int r = r0 + e / n, c = e - (r - r0) * n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(A[r * n + k], B[k * n + c], acc);
            for (int q = 0; q < nr; ++q) dst[q][r * n + c] = acc;
        }
        cl.sync();
    }
};

// E = exp(M) with M given in W.b[0]; returns the buffer holding E.
template <typename MM>
__device__ double *expm_block(int n, PhiWork &W, const MM &mm) {
    double *X = W.b[0], *X2 = W.b[1], *X4 = W.b[2], *X6 = W.b[3], *T4 = W.b[4], *T5 = W.b[5];
    const int nn = n * n;
    // ||M||_1 (max column sum)
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += fabs(X[r * n + c]);
        W.colsum[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int c = 0; c < n; ++c) m = fmax(m, W.colsum[c]);
        W.norm1 = m;
    }
    __syncthreads();
    const double theta13 = 5.371920351148152;   // Higham (2005), Table 2.3
    int sq = 0;
    double scaled = W.norm1;
    while (scaled > theta13 && sq < 1100) { scaled *= 0.5; ++sq; }
    const double scale = ldexp(1.0, -sq);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) X[e] *= scale;
    __syncthreads();
    mm(n, X, X, X2, true);     // another CTA may still be in the previous exponential
    mm(n, X2, X2, X4);
    mm(n, X4, X2, X6);
    const double *c = W.c;
    for (int e = threadIdx.x; e < nn; e += blockDim.x)
        T4[e] = c[13] * X6[e] + c[11] * X4[e] + c[9] * X2[e];
    __syncthreads();
    mm(n, X6, T4, T5);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int r = e / n;
        T5[e] += c[7] * X6[e] + c[5] * X4[e] + c[3] * X2[e] + ((r * n + r == e) ? c[1] : 0.0);
    }
    __syncthreads();
    mm(n, X, T5, T4);                                   // T4 = U
    for (int e = threadIdx.x; e < nn; e += blockDim.x)
        T5[e] = c[12] * X6[e] + c[10] * X4[e] + c[8] * X2[e];
    __syncthreads();
    mm(n, X6, T5, X);                                   // X = V (nonlinear part)
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int r = e / n;
        const double v = X[e] + c[6] * X6[e] + c[4] * X4[e] + c[2] * X2[e] +
                         ((r * n + r == e) ? c[0] : 0.0);
        X2[e] = v - T4[e];                              // P = V - U
        X4[e] = v + T4[e];                              // Q = V + U
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting on [P | Q]: Q <- P^{-1} Q.  Two barriers per column:
    // warp 0 finds the pivot row pv and stages, in the free buffers T4 and T5, the scaled
    // pivot row, the old row k and the multipliers; then every element is updated in place,
    // rows k and pv exchanging their roles (the same operations as swapping the rows, scaling
    // row k and eliminating).  Columns left of k of P are zero outside the unit entries and
    // are not touched.
    double *P = X2, *Q = X4;
    double *prowP = T4, *prowQ = T4 + n, *rowkP = T5, *rowkQ = T5 + n;   // 2n <= n*n for n >= 2
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            const int lane = (int)threadIdx.x;
            double best = -1.0;
            int bi = k;
            for (int i = k + lane; i < n; i += 32) {
                const double a = fabs(P[i * n + k]);
                if (a > best) { best = a; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            const int pv = __shfl_sync(0xffffffffu, bi, 0);
            const double pinv = 1.0 / P[pv * n + k];
            for (int c = lane; c < n; c += 32) {
                prowP[c] = P[pv * n + c] * pinv;
                prowQ[c] = Q[pv * n + c] * pinv;
                rowkP[c] = P[k * n + c];
                rowkQ[c] = Q[k * n + c];
                W.fcol[c] = c == pv ? P[k * n + k] : P[c * n + k];
            }
            if (lane == 0) W.piv = pv;
        }
        __syncthreads();
        const int pv = W.piv;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, cc = e - i * n;
            if (i == k) {
                if (cc >= k) P[e] = prowP[cc];
                Q[e] = prowQ[cc];
            } else {
                const double f = W.fcol[i];
                const double p0 = i == pv ? rowkP[cc] : P[e], q0 = i == pv ? rowkQ[cc] : Q[e];
                if (cc >= k) P[e] = fma(-f, prowP[cc], p0);
                Q[e] = fma(-f, prowQ[cc], q0);
            }
        }
        __syncthreads();
    }
    double *R = Q, *S = X6;
    // R = exp(M / 2^sq); record its (n-2, n-1) entry (the residual entry of Fig. 2)
    // for s / 2^sq, then after each squaring for s / 2^(sq-k-1)
    if (threadIdx.x == 0) {
        W.sq = sq;
        if (sq < 64) W.chain[sq] = R[(n - 2) * n + (n - 1)];
    }
    for (int k = 0; k < sq; ++k) {
        mm(n, R, R, S, k == 0);   // the P, Q step above still reads X6 (= S) in other CTAs
        double *t = R; R = S; S = t;
        if (threadIdx.x == 0 && sq - k - 1 < 64) W.chain[sq - k - 1] = R[(n - 2) * n + (n - 1)];
    }
    __syncthreads();
    return R;
}

// u = s phi(-s H_j) e_1 (written to `u` when u != nullptr, else kept in W.fcol); returns
// resnorm = h_{j+1,j} |e_j^T u| (Fig. 2).
template <typename MM>
__device__ double phi_eval(int j, const double *H, int ldh, double hnext, double s, double *u,
                           PhiWork &W, const MM &mm) {
    const int n = j + 1;
    double *M = W.b[0];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        double v = 0.0;
        if (r < j && c < j) v = -s * H[r * ldh + c];
        else if (r == 0 && c == j) v = s;
        M[e] = v;
    }
    __syncthreads();
    const double *E = expm_block(n, W, mm);
    const double last = E[(j - 1) * n + j];
    if (u)
        for (int r = threadIdx.x; r < j; r += blockDim.x) u[r] = E[r * n + j];
    __syncthreads();
    return hnext * fabs(last);                          // resnorm of Fig. 2
}

// Fig. 2 after the Arnoldi process, for iteration j, on one CTA (MM = MatmulBlock) or one cluster (every
// CTA runs the same control flow on identical data; rank 0 alone writes results).
template <typename MM>
__device__ void phi_step(Ctrl *ctrl, double *H, int ldh, int j, int mmax, double *u,
                         double *base, bool writer, const MM &mm, bool base_has_slots) {
    __shared__ PhiWork W;
    const int n = j + 1;
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) W.b[k] = base + (size_t)k * n * n;
        W.fcol = base + (size_t)6 * n * n;
        W.colsum = W.fcol + n;
        const bool trace_slots = (j == mmax) && n <= kTraceMaxN && base_has_slots;
        double *sb = W.colsum + n;
        for (int k = 0; k < kTraceSlots; ++k) W.slot[k] = trace_slots ? sb + (size_t)k * n * n : nullptr;
        W.cur = trace_slots ? sb + (size_t)kTraceSlots * n * n : nullptr;
        W.tmp = trace_slots ? W.cur + (size_t)n * n : nullptr;
        W.c[0] = 1.0;
        for (int k = 1; k <= 13; ++k)
            W.c[k] = W.c[k - 1] * (double)(13 - k + 1) / ((double)(2 * 13 - k + 1) * k);
    }
    __syncthreads();
    const double hnext = H[j * ldh + (j - 1)];           // h_{j+1,j} (last MGS pass)
    const double tau0 = ctrl->tau0, tol = ctrl->tol_phi;
    double *uo = writer ? u : nullptr;
    int evals = 1;
    double res = phi_eval(j, H, ldh, hnext, tau0, uo, W, mm);  // phi and resnorm at tau0
    int done = 0, shrunk = 0, status = 0;
    double tau = tau0;
    if (!isfinite(hnext) || !isfinite(res)) {
        status = CH_ENONFINITE;
        done = 1;
    } else if (res <= tol) {                                // converged
        done = 1;
    } else if (j == mmax) {                                 // step trace
        // Halve s from tau0 until resnorm(s) <= tol_phi: the trials s = tau0/2^k with
        // k <= sq are the intermediate squarings of the evaluation at tau0 (same arithmetic
        // as a fresh evaluation, whose scaling exponent is sq - k), recorded in W.chain.
        const int sq0 = W.sq;
        int k = 0, ok = 0;
        for (k = 1; k <= kMaxHalvings; ++k) {
            double r;
            if (k <= sq0 && k < 64) {
                r = hnext * fabs(W.chain[k]);
            } else {
                ++evals;
                r = phi_eval(j, H, ldh, hnext, ldexp(tau0, -k), nullptr, W, mm);
            }
            if (r <= tol) { ok = 1; break; }
        }
        if (!ok) {
            status = CH_ENOTCONV;
        } else if (W.slot[0] != nullptr) {
            // Bisection between lo0 = tau0/2^k (admissible) and 2 lo0: the trials are
            // lo + lo0/2^b, and M(s) is linear in s, so exp(M(lo + d)) = exp(M(lo)) exp(M(d)).
            // slot[b] = exp(M(lo0/2^b)) comes from one evaluation at lo0/2^12 and squarings.
            const double lo0 = ldexp(tau0, -k);
            ++evals;
            phi_eval(j, H, ldh, hnext, ldexp(lo0, -kBisections), nullptr, W, mm);
            const double *E = (W.sq % 2 == 0) ? W.b[2] : W.b[3];
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) W.slot[kBisections][e] = E[e];
            __syncthreads();
            for (int b = kBisections - 1; b >= 0; --b) mm(n, W.slot[b + 1], W.slot[b + 1], W.slot[b]);
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) W.cur[e] = W.slot[0][e];
            __syncthreads();
            double lo = lo0;
            for (int b = 1; b <= kBisections; ++b) {
                if (threadIdx.x == 0) {          // (j-1, j) entry of exp(M(lo)) exp(M(lo0/2^b))
                    double acc = 0.0;
                    for (int c = 0; c < n; ++c) acc = fma(W.cur[(j - 1) * n + c], W.slot[b][c * n + j], acc);
                    W.entry = acc;
                }
                __syncthreads();
                if (hnext * fabs(W.entry) <= tol) {
                    mm(n, W.cur, W.slot[b], W.tmp);
                    if (threadIdx.x == 0) { double *t = W.cur; W.cur = W.tmp; W.tmp = t; }
                    __syncthreads();
                    lo += ldexp(lo0, -b);
                }
            }
            if (uo)                                      // u = s phi(-s H) e_1 at s = lo
                for (int r = threadIdx.x; r < j; r += blockDim.x) uo[r] = W.cur[r * n + j];
            __syncthreads();
            tau = lo;
            shrunk = 1;
        } else {
            double lo = ldexp(tau0, -k), hi = 2.0 * lo;
            for (int b = 0; b < kBisections; ++b) {
                const double mid = 0.5 * (lo + hi);
                ++evals;
                if (phi_eval(j, H, ldh, hnext, mid, uo, W, mm) <= tol) lo = mid;
                else hi = mid;
            }
            ++evals;
            phi_eval(j, H, ldh, hnext, lo, uo, W, mm);      // u at s = lo
            tau = lo;
            shrunk = 1;
        }
        done = 1;
    }
    if (!writer) return;
    if (threadIdx.x == 0) {
        H[j * ldh + (j - 1)] = hnext;
        ctrl->phi_evals += evals;
        ctrl->resnorm = res;
        if (done) {
            ctrl->active = 0;
            if (status) {
                ctrl->status = status;
                ctrl->jexit = 0;
            } else {
                ctrl->jexit = j;
                ctrl->tau = tau;
                ctrl->converged = shrunk ? 0 : 1;
                ctrl->shrunk = shrunk;
            }
        } else {
            ctrl->gam[j] = 1.0 / hnext;                      // v_{j+1} = w / h_{j+1,j}
        }
    }
    if (done && !status)
        for (int c = threadIdx.x; c < j; c += blockDim.x)
            ctrl->coef[c] = ctrl->beta * ctrl->gam[c] * u[c];   // Krylov combine
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi(Ctrl *ctrl, double *H, int ldh, int j, int mmax, double *u, double *gscratch,
      int use_smem) {
    if (!ctrl->active) return;
    extern __shared__ double smem[];
    phi_step(ctrl, H, ldh, j, mmax, u, use_smem ? smem : gscratch, true, MatmulBlock(),
             use_smem != 0);
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi_cluster(Ctrl *ctrl, double *H, int ldh, int j, int mmax, double *u) {
    if (!ctrl->active) return;                 // same value in every CTA of the cluster
    extern __shared__ double smem[];
    const bool writer = cg::this_cluster().block_rank() == 0;
    phi_step(ctrl, H, ldh, j, mmax, u, smem, writer, MatmulCluster(), true);
}

// Batched form: one cluster per instance (cluster index = instance), each with its own
// control block, Hessenberg matrix (stride hstride) and u (stride ustride).
__global__ void __launch_bounds__(kPhiThreads)
k_phi_batch(Ctrl *ctrls, double *Hs, int64_t hstride, double *us, int64_t ustride, int ldh,
            int j, int mmax) {
    cg::cluster_group cl = cg::this_cluster();
    const int inst = (int)(blockIdx.x / cl.num_blocks());
    Ctrl *ctrl = ctrls + inst;
    if (!ctrl->active) return;                 // same value in every CTA of this cluster
    extern __shared__ double smem[];
    const bool writer = cl.block_rank() == 0;
    phi_step(ctrl, Hs + inst * hstride, ldh, j, mmax, us + inst * ustride, smem, writer,
             MatmulCluster(), true);
}

// ---- block-parallel evaluation: resnorm(tau0) and u for one Krylov dimension j -------------
template <typename MM>
__device__ void phi_eval_only(Ctrl *ctrl, const double *H, int ldh, int j, double *ub_j,
                              double *base, bool writer, const MM &mm) {
    __shared__ PhiWork W;
    const int n = j + 1;
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) W.b[k] = base + (size_t)k * n * n;
        W.fcol = base + (size_t)6 * n * n;
        W.colsum = W.fcol + n;
        for (int k = 0; k < kTraceSlots; ++k) W.slot[k] = nullptr;
        W.cur = W.tmp = nullptr;
        W.c[0] = 1.0;
        for (int k = 1; k <= 13; ++k)
            W.c[k] = W.c[k - 1] * (double)(13 - k + 1) / ((double)(2 * 13 - k + 1) * k);
    }
    __syncthreads();
    const double hnext = H[j * ldh + (j - 1)];
    const double res = phi_eval(j, H, ldh, hnext, ctrl->tau0, writer ? ub_j : nullptr, W, mm);
    if (writer && threadIdx.x == 0) ctrl->resj[j] = (isfinite(hnext) && isfinite(res)) ? res : NAN;
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi_multi_cluster(Ctrl *ctrl, const double *H, int ldh, int j0, double *ub, int ldu) {
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)(blockIdx.x / cl.num_blocks());
    if (!ctrl->active) return;
    extern __shared__ double smem[];
    phi_eval_only(ctrl, H, ldh, j0 + c, ub + (size_t)c * ldu, smem, cl.block_rank() == 0,
                  MatmulCluster());
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi_multi_block(Ctrl *ctrl, const double *H, int ldh, int j0, double *ub, int ldu) {
    if (!ctrl->active) return;
    extern __shared__ double smem[];
    phi_eval_only(ctrl, H, ldh, j0 + (int)blockIdx.x, ub + (size_t)blockIdx.x * ldu, smem, true,
                  MatmulBlock());
}

// First j in [j0, jlast] whose residual test passed (Fig. 2): that j ends the
// run, exactly as the per-iteration test would; a non-finite residual first ends it with an
// error.  Returns true when the run ended.
__device__ bool decide_first(Ctrl *ctrl, int j0, int jlast, const double *ub, int ldu,
                             bool writer) {
    __shared__ int dj;
    if (threadIdx.x == 0) {
        dj = 0;
        for (int j = j0; j <= jlast; ++j) {
            const double r = ctrl->resj[j];
            if (!isfinite(r)) { dj = -1; break; }
            if (r <= ctrl->tol_phi) { dj = j; break; }
        }
    }
    __syncthreads();
    const int d = dj;
    if (d == 0) return false;
    if (writer) {
        if (threadIdx.x == 0) {
            ctrl->phi_evals += (d > 0 ? d : jlast) - j0 + 1;
            ctrl->active = 0;
            if (d < 0) {
                ctrl->status = CH_ENONFINITE;
                ctrl->jexit = 0;
            } else {
                ctrl->jexit = d;
                ctrl->tau = ctrl->tau0;
                ctrl->converged = 1;
                ctrl->shrunk = 0;
                ctrl->resnorm = ctrl->resj[d];
            }
        }
        if (d > 0)
            for (int c = threadIdx.x; c < d; c += blockDim.x)
                ctrl->coef[c] = ctrl->beta * ctrl->gam[c] * ub[(size_t)(d - j0) * ldu + c];  // Krylov combine
    }
    __syncthreads();
    return true;
}

__global__ void k_phi_decide(Ctrl *ctrl, int j0, int j1, const double *ub, int ldu) {
    if (!ctrl->active) return;
    if (!decide_first(ctrl, j0, j1, ub, ldu, true) && threadIdx.x == 0)
        ctrl->phi_evals += j1 - j0 + 1;
}

// Last block of the run (j1 == mmax): decide among j0..mmax-1, else Fig. 2 at mmax with the
// step trace (the evaluation at tau0 is repeated to obtain its squaring chain).
__global__ void __launch_bounds__(kPhiThreads)
k_phi_decide_trace(Ctrl *ctrl, double *H, int ldh, int j0, int mmax, double *u, const double *ub,
                   int ldu) {
    if (!ctrl->active) return;
    extern __shared__ double smem[];
    const bool writer = cg::this_cluster().block_rank() == 0;
    if (j0 < mmax && decide_first(ctrl, j0, mmax - 1, ub, ldu, writer)) return;
    if (writer && threadIdx.x == 0) ctrl->phi_evals += mmax - j0;
    phi_step(ctrl, H, ldh, mmax, mmax, u, smem, writer, MatmulCluster(), true);
}

// Dynamic shared memory of one phi launch: six work matrices and two vectors, plus the
// trace matrices when j == mmax and n <= 32.
static size_t phi_smem_bytes(int n, int j, int mmax) {
    size_t words = (size_t)6 * n * n + 2 * n;
    if (j == mmax && n <= kTraceMaxN) words += (size_t)(kTraceSlots + 2) * n * n;
    return words * sizeof(double);
}

int phi_setup() {
    const size_t bytes = (size_t)(6 * kPhiSmemMaxN * kPhiSmemMaxN + 2 * kPhiSmemMaxN) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_phi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_phi_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_phi_multi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_phi_multi_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_phi_decide_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return (int)e;
}

// Small systems (n <= 8) stay on one CTA; up to 64 they use an 8-CTA cluster with the
// matrices in shared memory; beyond 64 one CTA works from global scratch.
void launch_phi(const Launch &L, double *H, int ldh, int j, int mmax, double *u,
                double *scratch) {
    const int n = j + 1;
    LaunchScope scope(L, CH_K_PHI);
    if (n > 8 && n <= kPhiSmemMaxN) {
        const size_t bytes = phi_smem_bytes(n, j, mmax);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kPhiCluster, 1, 1);
        cfg.blockDim = dim3(kPhiThreads, 1, 1);
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = L.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kPhiCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_phi_cluster, L.ctrl, H, ldh, j, mmax, u);
        return;
    }
    const int use_smem = n <= kPhiSmemMaxN;
    const size_t bytes = use_smem ? phi_smem_bytes(n, j, mmax) : 0;
    k_phi<<<1, kPhiThreads, bytes, L.stream>>>(L.ctrl, H, ldh, j, mmax, u, scratch, use_smem);
}

static void launch_cluster(const void *fn, int clusters, size_t bytes, cudaStream_t st, void **args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPhiCluster * clusters, 1, 1);
    cfg.blockDim = dim3(kPhiThreads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kPhiCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, fn, args);
}

void launch_phi_block(const Launch &L, double *H, int ldh, int j0, int j1, int mmax, double *u,
                      double *ub, int ldu) {
    const int nj = j1 - j0 + 1;
    const int n1 = j1 + 1;
    {
        LaunchScope scope(L, CH_K_PHI);
        const size_t bytes = (size_t)(6 * n1 * n1 + 2 * n1) * sizeof(double);
        if (n1 <= 8) {
            k_phi_multi_block<<<nj, kPhiThreads, bytes, L.stream>>>(L.ctrl, H, ldh, j0, ub, ldu);
        } else {
            Ctrl *c = L.ctrl;
            const double *Hc = H;
            void *args[] = {&c, &Hc, &ldh, &j0, &ub, &ldu};
            launch_cluster((const void *)k_phi_multi_cluster, nj, bytes, L.stream, args);
        }
    }
    LaunchScope scope(L, CH_K_PHI);
    if (j1 < mmax) {
        k_phi_decide<<<1, 128, 0, L.stream>>>(L.ctrl, j0, j1, ub, ldu);
    } else {
        Ctrl *c = L.ctrl;
        const double *ubc = ub;
        void *args[] = {&c, &H, &ldh, &j0, &mmax, &u, &ubc, &ldu};
        launch_cluster((const void *)k_phi_decide_trace, 1, phi_smem_bytes(mmax + 1, mmax, mmax),
                       L.stream, args);
    }
}

void launch_phi_batch(const Launch &L, Ctrl *ctrls, double *Hs, int64_t hstride, double *us,
                      int64_t ustride, int ldh, int j, int mmax, int count) {
    const int n = j + 1;
    LaunchScope scope(L, CH_K_PHI);
    const size_t bytes = phi_smem_bytes(n, j, mmax);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPhiCluster * count, 1, 1);
    cfg.blockDim = dim3(kPhiThreads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kPhiCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_phi_batch, ctrls, Hs, hstride, us, ustride, ldh, j, mmax);
}

}  // namespace ch
