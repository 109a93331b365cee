// ch_batch.cu -- many independent Cahn-Hilliard instances (uneven sizes, own eps, own time,
// own adaptive step and Krylov state) advanced together with adaptive EE2 (Fig. 4).
//
// Layout in HBM: the instances' vectors are concatenated, instance i at [off_i, off_i + N_i)
// with off_{i+1} = off_i + N_i rounded up to 64 values.  Every kernel runs over a table of
// chunks (instance, local range); the chunk length is picked at creation by timing a stencil
// pass for a few candidates.  Reductions close per instance: each chunk writes its partial,
// and the last chunk of an instance to arrive (per-instance arrival counter) sums that
// instance's partials in chunk order, so results do not depend on scheduling.  Each
// instance has its own control block (Ctrl), Hessenberg matrix and step state; the
// projected phi runs as one 8-CTA cluster per instance, and the step controller of Fig. 4
// runs on the device.  The host only polls "any Krylov run active" per Arnoldi iteration
// and "any instance before T" per step.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "ch_internal.cuh"

namespace ch {
void set_error(const char *msg);
}

namespace {

using ch::Ctrl;
using ch::Launch;
using ch::LaunchScope;
using ch::kThreads;

struct Inst {
    int n[3];
    int dim;
    int64_t off, N;
    double s[3], kap[3], sigma, eps2;
    int first_chunk, nchunks;
};

struct Chunk {
    int inst;
    int begin, end;      // local index range of the instance
    int pad;
};

// Per-instance step state (Fig. 4) and counters.
struct BState {
    double t, tau, est;
    int done, clipped, status, pad;
    long long steps, matvecs, rhs_evals, krylov_iters, tau_shrinks, phi_evals;
};

ch_status bfail(ch_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ch::set_error(buf);
    return st;
}

#define BCUDA(expr)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(CH_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                         __FILE__, __LINE__);                                               \
    } while (0)
#define BTRY(expr)                  \
    do {                            \
        ch_status s_ = (expr);      \
        if (s_ != CH_OK) return s_; \
    } while (0)

__device__ __forceinline__ unsigned bnp(unsigned i, unsigned c, unsigned n, unsigned st) {
    return (c + 1u == n) ? i - (n - 1u) * st : i + st;
}
__device__ __forceinline__ unsigned bnm(unsigned i, unsigned c, unsigned n, unsigned st) {
    return (c == 0u) ? i + (n - 1u) * st : i - st;
}

template <int DIM, typename T>
__device__ __forceinline__ void pair_sums_inst(const Inst &I, const T *__restrict__ x, unsigned l,
                                               T (&ps)[3]) {
    const unsigned n0 = (unsigned)I.n[0], n1 = (unsigned)I.n[1];
    const unsigned c0 = l % n0, r = l / n0, c1 = r % n1;
    ps[0] = x[bnp(l, c0, n0, 1u)] + x[bnm(l, c0, n0, 1u)];
    ps[1] = x[bnp(l, c1, n1, n0)] + x[bnm(l, c1, n1, n0)];
    if (DIM == 3) {
        const unsigned n2 = (unsigned)I.n[2], s2 = n0 * n1, c2 = r / n1;
        ps[2] = x[bnp(l, c2, n2, s2)] + x[bnm(l, c2, n2, s2)];
    } else {
        ps[2] = T(0);
    }
}

// Differences (x_l - x_{l+a}) + (x_l - x_{l-a}) along every axis of an instance (FP32 stages).
template <int DIM, typename T>
__device__ __forceinline__ void pair_diffs_inst(const Inst &I, const T *__restrict__ x, unsigned l,
                                                T (&pd)[3]) {
    const unsigned n0 = (unsigned)I.n[0], n1 = (unsigned)I.n[1];
    const unsigned c0 = l % n0, r = l / n0, c1 = r % n1;
    const T xl = x[l];
    pd[0] = (xl - x[bnp(l, c0, n0, 1u)]) + (xl - x[bnm(l, c0, n0, 1u)]);
    pd[1] = (xl - x[bnp(l, c1, n1, n0)]) + (xl - x[bnm(l, c1, n1, n0)]);
    if (DIM == 3) {
        const unsigned n2 = (unsigned)I.n[2], s2 = n0 * n1, c2 = r / n1;
        pd[2] = (xl - x[bnp(l, c2, n2, s2)]) + (xl - x[bnm(l, c2, n2, s2)]);
    } else {
        pd[2] = T(0);
    }
}

// The same differences for the four consecutive points 4q..4q+3 of an instance whose rows
// hold a multiple of four points (one row per group): 16-byte loads of the group's row and
// of the neighbouring rows (planes), two scalars across the row ends, and per point the same
// operations as pair_diffs_inst.
template <int DIM>
__device__ __forceinline__ void group_diffs_inst(const Inst &I, const float *__restrict__ x, unsigned q,
                                                 float4 &xc, float4 (&d)[3]) {
    const unsigned n0 = (unsigned)I.n[0], n1 = (unsigned)I.n[1];
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
        const unsigned n2 = (unsigned)I.n[2], c2 = r / n1, p4 = r4 * n1;
        const float4 zp = x4[c2 + 1u == n2 ? q - (n2 - 1u) * p4 : q + p4];
        const float4 zm = x4[c2 == 0u ? q + (n2 - 1u) * p4 : q - p4];
        d[2] = make_float4((xc.x - zp.x) + (xc.x - zm.x), (xc.y - zp.y) + (xc.y - zm.y),
                           (xc.z - zp.z) + (xc.z - zm.z), (xc.w - zp.w) + (xc.w - zm.w));
    } else {
        d[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ float dot4f(const float4 &a, const float4 &b) {
    return __fmaf_rn(a.w, b.w, __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x))));
}

template <typename VT> struct BDot;
template <> struct BDot<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct BDot<float> {     // exact products, compensated FP32 sum (as ch_stencil.cu)
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
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Per-instance reduction: chunk partials, then the instance's last chunk sums them in order.
template <int K, typename Fin>
__device__ __forceinline__ void inst_sum(double (&v)[K], const Inst &I, int inst, double *partials,
                                         int nchunks_total, unsigned int *tickets, Fin fin) {
    __shared__ bool last;
    ch::block_sum<K>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[(size_t)k * nchunks_total + blockIdx.x] = v[k];
        __threadfence();
        last = (atomicAdd(&tickets[inst], 1u) == (unsigned)I.nchunks - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        for (int c = threadIdx.x; c < I.nchunks; c += blockDim.x)
            acc[k] += __ldcg(&partials[(size_t)k * nchunks_total + I.first_chunk + c]);
    }
    ch::block_sum<K>(acc);
    if (threadIdx.x == 0) {
        fin(acc);
        tickets[inst] = 0u;
    }
}

#define CHUNK_BEGIN                                        \
    const Chunk ck = chunks[blockIdx.x];                   \
    const Inst I = insts[ck.inst];

#define CHUNK_LOOP(l) for (unsigned l = ck.begin + threadIdx.x; l < (unsigned)ck.end; l += blockDim.x)

// ---- per-step coefficients in the basis precision: FP64 D = 3y^2 - 1 + eps^2 sigma for the
// pair-sum stages, FP32 J = 3y^2 - 1 for the difference-form stages (see kb_tstage) --------
template <typename VT>
__global__ void __launch_bounds__(kThreads)
kb_prep(const Inst *insts, const Chunk *chunks, const BState *bs, const double *__restrict__ y,
        VT *__restrict__ D) {
    CHUNK_BEGIN
    if (bs[ck.inst].done) return;
    const double dconst = sizeof(VT) == 8 ? -1.0 + I.eps2 * I.sigma : -1.0;
    CHUNK_LOOP(l) {
        const double yi = y[I.off + l];
        D[I.off + l] = (VT)fma(3.0, yi * yi, dconst);
    }
}

// ---- f(y) of Eq. (IVP), FP64; stage 1 ------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
kb_rhs1(const Inst *insts, const Chunk *chunks, const BState *bs, const double *__restrict__ y,
        double *__restrict__ mu, double *__restrict__ q) {
    CHUNK_BEGIN
    if (bs[ck.inst].done) return;
    const double *yi_ = y + I.off;
    const double cshift = I.eps2 * I.sigma - 1.0;
    CHUNK_LOOP(l) {
        double ps[3];
        pair_sums_inst<DIM>(I, yi_, l, ps);
        const double yi = yi_[l];
        const double y2 = yi * yi;
        double m = (y2 + cshift) * yi;
        m = fma(-I.kap[0], ps[0], m);
        m = fma(-I.kap[1], ps[1], m);
        if (DIM == 3) m = fma(-I.kap[2], ps[2], m);
        mu[I.off + l] = m;
        q[I.off + l] = 2.0 * y2 * yi;
    }
}

// stage 2: f (FP64 and basis precision), ||f||^2, ||g_hat||^2 and, with `est`, the sums of
// Eq. (LIMest) for the step the instance's Krylov run took (ctrl->tau).
template <int DIM, typename VT>
__global__ void __launch_bounds__(kThreads)
kb_rhs2(const Inst *insts, const Chunk *chunks, const BState *bs, Ctrl *ctrls,
        const double *__restrict__ mu, const double *__restrict__ q, double *__restrict__ f,
        VT *__restrict__ fvt, const double *__restrict__ y0, const double *__restrict__ f0,
        const double *__restrict__ y1, int est, double *partials, int nct, unsigned int *tickets) {
    CHUNK_BEGIN
    if (bs[ck.inst].done) return;
    const double *mu_ = mu + I.off, *q_ = q + I.off;
    const double half_tau = 0.5 * ctrls[ck.inst].tau;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    CHUNK_LOOP(l) {
        double ps[3], qs[3];
        pair_sums_inst<DIM>(I, mu_, l, ps);
        double r = -I.sigma * mu_[l];
        r = fma(I.s[0], ps[0], r);
        r = fma(I.s[1], ps[1], r);
        if (DIM == 3) r = fma(I.s[2], ps[2], r);
        const int64_t gi = I.off + l;
        f[gi] = r;
        if (fvt) fvt[gi] = (VT)r;
        acc[0] = fma(r, r, acc[0]);
        pair_sums_inst<DIM>(I, q_, l, qs);
        double gh = I.sigma * q_[l];
        gh = fma(-I.s[0], qs[0], gh);
        gh = fma(-I.s[1], qs[1], gh);
        if (DIM == 3) gh = fma(-I.s[2], qs[2], gh);
        acc[1] = fma(gh, gh, acc[1]);
        if (est) {
            const double ypc = fma(half_tau, f0[gi] + r, y0[gi]);
            const double d = y1[gi] - ypc;
            acc[2] = fma(d, d, acc[2]);
            acc[3] = fma(ypc, ypc, acc[3]);
        }
    }
    Ctrl *ctrl = ctrls + ck.inst;
    inst_sum<4>(acc, I, ck.inst, partials, nct, tickets, [&](double (&tot)[4]) {
        for (int k = 0; k < 4; ++k) ctrl->red[k] = tot[k];
    });
}

// ---- Krylov start of every instance still before T: clipping (Fig. 4), start vector (Fig. 2)
// A device-driven run passes its step counter: once max_steps batch steps are taken the
// remaining steps of the graph pass leave every instance where it is (no Krylov run, the
// combine carries y over, the control skips the instance).
__global__ void kb_arm(Ctrl *ctrls, BState *bs, int count, double T, double tol_phi_fixed,
                       double tol, const long long *steps, long long max_steps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Ctrl *c = ctrls + i;
    BState *b = bs + i;
    c->jexit = 0; c->converged = 0; c->shrunk = 0; c->phi_evals = 0;
    c->hnext2 = 0.0; c->resnorm = 0.0;
    if (b->done || (steps && *steps >= max_steps)) { c->active = 0; return; }
    b->clipped = 0;
    if (b->t + b->tau > T) { b->tau = T - b->t; b->clipped = 1; }
    const double beta = sqrt(c->red[0]);
    c->beta = beta;
    c->tau0 = b->tau;
    c->tau = b->tau;
    double tp = tol_phi_fixed;
    if (!(tp > 0.0)) {                                       // Eq. (tol_phi)
        const double a = sqrt(c->red[1]) / (10.0 * beta);
        double m = a < 0.1 ? a : 0.1;
        if (10.0 * tol < m) m = 10.0 * tol;
        tp = m > 1e-7 ? m : 1e-7;
    }
    c->tol_phi = tp;
    if (!isfinite(beta)) { c->status = CH_ENONFINITE; c->active = 0; return; }
    c->active = beta > 0.0 ? 1 : 0;
    c->gam[0] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// ---- Arnoldi iteration (Fig. 2), per chunk of the still-active instances ------------------
template <int DIM, typename VT>
__global__ void __launch_bounds__(kThreads)
kb_tstage(const Inst *insts, const Chunk *chunks, const Ctrl *ctrls, const VT *__restrict__ x,
          const VT *__restrict__ D, VT *__restrict__ t) {
    CHUNK_BEGIN
    if (!ctrls[ck.inst].active) return;
    const VT *xi = x + I.off;
    const VT k0 = (VT)I.kap[0], k1 = (VT)I.kap[1], k2 = (VT)I.kap[2];
    if constexpr (sizeof(VT) == 4) {
        if ((I.n[0] & 3) == 0) {      // rows of whole groups of four: 16-byte accesses
            const float4 *D4 = reinterpret_cast<const float4 *>(D + I.off);
            float4 *t4 = reinterpret_cast<float4 *>(t + I.off);
            const unsigned ge = (unsigned)ck.end >> 2;
            for (unsigned q = ((unsigned)ck.begin >> 2) + threadIdx.x; q < ge; q += blockDim.x) {
                float4 xc, d[3];
                group_diffs_inst<DIM>(I, xi, q, xc, d);
                const float4 dq = D4[q];
                float4 r = make_float4(dq.x * xc.x, dq.y * xc.y, dq.z * xc.z, dq.w * xc.w);
                r.x = fmaf(k0, d[0].x, r.x); r.y = fmaf(k0, d[0].y, r.y);
                r.z = fmaf(k0, d[0].z, r.z); r.w = fmaf(k0, d[0].w, r.w);
                r.x = fmaf(k1, d[1].x, r.x); r.y = fmaf(k1, d[1].y, r.y);
                r.z = fmaf(k1, d[1].z, r.z); r.w = fmaf(k1, d[1].w, r.w);
                if (DIM == 3) {
                    r.x = fmaf(k2, d[2].x, r.x); r.y = fmaf(k2, d[2].y, r.y);
                    r.z = fmaf(k2, d[2].z, r.z); r.w = fmaf(k2, d[2].w, r.w);
                }
                t4[q] = r;
            }
            return;
        }
    }
    // FP64: pair-sum form with D; FP32: difference form with J (no cancellation of the
    // eps^2 sigma x term or of the smooth part of the neighbour sums in FP32 rounding)
    CHUNK_LOOP(l) {
        VT q[3];
        VT acc = D[I.off + l] * xi[l];
        if constexpr (sizeof(VT) == 8) {
            pair_sums_inst<DIM>(I, xi, l, q);
            acc = fma(-k0, q[0], acc);
            acc = fma(-k1, q[1], acc);
            if (DIM == 3) acc = fma(-k2, q[2], acc);
        } else {
            pair_diffs_inst<DIM>(I, xi, l, q);
            acc = fma(k0, q[0], acc);
            acc = fma(k1, q[1], acc);
            if (DIM == 3) acc = fma(k2, q[2], acc);
        }
        t[I.off + l] = acc;
    }
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kThreads)
kb_wstage(const Inst *insts, const Chunk *chunks, Ctrl *ctrls, const VT *__restrict__ t,
          VT *__restrict__ w, const VT *__restrict__ v1, double *Hs, int64_t hstride, int ldh,
          int j, double *partials, int nct, unsigned int *tickets) {
    CHUNK_BEGIN
    Ctrl *ctrl = ctrls + ck.inst;
    if (!ctrl->active) return;
    const double gam = ctrl->gam[j - 1];
    const VT c0 = (VT)(gam * I.sigma), c1 = (VT)(gam * I.s[0]), c2 = (VT)(gam * I.s[1]),
             c3 = (VT)(gam * I.s[2]);
    const VT *ti = t + I.off;
    BDot<VT> acc;
    CHUNK_LOOP(l) {
        VT q[3];
        VT r;
        if constexpr (sizeof(VT) == 8) {
            pair_sums_inst<DIM>(I, ti, l, q);
            r = c0 * ti[l];
            r = fma(-c1, q[0], r);
            r = fma(-c2, q[1], r);
            if (DIM == 3) r = fma(-c3, q[2], r);
        } else {
            pair_diffs_inst<DIM>(I, ti, l, q);
            r = c1 * q[0];
            r = fma(c2, q[1], r);
            if (DIM == 3) r = fma(c3, q[2], r);
        }
        w[I.off + l] = r;
        acc.add(r, v1[I.off + l]);
    }
    double v[1] = {acc.value()};
    double *H = Hs + ck.inst * hstride;
    inst_sum<1>(v, I, ck.inst, partials, nct, tickets,
                [&](double (&tot)[1]) { H[0 * ldh + (j - 1)] = ctrl->gam[0] * tot[0]; });
}

template <typename VT>
__global__ void __launch_bounds__(kThreads)
kb_mgs(const Inst *insts, const Chunk *chunks, Ctrl *ctrls, VT *__restrict__ w,
       const VT *__restrict__ vk, const VT *__restrict__ vk1, double *Hs, int64_t hstride,
       int ldh, int j, int k, int last, double *partials, int nct, unsigned int *tickets) {
    CHUNK_BEGIN
    Ctrl *ctrl = ctrls + ck.inst;
    if (!ctrl->active) return;
    double *H = Hs + ck.inst * hstride;
    const VT c = (VT)(H[(k - 1) * ldh + (j - 1)] * ctrl->gam[k - 1]);
    BDot<VT> acc;
    if (!last) {
        CHUNK_LOOP(l) {
            const int64_t gi = I.off + l;
            const VT r = fma(-c, vk[gi], w[gi]);
            w[gi] = r;
            acc.add(r, vk1[gi]);
        }
        double v[1] = {acc.value()};
        inst_sum<1>(v, I, ck.inst, partials, nct, tickets,
                    [&](double (&tot)[1]) { H[k * ldh + (j - 1)] = ctrl->gam[k] * tot[0]; });
    } else {
        CHUNK_LOOP(l) {
            const int64_t gi = I.off + l;
            const VT r = fma(-c, vk[gi], w[gi]);
            w[gi] = r;
            acc.add(r, r);
        }
        double v[1] = {acc.value()};
        inst_sum<1>(v, I, ck.inst, partials, nct, tickets, [&](double (&tot)[1]) {
            ctrl->hnext2 = tot[0];
            H[j * ldh + (j - 1)] = sqrt(tot[0]);          // h_{j+1,j} (Fig. 2)
        });
    }
}

// ---- Gram-corrected Arnoldi iteration of FP32 batches (mixed precision, j <= kBGsMaxJ) ----
// The coefficients of Fig. 2's modified Gram-Schmidt satisfy, for any computed basis,
//     h_kj = c_k - sum_{i<k} G_ki h_ij,   c_k = v_k . w,   G_ki = v_k . v_i,
// so one sweep over the basis gives every c_k and the Gram row of v_j, a forward
// substitution per instance gives the h_kj, and a second sweep applies the update and
// forms the new norm: three launches per iteration whatever j, instead of j + 2.
//   kbg_stage2A: w = gam_j A (stage-1 output), c_k and G_jk partials per chunk; the last
//                chunk of an instance sums its chunks' partials in chunk order and solves
//                for h_kj (H, update coefficients upd_k = h_kj gam_{k-1});
//   kbg_roundB:  w -= sum_k upd_k W_k, ||w||^2; the instance's last chunk stores h_{j+1,j}.
// j comes from the kernel argument, or from *jp when jp is given (device-driven loop).
constexpr int kBGsMaxJ = 31;
constexpr int kBGsSlots = 64;         // partials per chunk: c_k in [0, 32), G_jk in [32, 64)

// Block sums (256 threads) of nv <= 8 compensated per-thread pairs acc[q], written as
// double-float pairs to out[q] (fixed order: deterministic).
__device__ __forceinline__ void bgs_block_sums(const float2 (&acc)[8], int nv, float2 *out) {
    __shared__ float2 red[8][kThreads];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) red[q][tid] = acc[q];
    __syncthreads();
    const int q1 = tid >> 5, lane = tid & 31;                 // warp q1 adds value q1
    if (q1 < nv) {
        const float2 *p = &red[q1][lane * 8];
        float2 a = ch::ff_add(ch::ff_add(ch::ff_add(p[0], p[1]), ch::ff_add(p[2], p[3])),
                              ch::ff_add(ch::ff_add(p[4], p[5]), ch::ff_add(p[6], p[7])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 c;
            c.x = __shfl_down_sync(0xffffffffu, a.x, o);
            c.y = __shfl_down_sync(0xffffffffu, a.y, o);
            a = ch::ff_add(a, c);
        }
        if (lane == 0) out[q1] = a;
    }
    __syncthreads();
}

// compensated running sum of FP32 values (two-sum), kept as a (sum, correction) pair
__device__ __forceinline__ void bgs_acc(float2 &a, float p) {
    const float t = __fadd_rn(a.x, p);
    const float bp = __fsub_rn(t, a.x);
    a.y = __fadd_rn(a.y, __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
    a.x = t;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads)
kbg_stage2A(const Inst *insts, const Chunk *chunks, Ctrl *ctrls, const float *__restrict__ t,
            float *__restrict__ V, int64_t ldv, const float *__restrict__ slot0, int jarg,
            const int *jp, float2 *gpart, unsigned int *tickets, double *Hs, int64_t hstride,
            int ldh, double *grams, int64_t gstride, int ldg) {
    CHUNK_BEGIN
    Ctrl *ctrl = ctrls + ck.inst;
    if (!ctrl->active) return;
    const int j = jp ? *jp : jarg;
    auto W = [&](int c) -> const float * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    float *w = V + (int64_t)(j - 1) * ldv;                   // slot of W_{j+1}
    const float gam = (float)ctrl->gam[j - 1];
    const float c1 = gam * (float)I.s[0], c2 = gam * (float)I.s[1], c3 = gam * (float)I.s[2];
    const float *ti = t + I.off;
    const float *xj = W(j);
    float2 *part = gpart + (size_t)blockIdx.x * kBGsSlots;
    if ((I.n[0] & 3) == 0) {
        // ---- rows of whole groups of four: stage 2 fused into round A.  Tiles of two groups
        //      per thread; the tile's w is written once and kept with v_j in shared memory
        //      while the columns pass (v_j serves as column j), and the per-thread partials of
        //      each (tile, four columns) are added across the warp by a transposing shuffle
        //      tree into the warp's slots (c_k in [0, 32), G_jk in [32, 64)).
        __shared__ float4 wsm[2][kThreads], xsm[2][kThreads];
        __shared__ float2 accw[kThreads / 32][kBGsSlots];
        const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
        accw[wid][lane] = make_float2(0.f, 0.f);
        accw[wid][32 + lane] = make_float2(0.f, 0.f);
        __syncwarp();
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 *x4 = reinterpret_cast<const float4 *>(xj + I.off);
        float4 *w4 = reinterpret_cast<float4 *>(w + I.off);
        auto stage2 = [&](unsigned q) -> float4 {
            float4 tc, d[3];
            group_diffs_inst<DIM>(I, ti, q, tc, d);
            float4 r = make_float4(c1 * d[0].x, c1 * d[0].y, c1 * d[0].z, c1 * d[0].w);
            r.x = fmaf(c2, d[1].x, r.x); r.y = fmaf(c2, d[1].y, r.y);
            r.z = fmaf(c2, d[1].z, r.z); r.w = fmaf(c2, d[1].w, r.w);
            if (DIM == 3) {
                r.x = fmaf(c3, d[2].x, r.x); r.y = fmaf(c3, d[2].y, r.y);
                r.z = fmaf(c3, d[2].z, r.z); r.w = fmaf(c3, d[2].w, r.w);
            }
            return r;
        };
        const unsigned gb = (unsigned)ck.begin >> 2, ge = (unsigned)ck.end >> 2;
        // the same number of trips in every thread (the shuffle tree needs whole warps)
        for (unsigned base = gb; base < ge; base += 2u * kThreads) {
            const unsigned qa = base + threadIdx.x, qb = qa + kThreads;
            const bool ha = qa < ge, hb = qb < ge;
            const float4 wa = ha ? stage2(qa) : zero4, wb = hb ? stage2(qb) : zero4;
            if (ha) w4[qa] = wa;
            if (hb) w4[qb] = wb;
            wsm[0][threadIdx.x] = wa;
            wsm[1][threadIdx.x] = wb;
            xsm[0][threadIdx.x] = ha ? x4[qa] : zero4;
            xsm[1][threadIdx.x] = hb ? x4[qb] : zero4;
            for (int k0 = 1; k0 <= j; k0 += 4) {
                const int nk = min(4, j - k0 + 1);
                float4 va[4], vb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < nk && k0 + u < j) {
                        const float4 *c4 = reinterpret_cast<const float4 *>(W(k0 + u) + I.off);
                        va[u] = ha ? c4[qa] : zero4;
                        vb[u] = hb ? c4[qb] : zero4;
                    } else if (u < nk) {                    // column j is v_j itself
                        va[u] = xsm[0][threadIdx.x];
                        vb[u] = xsm[1][threadIdx.x];
                    } else {
                        va[u] = vb[u] = zero4;
                    }
                }
                float2 p[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) p[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 wv = wsm[r][threadIdx.x], xv = xsm[r][threadIdx.x];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        bgs_acc(p[u], dot4f(wv, r == 0 ? va[u] : vb[u]));
                        bgs_acc(p[4 + u], dot4f(xv, r == 0 ? va[u] : vb[u]));
                    }
                }
                // after the exchanges at lane distances 16, 8 and 4 a lane holds value
                // (lane >> 2) of its group of four lanes; distances 2 and 1 finish the sum
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool hi = (lane & 16u) != 0;
                    const float2 keep = hi ? p[i + 4] : p[i], send = hi ? p[i] : p[i + 4];
                    float2 rv;
                    rv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
                    rv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
                    p[i] = ch::ff_add(keep, rv);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const bool hi = (lane & 8u) != 0;
                    const float2 keep = hi ? p[i + 2] : p[i], send = hi ? p[i] : p[i + 2];
                    float2 rv;
                    rv.x = __shfl_xor_sync(0xffffffffu, send.x, 8);
                    rv.y = __shfl_xor_sync(0xffffffffu, send.y, 8);
                    p[i] = ch::ff_add(keep, rv);
                }
                float2 sv;
                {
                    const bool hi = (lane & 4u) != 0;
                    const float2 keep = hi ? p[1] : p[0], send = hi ? p[0] : p[1];
                    float2 rv;
                    rv.x = __shfl_xor_sync(0xffffffffu, send.x, 4);
                    rv.y = __shfl_xor_sync(0xffffffffu, send.y, 4);
                    sv = ch::ff_add(keep, rv);
                }
#pragma unroll
                for (int o = 2; o > 0; o >>= 1) {
                    float2 rv;
                    rv.x = __shfl_xor_sync(0xffffffffu, sv.x, o);
                    rv.y = __shfl_xor_sync(0xffffffffu, sv.y, o);
                    sv = ch::ff_add(sv, rv);
                }
                const int v = (int)(lane >> 2), u = v & 3;
                if ((lane & 3u) == 0 && u < nk && (v < 4 || k0 + u < j)) {
                    const int slot = (v < 4 ? 0 : 32) + k0 - 1 + u;
                    accw[wid][slot] = ch::ff_add(accw[wid][slot], sv);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < kBGsSlots) {          // the chunk's partials, warps added in order
            const int v = threadIdx.x, k = v < 32 ? v : v - 32;
            if (v < 32 ? k < j : k < j - 1) {
                float2 a = accw[0][v];
#pragma unroll
                for (int q = 1; q < kThreads / 32; ++q) a = ch::ff_add(a, accw[q][v]);
                part[v] = a;
                __threadfence();
            }
        }
        __syncthreads();
    } else {
    // ---- stage 2: w = gam_j A t (difference form, FP32)
    CHUNK_LOOP(l) {
        float q[3];
        pair_diffs_inst<DIM>(I, ti, l, q);
        float r = c1 * q[0];
        r = fmaf(c2, q[1], r);
        if (DIM == 3) r = fmaf(c3, q[2], r);
        w[I.off + l] = r;
    }
    // ---- round A: per-chunk partials of W_k . w (k <= j) and W_j . W_k (k < j), four
    //      columns per sweep over this thread's points (its own w values: no barrier)
    __shared__ float2 bout[8];
    for (int k0 = 1; k0 <= j; k0 += 4) {
        const int nk = min(4, j - k0 + 1);
        float2 acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
        CHUNK_LOOP(l) {
            const int64_t gi = I.off + l;
            const float wv = w[gi], xv = xj[gi];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < nk) {
                    const float v = W(k0 + u)[gi];
                    bgs_acc(acc[u], wv * v);
                    if (k0 + u < j) bgs_acc(acc[4 + u], xv * v);
                }
        }
        bgs_block_sums(acc, 8, bout);
        if (threadIdx.x == 0)
            for (int u = 0; u < nk; ++u) {
                part[k0 - 1 + u] = bout[u];
                if (k0 + u < j) part[32 + k0 - 1 + u] = bout[4 + u];
            }
    }
    }
    // ---- the instance's last chunk: sums over its chunks in order, then h_kj
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&tickets[ck.inst], 1u) == (unsigned)I.nchunks - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double cs[kBGsMaxJ + 1];
    __shared__ float gs[kBGsMaxJ][kBGsMaxJ + 2];       // G_ki (k > i), 0-based
    __shared__ double gms[kBGsMaxJ + 1];
    double *gram = grams + ck.inst * gstride;
    for (int e = threadIdx.x; e < j; e += blockDim.x) gms[e] = ctrl->gam[e];
    for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
        const int k = e / j, i = e % j;
        gs[k][i] = (i < k && k < j - 1) ? (float)gram[(size_t)k * ldg + i] : 0.f;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 64; v += blockDim.x) {
        const bool isc = v < 32;
        const int k = isc ? v : v - 32;                   // 0-based column
        if ((isc && k < j) || (!isc && k < j - 1)) {
            double sum = 0.0;
            for (int c = 0; c < I.nchunks; ++c) {
                const float2 pv = __ldcg(gpart + (size_t)(I.first_chunk + c) * kBGsSlots + v);
                sum += (double)pv.x + (double)pv.y;
            }
            if (isc) {
                cs[k] = gms[k] * sum;                                  // c_k = v_k . w
            } else {
                const double gji = gms[j - 1] * gms[k] * sum;          // G_jk = v_j . v_k
                gs[j - 1][k] = (float)gji;
                gram[(size_t)(j - 1) * ldg + k] = gji;
            }
        }
    }
    __syncthreads();
    // forward substitution h_k = c_k - sum_{i<k} G_ki h_i (lane k-1 of warp 0): the sweeps
    // h <- c - G h (FP32 corrections, small next to c_k) until they no longer change, else the
    // sequential substitution; h_k itself is FP64
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        __shared__ float hsm[32];
        const double r = l < j ? cs[l] : 0.0;
        const float rf = (float)r;
        float corr = 0.f;
        bool done = false;
        for (int sweep = 0; sweep < 4 && !done; ++sweep) {
            hsm[l] = __fsub_rn(rf, corr);
            __syncwarp();
            float c2s = 0.f;
            if (l < j)
                for (int i = 0; i < l; ++i) c2s = __fmaf_rn(gs[l][i], hsm[i], c2s);
            __syncwarp();
            done = __all_sync(0xffffffffu, c2s == corr);
            corr = c2s;
        }
        if (!done) {
            corr = 0.f;
            for (int i = 0; i < j; ++i) {
                const float gcur = (l > i && l < j) ? gs[l][i] : 0.f;
                const float hi = __shfl_sync(0xffffffffu, __fsub_rn(rf, corr), i);
                corr = __fmaf_rn(gcur, hi, corr);
            }
        }
        if (l < j) {
            const double h = r - (double)corr;
            ctrl->upd[l] = h * gms[l];
            Hs[ck.inst * hstride + (size_t)l * ldh + (j - 1)] = h;
        }
    }
    if (threadIdx.x == 0) tickets[ck.inst] = 0u;
}

__global__ void __launch_bounds__(kThreads)
kbg_roundB(const Inst *insts, const Chunk *chunks, Ctrl *ctrls, float *__restrict__ V, int64_t ldv,
           const float *__restrict__ slot0, int jarg, const int *jp, float2 *gpart,
           unsigned int *tickets, double *Hs, int64_t hstride, int ldh) {
    CHUNK_BEGIN
    Ctrl *ctrl = ctrls + ck.inst;
    if (!ctrl->active) return;
    const int j = jp ? *jp : jarg;
    auto W = [&](int c) -> const float * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * ldv; };
    float *w = V + (int64_t)(j - 1) * ldv;
    __shared__ float as[kBGsMaxJ];
    for (int e = threadIdx.x; e < j; e += blockDim.x) as[e] = (float)ctrl->upd[e];
    __syncthreads();
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
    if ((I.n[0] & 3) == 0) {          // rows of whole groups of four: 16-byte accesses
        float4 *w4 = reinterpret_cast<float4 *>(w + I.off);
        const unsigned ge = (unsigned)ck.end >> 2;
        for (unsigned q = ((unsigned)ck.begin >> 2) + threadIdx.x; q < ge; q += blockDim.x) {
            float4 x = w4[q];
            for (int k0 = 1; k0 <= j; k0 += 8) {       // eight column loads in flight
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = k0 + u <= j ? reinterpret_cast<const float4 *>(W(k0 + u) + I.off)[q]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
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
            w4[q] = x;
            bgs_acc(acc[0], dot4f(x, x));
        }
    } else
    CHUNK_LOOP(l) {
        const int64_t gi = I.off + l;
        float x = w[gi];
        for (int k0 = 1; k0 <= j; k0 += 8) {           // eight column loads in flight
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = k0 + u <= j ? W(k0 + u)[gi] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k0 + u <= j) x = __fmaf_rn(-as[k0 + u - 1], v[u], x);
        }
        w[gi] = x;
        bgs_acc(acc[0], x * x);
    }
    __shared__ float2 bout[8];
    bgs_block_sums(acc, 1, bout);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        gpart[(size_t)blockIdx.x * kBGsSlots] = bout[0];
        __threadfence();
        last = (atomicAdd(&tickets[ck.inst], 1u) == (unsigned)I.nchunks - 1u);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double nrm2 = 0.0;
    for (int c = 0; c < I.nchunks; ++c) {
        const float2 pv = __ldcg(gpart + (size_t)(I.first_chunk + c) * kBGsSlots);
        nrm2 += (double)pv.x + (double)pv.y;
    }
    ctrl->hnext2 = nrm2;
    Hs[ck.inst * hstride + (size_t)j * ldh + (j - 1)] = sqrt(nrm2);     // h_{j+1,j} (Fig. 2)
    tickets[ck.inst] = 0u;
}

// 1 in *flag when some instance's Krylov run is still active.
__global__ void kb_any(const Ctrl *ctrls, int count, int *flag) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        if (ctrls[i].active) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) *flag = any;
}

// Gate of Arnoldi iteration j in a device-driven step: the condition of that iteration's
// conditional node is 1 while some instance's Krylov run is still active, so iterations
// after every run has ended cost one small launch.  Kernel launches are tallied in *nlaunch
// (this one, plus the iteration's `iter_kernels` when it runs).
__global__ void kb_gate(const Ctrl *ctrls, int count, cudaGraphConditionalHandle h,
                        unsigned long long *nlaunch, int iter_kernels) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        if (ctrls[i].active) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        cudaGraphSetConditional(h, any ? 1u : 0u);
        atomicAdd(nlaunch, 1ull + (any ? (unsigned long long)iter_kernels : 0ull));
    }
}

// ---- Krylov combine of Fig. 2 per instance; finished instances carry y over ---------------
template <typename VT>
__global__ void __launch_bounds__(kThreads)
kb_combine(const Inst *insts, const Chunk *chunks, const BState *bs, Ctrl *ctrls,
           const double *__restrict__ y0, const VT *__restrict__ v0, const VT *__restrict__ V,
           int64_t ldv, double *__restrict__ ynext, float *__restrict__ dtmp, double *partials,
           int nct, unsigned int *tickets) {
    CHUNK_BEGIN
    Ctrl *ctrl = ctrls + ck.inst;
    const int j = bs[ck.inst].done ? 0 : ctrl->jexit;
    __shared__ double coef[130];
    for (int c = threadIdx.x; c < j; c += blockDim.x) coef[c] = ctrl->coef[c];
    __syncthreads();
    if (sizeof(VT) == 8) {
        CHUNK_LOOP(l) {
            const int64_t gi = I.off + l;
            double acc = 0.0;
            if (j > 0) acc = coef[0] * (double)v0[gi];
            for (int c = 1; c < j; ++c) acc = fma(coef[c], (double)V[(c - 1) * ldv + gi], acc);
            ynext[gi] = y0[gi] + acc;
        }
    } else {                           // mixed: FP32 increment, its mass removed in pass b
        BDot<float> m;
        CHUNK_LOOP(l) {
            const int64_t gi = I.off + l;
            float a = 0.f;
            if (j > 0) a = (float)coef[0] * (float)v0[gi];
            for (int c = 1; c < j; ++c) a = fmaf((float)coef[c], (float)V[(c - 1) * ldv + gi], a);
            dtmp[gi] = a;
            m.add(a, 1.0f);
        }
        double v[1] = {m.value()};
        inst_sum<1>(v, I, ck.inst, partials, nct, tickets,
                    [&](double (&tot)[1]) { ctrl->red[6] = tot[0]; });
    }
}

__global__ void __launch_bounds__(kThreads)
kb_combine32b(const Inst *insts, const Chunk *chunks, const BState *bs, const Ctrl *ctrls,
              const double *__restrict__ y0, const float *__restrict__ d,
              double *__restrict__ ynext) {
    CHUNK_BEGIN
    const bool moved = !bs[ck.inst].done && ctrls[ck.inst].jexit > 0;
    const double mean = moved ? ctrls[ck.inst].red[6] / (double)I.N : 0.0;
    CHUNK_LOOP(l) {
        const int64_t gi = I.off + l;
        ynext[gi] = moved ? y0[gi] + ((double)d[gi] - mean) : y0[gi];
    }
}

// ---- Fig. 4 per instance: est, time, next step size (Eq. EEdt), counters -----------------
// With `steps` (device-driven runs) the control also counts batch steps and, when cond_set,
// sets the condition of the graph's step loop: run on while an instance is before T and
// fewer than max_steps batch steps were taken.
__global__ void kb_control(Ctrl *ctrls, BState *bs, int count, double T, double tol,
                           int *remaining, long long *steps, long long max_steps, int cond_set,
                           cudaGraphConditionalHandle cond, unsigned long long *nlaunch,
                           int step_kernels) {
    __shared__ int rem;
    if (threadIdx.x == 0) rem = 0;
    __syncthreads();
    const bool halted = steps && *steps >= max_steps;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        Ctrl *c = ctrls + i;
        BState *b = bs + i;
        if (!b->done && !halted) {
            if (c->status != 0) {
                b->status = c->status;
                b->done = 1;
            } else {
                const double taken = c->tau;
                const double est = sqrt(c->red[2]) / sqrt(c->red[3]);
                b->est = est;
                b->matvecs += 1 + c->jexit;
                b->krylov_iters += c->jexit;
                b->tau_shrinks += c->shrunk;
                b->phi_evals += c->phi_evals;
                b->rhs_evals += 1;
                b->steps += 1;
                b->t = (b->clipped && taken == b->tau) ? T : b->t + taken;
                const double grow = 1.25 * taken;
                b->tau = (est > 0.0) ? fmin(grow, sqrt(tol / est) * taken) : grow;
                if (!isfinite(est)) { b->status = CH_ENONFINITE; b->done = 1; }
                else if (!(b->t < T)) b->done = 1;
                else if (!(b->tau > 0.0) || b->t + b->tau == b->t) { b->status = CH_ENOTCONV; b->done = 1; }
            }
        }
        if (!b->done) atomicAdd(&rem, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *remaining = rem;
        if (steps) {
            const long long k = halted ? *steps : *steps + 1;
            *steps = k;
            *nlaunch += (unsigned long long)step_kernels;
            if (cond_set) cudaGraphSetConditional(cond, (rem > 0 && k < max_steps) ? 1u : 0u);
        }
    }
}

__global__ void kb_init(BState *bs, Ctrl *ctrls, int count, double tau0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    BState b;
    memset(&b, 0, sizeof b);
    b.tau = tau0;
    bs[i] = b;
    ctrls[i].status = 0;
    ctrls[i].active = 0;
}

}  // namespace

// -------------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------------
struct ch_batch {
    int dim, count, precision, mmax_cap, nchunks, chunk_len;
    int64_t Ntot;
    cudaStream_t stream, cap_stream;
    std::vector<Inst> hinst;
    std::vector<int64_t> offsets;
    Inst *insts;
    Chunk *chunks;
    BState *bs;
    Ctrl *ctrls;
    double *H, *u;           // count x (mmax+1) x mmax, count x (mmax+1)
    double *ynew, *F[2], *mu, *q, *partials;
    unsigned int *tickets;
    void *D, *t, *V, *W[2];  // basis precision
    int *dflags;             // [0] any active, [1] remaining
    long long *dsteps;       // batch steps taken by a device-driven run
    float2 *gpart;           // mixed batches: chunk partials of the Gram-corrected iteration
    double *grams;           // mixed batches: Gram matrix of each instance's basis
    cudaGraphExec_t run_exec;               // device-driven integration (one graph launch)
    unsigned long long *dlaunch;            // kernels a device-driven run executed
    cudaStream_t cap_stream2;               // second capture stream (conditional bodies)
    std::vector<double> run_key;            // parameters the run graph was built for
    int *hflags;             // pinned: [0],[1] any active (alternating), [2] remaining
    cudaEvent_t ev[2];
    int64_t launches;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (slot, j) -> iteration graph
    int mmax_graphs;
    // pinned copies read back at the end of a device-driven run
    BState *hbs;                            // count per-instance states
    long long *hsteps;                      // batch steps taken
    unsigned long long *hran;               // kernels executed
    // Scheduling groups: a batch whose few stiffest instances would set its time runs them as
    // a group of their own, concurrently with the others, each group a batch object on its
    // own stream (the stiff group's of the highest priority) sharing the caller's layout.
    int ngroups;                            // 0: no groups (this object runs its instances)
    ch_batch *grp[2];
    std::vector<int> grp_idx[2];            // instance of this batch behind each group instance
    cudaStream_t grp_stream[2];
    cudaEvent_t grp_ev[3];
};

namespace {

template <typename VT> struct Kern;

Launch make_launch(ch_batch *b, cudaStream_t s) {
    Launch L;
    L.blocks = b->nchunks;
    L.stream = s;
    L.partials = b->partials;
    L.ctrl = b->ctrls;
    L.launches = &b->launches;
    L.timing = nullptr;
    return L;
}

#define BLAUNCH(KERNEL, ...)                                                               \
    do {                                                                                   \
        if (b->dim == 3) KERNEL<3><<<b->nchunks, kThreads, 0, s>>>(__VA_ARGS__);           \
        else KERNEL<2><<<b->nchunks, kThreads, 0, s>>>(__VA_ARGS__);                       \
        ++b->launches;                                                                     \
    } while (0)
#define BLAUNCH_T(KERNEL, VT, ...)                                                         \
    do {                                                                                   \
        if (b->dim == 3) KERNEL<3, VT><<<b->nchunks, kThreads, 0, s>>>(__VA_ARGS__);       \
        else KERNEL<2, VT><<<b->nchunks, kThreads, 0, s>>>(__VA_ARGS__);                   \
        ++b->launches;                                                                     \
    } while (0)

template <typename VT>
void rhs_b(ch_batch *b, cudaStream_t s, const double *y, int slot, int est, const double *y0,
           const double *f0) {
    VT *fvt = sizeof(VT) == 8 ? nullptr : (VT *)b->W[slot];
    BLAUNCH(kb_rhs1, b->insts, b->chunks, b->bs, y, b->mu, b->q);
    BLAUNCH_T(kb_rhs2, VT, b->insts, b->chunks, b->bs, b->ctrls, b->mu, b->q, b->F[slot], fvt,
              y0, f0, y, est, b->partials, b->nchunks, b->tickets);
}

template <typename VT>
VT *basis_col(ch_batch *b, int slot, int c) {   // W_c, 1-based
    if (c == 1) return sizeof(VT) == 8 ? (VT *)b->F[slot] : (VT *)b->W[slot];
    return (VT *)b->V + (int64_t)(c - 2) * b->Ntot;
}

// Kernels of Arnoldi iteration j of every active instance (Fig. 2) and the projected phi
// with its residual test: the Gram-corrected form (three launches) on FP32 batches with
// m_max <= kBGsMaxJ, the sequential modified Gram-Schmidt passes otherwise.  jp: the
// device-held j of a device-driven loop (nullptr: j as given).
template <typename VT>
void queue_arnoldi_kernels_b(ch_batch *b, cudaStream_t s, int slot, int j) {
    const int ldh = b->mmax_cap;
    const int64_t hs = (int64_t)(b->mmax_cap + 1) * b->mmax_cap;
    VT *Wj = basis_col<VT>(b, slot, j), *Wn = basis_col<VT>(b, slot, j + 1), *v1 = basis_col<VT>(b, slot, 1);
    BLAUNCH_T(kb_tstage, VT, b->insts, b->chunks, b->ctrls, Wj, (const VT *)b->D, (VT *)b->t);
    if (sizeof(VT) == 4 && b->gpart && j <= kBGsMaxJ) {
        const int ldg = b->mmax_cap + 1;
        const int64_t gst = (int64_t)ldg * ldg;
        BLAUNCH(kbg_stage2A, b->insts, b->chunks, b->ctrls, (const float *)b->t, (float *)b->V, b->Ntot,
                (const float *)v1, j, (const int *)nullptr, b->gpart, b->tickets, b->H, hs, ldh, b->grams,
                gst, ldg);
        kbg_roundB<<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->ctrls, (float *)b->V, b->Ntot,
                                                   (const float *)v1, j, nullptr, b->gpart, b->tickets, b->H,
                                                   hs, ldh);
        ++b->launches;
    } else {
        BLAUNCH_T(kb_wstage, VT, b->insts, b->chunks, b->ctrls, (const VT *)b->t, Wn, v1, b->H, hs, ldh,
                  j, b->partials, b->nchunks, b->tickets);
        for (int k = 1; k <= j; ++k) {
            const int last = k == j;
            kb_mgs<VT><<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->ctrls, Wn,
                                                        basis_col<VT>(b, slot, k),
                                                        last ? nullptr : basis_col<VT>(b, slot, k + 1),
                                                        b->H, hs, ldh, j, k, last, b->partials,
                                                        b->nchunks, b->tickets);
            ++b->launches;
        }
    }
}

template <typename VT>
void queue_arnoldi_b(ch_batch *b, cudaStream_t s, int slot, int j, int mmax) {
    const int ldh = b->mmax_cap;
    const int64_t hs = (int64_t)(b->mmax_cap + 1) * b->mmax_cap;
    queue_arnoldi_kernels_b<VT>(b, s, slot, j);
    Launch L = make_launch(b, s);
    ch::launch_phi_batch(L, b->ctrls, b->H, hs, b->u, b->mmax_cap + 1, ldh, j, mmax, b->count);
}

// Host-driven form: iteration j, then the "any run active" flag copied to pinned memory.
template <typename VT>
void queue_iteration_b(ch_batch *b, cudaStream_t s, int slot, int j, int mmax) {
    queue_arnoldi_b<VT>(b, s, slot, j, mmax);
    kb_any<<<1, 256, 0, s>>>(b->ctrls, b->count, &b->dflags[0]);
    ++b->launches;
    cudaMemcpyAsync(&b->hflags[j & 1], &b->dflags[0], sizeof(int), cudaMemcpyDeviceToHost, s);
}

template <typename VT>
ch_status krylov_b(ch_batch *b, int slot, int mmax, bool use_graphs) {
    for (int j = 1; j <= mmax; ++j) {
        if (use_graphs) {
            auto key = std::make_pair(slot, j);
            auto it = b->graphs.find(key);
            cudaGraphExec_t exec;
            if (it == b->graphs.end()) {
                cudaGraph_t g;
                int64_t before = b->launches;
                BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
                queue_iteration_b<VT>(b, b->cap_stream, slot, j, mmax);
                BCUDA(cudaStreamEndCapture(b->cap_stream, &g));
                cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return bfail(CH_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
                b->launches = before;
                b->graphs[key] = exec;
            } else {
                exec = it->second;
            }
            BCUDA(cudaGraphLaunch(exec, b->stream));
            b->launches += 3 + j + 1;
        } else {
            queue_iteration_b<VT>(b, b->stream, slot, j, mmax);
        }
        BCUDA(cudaGetLastError());
        BCUDA(cudaEventRecord(b->ev[j & 1], b->stream));
        if (j >= 2) {
            BCUDA(cudaEventSynchronize(b->ev[(j - 1) & 1]));
            if (b->hflags[(j - 1) & 1] == 0) break;
        }
    }
    return CH_OK;
}

template <typename VT>
ch_status integrate_b(ch_batch *b, const ch_params *prm, double *y, ch_stats *stats) {
    cudaStream_t s = b->stream;
    if (b->mmax_graphs != prm->mmax) {       // graphs bake m_max into the phi step
        for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
        b->graphs.clear();
        b->mmax_graphs = prm->mmax;
    }
    const bool use_graphs = true;
    kb_init<<<(b->count + 255) / 256, 256, 0, s>>>(b->bs, b->ctrls, b->count, prm->tau0);
    double *ycur = y, *ynew = b->ynew;
    int cur = 0;
    rhs_b<VT>(b, s, ycur, cur, 0, nullptr, nullptr);                 // f(y^0), norms
    BCUDA(cudaGetLastError());
    int64_t steps = 0;
    ch_status rc = CH_OK;
    for (;;) {
        kb_arm<<<(b->count + 255) / 256, 256, 0, s>>>(b->ctrls, b->bs, b->count, prm->T,
                                                      prm->tol_phi, prm->tol, nullptr, 0);
        kb_prep<VT><<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->bs, ycur, (VT *)b->D);
        ++b->launches;
        BTRY(krylov_b<VT>(b, cur, prm->mmax, use_graphs));
        kb_combine<VT><<<b->nchunks, kThreads, 0, s>>>(
            b->insts, b->chunks, b->bs, b->ctrls, ycur, basis_col<VT>(b, cur, 1), (VT *)b->V,
            b->Ntot, ynew, (float *)b->t, b->partials, b->nchunks, b->tickets);
        if (sizeof(VT) == 4)
            kb_combine32b<<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->bs, b->ctrls,
                                                           ycur, (float *)b->t, ynew);
        rhs_b<VT>(b, s, ynew, 1 - cur, 1, ycur, b->F[cur]);           // est, f(y^{n+1})
        kb_control<<<1, 256, 0, s>>>(b->ctrls, b->bs, b->count, prm->T, prm->tol, &b->dflags[1], nullptr,
                                     0, 0, cudaGraphConditionalHandle{}, nullptr, 0);
        BCUDA(cudaGetLastError());
        BCUDA(cudaMemcpyAsync(&b->hflags[2], &b->dflags[1], sizeof(int), cudaMemcpyDeviceToHost, s));
        BCUDA(cudaStreamSynchronize(s));
        std::swap(ycur, ynew);
        cur = 1 - cur;
        ++steps;
        if (b->hflags[2] == 0) break;
        if (steps >= prm->max_steps) {   // y and stats still receive the state reached
            rc = bfail(CH_ENOTCONV, "max_steps reached before T");
            break;
        }
    }
    if (ycur != y) BCUDA(cudaMemcpyAsync(y, ycur, b->Ntot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<BState> hb(b->count);
    BCUDA(cudaMemcpyAsync(hb.data(), b->bs, b->count * sizeof(BState), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < b->count; ++i) {
        if (hb[i].status && rc == CH_OK)
            rc = bfail((ch_status)hb[i].status, "instance %d failed (status %d) at t = %g", i, hb[i].status, hb[i].t);
        if (stats) {
            ch_stats &st = stats[i];
            memset(&st, 0, sizeof st);
            st.steps = hb[i].steps; st.matvecs = hb[i].matvecs; st.rhs_evals = hb[i].rhs_evals;
            st.krylov_iters = hb[i].krylov_iters; st.tau_shrinks = hb[i].tau_shrinks;
            st.phi_evals = hb[i].phi_evals; st.t = hb[i].t; st.tau_next = hb[i].tau;
            st.last_est = hb[i].est;
        }
    }
    return rc;
}

// ---- device-driven integration: the whole run is one graph launch --------------------------
// One batch step (Fig. 4 for every instance still before T) with all m_max Arnoldi iterations
// unrolled: the kernels of iteration j return at once for instances whose Krylov run has
// ended, so no host decision is needed inside a step.  Slot `cur` holds f(y^n) and the start
// vector; ycur -> ynew.  kb_control counts the step and, with cond_set, sets the loop condition.
template <typename VT>
ch_status queue_step_dev(ch_batch *b, cudaStream_t s, const ch_params *prm, int cur, double *ycur,
                         double *ynew, int cond_set, cudaGraphConditionalHandle cond) {
    const int64_t l0 = b->launches;
    kb_arm<<<(b->count + 255) / 256, 256, 0, s>>>(b->ctrls, b->bs, b->count, prm->T, prm->tol_phi, prm->tol,
                                                  b->dsteps, prm->max_steps);
    kb_prep<VT><<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->bs, ycur, (VT *)b->D);
    b->launches += 2;
    queue_arnoldi_b<VT>(b, s, cur, 1, prm->mmax);
    int64_t fixed = b->launches - l0;
    for (int j = 2; j <= prm->mmax; ++j) {
        // gate kernel, then a conditional node holding iteration j (captured on a second stream)
        cudaStreamCaptureStatus st;
        cudaGraph_t cg = nullptr;
        BCUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        BCUDA(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
        const int64_t li = b->launches;
        const int iter_kernels = (sizeof(VT) == 4 && b->gpart && j <= kBGsMaxJ) ? 4 : 3 + j;
        kb_gate<<<1, 256, 0, s>>>(b->ctrls, b->count, h, b->dlaunch, iter_kernels);
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        BCUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        BCUDA(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
        BCUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        BCUDA(cudaStreamBeginCaptureToGraph(b->cap_stream2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
        queue_arnoldi_b<VT>(b, b->cap_stream2, cur, j, prm->mmax);
        cudaGraph_t tmp = nullptr;
        BCUDA(cudaStreamEndCapture(b->cap_stream2, &tmp));
        b->launches = li;                  // executed launches are tallied on the device
    }
    const int64_t l1 = b->launches;
    kb_combine<VT><<<b->nchunks, kThreads, 0, s>>>(
        b->insts, b->chunks, b->bs, b->ctrls, ycur, basis_col<VT>(b, cur, 1), (VT *)b->V, b->Ntot, ynew,
        (float *)b->t, b->partials, b->nchunks, b->tickets);
    ++b->launches;
    if (sizeof(VT) == 4) {
        kb_combine32b<<<b->nchunks, kThreads, 0, s>>>(b->insts, b->chunks, b->bs, b->ctrls, ycur,
                                                       (float *)b->t, ynew);
        ++b->launches;
    }
    rhs_b<VT>(b, s, ynew, 1 - cur, 1, ycur, b->F[cur]);                 // est, f(y^{n+1})
    fixed += b->launches - l1 + 1;
    kb_control<<<1, 256, 0, s>>>(b->ctrls, b->bs, b->count, prm->T, prm->tol, &b->dflags[1], b->dsteps,
                                 prm->max_steps, cond_set, cond, b->dlaunch, (int)fixed);
    BCUDA(cudaGetLastError());
    return CH_OK;
}

// The run graph: a conditional while node whose body takes two batch steps, y -> ynew and
// ynew -> y, so every pass ends with the state in the caller's y (instances that reached T
// are carried over by the combine).  The body repeats while the second step's control finds
// an instance before T and fewer than max_steps steps taken.  Kernel arguments (y, T, tol,
// tau0, m_max, max_steps) are baked in: the graph is rebuilt when they change.
template <typename VT>
ch_status build_run_graph(ch_batch *b, const ch_params *prm, double *y) {
    const std::vector<double> key = {(double)(uintptr_t)y, prm->T, prm->tau0, prm->tol, prm->tol_phi,
                                     (double)prm->mmax, (double)prm->max_steps};
    if (b->run_exec && key == b->run_key) return CH_OK;
    if (b->run_exec) { cudaGraphExecDestroy(b->run_exec); b->run_exec = nullptr; }
    cudaGraph_t graph = nullptr;
    BCUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return bfail(CH_ECUDA, "conditional graph node: %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const int64_t before = b->launches;
    e = cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        ch_status st = queue_step_dev<VT>(b, b->cap_stream, prm, 0, y, b->ynew, 0, cond);
        if (st == CH_OK) st = queue_step_dev<VT>(b, b->cap_stream, prm, 1, b->ynew, y, 1, cond);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(b->cap_stream, &captured);
        if (st != CH_OK && e == cudaSuccess) e = cudaErrorStreamCaptureInvalidated;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->run_exec, graph, 0);
    cudaGraphDestroy(graph);
    b->launches = before;
    if (e != cudaSuccess) {
        b->run_exec = nullptr;
        cudaGetLastError();
        return bfail(CH_ECUDA, "run graph: %s", cudaGetErrorString(e));
    }
    b->run_key = key;
    return CH_OK;
}

// Device-driven run, queued on the batch's stream: nothing here waits for the GPU, so the
// groups of a batch run concurrently.  finish_b_dev waits and reads the counters.
template <typename VT>
ch_status launch_b_dev(ch_batch *b, const ch_params *prm, double *y) {
    cudaStream_t s = b->stream;
    BTRY(build_run_graph<VT>(b, prm, y));
    kb_init<<<(b->count + 255) / 256, 256, 0, s>>>(b->bs, b->ctrls, b->count, prm->tau0);
    BCUDA(cudaMemsetAsync(b->dsteps, 0, sizeof(long long), s));
    BCUDA(cudaMemsetAsync(b->dlaunch, 0, sizeof(unsigned long long), s));
    rhs_b<VT>(b, s, y, 0, 0, nullptr, nullptr);                      // f(y^0), norms
    BCUDA(cudaGetLastError());
    BCUDA(cudaGraphLaunch(b->run_exec, s));
    BCUDA(cudaMemcpyAsync(&b->hflags[2], &b->dflags[1], sizeof(int), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaMemcpyAsync(b->hsteps, b->dsteps, sizeof(long long), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaMemcpyAsync(b->hran, b->dlaunch, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaMemcpyAsync(b->hbs, b->bs, b->count * sizeof(BState), cudaMemcpyDeviceToHost, s));
    return CH_OK;
}

ch_status finish_b_dev(ch_batch *b, ch_stats *stats) {
    BCUDA(cudaStreamSynchronize(b->stream));
    b->launches += 3 + (int64_t)*b->hran;       // kb_init, f(y^0) and the graph's executed kernels
    ch_status rc = CH_OK;
    if (b->hflags[2] != 0) rc = bfail(CH_ENOTCONV, "max_steps reached before T");
    const BState *hb = b->hbs;
    for (int i = 0; i < b->count; ++i) {
        if (hb[i].status && rc == CH_OK)
            rc = bfail((ch_status)hb[i].status, "instance %d failed (status %d) at t = %g", i, hb[i].status, hb[i].t);
        if (stats) {
            ch_stats &st = stats[i];
            memset(&st, 0, sizeof st);
            st.steps = hb[i].steps; st.matvecs = hb[i].matvecs; st.rhs_evals = hb[i].rhs_evals;
            st.krylov_iters = hb[i].krylov_iters; st.tau_shrinks = hb[i].tau_shrinks;
            st.phi_evals = hb[i].phi_evals; st.t = hb[i].t; st.tau_next = hb[i].tau;
            st.last_est = hb[i].est;
        }
    }
    return rc;
}

template <typename VT>
ch_status integrate_b_dev(ch_batch *b, const ch_params *prm, double *y, ch_stats *stats) {
    BTRY(launch_b_dev<VT>(b, prm, y));
    return finish_b_dev(b, stats);
}

// Chunk length candidates for the autotuner (values per chunk; a chunk is one thread block).
const int kChunkCandidates[] = {1024, 2048, 4096, 8192};

void build_chunks(ch_batch *b, int chunk_len, std::vector<Chunk> &ch) {
    ch.clear();
    for (int i = 0; i < b->count; ++i) {
        Inst &I = b->hinst[i];
        I.first_chunk = (int)ch.size();
        for (int64_t l = 0; l < I.N; l += chunk_len)
            ch.push_back(Chunk{i, (int)l, (int)std::min<int64_t>(I.N, l + chunk_len), 0});
        I.nchunks = (int)ch.size() - I.first_chunk;
    }
}

}  // namespace

extern "C" {

ch_status ch_destroy_batch(ch_batch *b) {
    if (!b) return CH_OK;
    if (b->ngroups) {
        for (int g = 0; g < 2; ++g) {
            ch_destroy_batch(b->grp[g]);
            if (b->grp_stream[g]) cudaStreamDestroy(b->grp_stream[g]);
        }
        for (int k = 0; k < 3; ++k)
            if (b->grp_ev[k]) cudaEventDestroy(b->grp_ev[k]);
        delete b;
        return CH_OK;
    }
    cudaStreamSynchronize(b->stream);
    void *bufs[] = {b->insts, b->chunks, b->bs, b->ctrls, b->H, b->u, b->ynew, b->F[0], b->F[1],
                    b->mu, b->q, b->partials, b->tickets, b->D, b->t, b->V, b->W[0], b->W[1],
                    b->dflags, b->dsteps, b->dlaunch, b->gpart, b->grams};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->hflags) cudaFreeHost(b->hflags);
    if (b->hbs) cudaFreeHost(b->hbs);
    if (b->hsteps) cudaFreeHost(b->hsteps);
    if (b->hran) cudaFreeHost(b->hran);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->ev[0]) cudaEventDestroy(b->ev[0]);
    if (b->ev[1]) cudaEventDestroy(b->ev[1]);
    if (b->run_exec) cudaGraphExecDestroy(b->run_exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->cap_stream2) cudaStreamDestroy(b->cap_stream2);
    delete b;
    return CH_OK;
}

// One batch object.  With ext_off the instances keep the given offsets in an array of
// ext_total values (a scheduling group of a larger batch, sharing the caller's layout);
// every per-point workspace then spans ext_total values.
static ch_status create_impl(int dim, int count, const int64_t *n, const double *eps, int precision,
                             int mmax_capacity, void *cuda_stream, const int64_t *ext_off,
                             int64_t ext_total, ch_batch **out) {
    if (!out || !n || !eps) return bfail(CH_EINVAL, "null argument");
    *out = nullptr;
    if (dim != 2 && dim != 3) return bfail(CH_EINVAL, "dim must be 2 or 3");
    if (count < 1 || count > 65536) return bfail(CH_EINVAL, "count must be in [1, 65536]");
    if (precision != CH_FP64 && precision != CH_MIXED) return bfail(CH_EINVAL, "unknown precision");
    if (mmax_capacity < 1 || mmax_capacity > 63)
        return bfail(CH_EINVAL, "batch mmax_capacity must be in [1, 63]");
    ch_batch *b = new ch_batch();
    b->dim = dim; b->count = count; b->precision = precision; b->mmax_cap = mmax_capacity;
    b->stream = (cudaStream_t)cuda_stream;
    b->launches = 0;
    b->mmax_graphs = -1;
    b->hinst.resize(count);
    b->offsets.resize(count + 1);
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        Inst &I = b->hinst[i];
        memset(&I, 0, sizeof I);
        I.dim = dim;
        int64_t N = 1;
        for (int a = 0; a < 3; ++a) {
            const int64_t na = a < dim ? n[3 * i + a] : 1;
            if (a < dim && (na < 4 || na > (1 << 20))) { delete b; return bfail(CH_EINVAL, "instance %d: n[%d] out of range [4, 2^20]", i, a); }
            I.n[a] = (int)na;
            N *= na;
        }
        if (!(eps[i] > 0.0) || !isfinite(eps[i])) { delete b; return bfail(CH_EINVAL, "instance %d: eps must be > 0", i); }
        I.N = N;
        I.off = ext_off ? ext_off[i] : off;
        I.eps2 = eps[i] * eps[i];
        I.sigma = 0.0;
        for (int a = 0; a < dim; ++a) {
            I.s[a] = (double)I.n[a] * (double)I.n[a];
            I.kap[a] = I.eps2 * I.s[a];
            I.sigma += 2.0 * I.s[a];
        }
        b->offsets[i] = I.off;
        off += (N + 63) / 64 * 64;
        if (off >= ((int64_t)1 << 31)) {   // checked per instance, before the sum can overflow
            delete b;
            return bfail(CH_EINVAL, "batch of more than 2^31 - 1 values (at instance %d)", i);
        }
    }
    if (ext_off) off = ext_total;
    b->offsets[count] = off;
    b->Ntot = off;
    if (off >= ((int64_t)1 << 31)) { delete b; return bfail(CH_EINVAL, "batch of %lld values exceeds 2^31 - 1", (long long)off); }
    auto cleanup = [&](const char *what, cudaError_t e) {
        ch_destroy_batch(b);
        return bfail(CH_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    };
    const size_t vb = (size_t)off * sizeof(double);
    const size_t eb = (size_t)off * (precision == CH_MIXED ? sizeof(float) : sizeof(double));
    // chunk table for the largest candidate count (most chunks)
    std::vector<Chunk> ch;
    build_chunks(b, kChunkCandidates[0], ch);
    const int max_chunks = (int)ch.size();
    struct { void **p; size_t bytes; } allocs[] = {
        {(void **)&b->insts, sizeof(Inst) * count}, {(void **)&b->chunks, sizeof(Chunk) * max_chunks},
        {(void **)&b->bs, sizeof(BState) * count}, {(void **)&b->ctrls, sizeof(Ctrl) * count},
        {(void **)&b->H, sizeof(double) * count * (size_t)(mmax_capacity + 1) * mmax_capacity},
        {(void **)&b->u, sizeof(double) * count * (size_t)(mmax_capacity + 1)},
        {(void **)&b->ynew, vb}, {(void **)&b->F[0], vb}, {(void **)&b->F[1], vb},
        {(void **)&b->mu, vb}, {(void **)&b->q, vb},
        {(void **)&b->partials, sizeof(double) * 4 * (size_t)max_chunks},
        {(void **)&b->tickets, sizeof(unsigned int) * count},
        {(void **)&b->D, eb}, {(void **)&b->t, std::max(eb, (size_t)off * sizeof(float))},
        {(void **)&b->V, eb * (size_t)mmax_capacity}, {(void **)&b->dflags, 2 * sizeof(int)},
        {(void **)&b->dsteps, sizeof(long long)}, {(void **)&b->dlaunch, sizeof(unsigned long long)},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) { cudaGetLastError(); return cleanup("cudaMalloc of batch workspace", e); }
    }
    if (precision == CH_MIXED) {
        for (int k = 0; k < 2; ++k) {
            cudaError_t e = cudaMalloc(&b->W[k], eb);
            if (e != cudaSuccess) { cudaGetLastError(); return cleanup("cudaMalloc of FP32 start vectors", e); }
        }
        if (mmax_capacity <= kBGsMaxJ) {    // the Gram-corrected iteration's workspace
            cudaError_t e = cudaMalloc((void **)&b->gpart, sizeof(float2) * kBGsSlots * (size_t)max_chunks);
            if (e == cudaSuccess)
                e = cudaMalloc((void **)&b->grams, sizeof(double) * count * (size_t)(mmax_capacity + 1) * (mmax_capacity + 1));
            if (e != cudaSuccess) { cudaGetLastError(); return cleanup("cudaMalloc of Gram workspace", e); }
        }
    }
    cudaError_t e = cudaMemset(b->tickets, 0, sizeof(unsigned int) * count);
    if (e == cudaSuccess) e = cudaMemset(b->ctrls, 0, sizeof(Ctrl) * count);
    if (e == cudaSuccess) e = cudaMemset(b->H, 0, sizeof(double) * count * (size_t)(mmax_capacity + 1) * mmax_capacity);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->hflags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->hbs, sizeof(BState) * count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->hsteps, sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->hran, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = (cudaError_t)ch::phi_setup();
    if (e != cudaSuccess) return cleanup("batch set-up", e);
    // ---- chunk-length autotuner: time the kernels of one Arnoldi iteration (j = 8: stencil
    // stages, orthogonalisation, per-instance reductions, without the chunk-independent
    // projected phi) over the whole batch for each candidate, on zero data
    {
        int one = 1;
        for (int i = 0; i < count; ++i)
            cudaMemcpy(&b->ctrls[i].active, &one, sizeof(int), cudaMemcpyHostToDevice);
        cudaMemset(b->D, 0, eb);
        cudaMemset(b->F[0], 0, vb);
        cudaMemset(b->V, 0, eb * (size_t)mmax_capacity);
        if (precision == CH_MIXED) cudaMemset(b->W[0], 0, eb);
        const int jt = std::min(8, mmax_capacity);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        int best = kChunkCandidates[0];
        for (int cand : kChunkCandidates) {
            build_chunks(b, cand, ch);
            b->nchunks = (int)ch.size();
            cudaMemcpy(b->chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice);
            cudaMemcpy(b->insts, b->hinst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice);
            cudaStream_t s = b->stream;
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) {
                    if (precision == CH_MIXED) queue_arnoldi_kernels_b<float>(b, s, 0, jt);
                    else queue_arnoldi_kernels_b<double>(b, s, 0, jt);
                }
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (ms < best_ms) { best_ms = ms; best = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int zero = 0;
        for (int i = 0; i < count; ++i)
            cudaMemcpy(&b->ctrls[i].active, &zero, sizeof(int), cudaMemcpyHostToDevice);
        b->launches = 0;
        // the timed iterations wrote Hessenberg and Gram entries of zero vectors: clear them
        cudaMemset(b->H, 0, sizeof(double) * count * (size_t)(mmax_capacity + 1) * mmax_capacity);
        if (b->grams)
            cudaMemset(b->grams, 0, sizeof(double) * count * (size_t)(mmax_capacity + 1) * (mmax_capacity + 1));
        b->chunk_len = best;
        build_chunks(b, best, ch);
        b->nchunks = (int)ch.size();
        cudaMemcpy(b->chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(b->insts, b->hinst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice);
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cleanup("chunk autotuning", e);
    }
    *out = b;
    return CH_OK;
}

// Scheduling groups.  The time of a batch is set by its stiffest instances: they take the
// most steps, each a Krylov run of iterations on a small part of the batch, bound by latency
// rather than bandwidth, while the rest of the batch is bandwidth-bound.  So a batch of at
// least kGroupMinCount instances whose instances within a factor 2 of the largest stiffness
// estimate are at most an eighth of it runs those as a second batch, concurrently with the
// rest on a stream of higher priority.  Stiffness estimate: the dominant terms of the closed
// form of ||A_hat||_1 at d = -1 (Sec. 3.2), eps^2 (sum_a 4 n_a^2)^2 + sum_a 4 n_a^2.
// Groups are taken only when CH_BATCH_GROUPS=2 at creation.  Measured on 256 2D instances
// they shorten an FP64 batch (whose bulk is the heavier part) but lengthen a mixed one,
// whose stiff instances take the most steps and slow down under contention.
constexpr int kGroupMinCount = 16;

ch_status ch_create_batch(int dim, int count, const int64_t *n, const double *eps, int precision,
                          int mmax_capacity, void *cuda_stream, ch_batch **out) {
    const char *env = getenv("CH_BATCH_GROUPS");
    bool valid = out && n && eps && (dim == 2 || dim == 3) && count >= kGroupMinCount && count <= 65536 &&
                 env && env[0] == '2';
    std::vector<double> lam;
    std::vector<int64_t> offs;
    if (valid) {
        lam.resize(count);
        offs.resize(count + 1);
        int64_t off = 0;
        for (int i = 0; i < count && valid; ++i) {
            int64_t N = 1;
            double s4 = 0.0;
            for (int a = 0; a < dim; ++a) {
                const int64_t na = n[3 * i + a];
                if (na < 4 || na > (1 << 20)) { valid = false; break; }
                N *= na;
                s4 += 4.0 * (double)na * (double)na;
            }
            if (!(eps[i] > 0.0) || !isfinite(eps[i])) valid = false;
            lam[i] = eps[i] * eps[i] * s4 * s4 + s4;
            offs[i] = off;
            off += (N + 63) / 64 * 64;
            if (off >= ((int64_t)1 << 31)) valid = false;
        }
        offs[count] = off;
    }
    std::vector<int> stiff, rest;
    if (valid) {
        const double lmax = *std::max_element(lam.begin(), lam.end());
        for (int i = 0; i < count; ++i) (lam[i] >= 0.5 * lmax ? stiff : rest).push_back(i);
        valid = !stiff.empty() && (int)stiff.size() * 8 <= count;
    }
    if (!valid)
        return create_impl(dim, count, n, eps, precision, mmax_capacity, cuda_stream, nullptr, 0, out);
    *out = nullptr;
    ch_batch *b = new ch_batch();
    b->dim = dim; b->count = count; b->precision = precision; b->mmax_cap = mmax_capacity;
    b->stream = (cudaStream_t)cuda_stream;
    b->offsets = offs;
    b->Ntot = offs[count];
    b->ngroups = 2;
    b->grp_idx[0] = stiff;
    b->grp_idx[1] = rest;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->grp_stream[0], cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->grp_stream[1], cudaStreamNonBlocking, least);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->grp_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ch_destroy_batch(b);
        return bfail(CH_ECUDA, "batch group streams: %s", cudaGetErrorString(e));
    }
    for (int g = 0; g < 2; ++g) {
        const std::vector<int> &idx = b->grp_idx[g];
        std::vector<int64_t> ng(3 * idx.size()), og(idx.size());
        std::vector<double> eg(idx.size());
        for (size_t k = 0; k < idx.size(); ++k) {
            for (int a = 0; a < 3; ++a) ng[3 * k + a] = n[3 * idx[k] + a];
            eg[k] = eps[idx[k]];
            og[k] = offs[idx[k]];
        }
        const ch_status st = create_impl(dim, (int)idx.size(), ng.data(), eg.data(), precision, mmax_capacity,
                                         b->grp_stream[g], og.data(), b->Ntot, &b->grp[g]);
        if (st != CH_OK) {
            ch_destroy_batch(b);
            return st;
        }
    }
    b->chunk_len = b->grp[1]->chunk_len;
    *out = b;
    return CH_OK;
}

int ch_batch_groups(const ch_batch *b) { return b ? (b->ngroups ? b->ngroups : 1) : 0; }

ch_status ch_batch_layout(const ch_batch *b, int64_t *offsets, int *chunk_len) {
    if (!b) return bfail(CH_EINVAL, "null batch");
    if (offsets)
        for (int i = 0; i <= b->count; ++i) offsets[i] = b->offsets[i];
    if (chunk_len) *chunk_len = b->chunk_len;
    return CH_OK;
}

ch_status ch_integrate_batch(ch_batch *b, const ch_params *prm, double *y, ch_stats *stats) {
    if (!b || !prm || !y) return bfail(CH_EINVAL, "null argument");
    if (prm->scheme != CH_EE2 || !prm->adaptive)
        return bfail(CH_EINVAL, "the batch integrator runs adaptive EE2 (Fig. 4)");
    if (prm->eyre) return bfail(CH_EINVAL, "the batch integrator has no Eyre splitting");
    if (!(prm->T > 0.0) || !(prm->tau0 > 0.0) || !(prm->tol > 0.0) || !isfinite(prm->T) ||
        !isfinite(prm->tau0))
        return bfail(CH_EINVAL, "T and tau0 must be finite and > 0, tol > 0");
    if (prm->mmax < 1 || prm->mmax > b->mmax_cap) return bfail(CH_EINVAL, "mmax outside [1, capacity]");
    if (prm->max_steps < 1) return bfail(CH_EINVAL, "max_steps must be >= 1");
    ch::NvtxRange range("ch_integrate_batch EE2");
    const char *env = getenv("CH_BATCH_HOST_LOOP");
    const bool host_loop = env && env[0] == '1';
    if (b->ngroups) {
        // both groups start after the caller's earlier work on its stream, run concurrently,
        // and the caller's stream waits for both
        BCUDA(cudaEventRecord(b->grp_ev[2], b->stream));
        for (int g = 0; g < 2; ++g) BCUDA(cudaStreamWaitEvent(b->grp_stream[g], b->grp_ev[2], 0));
        std::vector<ch_stats> gst[2];
        ch_status rc[2] = {CH_OK, CH_OK};
        bool queued[2] = {false, false};
        for (int g = 0; g < 2; ++g) {
            gst[g].resize(b->grp[g]->count);
            if (host_loop) continue;
            rc[g] = b->precision == CH_MIXED ? launch_b_dev<float>(b->grp[g], prm, y)
                                             : launch_b_dev<double>(b->grp[g], prm, y);
            queued[g] = rc[g] == CH_OK;
        }
        for (int g = 0; g < 2; ++g) {
            if (queued[g]) rc[g] = finish_b_dev(b->grp[g], gst[g].data());
            else if (host_loop || (rc[g] == CH_ECUDA && !b->grp[g]->run_exec))
                rc[g] = b->precision == CH_MIXED ? integrate_b<float>(b->grp[g], prm, y, gst[g].data())
                                                 : integrate_b<double>(b->grp[g], prm, y, gst[g].data());
        }
        for (int g = 0; g < 2; ++g) {
            BCUDA(cudaEventRecord(b->grp_ev[g], b->grp_stream[g]));
            BCUDA(cudaStreamWaitEvent(b->stream, b->grp_ev[g], 0));
            if (stats)
                for (size_t k = 0; k < b->grp_idx[g].size(); ++k) stats[b->grp_idx[g][k]] = gst[g][k];
        }
        return rc[0] != CH_OK ? rc[0] : rc[1];
    }
    // The run is one graph launch (device-driven steps and Krylov iterations); CH_BATCH_HOST_LOOP=1
    // selects the host-driven loop (one graph per Arnoldi iteration, the host reading a
    // device flag after each), which is also taken if the run graph cannot be built.
    if (!host_loop) {
        const ch_status st = b->precision == CH_MIXED ? integrate_b_dev<float>(b, prm, y, stats)
                                                      : integrate_b_dev<double>(b, prm, y, stats);
        if (st != CH_ECUDA || b->run_exec) return st;
    }
    return b->precision == CH_MIXED ? integrate_b<float>(b, prm, y, stats)
                                    : integrate_b<double>(b, prm, y, stats);
}

int64_t ch_batch_kernel_launches(const ch_batch *b) {
    if (!b) return 0;
    return b->ngroups ? b->grp[0]->launches + b->grp[1]->launches : b->launches;
}

}  // extern "C"
