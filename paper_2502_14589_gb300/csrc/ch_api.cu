// ch_api.cu -- C ABI (include/ch.h) and host orchestration of the Cahn-Hilliard hot path.
//
// The host queues kernels on the grid's stream and reads back a few scalars once per time
// step (step size taken, error estimate, lambda_max of the next LIM step).  Inside a Krylov
// run the host queues Arnoldi iteration j+1 before it waits for the result of iteration j
// (the device `active` flag, copied to pinned memory), so the GPU never idles on the host;
// kernels of an iteration queued after convergence return at once.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "ch_internal.cuh"

using ch::Ctrl;
using ch::Geom;
using ch::Launch;

static thread_local char g_last_error[512] = "";

static ch_status fail(ch_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return st;
}

namespace ch {
// error message shared by every entry point of the library (ch_last_error)
void set_error(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }
}

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(CH_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                \
    } while (0)

#define CH_TRY(expr)                        \
    do {                                    \
        ch_status s_ = (expr);              \
        if (s_ != CH_OK) return s_;         \
    } while (0)

struct StepRecord {
    double tau, est;
    int jexit, restarts, shrunk, p;
};

// One captured Arnoldi iteration (Fig. 2, a fixed j with its residual test) and what it launches.
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    int64_t counts[CH_K_COUNT] = {0};
};

struct ch_grid {
    Geom g;
    int precision;
    int mmax_cap;
    cudaStream_t stream;
    Launch L;
    int64_t launches;
    ch::Timing timing;
    cudaStream_t cap_stream;      // private non-blocking stream used only to capture graphs
    std::map<std::tuple<int, const void *, int, int, int>, IterGraph> graphs;
    int use_graphs;
    int fused_arnoldi;            // 1: one cooperative launch per Arnoldi iteration
    int g64;                      // FP64 grids: Gram-corrected iteration (j <= 31) instead of the
                                  // sequential passes (grids of at most kG64MaxPoints points)
    int arn_blocks;               // its grid
    double *mfb[3];               // variable-mobility grids: face mobilities (FP64)
    float *mffb[3];               // and their FP32 copies (mixed grids)
    int var_mobility;             // 1: created with room for a variable mobility
    float2 *gpart;                // reduction scratch of the Gram-corrected iterations (8-byte slots)
    double *gram;                 // Gram matrix of the Krylov basis (Gram-corrected iterations)
    // device workspace
    double *D, *G, *t, *q;        // per-step coefficients and stage scratch
    double *F[2];                 // rhs buffers; F[cur] is basis column 0 of a Krylov run
    double *V;                    // basis columns 1..mmax_cap, stride ldv
    int64_t ldv;
    double *y[3];                 // state scratch (ping-pong)
    float *Vf, *Wf[2], *Df, *tf;  // mixed precision: FP32 basis (slot 0 = Wf[cur]), D, stage
    double *H;                    // (mmax_cap + 1) x mmax_cap, row-major
    double *u;                    // mmax_cap
    double *ub;                   // kPhiBlock x (mmax_cap + 1): u of each j of a phi block
    double *phi_scratch;
    double *partials;
    Ctrl *ctrl;
    // pinned host mirrors
    Ctrl *hctrl;
    int *hflag;
    cudaEvent_t ev[2];
    // integration state: (t, tau) reached by the last ch_integrate, and an optional
    // resume point set by ch_set_state for the next one
    double t_last, tau_last;
    double t_resume, tau_resume;
    int resume;
    std::vector<StepRecord> rec;
    int64_t rec_cap;
};

// ---------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------
static ch_status sync_ctrl(ch_grid *g) {
    CUDA_TRY(cudaMemcpyAsync(g->hctrl, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->hctrl->status != 0) {
        const int st = g->hctrl->status;
        int zero = 0;
        CUDA_TRY(cudaMemcpyAsync(&g->ctrl->status, &zero, sizeof(int), cudaMemcpyHostToDevice, g->stream));
        if (st == CH_ETIMEOUT)   // a grid barrier gave up: its counters are no longer in step
            CUDA_TRY(cudaMemsetAsync(&g->ctrl->bar, 0, sizeof g->ctrl->bar, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        return fail((ch_status)st, st == CH_ENONFINITE ? "non-finite value in the solution or a reduction"
                                   : st == CH_ETIMEOUT ? "a grid barrier of the Arnoldi iteration timed out"
                                                       : "Krylov run found no admissible step size");
    }
    return CH_OK;
}

static ch_status check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CH_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return CH_OK;
}

// Grid geometry of the periodic unit square / cube, h_a = 1/n_a (arguments checked by the
// caller): s_a = 1/h_a^2, kap_a = eps^2 s_a, sigma = 2 sum_a s_a.
static void fill_geom(Geom &G, int dim, const int64_t n[3], double eps) {
    memset(&G, 0, sizeof G);
    G.dim = dim;
    int64_t N = 1;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = a < dim ? (int)n[a] : 1;
        N *= G.n[a];
    }
    G.N = N;
    G.st[0] = 1; G.st[1] = G.n[0]; G.st[2] = (int64_t)G.n[0] * G.n[1];
    G.eps2 = eps * eps;
    G.sigma = 0.0;
    for (int a = 0; a < dim; ++a) {
        G.s[a] = (double)n[a] * (double)n[a];
        G.kap[a] = G.eps2 * G.s[a];
        G.sigma += 2.0 * G.s[a];
    }
}

// The spectral bound of Fig. 1 in closed form: column j of A_hat has the entries
//   centre  d sigma + eps^2 (sigma^2 + 2 sum_a s_a^2),   +-e_a  -s_a (d + 2 eps^2 sigma),
//   +-2e_a  eps^2 s_a^2,   +-e_a +-e_b  2 eps^2 s_a s_b   (distinct when every n_a >= 4),
// so its absolute sum g(d) is convex in d and ||A_hat||_1 = max(g(d_min), g(d_max)).
static double col_abs_sum(const Geom &G, double d) {
    const double e2 = G.eps2, sg = G.sigma;
    double sq = 0.0;
    for (int a = 0; a < G.dim; ++a) sq += G.s[a] * G.s[a];
    double r = fabs(d * sg + e2 * (sg * sg + 2.0 * sq));
    for (int a = 0; a < G.dim; ++a) r += 2.0 * G.s[a] * fabs(d + 2.0 * e2 * sg);
    for (int a = 0; a < G.dim; ++a) r += 2.0 * e2 * G.s[a] * G.s[a];
    for (int a = 0; a < G.dim; ++a)
        for (int b = a + 1; b < G.dim; ++b) r += 8.0 * e2 * G.s[a] * G.s[b];
    return r;
}

static double lambda_from_minmax(const Geom &G, double y2min, double y2max, int eyre) {
    const double shift = eyre ? 1.0 : 0.0;
    const double dmin = 3.0 * y2min - 1.0 + shift, dmax = 3.0 * y2max - 1.0 + shift;
    return std::max(col_abs_sum(G, dmin), col_abs_sum(G, dmax));
}

// Fig. 1's spectral bound of A_hat(y), queued on the grid's stream: the closed form above
// from the extremes of y^2 on periodic constant-mobility grids, else the maximum of the
// explicit column sums (Neumann boundaries change the boundary columns, a variable mobility
// every column).  lambda_read gives the value once the control block is on the host.
static bool closed_form_bound(const Geom &G) { return G.bc == 0 && G.mf[0] == nullptr; }

static void lambda_queue(ch_grid *g, const double *y, int eyre) {
    if (closed_form_bound(g->g)) ch::launch_prep(g->L, g->g, y, eyre, g->D, nullptr, 1);
    else ch::launch_colmax(g->L, g->g, y, eyre);
}

static double lambda_read(const ch_grid *g, int eyre) {
    if (closed_form_bound(g->g)) return lambda_from_minmax(g->g, g->hctrl->red[4], g->hctrl->red[5], eyre);
    return g->hctrl->red[4];
}

// Eq. (p); -1 when tau * lambda_max is not finite or p would exceed 10^6 (checked on the
// double, before the conversion to int)
static int cheb_order(double tau, double lmax) {
    const double pi = 3.14159265358979323846;
    const double p = ceil((pi / 4.0) / (pi / 2.0 - atan(sqrt(tau * lmax))));
    return (p >= 1.0 && p <= 1e6) ? (int)p : -1;
}

// f = rhs(y) into out; mode bits of k_rhs2 (1: ||f||^2, 2: ||g_hat||^2, 4: est sums,
// 8: half_tau taken from ctrl->tau).
static void rhs(ch_grid *g, const double *y, double *out, int eyre, int mode,
                const double *y0 = nullptr, const double *f0 = nullptr, double half_tau = 0.0) {
    ch::launch_rhs1(g->L, g->g, y, eyre, g->t, (mode & 2) ? g->q : nullptr);
    ch::launch_rhs2(g->L, g->g, g->t, (mode & 2) ? g->q : nullptr, out, y0, f0, y, half_tau, mode);
}

// One Krylov run of Fig. 2.  Basis column W_1 is in slot0 and red[0] = ||W_1||^2 (and
// red[1] = ||g_hat||^2 when use_ghat).  Dm must hold the linearisation coefficients in the
// basis precision VT.  The result y0 + V_j (beta u) is written to ynext (FP64); the run's
// scalars are left in ctrl (not synchronised).
// Krylov dimensions evaluated together by one projected-phi launch (Fig. 2, projected phi and residual test for
// j0..j0+7 from the same H, one cluster each).  Iterations past the j at exit are
// speculative work: their A_hat products are not counted as matvecs and their basis
// columns are never combined.  Eight per launch halves the phi launches of a run to m_max
// = 30 against four, for at most four more speculative iterations when a run stops early.
constexpr int kPhiBlock = 8;
constexpr int64_t kG64MaxPoints = (int64_t)1 << 19;

// Krylov dimensions per projected-phi launch for this grid.  Speculative iterations cost
// an Arnoldi iteration each (about 1 us per 1e4 points: 3-4 ms at 512^3), a phi launch tens
// of microseconds whatever the grid, so large grids decide after every iteration and small
// ones (launch-latency bound) batch eight.
constexpr int64_t kPhiEveryIterPoints = (int64_t)1 << 22;
static int phi_block(const ch_grid *g) { return g->g.N >= kPhiEveryIterPoints ? 1 : kPhiBlock; }

// Kernels of Arnoldi iterations j0..j1 (Fig. 2), the projected phi and residual
// tests of those dimensions, and the copy of the device `active` flag to pinned memory.
template <typename VT>
static void queue_block(ch_grid *g, const Launch &L, VT *slot0, VT *V, const VT *Dm, VT *t,
                        int j0, int j1, int mmax, cudaStream_t stream) {
    const int ldh = g->mmax_cap;
    auto W = [&](int c) -> VT * { return c == 1 ? slot0 : V + (int64_t)(c - 2) * g->ldv; };
    for (int j = j0; j <= j1; ++j) {
        if (g->fused_arnoldi) {
            if constexpr (sizeof(VT) == 4) {
                if (j <= ch::kGsMaxJ) {
                    ch::launch_arnoldi_gmgs(L, g->arn_blocks, g->g, slot0, V, g->ldv, Dm, t, g->H, ldh, j,
                                            g->gpart, g->gram, g->mmax_cap + 1);
                    if (mmax > 63) ch::launch_phi(L, g->H, ldh, j, mmax, g->u, g->phi_scratch);
                    continue;
                }
            }
            if constexpr (sizeof(VT) == 8) {
                if (g->g64 && j <= ch::kGsMaxJ) {
                    ch::launch_arnoldi_g64(L, g->arn_blocks, g->g, slot0, V, g->ldv, Dm, t, g->H, ldh, j,
                                           (double *)g->gpart, g->gram, g->mmax_cap + 1);
                    if (mmax > 63) ch::launch_phi(L, g->H, ldh, j, mmax, g->u, g->phi_scratch);
                    continue;
                }
            }
            ch::launch_arnoldi<VT>(L, g->arn_blocks, g->g, slot0, V, g->ldv, Dm, t, g->H, ldh, j);
            if (mmax > 63) ch::launch_phi(L, g->H, ldh, j, mmax, g->u, g->phi_scratch);
            continue;
        }
        VT *Wj = W(j), *Wn = W(j + 1);
        ch::launch_tstage<VT>(L, g->g, Wj, Dm, t, 1);
        ch::launch_wstage<VT>(L, g->g, t, Wn, slot0, &g->H[0 * ldh + (j - 1)], j - 1, 1);
        for (int k = 1; k <= j; ++k) {
            const int last = (k == j);
            ch::launch_mgs<VT>(L, g->g.N, Wn, W(k), last ? nullptr : W(k + 1),
                               &g->H[(k - 1) * ldh + (j - 1)], last ? nullptr : &g->H[k * ldh + (j - 1)],
                               k, last, ldh);
        }
        if (mmax > 63) ch::launch_phi(L, g->H, ldh, j, mmax, g->u, g->phi_scratch);
    }
    if (mmax <= 63) ch::launch_phi_block(L, g->H, ldh, j0, j1, mmax, g->u, g->ub, g->mmax_cap + 1);
    cudaMemcpyAsync(&g->hflag[j1 & 1], &g->ctrl->active, sizeof(int), cudaMemcpyDeviceToHost, stream);
}

// The block as a CUDA graph, captured on the private stream the first time this
// (precision, start column, j0, j1, m_max) occurs and replayed afterwards.
template <typename VT>
static ch_status block_graph(ch_grid *g, VT *slot0, VT *V, const VT *Dm, VT *t, int j0, int j1,
                             int mmax, IterGraph **out) {
    auto key = std::make_tuple((int)sizeof(VT), (const void *)slot0, j0, j1, mmax);
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) { *out = &it->second; return CH_OK; }
    IterGraph ig;
    ch::Timing counter;                       // counts only (cls = -1), no events
    Launch Lc = g->L;
    Lc.stream = g->cap_stream;
    Lc.launches = &ig.launches;
    Lc.timing = &counter;
    cudaGraph_t graph;
    CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    queue_block<VT>(g, Lc, slot0, V, Dm, t, j0, j1, mmax, g->cap_stream);
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (e != cudaSuccess) return fail(CH_ECUDA, "graph capture of iterations %d-%d: %s", j0, j1, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ig.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(CH_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
    for (int k = 0; k < CH_K_COUNT; ++k) ig.counts[k] = counter.counts[k];
    *out = &(g->graphs[key] = ig);
    return CH_OK;
}

// One Krylov run of Fig. 2.  Basis column W_1 is in slot0 and red[0] = ||W_1||^2 (and
// red[1] = ||g_hat||^2 when use_ghat).  Dm must hold the linearisation coefficients in the
// basis precision VT.  The run's scalars are left in ctrl; the caller queues the combine.
// Block b+1 is queued before block b's flag is read, so the GPU never waits on the host.
template <typename VT>
static ch_status krylov_run_t(ch_grid *g, const double *y0, VT *slot0, VT *V, const VT *Dm,
                              VT *t, double tau0, double tol_phi_fixed, double tol, int use_ghat,
                              int mmax, double *ynext) {
    (void)y0; (void)ynext;
    const Launch &L = g->L;
    ch::launch_krylov_arm(L, tau0, tol_phi_fixed, tol, use_ghat);
    const bool graphs = g->use_graphs && g->timing.cls < 0;
    const int B = mmax <= 63 ? phi_block(g) : 1;
    int prev_j1 = 0;
    for (int j0 = 1; j0 <= mmax; j0 += B) {
        const int j1 = std::min(j0 + B - 1, mmax);
        IterGraph *ig = nullptr;
        if (graphs && block_graph<VT>(g, slot0, V, Dm, t, j0, j1, mmax, &ig) != CH_OK) {
            cudaGetLastError();               // capture not possible here: launch directly
            g->use_graphs = 0;
            ig = nullptr;
        }
        if (ig) {
            CUDA_TRY(cudaGraphLaunch(ig->exec, g->stream));
            g->launches += ig->launches;
            for (int k = 0; k < CH_K_COUNT; ++k) g->timing.counts[k] += ig->counts[k];
        } else {
            queue_block<VT>(g, L, slot0, V, Dm, t, j0, j1, mmax, g->stream);
        }
        CH_TRY(check_launch());
        CUDA_TRY(cudaEventRecord(g->ev[j1 & 1], g->stream));
        if (prev_j1 > 0) {
            CUDA_TRY(cudaEventSynchronize(g->ev[prev_j1 & 1]));
            if (g->hflag[prev_j1 & 1] == 0) break;
        }
        prev_j1 = j1;
    }
    return CH_OK;
}

// Krylov run on the grid's basis in its precision: slot `s` (0/1) holds W_1 in FP64 (F[s]);
// mixed grids first round it into the FP32 basis.  Ends with the combine into ynext.
static ch_status krylov_run(ch_grid *g, const double *y0, int s, double tau0,
                            double tol_phi_fixed, double tol, int use_ghat, int mmax,
                            double *ynext) {
    ch::NvtxRange range("Krylov run (Fig. 2)");
    if (g->precision == CH_FP64) {
        CH_TRY(krylov_run_t<double>(g, y0, g->F[s], g->V, g->D, g->t, tau0, tol_phi_fixed, tol,
                                    use_ghat, mmax, ynext));
        ch::launch_combine(g->L, g->g.N, y0, g->F[s], g->V, g->ldv, ynext);
    } else {
        ch::launch_to32(g->L, g->g.N, g->F[s], g->Wf[s]);
        CH_TRY(krylov_run_t<float>(g, y0, g->Wf[s], g->Vf, g->Df, g->tf, tau0, tol_phi_fixed, tol,
                                   use_ghat, mmax, ynext));
        ch::launch_combine32(g->L, g->g.N, y0, g->Wf[s], g->Vf, g->ldv, (float *)g->t, ynext);
    }
    return check_launch();
}

// Linearisation coefficients of A_hat_n at yn (and G for residuals / LIM) in FP64; mixed
// grids also keep J = D - eps^2 sigma in FP32 for the Krylov matvecs.
static void prep(ch_grid *g, const double *yn, int eyre, int want_G, int want_minmax) {
    ch::launch_prep(g->L, g->g, yn, eyre, g->D, want_G ? g->G : nullptr, want_minmax);
    // FP32 stages take J (+1 Eyre) = D - eps^2 sigma (the difference form of the stages)
    if (g->precision == CH_MIXED) ch::launch_to32(g->L, g->g.N, g->D, g->Df, -g->g.eps2 * g->g.sigma);
}

static void add_record(ch_grid *g, const StepRecord &r) {
    if ((int64_t)g->rec.size() < g->rec_cap) g->rec.push_back(r);
}

// ---------------------------------------------------------------------------------------
// EE2 step (Sec. 4).  On entry F[cur] = f(y_n) with red[0] = ||f||^2 (+ red[1]).
// adaptive: nonlinear RT step choice; else linear RT restarting over tau.
// With want_est, f(y_next) goes to F[1-cur] with the est sums of Eq. (LIMest).
// ---------------------------------------------------------------------------------------
struct EEOut {
    double tau, est;
    int jexit, restarts, shrunk, phi_evals;
    int64_t matvecs;
};

static ch_status ee_step_impl(ch_grid *g, const double *yn, int cur, double tau,
                              double tol_phi_fixed, double tol, int mmax, int linear_restart,
                              int eyre, double *ynext, int want_est, EEOut *out) {
    const Launch &L = g->L;
    const int use_ghat = !(tol_phi_fixed > 0.0);
    memset(out, 0, sizeof *out);
    prep(g, yn, eyre, linear_restart, 0);
    if (!linear_restart) {
        CH_TRY(krylov_run(g, yn, cur, tau, tol_phi_fixed, tol, use_ghat, mmax, ynext));
        if (want_est)   // Eq. (LIMest) for the step actually taken (ctrl->tau), f(y_{n+1}) -> F[1-cur]
            rhs(g, ynext, g->F[1 - cur], eyre, 1 | (use_ghat ? 2 : 0) | 4 | 8, yn, g->F[cur]);
        CH_TRY(check_launch());
        CH_TRY(sync_ctrl(g));
        out->tau = g->hctrl->tau;
        out->jexit = g->hctrl->jexit;
        out->shrunk = g->hctrl->shrunk;
        out->phi_evals = g->hctrl->phi_evals;
        out->matvecs = 1 + g->hctrl->jexit;
    } else {
        // Linear residual-time restarting over the whole step: A_hat_n, g_hat^n stay at y_n;
        // tol_phi is fixed for the step by the first run (Eq. tol_phi uses beta at y_n).
        double remaining = tau, tphi = tol_phi_fixed;
        const double *ycur = yn;
        int slot = cur;
        double *dst = ynext;
        int restarts = 0;
        for (;;) {
            CH_TRY(krylov_run(g, ycur, slot, remaining, tphi, tol, use_ghat && restarts == 0, mmax, dst));
            CH_TRY(sync_ctrl(g));
            tphi = g->hctrl->tol_phi;
            out->jexit = g->hctrl->jexit;
            out->phi_evals += g->hctrl->phi_evals;
            out->matvecs += 1 + g->hctrl->jexit;
            const double taken = g->hctrl->tau;
            if (taken >= remaining) break;
            remaining -= taken;
            ycur = dst;
            dst = (dst == ynext) ? g->y[0] : (dst == g->y[0] ? g->y[1] : g->y[0]);
            if (++restarts > 100000) return fail(CH_ENOTCONV, "linear restart cap reached");
            // restart vector W_1 = g_hat^n - A_hat_n y_cur (the start vector of Fig. 2)
            slot = 1 - cur;
            ch::launch_resid1(L, g->g, ycur, g->D, g->G, g->t);
            ch::launch_resid2(L, g->g, g->t, g->F[slot]);
        }
        if (dst != ynext)
            CUDA_TRY(cudaMemcpyAsync(ynext, dst, g->g.N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     g->stream));
        out->restarts = restarts;
        out->tau = tau;
        if (want_est) {
            rhs(g, ynext, g->F[1 - cur], eyre, 1 | (use_ghat ? 2 : 0) | 4, yn, g->F[cur], 0.5 * tau);
            CH_TRY(check_launch());
            CH_TRY(sync_ctrl(g));
        }
    }
    if (want_est) out->est = sqrt(g->hctrl->red[2]) / sqrt(g->hctrl->red[3]);
    return CH_OK;
}

// ---------------------------------------------------------------------------------------
// Order of the Chebyshev parameters (Fig. 1 fixes only beta_1 first).  The factors
// of the LIM iterations commute, so the order changes only the growth of rounding errors;
// this is the recursive mirror-pair order of Lebedev and Finogenov (1971), extended to odd
// p by placing the middle index right after the first pair.  1-based indices, cached per p.
// ---------------------------------------------------------------------------------------
static void mirror_pair_order(int p, std::vector<int> &out) {
    out.clear();
    if (p == 1) { out.push_back(1); return; }
    std::vector<int> half;
    mirror_pair_order(p / 2, half);
    for (size_t i = 0; i < half.size(); ++i) {
        out.push_back(half[i]);
        out.push_back(p + 1 - half[i]);
        if (i == 0 && (p % 2 == 1)) out.push_back(p / 2 + 1);
    }
}

static const std::vector<int> &cheb_param_order(int p) {
    static std::mutex mu;
    static std::map<int, std::vector<int>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(p);
    if (it != cache.end()) return it->second;
    std::vector<int> o;
    mirror_pair_order(p, o);
    return cache.emplace(p, std::move(o)).first->second;
}

// ---------------------------------------------------------------------------------------
// LIM step (Sec. 3.1, Fig. 1) with lambda_max given.
// ---------------------------------------------------------------------------------------
// Fig. 1 on the host: p by Eq. (p) and a_m = lmax (z_1 - beta_m)/(1 + z_1)
// for m = 1..p with beta_m = cos(pi (2m - 1) / (2p)) and z_1 = beta_1.
static ch_status lim_schedule(double tau, double lmax, int *p_out, std::vector<double> &a) {
    const double pi = 3.14159265358979323846;
    const int p = cheb_order(tau, lmax);                                   // Eq. (p)
    if (p < 1)
        return fail(isfinite(lmax) ? CH_EINVAL : CH_ENONFINITE,
                    "Chebyshev order for tau * lambda_max = %g out of range", tau * lmax);
    std::vector<double> beta(p);
    a.assign(p, 0.0);
    for (int i = 1; i <= p; ++i) beta[i - 1] = cos(pi * (2.0 * i - 1.0) / (2.0 * p));   // 2
    const double z1 = beta[0];                                             // z_1
    for (int m = 1; m <= p; ++m) a[m - 1] = lmax / (1.0 + z1) * (z1 - beta[m - 1]);     // 5
    *p_out = p;
    return CH_OK;
}

// Mixed-precision grids run the LIM iterations on the FP32 increment d = y_prev - y^n (the
// increment form of launch_lim32) while the rounding growth of the iterates, at most
// 3 (tau lambda_max)^2 with the mirror-pair order, times the FP32 unit roundoff stays below
// kLim32Growth; a step beyond that (stiff tau) runs the FP64 iterations.
constexpr double kLim32Growth = 1e-5;
static bool lim_in_fp32(const ch_grid *g, double tau, double lmax) {
    const double x = tau * lmax;
    return g->precision == CH_MIXED && 3.0 * x * x * 0x1p-24 <= kLim32Growth;
}

// fn: f(y^n) when the caller has it (the adaptive driver keeps it from the estimate), else
// nullptr; *rhs_used is set when the step evaluated f itself.
static ch_status lim_step_impl(ch_grid *g, const double *yn, double tau, double lmax, int eyre,
                               double *ynext, int *p_out, const double *fn = nullptr,
                               int *rhs_used = nullptr) {
    const Launch &L = g->L;
    ch::NvtxRange range("LIM iterations (Fig. 1)");
    int p = 0;
    std::vector<double> a;
    CH_TRY(lim_schedule(tau, lmax, &p, a));
    const std::vector<int> &order = cheb_param_order(p);                   // ordered set
    const int total = 2 * p - 1;
    if (rhs_used) *rhs_used = 0;
    if (lim_in_fp32(g, tau, lmax)) {
        if (!fn) {                             // f(y^n) = g_hat - A_hat y^n, FP64
            rhs(g, yn, g->G, eyre, 0);
            fn = g->G;
            if (rhs_used) *rhs_used = 1;
        }
        ch::launch_prep(L, g->g, yn, eyre, g->D, nullptr, 0);
        ch::launch_to32(L, g->g.N, g->D, g->Df, -g->g.eps2 * g->g.sigma);   // J (+1 Eyre)
        const float *dprev = nullptr;
        int it = 0;
        for (int sweep = 0; sweep < 2; ++sweep) {                          // m = 1..p, 2..p
            for (int idx = (sweep == 0 ? 0 : 1); idx < p; ++idx) {
                float *dnext = g->Wf[it & 1];
                ++it;
                const double am = a[order[idx] - 1], alpha = 1.0 / (1.0 + tau * am);
                if (dprev) ch::launch_tstage<float>(L, g->g, dprev, g->Df, g->tf, 0);
                ch::launch_lim32(L, g->g, g->tf, fn, dprev, dnext, alpha * tau * am, alpha * tau);
                dprev = dnext;
            }
        }
        ch::launch_add_increment(L, g->g.N, yn, dprev, ynext);
        *p_out = p;
        return check_launch();
    }
    ch::launch_prep(L, g->g, yn, eyre, g->D, g->G, 0);
    const double *prev = yn;
    int it = 0;
    for (int sweep = 0; sweep < 2; ++sweep) {                              // m = 1..p, 2..p
        for (int idx = (sweep == 0 ? 0 : 1); idx < p; ++idx) {
            ++it;
            double *next = (it == total) ? ynext : g->y[it & 1];
            const double am = a[order[idx] - 1];
            ch::launch_resid1(L, g->g, prev, g->D, g->G, g->t);
            ch::launch_lim2(L, g->g, g->t, yn, prev, next, tau * am, tau, 1.0 / (1.0 + tau * am));
            prev = next;
        }
    }
    *p_out = p;
    return check_launch();
}

void ch::Timing::harvest() {
    if (used == 0) return;
    cudaEventSynchronize(ev[2 * used - 1]);
    for (size_t k = 0; k < used; ++k) {
        if (cls == CH_K_ARNOLDI && active && active[k] == 0) continue;    // returned at once
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) total_ms += ms;
        ++timed;
        flops += wflops[k];
        bytes += wbytes[k];
    }
    used = 0;
}

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

ch_status ch_timing_start(ch_grid *g, int kernel_class) {
    if (!g || kernel_class < -1 || kernel_class >= CH_K_COUNT) return fail(CH_EINVAL, "bad kernel class");
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->timing.harvest();
    if (kernel_class >= 0 && g->timing.ev.empty()) {
        const size_t slots = 4096;
        g->timing.ev.resize(2 * slots);
        for (auto &e : g->timing.ev) CUDA_TRY(cudaEventCreate(&e));
        g->timing.wflops.assign(slots, 0.0);
        g->timing.wbytes.assign(slots, 0.0);
        CUDA_TRY(cudaMallocHost((void **)&g->timing.active, slots * sizeof(int)));
    }
    g->timing.cls = kernel_class;
    g->timing.used = 0;
    g->timing.total_ms = 0.0;
    g->timing.timed = 0;
    g->timing.flops = g->timing.bytes = 0.0;
    for (auto &c : g->timing.counts) c = 0;
    return CH_OK;
}

ch_status ch_timing_work(ch_grid *g, double *flops, double *bytes) {
    if (!g) return fail(CH_EINVAL, "null grid");
    if (flops) *flops = g->timing.flops;
    if (bytes) *bytes = g->timing.bytes;
    return CH_OK;
}

ch_status ch_bench_kernel(ch_grid *g, int kernel_class, int reps, double *avg_us,
                          double *bytes_per_launch, double *flops_per_launch,
                          double *fp64_instr_per_launch) {
    if (!g || reps < 1 || reps > 100000) return fail(CH_EINVAL, "bad arguments");
    ch::NvtxRange range("ch_bench_kernel");      // lets a profiler select these launches
    if (kernel_class == CH_K_ARNOLDI && !g->fused_arnoldi)
        return fail(CH_EINVAL, "this grid runs Arnoldi iterations as separate kernels");
    const int d = g->g.dim;
    const double N = (double)g->g.N;
    const bool mixed = g->precision == CH_MIXED;
    const double vb = mixed ? 4.0 : 8.0;           // bytes of one Krylov-vector value
    double bytes = 0, flops = 0, instr = 0;
    Launch Lc = g->L;
    ch::Timing counter;
    int64_t cnt = 0;
    Lc.stream = g->cap_stream;
    Lc.launches = &cnt;
    Lc.timing = &counter;
    int one = 1;
    CUDA_TRY(cudaMemcpyAsync(&g->ctrl->active, &one, sizeof(int), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    cudaGraph_t graph;
    CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < reps; ++r) {
        switch (kernel_class) {
        case CH_K_TSTAGE:   // t = D x - sum kap (pairs): 1 mul + d (add + fma)
            if (mixed) ch::launch_tstage<float>(Lc, g->g, g->Wf[0], g->Df, g->tf, 0);
            else ch::launch_tstage<double>(Lc, g->g, g->F[0], g->D, g->t, 0);
            bytes = 3 * vb * N; flops = (1 + 3.0 * d) * N; instr = mixed ? 0 : (1 + 2.0 * d) * N;
            break;
        case CH_K_WSTAGE:   // w = c0 t - sum c (pairs), dot with v1: 1 mul + d (add + fma) + fma
            if (mixed) ch::launch_wstage<float>(Lc, g->g, g->tf, g->Vf, g->Wf[0], &g->H[0], 0, 0);
            else ch::launch_wstage<double>(Lc, g->g, g->t, g->V, g->F[0], &g->H[0], 0, 0);
            bytes = 3 * vb * N; flops = (3 + 3.0 * d) * N; instr = mixed ? 0 : (2 + 2.0 * d) * N;
            break;
        case CH_K_MGS:      // w -= c v_k, dot(w, v_{k+1}): 2 fma
            if (mixed) ch::launch_mgs<float>(Lc, g->g.N, g->Vf, g->Wf[0], g->Wf[1], &g->H[0], &g->H[1], 1, 0, 0);
            else ch::launch_mgs<double>(Lc, g->g.N, g->V, g->F[0], g->F[1], &g->H[0], &g->H[1], 1, 0, 0);
            bytes = 4 * vb * N; flops = 4.0 * N; instr = mixed ? 0 : 2.0 * N;
            break;
        case CH_K_RESID1:   // t = G - D x + sum kap (pairs): fma + d (add + fma)
            ch::launch_resid1(Lc, g->g, g->y[0], g->D, g->G, g->t);
            bytes = 32.0 * N; flops = (2 + 3.0 * d) * N; instr = (1 + 2.0 * d) * N;
            break;
        case CH_K_LIM2:     // r = c0 t - sum c (pairs); fma(ca, prev, fma(alpha, yn, r))
            ch::launch_lim2(Lc, g->g, g->t, g->y[2], g->y[0], g->y[1], 0.5, 1e-3, 0.9);
            bytes = 32.0 * N; flops = (5 + 3.0 * d) * N; instr = (3 + 2.0 * d) * N;
            break;
        case CH_K_RHS1:     // mu = (y^2 + c) y - sum kap (pairs): fma, mul, d (add + fma)
            ch::launch_rhs1(Lc, g->g, g->y[2], 0, g->t, nullptr);
            bytes = 16.0 * N; flops = (3 + 3.0 * d) * N; instr = (2 + 2.0 * d) * N;
            break;
        case CH_K_RHS2:     // f = -(sigma mu - sum s (pairs)), ||f||^2
            ch::launch_rhs2(Lc, g->g, g->t, nullptr, g->y[1], nullptr, nullptr, g->y[2], 0.0, 1);
            bytes = 16.0 * N; flops = (3 + 3.0 * d) * N; instr = (2 + 2.0 * d) * N;
            break;
        case CH_K_ARNOLDI: {  // one whole Arnoldi iteration with j = min(10, capacity) passes
            const int j = std::min(10, g->mmax_cap);
            if (mixed) ch::launch_arnoldi_gmgs(Lc, g->arn_blocks, g->g, g->Wf[0], g->Vf, g->ldv, g->Df, g->tf,
                                               g->H, g->mmax_cap, j, g->gpart, g->gram, g->mmax_cap + 1);
            else if (g->g64 && j <= ch::kGsMaxJ)
                ch::launch_arnoldi_g64(Lc, g->arn_blocks, g->g, g->F[0], g->V, g->ldv, g->D, g->t, g->H, g->mmax_cap, j,
                                       (double *)g->gpart, g->gram, g->mmax_cap + 1);
            else ch::launch_arnoldi<double>(Lc, g->arn_blocks, g->g, g->F[0], g->V, g->ldv, g->D, g->t, g->H, g->mmax_cap, j);
            bytes = mixed ? (6.0 + 2.0 * j) * vb * N : (5.0 + j) * vb * N;
            flops = mixed ? ((1 + 3.0 * d) + (1 + 3.0 * d) + 6.0 * j + 2.0) * N
                          : ((1 + 3.0 * d) + (3 + 3.0 * d) + 4.0 * j) * N;
            instr = mixed ? 0 : ((1 + 2.0 * d) + (2 + 2.0 * d) + 2.0 * j) * N;
            break;
        }
        default:
            cudaStreamEndCapture(g->cap_stream, &graph);
            return fail(CH_EINVAL, "kernel class %d cannot be benchmarked", kernel_class);
        }
    }
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (e != cudaSuccess) return fail(CH_ECUDA, "capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(CH_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaGraphLaunch(exec, g->stream));              // warm-up
    CUDA_TRY(cudaEventRecord(e0, g->stream));
    CUDA_TRY(cudaGraphLaunch(exec, g->stream));
    CUDA_TRY(cudaEventRecord(e1, g->stream));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    int zero = 0;
    CUDA_TRY(cudaMemcpyAsync(&g->ctrl->active, &zero, sizeof(int), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->launches += 2 * cnt;
    if (avg_us) *avg_us = 1e3 * ms / reps;
    if (bytes_per_launch) *bytes_per_launch = bytes;
    if (flops_per_launch) *flops_per_launch = flops;
    if (fp64_instr_per_launch) *fp64_instr_per_launch = instr;
    return CH_OK;
}

ch_status ch_timing_read(ch_grid *g, double *total_ms, int64_t *timed_launches, int64_t *counts) {
    if (!g) return fail(CH_EINVAL, "null grid");
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->timing.harvest();
    if (total_ms) *total_ms = g->timing.total_ms;
    if (timed_launches) *timed_launches = g->timing.timed;
    if (counts) for (int k = 0; k < CH_K_COUNT; ++k) counts[k] = g->timing.counts[k];
    return CH_OK;
}

const char *ch_last_error(void) { return g_last_error; }

int64_t ch_kernel_launches(const ch_grid *g) { return g ? g->launches : 0; }

ch_status ch_lim_schedule(double tau, double lambda_max, int capacity, int *p, int *order,
                          double *a) {
    if (!p) return fail(CH_EINVAL, "null argument");
    if (!(tau > 0.0) || !isfinite(tau) || !(lambda_max >= 0.0))
        return fail(CH_EINVAL, "tau must be finite and > 0, lambda_max >= 0");
    int pp = 0;
    std::vector<double> av;
    CH_TRY(lim_schedule(tau, lambda_max, &pp, av));
    *p = pp;
    if (capacity < pp) return capacity == 0 ? CH_OK : fail(CH_EINVAL, "capacity %d < p = %d", capacity, pp);
    const std::vector<int> &o = cheb_param_order(pp);
    for (int k = 0; k < pp; ++k) {
        if (order) order[k] = o[k];
        if (a) a[k] = av[k];
    }
    return CH_OK;
}

ch_status ch_lambda_max_bound(int dim, const int64_t n[3], double eps, int eyre, double y2min,
                              double y2max, double *lambda_max) {
    if (!n || !lambda_max) return fail(CH_EINVAL, "null argument");
    if (dim != 2 && dim != 3) return fail(CH_EINVAL, "dim must be 2 or 3");
    for (int a = 0; a < dim; ++a)
        if (n[a] < 4 || n[a] > (1 << 20)) return fail(CH_EINVAL, "n[%d] out of range [4, 2^20]", a);
    if (!(eps > 0.0) || !isfinite(eps)) return fail(CH_EINVAL, "eps must be finite and > 0");
    if (!(y2min >= 0.0) || !(y2max >= y2min)) return fail(CH_EINVAL, "need 0 <= y2min <= y2max");
    Geom G;
    fill_geom(G, dim, n, eps);
    *lambda_max = lambda_from_minmax(G, y2min, y2max, eyre);
    return CH_OK;
}

ch_status ch_create_grid(int dim, const int64_t n[3], double eps, int precision,
                         int mmax_capacity, void *cuda_stream, ch_grid **out) {
    return ch_create_grid_ex(dim, n, eps, precision, mmax_capacity, nullptr, cuda_stream, out);
}

ch_status ch_create_grid_ex(int dim, const int64_t n[3], double eps, int precision,
                            int mmax_capacity, const ch_grid_options *opts, void *cuda_stream,
                            ch_grid **out) {
    g_last_error[0] = 0;
    if (!out || !n) return fail(CH_EINVAL, "null argument");
    *out = nullptr;
    const int bc = opts ? opts->bc : CH_BC_PERIODIC;
    const int var_mob = opts ? opts->variable_mobility : 0;
    if (bc != CH_BC_PERIODIC && bc != CH_BC_NEUMANN) return fail(CH_EINVAL, "unknown boundary condition");
    if (var_mob != 0 && var_mob != 1) return fail(CH_EINVAL, "variable_mobility must be 0 or 1");
    if (dim != 2 && dim != 3) return fail(CH_EINVAL, "dim must be 2 or 3");
    int64_t N = 1;
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 4 || n[a] > (1 << 20)) return fail(CH_EINVAL, "n[%d] = %lld out of range [4, 2^20]", a, (long long)n[a]);
        N *= n[a];
    }
    if (N >= (int64_t)1 << 31) return fail(CH_EINVAL, "grid of %lld points exceeds 2^31 - 1", (long long)N);
    if (!(eps > 0.0) || !isfinite(eps)) return fail(CH_EINVAL, "eps must be finite and > 0");
    if (precision != CH_FP64 && precision != CH_MIXED) return fail(CH_EINVAL, "unknown precision");
    if (mmax_capacity < 1 || mmax_capacity > 128) return fail(CH_EINVAL, "mmax_capacity must be in [1, 128]");

    ch_grid *g = new ch_grid();
    fill_geom(g->g, dim, n, eps);
    g->g.bc = bc;
    g->var_mobility = var_mob;
    g->precision = precision;
    g->mmax_cap = mmax_capacity;
    g->stream = (cudaStream_t)cuda_stream;
    g->launches = 0;
    g->rec_cap = 0;
    g->resume = 0;
    g->t_last = g->tau_last = 0.0;
    g->cap_stream = nullptr;
    {
        const char *env = getenv("CH_NO_GRAPHS");
        g->use_graphs = !(env && env[0] == '1');
        env = getenv("CH_NO_FUSED_ARNOLDI");
        g->fused_arnoldi = !(env && env[0] == '1');
        // FP64 sequential passes are bound by their j + 2 grid synchronisations on small grids
        // (a pass of 2 FMAs per point takes less than a barrier's few us): measured, the Gram
        // form took a batch of 64^2..512^2 grids one by one from 153 s to 133 s, but made EE2 on
        // 1024^2 8 % slower (46.7 s against 43.0 s), so it serves grids up to 512K points.
        env = getenv("CH_ARNOLDI_MGS");
        g->g64 = precision == CH_FP64 && N <= kG64MaxPoints && !(env && env[0] == '1');
    }

    auto cleanup_fail = [&](ch_status st, const char *what, cudaError_t e) {
        ch_destroy_grid(g);
        return fail(st, "%s: %s", what, cudaGetErrorString(e));
    };
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cleanup_fail(CH_ECUDA, "device query", e);
    const int64_t want = (N + ch::kThreads - 1) / ch::kThreads;
    g->L.blocks = (int)std::min<int64_t>(want, (int64_t)sms * ch::kBlocksPerSM);
    g->arn_blocks = precision == CH_MIXED ? ch::arnoldi_blocks<float>(dim, N)
                                          : ch::arnoldi_blocks<double>(dim, N);
    if (g->arn_blocks < 1) g->fused_arnoldi = 0;
    g->L.stream = g->stream;
    g->L.launches = &g->launches;
    g->L.timing = &g->timing;

    const int64_t ld = (N + 31) / 32 * 32;     // 256-byte aligned columns
    g->ldv = ld;
    const size_t vb = (size_t)ld * sizeof(double);
    struct { double **p; size_t bytes; } allocs[] = {
        {&g->D, vb}, {&g->G, vb}, {&g->t, vb}, {&g->q, vb}, {&g->F[0], vb}, {&g->F[1], vb},
        {&g->y[0], vb}, {&g->y[1], vb}, {&g->y[2], vb},
        {&g->V, vb * (size_t)mmax_capacity},
        {&g->H, sizeof(double) * (size_t)(mmax_capacity + 1) * mmax_capacity},
        {&g->u, sizeof(double) * (size_t)(mmax_capacity + 1)},
        {&g->ub, sizeof(double) * (size_t)kPhiBlock * (mmax_capacity + 1)},
        {&g->phi_scratch, sizeof(double) * (size_t)(6 * (mmax_capacity + 1) * (mmax_capacity + 1) + 2 * (mmax_capacity + 1))},
        {&g->partials, sizeof(double) * (size_t)std::max(ch::kMaxRed * g->L.blocks, 2 * g->arn_blocks)},
    };
    for (auto &a : allocs) {
        if (precision == CH_MIXED && a.p == &g->V) continue;     // FP32 basis instead
        e = cudaMalloc((void **)a.p, a.bytes);
        if (e != cudaSuccess) { cudaGetLastError(); return cleanup_fail(CH_ENOMEM, "cudaMalloc of grid workspace", e); }
    }
    if (precision == CH_MIXED) {
        const size_t fb = (size_t)ld * sizeof(float);
        struct { float **p; size_t bytes; } fallocs[] = {
            {&g->Vf, fb * (size_t)mmax_capacity}, {&g->Wf[0], fb}, {&g->Wf[1], fb}, {&g->Df, fb}, {&g->tf, fb}};
        for (auto &a : fallocs) {
            e = cudaMalloc((void **)a.p, a.bytes);
            if (e != cudaSuccess) { cudaGetLastError(); return cleanup_fail(CH_ENOMEM, "cudaMalloc of FP32 basis", e); }
        }
    }
    if (precision == CH_MIXED || g->g64) {
        e = cudaMalloc((void **)&g->gpart, sizeof(float2) * 3 * (ch::kGsMaxJ + 1) * (size_t)std::max(g->arn_blocks, 1));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&g->gram, sizeof(double) * (size_t)(mmax_capacity + 1) * (mmax_capacity + 1));
        if (e != cudaSuccess) { cudaGetLastError(); return cleanup_fail(CH_ENOMEM, "cudaMalloc of Gram workspace", e); }
    }
    if (var_mob) {    // face mobilities per axis (FP64, and FP32 on mixed grids)
        for (int a = 0; a < dim; ++a) {
            e = cudaMalloc((void **)&g->mfb[a], vb);
            if (e == cudaSuccess && precision == CH_MIXED) e = cudaMalloc((void **)&g->mffb[a], (size_t)ld * sizeof(float));
            if (e != cudaSuccess) { cudaGetLastError(); return cleanup_fail(CH_ENOMEM, "cudaMalloc of face mobilities", e); }
        }
    }
    e = cudaMalloc((void **)&g->ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) { cudaGetLastError(); return cleanup_fail(CH_ENOMEM, "cudaMalloc of control block", e); }
    e = cudaMemset(g->ctrl, 0, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMemset(g->H, 0, sizeof(double) * (size_t)(mmax_capacity + 1) * mmax_capacity);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->hctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->hflag, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = (cudaError_t)ch::phi_setup();
    if (e == cudaSuccess) e = (cudaError_t)ch::arnoldi_setup();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cleanup_fail(CH_ECUDA, "grid set-up", e);
    g->L.partials = g->partials;
    g->L.ctrl = g->ctrl;
    *out = g;
    return CH_OK;
}

ch_status ch_destroy_grid(ch_grid *g) {
    if (!g) return CH_OK;
    cudaStreamSynchronize(g->stream);
    double *bufs[] = {g->D, g->G, g->t, g->q, g->F[0], g->F[1], g->y[0], g->y[1], g->y[2],
                      g->V, g->H, g->u, g->ub, g->phi_scratch, g->partials};
    for (double *b : bufs)
        if (b) cudaFree(b);
    float *fbufs[] = {g->Vf, g->Wf[0], g->Wf[1], g->Df, g->tf};
    for (float *b : fbufs)
        if (b) cudaFree(b);
    for (int a = 0; a < 3; ++a) {
        if (g->mfb[a]) cudaFree(g->mfb[a]);
        if (g->mffb[a]) cudaFree(g->mffb[a]);
    }
    if (g->gpart) cudaFree(g->gpart);
    if (g->gram) cudaFree(g->gram);
    if (g->ctrl) cudaFree(g->ctrl);
    if (g->hctrl) cudaFreeHost(g->hctrl);
    if (g->hflag) cudaFreeHost(g->hflag);
    if (g->ev[0]) cudaEventDestroy(g->ev[0]);
    if (g->ev[1]) cudaEventDestroy(g->ev[1]);
    for (auto &e : g->timing.ev) if (e) cudaEventDestroy(e);
    if (g->timing.active) cudaFreeHost(g->timing.active);
    for (auto &kv : g->graphs) if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
    return CH_OK;
}

ch_status ch_rhs(ch_grid *g, const double *y, double *f, int eyre, double *norm_f,
                 double *norm_ghat) {
    if (!g || !y || !f) return fail(CH_EINVAL, "null argument");
    const int mode = (norm_f ? 1 : 0) | (norm_ghat ? 2 : 0);
    rhs(g, y, f, eyre, mode);
    CH_TRY(check_launch());
    if (mode) {
        CH_TRY(sync_ctrl(g));
        if (norm_f) *norm_f = sqrt(g->hctrl->red[0]);
        if (norm_ghat) *norm_ghat = sqrt(g->hctrl->red[1]);
    }
    return CH_OK;
}

ch_status ch_jacvec(ch_grid *g, const double *y_lin, const double *v, double *w, int eyre) {
    if (!g || !y_lin || !v || !w) return fail(CH_EINVAL, "null argument");
    ch::launch_prep(g->L, g->g, y_lin, eyre, g->D, nullptr, 0);
    ch::launch_tstage<double>(g->L, g->g, v, g->D, g->t, 0);
    ch::launch_wstage<double>(g->L, g->g, g->t, w, nullptr, nullptr, 0, 0);
    return check_launch();
}

ch_status ch_set_mobility(ch_grid *g, const double *M) {
    if (!g) return fail(CH_EINVAL, "null grid");
    if (!g->var_mobility) return fail(CH_EINVAL, "grid created without variable_mobility");
    const bool was = g->g.mf[0] != nullptr;
    if (M) {
        double *const mf[3] = {g->mfb[0], g->mfb[1], g->mfb[2]};
        float *const mff[3] = {g->mffb[0], g->mffb[1], g->mffb[2]};
        ch::launch_face_mob(g->L, g->g, M, mf, mff);
        for (int a = 0; a < 3; ++a) { g->g.mf[a] = g->mfb[a]; g->g.mff[a] = g->mffb[a]; }
    } else {
        for (int a = 0; a < 3; ++a) { g->g.mf[a] = nullptr; g->g.mff[a] = nullptr; }
    }
    // captured Arnoldi graphs hold the geometry by value: drop them when the operator form changes
    if (was != (M != nullptr)) {
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        for (auto &kv : g->graphs) if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        g->graphs.clear();
    }
    return check_launch();
}

ch_status ch_lambda_max(ch_grid *g, const double *y, int eyre, double *lambda_max) {
    if (!g || !y || !lambda_max) return fail(CH_EINVAL, "null argument");
    lambda_queue(g, y, eyre);
    CH_TRY(check_launch());
    CH_TRY(sync_ctrl(g));
    *lambda_max = lambda_read(g, eyre);
    return CH_OK;
}

ch_status ch_estimate(ch_grid *g, const double *y0, const double *y1, double tau, double *est) {
    if (!g || !y0 || !y1 || !est) return fail(CH_EINVAL, "null argument");
    rhs(g, y0, g->F[0], 0, 0);
    rhs(g, y1, g->F[1], 0, 4, y0, g->F[0], 0.5 * tau);
    CH_TRY(check_launch());
    CH_TRY(sync_ctrl(g));
    *est = sqrt(g->hctrl->red[2]) / sqrt(g->hctrl->red[3]);
    return CH_OK;
}

ch_status ch_phi_krylov(ch_grid *g, const double *y_n, double tau0, double tol_phi, int mmax,
                        int linear_restart, int eyre, double *y_next, double *tau_used,
                        ch_stats *stats) {
    if (!g || !y_n || !y_next) return fail(CH_EINVAL, "null argument");
    if (y_n == y_next) return fail(CH_EINVAL, "y_next may not alias y_n");
    if (mmax < 1 || mmax > g->mmax_cap) return fail(CH_EINVAL, "mmax outside [1, capacity]");
    if (!(tau0 > 0.0) || !(tol_phi > 0.0) || !isfinite(tau0))
        return fail(CH_EINVAL, "tau0 must be finite and > 0, tol_phi > 0");
    rhs(g, y_n, g->F[0], eyre, 1);
    EEOut o;
    CH_TRY(ee_step_impl(g, y_n, 0, tau0, tol_phi, 0.0, mmax, linear_restart, eyre, y_next, 0, &o));
    if (tau_used) *tau_used = o.tau;
    if (stats) {
        stats->matvecs += o.matvecs;
        stats->krylov_iters += o.matvecs - 1 - o.restarts;
        stats->restarts += o.restarts;
        stats->tau_shrinks += o.shrunk;
        stats->phi_evals += o.phi_evals;
        stats->rhs_evals += 1;
    }
    return CH_OK;
}

static ch_status check_params(ch_grid *g, const ch_params *p) {
    if (!p) return fail(CH_EINVAL, "null params");
    if (p->scheme != CH_EE2 && p->scheme != CH_LIM) return fail(CH_EINVAL, "unknown scheme");
    if (!(p->T > 0.0) || !(p->tau0 > 0.0) || !isfinite(p->T) || !isfinite(p->tau0))
        return fail(CH_EINVAL, "T and tau0 must be finite and > 0");
    if (p->adaptive && !(p->tol > 0.0)) return fail(CH_EINVAL, "tol must be > 0 for adaptive runs");
    if (p->scheme == CH_EE2 && (p->mmax < 1 || p->mmax > g->mmax_cap))
        return fail(CH_EINVAL, "mmax outside [1, capacity]");
    if (p->scheme == CH_EE2 && !(p->tol_phi > 0.0) && !(p->tol > 0.0))
        return fail(CH_EINVAL, "need tol_phi > 0 or tol > 0");
    if (p->max_steps < 1) return fail(CH_EINVAL, "max_steps must be >= 1");
    return CH_OK;
}

ch_status ch_ee_step(ch_grid *g, const double *y_n, double tau, const ch_params *prm,
                     double *y_next, double *tau_used, double *est) {
    if (!g || !y_n || !y_next) return fail(CH_EINVAL, "null argument");
    if (y_n == y_next) return fail(CH_EINVAL, "y_next may not alias y_n");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(CH_EINVAL, "tau must be finite and > 0");
    CH_TRY(check_params(g, prm));
    const int use_ghat = !(prm->tol_phi > 0.0);
    rhs(g, y_n, g->F[0], prm->eyre, 1 | (use_ghat ? 2 : 0));
    EEOut o;
    CH_TRY(ee_step_impl(g, y_n, 0, tau, prm->tol_phi, prm->tol, prm->mmax, !prm->adaptive,
                        prm->eyre, y_next, 1, &o));
    if (tau_used) *tau_used = o.tau;
    if (est) *est = o.est;
    return CH_OK;
}

ch_status ch_lim_step(ch_grid *g, const double *y_n, double tau, int eyre, double *y_next,
                      int *p_used, double *lambda_max) {
    if (!g || !y_n || !y_next) return fail(CH_EINVAL, "null argument");
    if (y_n == y_next) return fail(CH_EINVAL, "y_next may not alias y_n");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(CH_EINVAL, "tau must be finite and > 0");
    double lmax;
    CH_TRY(ch_lambda_max(g, y_n, eyre, &lmax));
    int p = 0;
    CH_TRY(lim_step_impl(g, y_n, tau, lmax, eyre, y_next, &p));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (p_used) *p_used = p;
    if (lambda_max) *lambda_max = lmax;
    return CH_OK;
}

ch_status ch_set_record_capacity(ch_grid *g, int64_t capacity) {
    if (!g || capacity < 0) return fail(CH_EINVAL, "bad argument");
    g->rec_cap = capacity;
    g->rec.clear();
    g->rec.reserve((size_t)std::min<int64_t>(capacity, 1 << 20));
    return CH_OK;
}

ch_status ch_get_records(ch_grid *g, int64_t max, double *tau, int *jexit, int *restarts,
                         int *shrunk, int *p, double *est, int64_t *count) {
    if (!g) return fail(CH_EINVAL, "null grid");
    const int64_t n = std::max<int64_t>(0, std::min<int64_t>(max, (int64_t)g->rec.size()));
    for (int64_t k = 0; k < n; ++k) {
        const StepRecord &r = g->rec[(size_t)k];
        if (tau) tau[k] = r.tau;
        if (jexit) jexit[k] = r.jexit;
        if (restarts) restarts[k] = r.restarts;
        if (shrunk) shrunk[k] = r.shrunk;
        if (p) p[k] = r.p;
        if (est) est[k] = r.est;
    }
    if (count) *count = n;
    return CH_OK;
}

ch_status ch_get_state(ch_grid *g, double *t, double *tau) {
    if (!g) return fail(CH_EINVAL, "null grid");
    if (t) *t = g->t_last;
    if (tau) *tau = g->tau_last;
    return CH_OK;
}

ch_status ch_set_state(ch_grid *g, double t, double tau) {
    if (!g || !(t >= 0.0) || !(tau > 0.0)) return fail(CH_EINVAL, "bad state");
    g->t_resume = t;
    g->tau_resume = tau;
    g->resume = 1;
    return CH_OK;
}

ch_status ch_energy_mass(ch_grid *g, const double *y, double *energy, double *mass) {
    if (!g || !y) return fail(CH_EINVAL, "null argument");
    ch::launch_energy(g->L, g->g, y);
    CH_TRY(check_launch());
    CH_TRY(sync_ctrl(g));
    double vol = 1.0;
    for (int a = 0; a < g->g.dim; ++a) vol /= (double)g->g.n[a];
    if (energy) *energy = vol * g->hctrl->red[6];
    if (mass) *mass = vol * g->hctrl->red[7];
    return CH_OK;
}

// Step size of constant-step step k: tau0, the last of ceil(T/tau0) steps ending at T.
static int64_t const_nsteps(double T, double tau0) { return (int64_t)ceil(T / tau0 - 1e-9); }
static double const_tau(double T, double tau0, int64_t k) {
    const int64_t n = const_nsteps(T, tau0);
    if (k < n - 1) return tau0;
    const double last = T - (double)(n - 1) * tau0;
    return fabs(last - tau0) <= 1e-9 * tau0 ? tau0 : last;
}

ch_status ch_integrate(ch_grid *g, const ch_params *prm, double *y, ch_stats *stats) {
    if (!g || !y) return fail(CH_EINVAL, "null argument");
    CH_TRY(check_params(g, prm));
    ch::NvtxRange range(prm->scheme == CH_EE2 ? "ch_integrate EE2" : "ch_integrate LIM");
    ch_stats st;
    memset(&st, 0, sizeof st);
    g->rec.clear();
    double t = g->resume ? g->t_resume : 0.0;                              // t := 0
    double tau = g->resume ? g->tau_resume : prm->tau0;
    g->resume = 0;
    const int adaptive = prm->adaptive, eyre = prm->eyre;
    const int64_t nconst = adaptive ? 0 : const_nsteps(prm->T, prm->tau0);
    const int use_ghat = prm->scheme == CH_EE2 && !(prm->tol_phi > 0.0);
    // state: ycur (the caller's y, updated in place at the end of each step via swap)
    double *ycur = y, *ynew = g->y[2];
    int cur = 0;
    double lmax = 0.0;
    // f(y_0) for the first Krylov start vector / the first PC estimate
    if (prm->scheme == CH_EE2 || adaptive) {
        rhs(g, ycur, g->F[cur], eyre, 1 | (use_ghat ? 2 : 0));
        st.rhs_evals += 1;
    }
    if (prm->scheme == CH_LIM) {
        lambda_queue(g, ycur, eyre);
        CH_TRY(check_launch());
        CH_TRY(sync_ctrl(g));
        lmax = lambda_read(g, eyre);
    }
    ch_status rc = CH_OK;
    for (;;) {
        if (adaptive ? !(t < prm->T) : st.steps >= nconst) break;         // while t < T
        int clipped = 0;
        if (adaptive) {
            if (t + tau > prm->T) { tau = prm->T - t; clipped = 1; }      // clip to T
        } else {
            tau = const_tau(prm->T, prm->tau0, st.steps);
        }
        StepRecord r = {tau, 0.0, 0, 0, 0, 0};
        double taken = tau, est = 0.0;
        if (prm->scheme == CH_EE2) {                                       // EE2 step, Fig. 4
            EEOut o;
            rc = ee_step_impl(g, ycur, cur, tau, prm->tol_phi, prm->tol, prm->mmax, !adaptive,
                              eyre, ynew, adaptive, &o);
            if (rc != CH_OK) break;
            taken = o.tau; est = o.est;
            r.jexit = o.jexit; r.restarts = o.restarts; r.shrunk = o.shrunk;
            st.matvecs += o.matvecs;
            st.krylov_iters += o.matvecs - 1 - o.restarts;
            st.restarts += o.restarts;
            st.tau_shrinks += o.shrunk;
            st.phi_evals += o.phi_evals;
            if (adaptive) { st.rhs_evals += 1; cur = 1 - cur; }
            else {
                rhs(g, ynew, g->F[cur], eyre, 1 | (use_ghat ? 2 : 0));
                st.rhs_evals += 1;
            }
        } else {                                                           // LIM step, Fig. 3
            int p = 0;
            int rhs_used = 0;
            rc = lim_step_impl(g, ycur, tau, lmax, eyre, ynew, &p, adaptive ? g->F[cur] : nullptr, &rhs_used);
            if (rc != CH_OK) break;
            st.rhs_evals += rhs_used;
            r.p = p;
            st.matvecs += 2 * p - 1;
            // f(y_{n+1}) with the est sums, and lambda_max of the next step
            if (adaptive) {
                ch::launch_rhs1(g->L, g->g, ynew, eyre, g->t, nullptr);
                ch::launch_rhs2(g->L, g->g, g->t, nullptr, g->F[1 - cur], ycur, g->F[cur], ynew,
                                0.5 * tau, 4);
                st.rhs_evals += 1;
            }
            lambda_queue(g, ynew, eyre);
            rc = check_launch();
            if (rc != CH_OK) break;
            rc = sync_ctrl(g);
            if (rc != CH_OK) break;
            if (adaptive) {
                est = sqrt(g->hctrl->red[2]) / sqrt(g->hctrl->red[3]);
                cur = 1 - cur;
            }
            lmax = lambda_read(g, eyre);
        }
        if (adaptive && !isfinite(est)) { rc = fail(CH_ENONFINITE, "non-finite error estimate"); break; }
        r.tau = taken; r.est = est;
        add_record(g, r);
        std::swap(ycur, ynew);                                             // accept
        if (adaptive) t = (clipped && taken == tau) ? prm->T : t + taken;
        else t = (st.steps + 1 == nconst) ? prm->T : t + taken;
        ++st.steps;
        if (adaptive) {                                                    // next tau
            if (prm->scheme == CH_EE2) {                                   // Eq. (EEdt)
                const double grow = 1.25 * taken;
                tau = (est > 0.0) ? std::min(grow, sqrt(prm->tol / est) * taken) : grow;
            } else {                                                       // Eq. (LIMdt)
                tau = (est > 0.0) ? (prm->tol / est) * taken : taken;
            }
        }
        if (adaptive && t < prm->T && (!(tau > 0.0) || !isfinite(tau) || t + tau == t)) {
            rc = fail(CH_ENOTCONV, "step size %g makes no progress at t = %g", tau, t);
            break;
        }
        if (st.steps >= prm->max_steps && (adaptive ? t < prm->T : st.steps < nconst)) {
            rc = fail(CH_ENOTCONV, "max_steps reached before T");
            break;
        }
    }
    if (ycur != y) {
        cudaError_t e = cudaMemcpyAsync(y, ycur, g->g.N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess && rc == CH_OK) rc = fail(CH_ECUDA, "copy of the result: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess && rc == CH_OK) rc = fail(CH_ECUDA, "stream sync: %s", cudaGetErrorString(e));
    st.t = t;
    st.tau_next = tau;
    st.last_est = g->rec.empty() ? 0.0 : g->rec.back().est;
    g->t_last = t;
    g->tau_last = tau;
    if (stats) *stats = st;
    return rc;
}

}  // extern "C"
