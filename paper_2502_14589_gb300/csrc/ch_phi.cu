// ch_phi.cu -- projected phi evaluation, residual test and residual-time step choice of the
// Krylov method of Fig. 2 (lines 9-20), in FP64 on one thread block.
//
// u = s phi(-s H_j) e_1 (Eqs. phi, yt_m) is the last column of exp([[-s H_j, s e_1], [0, 0]]).
// The exponential uses the diagonal Pade approximant of degree 13 with scaling and squaring
// (N.J. Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005); the scaling exponent is the least
// integer sq >= 0 with ||M||_1 / 2^sq <= theta_13, found by exact halving.  The Pade
// denominator system is solved by Gauss-Jordan elimination with partial pivoting.
// All matrices (n = j+1 <= 129) live in shared memory when n <= 64, else in global scratch.
#include <math.h>

#include "ch_internal.cuh"

namespace ch {

constexpr int kPhiThreads = 512;
constexpr int kPhiSmemMaxN = 64;
constexpr int kMaxHalvings = 60;   // fixed trace rule of Fig. 2 lines 16-17
constexpr int kBisections = 12;

struct PhiWork {
    double *b[6];       // six n x n buffers (row-major, ld = n)
    double *fcol;       // n
    double *colsum;     // n
    double c[14];       // Pade coefficients
    int piv;
    double pinv;
    double norm1;
    double res;
};

__device__ __forceinline__ void mm(int n, const double *A, const double *B, double *C) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(A[r * n + k], B[k * n + c], acc);
        C[e] = acc;
    }
    __syncthreads();
}

// E = exp(M) with M given in W.b[0]; returns the buffer holding E.
__device__ double *expm_block(int n, PhiWork &W) {
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
    mm(n, X, X, X2);
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
    // Gauss-Jordan with partial pivoting on [P | Q]: Q <- P^{-1} Q
    double *P = X2, *Q = X4;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + (int)threadIdx.x; i < n; i += 32) {
                const double a = fabs(P[i * n + k]);
                if (a > best) { best = a; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) W.piv = bi;
        }
        __syncthreads();
        const int pv = W.piv;
        if (pv != k) {
            for (int cc = threadIdx.x; cc < n; cc += blockDim.x) {
                double t = P[k * n + cc]; P[k * n + cc] = P[pv * n + cc]; P[pv * n + cc] = t;
                t = Q[k * n + cc]; Q[k * n + cc] = Q[pv * n + cc]; Q[pv * n + cc] = t;
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) W.fcol[i] = P[i * n + k];
        if (threadIdx.x == 0) W.pinv = 1.0 / P[k * n + k];
        __syncthreads();
        const double pinv = W.pinv;
        for (int cc = threadIdx.x; cc < n; cc += blockDim.x) {
            P[k * n + cc] *= pinv;
            Q[k * n + cc] *= pinv;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, cc = e - i * n;
            if (i == k) continue;
            const double f = W.fcol[i];
            if (cc >= k) P[e] = fma(-f, P[k * n + cc], P[e]);
            Q[e] = fma(-f, Q[k * n + cc], Q[e]);
        }
        __syncthreads();
    }
    double *R = Q, *S = X6;
    for (int k = 0; k < sq; ++k) {
        mm(n, R, R, S);
        double *t = R; R = S; S = t;
    }
    return R;
}

// u = s phi(-s H_j) e_1 into W.fcol[0..j-1]... (u written to `u`), returns resnorm.
__device__ double phi_eval(int j, const double *H, int ldh, double hnext, double s, double *u,
                           PhiWork &W) {
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
    const double *E = expm_block(n, W);
    for (int r = threadIdx.x; r < j; r += blockDim.x) u[r] = E[r * n + j];
    __syncthreads();
    return hnext * fabs(u[j - 1]);                      // Fig. 2 line 12
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi(Ctrl *ctrl, double *H, int ldh, int j, int mmax, double *u, double *gscratch,
      int use_smem) {
    if (!ctrl->active) return;
    extern __shared__ double smem[];
    __shared__ PhiWork W;
    const int n = j + 1;
    if (threadIdx.x == 0) {
        double *base = use_smem ? smem : gscratch;
        for (int k = 0; k < 6; ++k) W.b[k] = base + (size_t)k * n * n;
        W.fcol = base + (size_t)6 * n * n;
        W.colsum = W.fcol + n;
        W.c[0] = 1.0;
        for (int k = 1; k <= 13; ++k)
            W.c[k] = W.c[k - 1] * (double)(13 - k + 1) / ((double)(2 * 13 - k + 1) * k);
    }
    __syncthreads();
    const double hnext = sqrt(ctrl->hnext2);             // Fig. 2 line 9
    const double tau0 = ctrl->tau0, tol = ctrl->tol_phi;
    if (threadIdx.x == 0) H[j * ldh + (j - 1)] = hnext;
    __syncthreads();
    int evals = 1;
    double res = phi_eval(j, H, ldh, hnext, tau0, u, W);  // lines 10-12
    int done = 0, shrunk = 0, status = 0;
    double tau = tau0;
    if (!isfinite(hnext) || !isfinite(res)) {
        status = CH_ENONFINITE;
        done = 1;
    } else if (res <= tol) {                                // lines 13-14
        done = 1;
    } else if (j == mmax) {                                 // lines 15-19
        double lo = tau0, hi = tau0;
        int ok = 0;
        for (int k = 0; k < kMaxHalvings; ++k) {
            hi = lo;
            lo = 0.5 * lo;
            ++evals;
            if (phi_eval(j, H, ldh, hnext, lo, u, W) <= tol) { ok = 1; break; }
        }
        if (ok) {
            for (int k = 0; k < kBisections; ++k) {
                const double mid = 0.5 * (lo + hi);
                ++evals;
                if (phi_eval(j, H, ldh, hnext, mid, u, W) <= tol) lo = mid;
                else hi = mid;
            }
            ++evals;
            phi_eval(j, H, ldh, hnext, lo, u, W);           // line 18
            tau = lo;
            shrunk = 1;
        } else {
            status = CH_ENOTCONV;
        }
        done = 1;
    }
    if (threadIdx.x == 0) {
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
            ctrl->gam[j] = 1.0 / hnext;                      // v_{j+1} = w / h_{j+1,j}, line 21
        }
    }
    if (done && !status)
        for (int c = threadIdx.x; c < j; c += blockDim.x)
            ctrl->coef[c] = ctrl->beta * ctrl->gam[c] * u[c];   // line 23
}

int phi_setup() {
    const size_t bytes = (size_t)(6 * kPhiSmemMaxN * kPhiSmemMaxN + 2 * kPhiSmemMaxN) * sizeof(double);
    return (int)cudaFuncSetAttribute(k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_phi(const Launch &L, double *H, int ldh, int j, int mmax, double *u,
                double *scratch) {
    const int n = j + 1;
    const int use_smem = n <= kPhiSmemMaxN;
    const size_t bytes = use_smem ? (size_t)(6 * n * n + 2 * n) * sizeof(double) : 0;
    LaunchScope scope(L, CH_K_PHI);
    k_phi<<<1, kPhiThreads, bytes, L.stream>>>(L.ctrl, H, ldh, j, mmax, u, scratch, use_smem);
}

}  // namespace ch
