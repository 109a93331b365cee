/*
 * ch_oracle.c -- plain, slow, single-threaded FP64 reference ("the oracle") for the
 * explicit Cahn-Hilliard time integrators of M.A. Botchev, "Explicit adaptive time
 * stepping for the Cahn-Hilliard equation by exponential Krylov subspace and Chebyshev
 * polynomial methods" (arXiv:2502.14589).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
 * check of __graft_entry__ and the CPU-baseline / reference arm of bench.py may build,
 * load or call it.  It shares no code, header, table or helper with the CUDA library;
 * the two meet only in the seeded input arrays that the tests hand to both.
 *
 * Every routine follows one passage of the paper and says which.  Loops are written out
 * in the order the paper states the algorithm, with no blocking or fusion, so a reader
 * can check them against the paper by eye.  The spatial discretisation is the second-order
 * finite-difference Laplacian on the unit square / cube, h_a = 1/n_a, with periodic
 * boundaries or with the paper's homogeneous Neumann conditions of Eq. (CH) on cell-centred
 * nodes (Sec. 5.1: x_i = (i - 1/2) h), where a neighbour beyond the boundary is the mirror
 * image of the point inside it.
 *
 * Readings of points where the paper is silent:
 *  - periodic boundary conditions for the benchmark workloads; the paper's Neumann
 *    conditions are the other choice of or_grid.bc;
 *  - the residual trace over s in [0, tau0] of Fig. 2 (left unspecified) = halve s from
 *    the upper end until the residual test passes, then bisect a fixed number of times
 *    keeping the admissible end;
 *  - constant-step EE2 uses linear residual-time restarting over the whole step with
 *    A_hat, g_hat frozen at y^n;
 *  - the order of beta_2..beta_p (left open by Fig. 1) bounds round-off growth (or_lim_order);
 *  - beta == 0 gives y^{n+1} = y^n; est == 0 keeps tau (LIM) or takes 5/4 tau (EE2);
 *  - a step clipped to end at T sets t := T exactly;
 *  - variable mobility (the Remark on Eq. CHmob): conservative flux form with each face's
 *    mobility the mean of its two nodes, nodal values supplied by the caller.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Grid description.  Points are stored x fastest: index = i0 + n0*(i1 + n1*i2).         */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int dim;        /* 2 or 3 */
    long n[3];      /* points per axis; n[2] == 1 when dim == 2 */
    double eps;     /* epsilon of the IVP (Sec. 2, Eq. IVP) */
    int eyre;       /* 0: A_hat, g_hat of Eq. (A_g); 1: Eyre splitting, Eq. (A_g_cs) */
    int bc;         /* 0: periodic; 1: homogeneous Neumann (Eq. CH), cell-centred nodes */
    const double *mob; /* NULL: unit mobility (Eq. IVP); else the nodal mobility M(y^n_i) >= 0
                          of Eq. (CHmob), frozen over the step as the Remark on it allows */
} or_grid;

typedef struct {            /* counters of work, as the paper counts it (Sec. 5.1) */
    long steps;             /* accepted time steps */
    long matvecs;           /* products with A_hat_n (the paper's cost measure) */
    long rhs_evals;         /* evaluations of the CH right-hand side */
    long krylov_iters;      /* Arnoldi iterations over all steps */
    long restarts;          /* linear residual-time restarts (constant-step EE2) */
    long tau_shrinks;       /* steps whose size the Krylov residual test reduced */
    long phi_evals;         /* projected phi evaluations */
    int status;             /* 0 ok, 4 not converged, 5 non-finite */
} or_stats;

static long or_N(const or_grid *g) { return g->n[0] * g->n[1] * g->n[2]; }

static double or_s(const or_grid *g, int a) { /* 1/h_a^2 with h_a = 1/n_a */
    return (double)g->n[a] * (double)g->n[a];
}

static long wrap(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }

/* Cell-centred Neumann: the node beyond a face is the mirror image of the node inside it
 * (index -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2), so every one-sided difference across
 * the boundary vanishes, the discrete form of dc/dn = dmu/dn = 0 in Eq. (CH).            */
static long mirror(long i, long n) {
    if (i < 0) return -i - 1;
    if (i >= n) return 2 * n - i - 1;
    return i;
}

/* index of the point shifted by `off` along axis a (|off| <= n_a) */
static long shift(const or_grid *g, long idx, int a, long off) {
    long i[3];
    i[0] = idx % g->n[0];
    i[1] = (idx / g->n[0]) % g->n[1];
    i[2] = idx / (g->n[0] * g->n[1]);
    i[a] = g->bc ? mirror(i[a] + off, g->n[a]) : wrap(i[a] + off, g->n[a]);
    return i[0] + g->n[0] * (i[1] + g->n[1] * i[2]);
}

/* Sec. 2, Eq. (IVP): A is symmetric positive semidefinite and -A is the discrete
 * Laplacian.  Standard second-order differences (Sec. 5.1), neighbours by shift():
 * (A v)_i = sum_a (2 v_i - v_{i+e_a} - v_{i-e_a}) / h_a^2.                            */
void or_apply_A(const or_grid *g, const double *v, double *out) {
    long N = or_N(g);
    for (long i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int a = 0; a < g->dim; ++a) {
            double s = or_s(g, a);
            acc += s * (2.0 * v[i] - v[shift(g, i, a, +1)] - v[shift(g, i, a, -1)]);
        }
        out[i] = acc;
    }
}

/* The Remark on Eq. (CHmob): with a mobility M(c), the outer operator becomes A_M(y^n), a
 * discretisation of -div(M grad .), frozen over the step.  Conservative flux form with the
 * mobility of a cell face taken as the mean of its two nodes:
 *   (A_M v)_i = sum_a (1/h_a^2) sum_{+-} (M_i + M_{i+-e_a})/2 (v_i - v_{i+-e_a}),
 * symmetric, positive semidefinite for M >= 0, with zero column sums (mass).  A Neumann face
 * has the node itself as its mirror neighbour, so its flux vanishes.  Unit mobility is A. */
void or_apply_AM(const or_grid *g, const double *v, double *out) {
    if (!g->mob) { or_apply_A(g, v, out); return; }
    long N = or_N(g);
    const double *M = g->mob;
    for (long i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int a = 0; a < g->dim; ++a) {
            double s = or_s(g, a);
            long ip = shift(g, i, a, +1), im = shift(g, i, a, -1);
            acc += s * (0.5 * (M[i] + M[ip]) * (v[i] - v[ip]) + 0.5 * (M[i] + M[im]) * (v[i] - v[im]));
        }
        out[i] = acc;
    }
}

/* Eq. (F): F(c) = (1 - c^2)^2 / 4,  F'(c) = c (c^2 - 1). *//* Eq. (F): F(c) = (1 - c^2)^2 / 4,  F'(c) = c (c^2 - 1). */
static double F(double c) { double t = 1.0 - c * c; return 0.25 * t * t; }
static double Fp(double c) { return c * (c * c - 1.0); }

/* Eq. (J): J_n = 3 diag((y^n)^2) - I, returned as its diagonal. */
static double Jdiag(double y) { return 3.0 * y * y - 1.0; }

/* Sec. 2, Eq. (IVP): f(y) = -A (F'(y) + eps^2 A y). */
void or_rhs(const or_grid *g, const double *y, double *f) {
    long N = or_N(g);
    double *Ay = malloc(N * sizeof(double)), *mu = malloc(N * sizeof(double));
    or_apply_A(g, y, Ay);
    for (long i = 0; i < N; ++i) mu[i] = Fp(y[i]) + g->eps * g->eps * Ay[i];
    or_apply_AM(g, mu, f);
    for (long i = 0; i < N; ++i) f[i] = -f[i];
    free(Ay); free(mu);
}

/* Eq. (A_g): g_hat^n = A (J_n y^n - F'(y^n));
 * Eq. (A_g_cs) with the Eyre splitting: g_hat^n = A (J_n y^n + y^n - F'(y^n)).       */
void or_ghat(const or_grid *g, const double *yn, double *ghat) {
    long N = or_N(g);
    double *t = malloc(N * sizeof(double));
    for (long i = 0; i < N; ++i) {
        t[i] = Jdiag(yn[i]) * yn[i] - Fp(yn[i]);
        if (g->eyre) t[i] += yn[i];
    }
    or_apply_AM(g, t, ghat);
    free(t);
}

/* Eq. (A_g): A_hat_n v = A (J_n + eps^2 A) v;
 * Eq. (A_g_cs): A_hat_n v = A (J_n + eps^2 A + I) v.                                   */
void or_jacvec(const or_grid *g, const double *yn, const double *v, double *w) {
    long N = or_N(g);
    double *Av = malloc(N * sizeof(double)), *t = malloc(N * sizeof(double));
    or_apply_A(g, v, Av);
    for (long i = 0; i < N; ++i) {
        t[i] = Jdiag(yn[i]) * v[i] + g->eps * g->eps * Av[i];
        if (g->eyre) t[i] += v[i];
    }
    or_apply_AM(g, t, w);
    free(Av); free(t);
}

/* ------------------------------------------------------------------------------------ */
/* LIM (Sec. 3, Fig. 1)                                                                 */
/* ------------------------------------------------------------------------------------ */

/* Fig. 1, spectral bound: lambda_max := ||A_hat_n||_1 = max_j sum_i |a_ij|, computed by forming
 * every column A_hat_n e_j explicitly.  A column has at most 13 (2D) or 25 (3D) nonzeros;
 * they are gathered into a small list, summing entries whose periodic indices coincide
 * (which happens on grids with fewer than 5 points along an axis).                      */
typedef struct { long idx; double val; } or_entry;

static int add_entry(or_entry *list, int cnt, long idx, double val) {
    for (int k = 0; k < cnt; ++k)
        if (list[k].idx == idx) { list[k].val += val; return cnt; }
    list[cnt].idx = idx; list[cnt].val = val; return cnt + 1;
}

/* A applied to a sparse vector given as an entry list */
static int sparse_apply_A(const or_grid *g, const or_entry *in, int nin, or_entry *out) {
    int cnt = 0;
    for (int k = 0; k < nin; ++k) {
        for (int a = 0; a < g->dim; ++a) {
            double s = or_s(g, a);
            cnt = add_entry(out, cnt, in[k].idx, 2.0 * s * in[k].val);
            cnt = add_entry(out, cnt, shift(g, in[k].idx, a, +1), -s * in[k].val);
            cnt = add_entry(out, cnt, shift(g, in[k].idx, a, -1), -s * in[k].val);
        }
    }
    return cnt;
}

/* A_M applied to a sparse vector (column k of A_M for each input entry k; A_M is symmetric) */
static int sparse_apply_AM(const or_grid *g, const or_entry *in, int nin, or_entry *out) {
    if (!g->mob) return sparse_apply_A(g, in, nin, out);
    const double *M = g->mob;
    int cnt = 0;
    for (int k = 0; k < nin; ++k) {
        long c = in[k].idx;
        for (int a = 0; a < g->dim; ++a) {
            double s = or_s(g, a);
            for (int off = -1; off <= 1; off += 2) {
                long nb = shift(g, c, a, off);
                double mf = 0.5 * (M[c] + M[nb]);
                cnt = add_entry(out, cnt, c, s * mf * in[k].val);
                cnt = add_entry(out, cnt, nb, -s * mf * in[k].val);
            }
        }
    }
    return cnt;
}

/* Absolute sum of column j of A_hat_n, formed explicitly. */
double or_column_abs_sum(const or_grid *g, const double *yn, long j) {
    or_entry e[1], Ae[8], AAe[64], Me[8], col[64];
    double dj = Jdiag(yn[j]) + (g->eyre ? 1.0 : 0.0);
    e[0].idx = j; e[0].val = 1.0;
    int nA = sparse_apply_A(g, e, 1, Ae);          /* A e_j */
    int nAA = sparse_apply_AM(g, Ae, nA, AAe);     /* A_M A e_j (A A e_j at unit mobility) */
    int nM = sparse_apply_AM(g, e, 1, Me);         /* A_M e_j */
    /* column j of A_hat = A_M (D + eps^2 A) e_j = d_j A_M e_j + eps^2 A_M A e_j */
    int nc = 0;
    for (int k = 0; k < nM; ++k) nc = add_entry(col, nc, Me[k].idx, dj * Me[k].val);
    for (int k = 0; k < nAA; ++k)
        nc = add_entry(col, nc, AAe[k].idx, g->eps * g->eps * AAe[k].val);
    double sum = 0.0;
    for (int k = 0; k < nc; ++k) sum += fabs(col[k].val);
    return sum;
}

double or_lambda_max(const or_grid *g, const double *yn) {
    long N = or_N(g);
    double best = 0.0;
    for (long j = 0; j < N; ++j) {
        double sum = or_column_abs_sum(g, yn, j);
        if (sum > best) best = sum;
    }
    return best;
}

/* Eq. (p): p = ceil( (pi/4) / (pi/2 - arctan sqrt(tau lambda_max)) ). */
int or_cheb_order(double tau, double lambda_max) {
    const double pi = 3.14159265358979323846;
    double x = (pi / 4.0) / (pi / 2.0 - atan(sqrt(tau * lambda_max)));
    return (int)ceil(x);
}

/* A linear operator y -> A_hat y, so that the LIM and Krylov cores below can be run on
 * the Cahn-Hilliard grid operator and, in tests, on small dense matrices.             */
typedef void (*or_matvec_fn)(void *ctx, const double *v, double *w);

typedef struct { const or_grid *g; const double *yn; } or_grid_op;
static void grid_matvec(void *ctx, const double *v, double *w) {
    or_grid_op *op = ctx; or_jacvec(op->g, op->yn, v, w);
}

typedef struct { long N; const double *M; } or_dense_op;   /* row-major N x N */
static void dense_matvec(void *ctx, const double *v, double *w) {
    or_dense_op *op = ctx;
    for (long i = 0; i < op->N; ++i) {
        double acc = 0.0;
        for (long k = 0; k < op->N; ++k) acc += op->M[i * op->N + k] * v[k];
        w[i] = acc;
    }
}

/* Fig. 1 asks for an ORDERED set {beta_m} and fixes only beta_1 = cos(pi/2p) (so
 * that a_1 = 0 comes first).  Every LIM iteration maps the error against the implicit-
 * Euler solution of Eq. (EBlin) by the factor (tau a_m - tau A_hat)/(1 + tau a_m); these
 * factors commute, so the order of beta_2..beta_p does not change the step in exact
 * arithmetic, only how far the intermediate iterates grow and how much later factors
 * amplify the rounding errors made on them.  In the natural order i = 2..p the iterates
 * grow by 1e10 at tau*lambda_max = 700 (1e63 at 2.5e4), which makes the step useless in
 * FP64 on fine grids.  The order used here is the recursive mirror-pair ordering of
 * Lebedev and Finogenov (USSR Comput. Math. Math. Phys. 11(2), 1971) for Chebyshev
 * iteration parameters, extended to odd p:
 *   order(1) = (1);
 *   order(p), m = floor(p/2): for each j of order(m) in turn, the pair (j, p + 1 - j);
 *   for odd p the middle index m + 1 is inserted right after the first pair.
 * It starts with m = 1, as Fig. 1 requires, and keeps the growth of iterates times the
 * amplification of later factors near (tau*lambda_max)^2.  The second sweep (m = 2..p)
 * reuses the order without m = 1.  order[] receives 0-based m.                          */
#define OR_LIM_MAX_P 1000000
static void lim_order_rec(int p, int *out) {               /* 1-based, length p */
    if (p == 1) { out[0] = 1; return; }
    int m = p / 2, k = 0;
    int *inner = malloc(m * sizeof(int));
    lim_order_rec(m, inner);
    for (int i = 0; i < m; ++i) {
        out[k++] = inner[i];
        out[k++] = p + 1 - inner[i];
        if (i == 0 && (p % 2) == 1) out[k++] = m + 1;
    }
    free(inner);
}

int or_lim_order(int p, int *order) {
    if (p < 1 || p > OR_LIM_MAX_P) return -1;
    lim_order_rec(p, order);
    for (int i = 0; i < p; ++i) order[i] -= 1;
    return 0;
}

/* Fig. 1: one LIM step for y' = -A_hat y + g_hat, y(0) = y^n, with a given
 * spectral bound lambda_max.  Returns p (or -1 when p exceeds OR_LIM_MAX_P).           */
static int lim_core(or_matvec_fn mv, void *ctx, long N, const double *ghat,
                    const double *yn, double tau, double lambda_max, double *ynext,
                    long *matvecs) {
    const double pi = 3.14159265358979323846;
    int p = or_cheb_order(tau, lambda_max);                        /* Eq. (p) */
    int *order = malloc(p * sizeof(int));
    if (or_lim_order(p, order) != 0) { free(order); return -1; }   /* ordered set */
    double *beta = malloc(p * sizeof(double)), *a = malloc(p * sizeof(double));
    for (int i = 1; i <= p; ++i) beta[i - 1] = cos(pi * (2.0 * i - 1.0) / (2.0 * p));
    double z1 = beta[0];                                           /* z_1 */
    for (int m = 1; m <= p; ++m) a[m - 1] = lambda_max / (1.0 + z1) * (z1 - beta[m - 1]); /* a_m */
    double *prev = malloc(N * sizeof(double)), *Ay = malloc(N * sizeof(double));
    memcpy(prev, yn, N * sizeof(double));                          /* y(prev) := y^n */
    for (int sweep = 0; sweep < 2; ++sweep) {                      /* m = 1..p, then 2..p */
        for (int idx = (sweep == 0 ? 0 : 1); idx < p; ++idx) {
            double am = a[order[idx]];
            mv(ctx, prev, Ay); ++*matvecs;
            for (long i = 0; i < N; ++i)                           /* the LIM update */
                ynext[i] = (yn[i] + tau * am * prev[i] + tau * (ghat[i] - Ay[i]))
                           / (1.0 + tau * am);
            memcpy(prev, ynext, N * sizeof(double));               /* y(prev) := y(next) */
        }
    }
    free(order); free(beta); free(a); free(prev); free(Ay);
    return p;
}

/* Fig. 1 on the Cahn-Hilliard grid operator: A_hat_n, g_hat^n from y^n (Eq. A_g or
 * Eq. A_g_cs), lambda_max = ||A_hat_n||_1.                                            */
int or_lim_step(const or_grid *g, const double *yn, double tau, double *ynext,
                double *lambda_max_out, long *matvecs) {
    long N = or_N(g);
    double *ghat = malloc(N * sizeof(double));
    or_ghat(g, yn, ghat);
    double lmax = or_lambda_max(g, yn);
    or_grid_op op = { g, yn };
    long mv = 0;
    int p = lim_core(grid_matvec, &op, N, ghat, yn, tau, lmax, ynext, &mv);
    if (lambda_max_out) *lambda_max_out = lmax;
    if (matvecs) *matvecs += mv;
    free(ghat);
    return p;
}

/* Dense-matrix entry for tests: LIM step for y' = -M y + g. */
int or_lim_dense(long N, const double *M, const double *ghat, const double *yn, double tau,
                 double lambda_max, double *ynext) {
    or_dense_op op = { N, M };
    long mv = 0;
    return lim_core(dense_matvec, &op, N, ghat, yn, tau, lambda_max, ynext, &mv);
}

/* ------------------------------------------------------------------------------------ */
/* Small dense matrix exponential: diagonal Pade approximant of degree 13 with scaling   */
/* and squaring, after N.J. Higham, "The scaling and squaring method for the matrix      */
/* exponential revisited", SIAM J. Matrix Anal. Appl. 26(4), 2005.  The degree is fixed  */
/* at 13 (accurate for every norm; only the cost differs from the paper's cheaper        */
/* choices for small norms).                                                            */
/* ------------------------------------------------------------------------------------ */
static void mat_mul(int n, const double *X, const double *Y, double *Z) {  /* Z = X Y */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += X[i * n + k] * Y[k * n + j];
            Z[i * n + j] = acc;
        }
}

/* Solve P X = Q (n x n, n right-hand sides) by Gaussian elimination with partial
 * pivoting; P and Q are overwritten, the solution is left in Q.  Returns 0 on success. */
static int solve_lu(int n, double *P, double *Q) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i) if (fabs(P[i * n + k]) > fabs(P[piv * n + k])) piv = i;
        if (P[piv * n + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = P[k * n + j]; P[k * n + j] = P[piv * n + j]; P[piv * n + j] = t;
                t = Q[k * n + j]; Q[k * n + j] = Q[piv * n + j]; Q[piv * n + j] = t;
            }
        }
        for (int i = k + 1; i < n; ++i) {
            double l = P[i * n + k] / P[k * n + k];
            for (int j = k; j < n; ++j) P[i * n + j] -= l * P[k * n + j];
            for (int j = 0; j < n; ++j) Q[i * n + j] -= l * Q[k * n + j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < n; ++j) {
            double acc = Q[k * n + j];
            for (int i = k + 1; i < n; ++i) acc -= P[k * n + i] * Q[i * n + j];
            Q[k * n + j] = acc / P[k * n + k];
        }
    return 0;
}

/* E = exp(M), row-major n x n. */
int or_expm(int n, const double *M, double *E) {
    const int m = 13;
    const double theta13 = 5.371920351148152;   /* Higham (2005), Table 2.3 */
    double c[14];                                /* Pade coefficients, c_0 = 1:        */
    c[0] = 1.0;                                  /* c_k = (2m-k)! m! / ((2m)! k! (m-k)!) */
    for (int k = 1; k <= m; ++k) c[k] = c[k - 1] * (double)(m - k + 1) / ((double)(2 * m - k + 1) * k);
    size_t sz = (size_t)n * n * sizeof(double);
    double *X = malloc(sz), *X2 = malloc(sz), *X4 = malloc(sz), *X6 = malloc(sz);
    double *T = malloc(sz), *U = malloc(sz), *V = malloc(sz), *P = malloc(sz), *Q = malloc(sz);
    double norm1 = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(M[i * n + j]);
        if (s > norm1) norm1 = s;
    }
    int sq = 0;                                  /* least sq >= 0 with norm1/2^sq <= theta13 */
    for (double sc = norm1; sc > theta13 && sq < 1100; sc *= 0.5) ++sq;
    double scale = ldexp(1.0, -sq);
    for (int i = 0; i < n * n; ++i) X[i] = M[i] * scale;
    mat_mul(n, X, X, X2); mat_mul(n, X2, X2, X4); mat_mul(n, X4, X2, X6);
    /* U = X [X6 (c13 X6 + c11 X4 + c9 X2) + c7 X6 + c5 X4 + c3 X2 + c1 I] */
    for (int i = 0; i < n * n; ++i) T[i] = c[13] * X6[i] + c[11] * X4[i] + c[9] * X2[i];
    mat_mul(n, X6, T, U);
    for (int i = 0; i < n * n; ++i) U[i] += c[7] * X6[i] + c[5] * X4[i] + c[3] * X2[i];
    for (int i = 0; i < n; ++i) U[i * n + i] += c[1];
    memcpy(T, U, sz);
    mat_mul(n, X, T, U);
    /* V = X6 (c12 X6 + c10 X4 + c8 X2) + c6 X6 + c4 X4 + c2 X2 + c0 I */
    for (int i = 0; i < n * n; ++i) T[i] = c[12] * X6[i] + c[10] * X4[i] + c[8] * X2[i];
    mat_mul(n, X6, T, V);
    for (int i = 0; i < n * n; ++i) V[i] += c[6] * X6[i] + c[4] * X4[i] + c[2] * X2[i];
    for (int i = 0; i < n; ++i) V[i * n + i] += c[0];
    /* r_13 = (V - U)^{-1} (V + U) */
    for (int i = 0; i < n * n; ++i) { P[i] = V[i] - U[i]; Q[i] = V[i] + U[i]; }
    int rc = solve_lu(n, P, Q);
    for (int k = 0; k < sq; ++k) { mat_mul(n, Q, Q, T); memcpy(Q, T, sz); }
    memcpy(E, Q, sz);
    free(X); free(X2); free(X4); free(X6); free(T); free(U); free(V); free(P); free(Q);
    return rc;
}

/* Sec. 4.1, Eqs. (phi), (yt_m): u = s phi(-s H_j) e_1 for the leading j x j block of the
 * Hessenberg matrix H (leading dimension ldh, row-major), via the exponential of the
 * augmented matrix [[-s H_j, s e_1], [0, 0]], whose last column holds s phi(-s H_j) e_1. */
int or_phi_e1(int j, const double *H, int ldh, double s, double *u) {
    int n = j + 1;
    double *M = calloc((size_t)n * n, sizeof(double)), *E = malloc((size_t)n * n * sizeof(double));
    for (int r = 0; r < j; ++r)
        for (int c = 0; c < j; ++c) M[r * n + c] = -s * H[r * ldh + c];
    M[0 * n + j] = s;
    int rc = or_expm(n, M, E);
    for (int r = 0; r < j; ++r) u[r] = E[r * n + j];
    free(M); free(E);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Krylov subspace method of Fig. 2 (Sec. 4.1): Arnoldi with modified Gram-Schmidt,      */
/* the residual norm of Eq. (rm), and the residual-time step choice of Eq. (phi_stop).   */
/* ------------------------------------------------------------------------------------ */
static double dot(long N, const double *a, const double *b) {
    double acc = 0.0;
    for (long i = 0; i < N; ++i) acc += a[i] * b[i];
    return acc;
}

/* Fixed search rule for the step trace of Fig. 2 (the residual as a function of s in [0, tau0]):
 * halve s from s_max until resnorm(s) <= tol, at most OR_MAX_HALVINGS times, then
 * OR_BISECTIONS bisection steps between that admissible s and the last rejected one,
 * keeping the admissible end.                                                           */
#define OR_MAX_HALVINGS 60
#define OR_BISECTIONS 12

static double resnorm_at(int j, const double *H, int ldh, double hnext, double s,
                         double *u, long *phi_evals) {
    or_phi_e1(j, H, ldh, s, u); ++*phi_evals;
    return hnext * fabs(u[j - 1]);                     /* resnorm of Fig. 2 */
}

/* One run of the Arnoldi loop of Fig. 2 for y' = -A_hat y + g, y(0) = y0, with starting
 * vector v_1 = g - A_hat y0.  The tentative step is tau0.  On return *tau is
 * the step taken (tau0, or the largest admissible s < tau0 found by the trace) and
 * ynext = y0 + V_j (beta u).  *jexit is the Krylov dimension j at exit.
 * Returns 0 ok, 4 when no admissible s is found.                                        */
static int krylov_core(or_matvec_fn mv, void *ctx, long N, const double *g,
                       const double *y0, double tau0, double tol_phi, int mmax,
                       double *ynext, double *tau, int *jexit, or_stats *st) {
    int ldh = mmax;                                                /* H is (mmax+1) x mmax */
    double *H = calloc((size_t)(mmax + 1) * mmax, sizeof(double)); /* H := 0 */
    double *V = calloc((size_t)N * (mmax + 1), sizeof(double));    /* column k at V + k*N */
    double *w = malloc(N * sizeof(double)), *u = calloc(mmax, sizeof(double));
    int rc = 0;
    mv(ctx, y0, w); ++st->matvecs;                                 /* start vector */
    for (long i = 0; i < N; ++i) V[i] = g[i] - w[i];
    double beta = sqrt(dot(N, V, V));
    *tau = tau0;
    *jexit = 0;
    if (beta == 0.0) {                       /* stationary point of the linear IVP */
        memcpy(ynext, y0, N * sizeof(double));
        goto done;
    }
    for (long i = 0; i < N; ++i) V[i] /= beta;
    int j;
    for (j = 1; j <= mmax; ++j) {                                  /* Arnoldi loop */
        double *vj = V + (size_t)(j - 1) * N;
        mv(ctx, vj, w); ++st->matvecs; ++st->krylov_iters;          /* w := A_hat v_j */
        for (int i = 1; i <= j; ++i) {                             /* modified Gram-Schmidt */
            double *vi = V + (size_t)(i - 1) * N;
            double hij = dot(N, w, vi);
            H[(i - 1) * ldh + (j - 1)] = hij;
            for (long k = 0; k < N; ++k) w[k] -= hij * vi[k];
        }
        double hnext = sqrt(dot(N, w, w));                         /* h_{j+1,j} */
        H[j * ldh + (j - 1)] = hnext;
        double s = tau0;                                           /* s := tau0 */
        double resnorm = resnorm_at(j, H, ldh, hnext, s, u, &st->phi_evals); /* resnorm */
        if (resnorm <= tol_phi) {                                  /* converged */
            *tau = tau0;
            break;
        } else if (j == mmax) {                                    /* step trace */
            double lo = tau0, hi = tau0;
            int ok = 0;
            for (int k = 0; k < OR_MAX_HALVINGS; ++k) {
                hi = lo; lo = 0.5 * lo;
                if (resnorm_at(j, H, ldh, hnext, lo, u, &st->phi_evals) <= tol_phi) { ok = 1; break; }
            }
            if (!ok) { rc = 4; *tau = 0.0; break; }
            for (int k = 0; k < OR_BISECTIONS; ++k) {
                double mid = 0.5 * (lo + hi);
                if (resnorm_at(j, H, ldh, hnext, mid, u, &st->phi_evals) <= tol_phi) lo = mid;
                else hi = mid;
            }
            *tau = lo;                                             /* tau := s */
            resnorm_at(j, H, ldh, hnext, lo, u, &st->phi_evals);   /* u at s */
            break;
        }
        double *vnext = V + (size_t)j * N;                         /* v_{j+1} := w / h_{j+1,j} */
        for (long k = 0; k < N; ++k) vnext[k] = w[k] / hnext;
    }
    if (j > mmax) j = mmax;
    *jexit = j;
    if (rc == 0) {                                                 /* y0 + V_j (beta u) */
        for (long k = 0; k < N; ++k) {
            double acc = 0.0;
            for (int c = 0; c < j; ++c) acc += V[(size_t)c * N + k] * (beta * u[c]);
            ynext[k] = y0[k] + acc;
        }
    } else {
        memcpy(ynext, y0, N * sizeof(double));
    }
done:
    free(H); free(V); free(w); free(u);
    return rc;
}

/* Dense-matrix entry for tests: one Fig. 2 run for y' = -M y + g, y(0) = y0. */
int or_krylov_dense(long N, const double *M, const double *g, const double *y0, double tau0,
                    double tol_phi, int mmax, double *ynext, double *tau, int *jexit) {
    or_dense_op op = { N, M };
    or_stats st; memset(&st, 0, sizeof st);
    return krylov_core(dense_matvec, &op, N, g, y0, tau0, tol_phi, mmax, ynext, tau, jexit, &st);
}

/* Arnoldi relation check for tests: runs the Arnoldi process of Fig. 2 for exactly m
 * iterations (no residual test) and returns V (N x (m+1), column-major by vector) and
 * H ((m+1) x m row-major).                                                            */
int or_arnoldi_dense(long N, const double *M, const double *v1, int m, double *V, double *H) {
    or_dense_op op = { N, M };
    double *w = malloc(N * sizeof(double));
    double beta = sqrt(dot(N, v1, v1));
    for (long i = 0; i < N; ++i) V[i] = v1[i] / beta;
    memset(H, 0, (size_t)(m + 1) * m * sizeof(double));
    for (int j = 1; j <= m; ++j) {
        dense_matvec(&op, V + (size_t)(j - 1) * N, w);
        for (int i = 1; i <= j; ++i) {
            double *vi = V + (size_t)(i - 1) * N;
            double hij = dot(N, w, vi);
            H[(i - 1) * m + (j - 1)] = hij;
            for (long k = 0; k < N; ++k) w[k] -= hij * vi[k];
        }
        double hn = sqrt(dot(N, w, w));
        H[j * m + (j - 1)] = hn;
        for (long k = 0; k < N; ++k) V[(size_t)j * N + k] = w[k] / hn;
    }
    free(w);
    return 0;
}

/* Eq. (tol_phi): tol_phi = max{ min{ ||g_hat||/(10 beta), 1/10, 10 tol }, 1e-7 }. */
double or_tol_phi(double norm_ghat, double beta, double tol) {
    double a = norm_ghat / (10.0 * beta);
    double m = a < 0.1 ? a : 0.1;
    if (10.0 * tol < m) m = 10.0 * tol;
    return m > 1e-7 ? m : 1e-7;
}

/* One EE2 step (Sec. 4.1, Eqs. IVPlin, EE2, Fig. 2) on the grid operator.
 * linear_restart = 0: nonlinear RT restarting -- the Krylov run may shrink tau and the
 *   shrunken step is taken (the adaptive scheme of Fig. 4 takes the step the Krylov run returns).
 * linear_restart = 1: linear RT restarting over the whole step tau (constant-step use,
 *   end of Sec. 4.1): A_hat_n, g_hat^n stay frozen at y^n; whenever a run cannot reach
 *   the remaining time it advances by its admissible s and restarts from there with
 *   v_1 = g_hat^n - A_hat_n y_cur and its own beta.
 * tol_phi_fixed > 0 overrides Eq. (tol_phi) (tol is then unused).                      */
#define OR_MAX_RESTARTS 100000
int or_ee_step(const or_grid *g, const double *yn, double tau_in, double tol,
               double tol_phi_fixed, int mmax, int linear_restart, double *ynext,
               double *tau_out, int *jexit, or_stats *st) {
    long N = or_N(g);
    double *ghat = malloc(N * sizeof(double)), *ycur = malloc(N * sizeof(double));
    double *f = malloc(N * sizeof(double));
    or_ghat(g, yn, ghat);
    or_grid_op op = { g, yn };
    /* beta = ||g_hat - A_hat y^n||, needed by Eq. (tol_phi) */
    or_jacvec(g, yn, yn, f);
    for (long i = 0; i < N; ++i) f[i] = ghat[i] - f[i];
    double beta = sqrt(dot(N, f, f));
    double tol_phi = tol_phi_fixed > 0.0 ? tol_phi_fixed
                                         : or_tol_phi(sqrt(dot(N, ghat, ghat)), beta, tol);
    int rc = 0;
    double tau = 0.0;
    if (!linear_restart) {
        rc = krylov_core(grid_matvec, &op, N, ghat, yn, tau_in, tol_phi, mmax, ynext, &tau,
                         jexit, st);
        if (rc == 0 && tau < tau_in) ++st->tau_shrinks;
        *tau_out = tau;
    } else {
        double remaining = tau_in;
        memcpy(ycur, yn, N * sizeof(double));
        long nrestart = 0;
        for (;;) {
            rc = krylov_core(grid_matvec, &op, N, ghat, ycur, remaining, tol_phi, mmax, ynext,
                             &tau, jexit, st);
            if (rc != 0) break;
            if (tau >= remaining) break;                 /* reached t_n + tau_in */
            remaining -= tau;
            memcpy(ycur, ynext, N * sizeof(double));
            ++st->restarts;
            if (++nrestart > OR_MAX_RESTARTS) { rc = 4; break; }
        }
        *tau_out = tau_in;
    }
    free(ghat); free(ycur); free(f);
    return rc;
}

/* Eq. (LIMest): y_PC = y^n - (tau/2) A (F'(y^n) + F'(y^{n+1}) + eps^2 A (y^n + y^{n+1})),
 * est = ||y^{n+1} - y_PC|| / ||y_PC||.  Returns est.                                    */
double or_estimate(const or_grid *g, const double *yn, const double *ynp1, double tau) {
    long N = or_N(g);
    double *sum = malloc(N * sizeof(double)), *Asum = malloc(N * sizeof(double));
    double *t = malloc(N * sizeof(double)), *ypc = malloc(N * sizeof(double));
    for (long i = 0; i < N; ++i) sum[i] = yn[i] + ynp1[i];
    or_apply_A(g, sum, Asum);
    for (long i = 0; i < N; ++i) t[i] = Fp(yn[i]) + Fp(ynp1[i]) + g->eps * g->eps * Asum[i];
    or_apply_AM(g, t, Asum);
    for (long i = 0; i < N; ++i) ypc[i] = yn[i] - 0.5 * tau * Asum[i];
    double num = 0.0, den = 0.0;
    for (long i = 0; i < N; ++i) {
        double d = ynp1[i] - ypc[i];
        num += d * d; den += ypc[i] * ypc[i];
    }
    free(sum); free(Asum); free(t); free(ypc);
    return sqrt(num) / sqrt(den);
}

/* ------------------------------------------------------------------------------------ */
/* Time-stepping drivers: Fig. 3 (adaptive LIM), Fig. 4 (adaptive EE2), and constant-step */
/* versions of both.  Per-step records (tau taken, Krylov j at exit, restarts, shrink      */
/* flag, LIM p, est) are written while there is room (max_rec).                          */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int scheme;          /* 0 = EE2, 1 = LIM */
    int adaptive;        /* 1: Figs. 3/4; 0: constant tau = tau0 */
    double T, tau0, tol; /* Given of Figs. 3 and 4 */
    int mmax;            /* Krylov dimension (EE2) */
    double tol_phi;      /* > 0: fixed Krylov tolerance; <= 0: Eq. (tol_phi) */
    long max_steps;      /* safety cap */
} or_params;

typedef struct {
    double *tau; int *jexit; int *restarts; int *shrunk; int *p; double *est;
    long max_rec;
} or_records;

/* Step size of step k (0-based) of a constant-step run over [0, T]: tau0, except that
 * the last of ceil(T/tau0) steps ends exactly at T (it is tau0 itself whenever T is a
 * multiple of tau0 up to 1e-9 relative).                                               */
long or_const_nsteps(double T, double tau0) { return (long)ceil(T / tau0 - 1e-9); }
double or_const_tau(double T, double tau0, long k) {
    long n = or_const_nsteps(T, tau0);
    if (k < n - 1) return tau0;
    double last = T - (double)(n - 1) * tau0;
    return fabs(last - tau0) <= 1e-9 * tau0 ? tau0 : last;
}

int or_integrate(const or_grid *g, const or_params *prm, double *y, or_stats *st,
                 or_records *rec, double *t_out) {
    long N = or_N(g);
    double *ynext = malloc(N * sizeof(double));
    double t = 0.0, tau = prm->tau0;                                 /* t := 0, tau := tau0 */
    long nconst = prm->adaptive ? 0 : or_const_nsteps(prm->T, prm->tau0);
    int rc = 0;
    memset(st, 0, sizeof *st);
    for (;;) {
        if (prm->adaptive ? !(t < prm->T) : st->steps >= nconst) break;   /* while t < T */
        int clipped = 0;
        if (prm->adaptive) {
            if (t + tau > prm->T) { tau = prm->T - t; clipped = 1; }       /* clip to T */
        } else {
            tau = or_const_tau(prm->T, prm->tau0, st->steps);
        }
        double taken = tau, est = 0.0, lmax = 0.0;
        int jexit = 0, p = 0;
        long restarts_before = st->restarts, shrinks_before = st->tau_shrinks;
        if (prm->scheme == 0) {                                      /* EE2 step, Fig. 4 */
            int lin = prm->adaptive ? 0 : 1;
            rc = or_ee_step(g, y, tau, prm->tol, prm->tol_phi, prm->mmax, lin, ynext,
                            &taken, &jexit, st);
        } else {                                                     /* LIM step, Fig. 3 */
            p = or_lim_step(g, y, tau, ynext, &lmax, &st->matvecs);
            if (p < 0) rc = 4;
        }
        if (rc != 0) break;
        for (long i = 0; i < N; ++i)
            if (!isfinite(ynext[i])) { rc = 5; break; }
        if (rc != 0) break;
        if (prm->adaptive) {                                         /* est, Eq. (LIMest) */
            est = or_estimate(g, y, ynext, taken);
            st->rhs_evals += 1;
            if (!isfinite(est)) { rc = 5; break; }
        }
        if (rec && st->steps < rec->max_rec) {
            long k = st->steps;
            rec->tau[k] = taken; rec->jexit[k] = jexit; rec->p[k] = p; rec->est[k] = est;
            rec->restarts[k] = (int)(st->restarts - restarts_before);
            rec->shrunk[k] = (int)(st->tau_shrinks - shrinks_before);
        }
        memcpy(y, ynext, N * sizeof(double));                        /* accept */
        if (prm->adaptive) t = (clipped && taken == tau) ? prm->T : t + taken;
        else t = (st->steps + 1 == nconst) ? prm->T : t + taken;
        ++st->steps;
        if (prm->adaptive) {                                         /* next tau */
            if (prm->scheme == 0) {                                  /* Eq. (EEdt) */
                double grow = 1.25 * taken;
                tau = (est > 0.0) ? fmin(grow, sqrt(prm->tol / est) * taken) : grow;
            } else {                                                 /* Eq. (LIMdt) */
                tau = (est > 0.0) ? (prm->tol / est) * taken : taken;
            }
        }
        if (st->steps >= prm->max_steps && (prm->adaptive ? t < prm->T : st->steps < nconst)) {
            rc = 4; break;
        }
    }
    st->status = rc;
    if (t_out) *t_out = t;
    free(ynext);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Diagnostics (Sec. 5.2): discrete energy, Eq. (Ediscr) read as the Riemann sum of the  */
/* energy functional of Eq. (Ee) with forward differences (periodic: n per axis; Neumann: */
/* the n-1 interior ones, as Eq. (Ediscr) sums them), and the mass of Eq. (m), h^d sum y. */
/* ------------------------------------------------------------------------------------ */
double or_energy(const or_grid *g, const double *y) {
    long N = or_N(g);
    double vol = 1.0;
    for (int a = 0; a < g->dim; ++a) vol /= (double)g->n[a];
    double sF = 0.0, sG = 0.0;
    for (long i = 0; i < N; ++i) {
        sF += F(y[i]);
        for (int a = 0; a < g->dim; ++a) {
            double d = (y[shift(g, i, a, +1)] - y[i]) * (double)g->n[a];
            sG += d * d;
        }
    }
    return vol * (sF + 0.5 * g->eps * g->eps * sG);
}

double or_mass(const or_grid *g, const double *y) {
    long N = or_N(g);
    double vol = 1.0, s = 0.0;
    for (int a = 0; a < g->dim; ++a) vol /= (double)g->n[a];
    for (long i = 0; i < N; ++i) s += y[i];
    return vol * s;
}
