/*
 * Plain FP64 CPU oracle for the GaBP SVM solver of Bickson, Yom-Tov and Dolev,
 * "A Gaussian Belief Propagation Solver for Large Scale Support Vector
 * Machines".
 *
 * TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library) never calls,
 * links or loads this file; only the tests, the smoke check and the CPU
 * baseline of the benchmark do.  It shares no code, header or constant with
 * the CUDA sources.
 *
 * Everything is double precision and written as the paper states it, with no
 * blocking or fusion: loops over nodes and pairs.  OpenMP only splits the
 * outer loop over nodes; it changes no summation order.
 *
 * Readings of points the paper leaves open (bias as an additive lambda^2 term,
 * the amount of diagonal weighting, the synchronous schedule, the residual
 * used as the convergence test) are documented at each function.
 *
 * Return codes: 0 ok, 1 numeric failure (a nonpositive or non-finite cavity
 * precision), 2 out of memory, 3 invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ENUMERIC 1
#define ORC_ENOMEM 2
#define ORC_EINVAL 3

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Index of the calling thread inside a parallel region (0 without OpenMP). */
static int orc_thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* RBF kernel value K(a, b) = exp(-gamma ||a - b||^2) by the direct difference
 * (Section 1.1 names the radial-basis kernel; Section 5 uses it for every
 * experiment). */
static double rbf(const double* a, const double* b, long m, double gamma)
{
    double d2 = 0.0;
    for (long k = 0; k < m; ++k) {
        double t = a[k] - b[k];
        d2 += t * t;
    }
    return exp(-gamma * d2);
}

/* One off-diagonal entry of the SVM matrix:
 *   D_ij = y_i y_j K'(x_i, x_j)                      (Section 1.1, dual)
 *   K'(x_i, x_j) = K(x_i, x_j) + lambda^2            (Section 3, bias)
 * The bias is the paper's extra constant feature lambda appended to every
 * pattern; for the RBF kernel a constant coordinate cancels in the distance,
 * so it enters as the additive lambda^2 of the augmented inner product. */
double orc_q_offdiag(const double* xi, const double* xj, double yi, double yj,
                     long m, double gamma, double lam)
{
    return yi * yj * (rbf(xi, xj, m, gamma) + lam * lam);
}

/* Diagonal weighting (Section 3.1).  The paper weights the main diagonal of D
 * until Q is diagonally dominant, and motivates it with the 2-norm soft margin
 * that adds 1/C to the diagonal.
 *   rule 1 ("soft2"):    Q_ii = D_ii + 1/C = 1 + lambda^2 + 1/C
 *   rule 0 ("dominant"): Q_ii = max(1 + lambda^2 + 1/C, (1 + delta) R_i),
 *                        R_i = sum_{j != i} |Q_ij|                        */
double orc_q_diag(double row_abs_sum, double lam, double C, int diag_rule, double delta)
{
    double base = 1.0 + lam * lam + 1.0 / C;
    if (diag_rule == 1) return base;
    double dom = (1.0 + delta) * row_abs_sum;
    return dom > base ? dom : base;
}

/* Full n x n matrix Q (row-major) of the SVM dual for an RBF kernel. */
int orc_build_q(const double* X, const double* y, long n, long m, double gamma,
                double lam, double C, int diag_rule, double delta, double* Q)
{
    if (n < 1 || m < 1 || !(gamma > 0) || !(C > 0)) return ORC_EINVAL;
#pragma omp parallel for schedule(dynamic, 8)
    for (long i = 0; i < n; ++i) {
        for (long j = i + 1; j < n; ++j) {
            double q = orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam);
            Q[i * n + j] = q;
            Q[j * n + i] = q;
        }
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double R = 0.0;
        for (long j = 0; j < n; ++j)
            if (j != i) R += fabs(Q[i * n + j]);
        Q[i * n + i] = orc_q_diag(R, lam, C, diag_rule, delta);
    }
    return ORC_OK;
}

/* The diagonal of Q and the off-diagonal absolute row sums R_i of every row,
 * without storing Q: each unordered pair's |Q_ij| is formed once and added to
 * both rows (per-thread row-sum arrays, summed at the end).  O(n^2 m) time,
 * O(n T) memory for T threads.  The diagonal follows orc_q_diag. */
int orc_q_diag_all(const double* X, const double* y, long n, long m, double gamma,
                   double lam, double C, int diag_rule, double delta, double* diag, double* R)
{
    if (n < 1 || m < 1 || !(gamma > 0) || !(C > 0)) return ORC_EINVAL;
    const int T = orc_threads();
    double* acc = (double*)calloc((size_t)T * (size_t)n, sizeof(double));
    if (!acc) return ORC_ENOMEM;
#pragma omp parallel
    {
        double* mine = acc + (size_t)orc_thread_id() * (size_t)n;
#pragma omp for schedule(dynamic, 16)
        for (long i = 0; i < n; ++i) {
            double ri = 0.0;
            for (long j = i + 1; j < n; ++j) {
                double q = fabs(orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam));
                ri += q;
                mine[j] += q;
            }
            mine[i] += ri;
        }
    }
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += acc[(size_t)t * (size_t)n + i];
        R[i] = s;
        diag[i] = orc_q_diag(s, lam, C, diag_rule, delta);
    }
    free(acc);
    return ORC_OK;
}

/* The diagonal, the off-diagonal absolute row sums R_i and, for the
 * tile-sparse reading of Section 6's sparsified kernel, the largest |Q_ij| of
 * every block x block tile (I <= J) of the upper triangle (pairs i < j only;
 * tile index L = I Nt - I (I - 1) / 2 + (J - I), Nt = ceil(n / block)), in one
 * pass over the pairs without storing Q.  Row i's pairs go to its own thread,
 * so each tile maximum is the plain maximum over its rows.  R and the diagonal
 * follow orc_q_diag_all. */
int orc_q_diag_tilemax(const double* X, const double* y, long n, long m, double gamma,
                       double lam, double C, int diag_rule, double delta, long block,
                       double* diag, double* R, double* tmax)
{
    if (n < 1 || m < 1 || block < 1 || !(gamma > 0) || !(C > 0)) return ORC_EINVAL;
    const long Nt = (n + block - 1) / block;
    const long ntiles = Nt * (Nt + 1) / 2;
    const int T = orc_threads();
    double* acc = (double*)calloc((size_t)T * (size_t)n, sizeof(double));
    double* tm = (double*)calloc((size_t)T * (size_t)ntiles, sizeof(double));
    if (!acc || !tm) { free(acc); free(tm); return ORC_ENOMEM; }
#pragma omp parallel
    {
        double* mine = acc + (size_t)orc_thread_id() * (size_t)n;
        double* mt = tm + (size_t)orc_thread_id() * (size_t)ntiles;
#pragma omp for schedule(dynamic, 16)
        for (long i = 0; i < n; ++i) {
            const long I = i / block;
            double ri = 0.0;
            for (long j = i + 1; j < n; ++j) {
                double q = fabs(orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam));
                ri += q;
                mine[j] += q;
                const long J = j / block;
                const long L = I * Nt - I * (I - 1) / 2 + (J - I);
                if (q > mt[L]) mt[L] = q;
            }
            mine[i] += ri;
        }
    }
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += acc[(size_t)t * (size_t)n + i];
        R[i] = s;
        diag[i] = orc_q_diag(s, lam, C, diag_rule, delta);
    }
    for (long L = 0; L < ntiles; ++L) {
        double v = 0.0;
        for (int t = 0; t < T; ++t)
            if (tm[(size_t)t * (size_t)ntiles + L] > v) v = tm[(size_t)t * (size_t)ntiles + L];
        tmax[L] = v;
    }
    free(acc);
    free(tm);
    return ORC_OK;
}

/* Residual r = 1 - Q mu of the tile-sparse matrix (the reading of Section 6's
 * sparsified kernel used with orc_q_diag_tilemax): Q_ii = diag[i], and Q_ij
 * (i != j) is the SVM entry where the block x block tile holding the pair is
 * kept (keep[I * Nt + J] != 0 for I <= J, the upper-triangle tile of the pair)
 * and 0 where it is dropped.  Only kept tiles are visited, O(kept pairs m).
 * Returns ||r||_inf. */
double orc_residual_tile_sparse(const double* X, const double* y, long n, long m, double gamma,
                                double lam, const double* diag, long block, const unsigned char* keep,
                                const double* mu, double* r)
{
    const long Nt = (n + block - 1) / block;
    double rmax = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : rmax)
    for (long i = 0; i < n; ++i) {
        const long I = i / block;
        double s = 1.0 - diag[i] * mu[i];
        for (long J = 0; J < Nt; ++J) {
            const long lo = I < J ? I : J, hi = I < J ? J : I;
            if (!keep[lo * Nt + hi]) continue;
            const long j1 = (J + 1) * block < n ? (J + 1) * block : n;
            for (long j = J * block; j < j1; ++j) {
                if (j == i) continue;
                s -= orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam) * mu[j];
            }
        }
        r[i] = s;
        const double a = fabs(s);
        if (a > rmax) rmax = a;
    }
    return rmax;
}

/* The same quantities for chosen rows only, for matrices too large for the
 * whole-matrix passes above: for each row i of rows[0 .. nrows), with I = i /
 * block, the largest |Q_ab| of every tile (I, J), J = 0 .. Nt - 1 (pairs a != b
 * of block I x block J: the tile of the pair, upper or lower, holds the same
 * entries), tmax_rows[k * Nt + J] for the k-th row; R[k] = sum_{j != i} |Q_ij|
 * over the whole row, diag[k] the diagonal rule's Q_ii from it; and the
 * residual r[k] = 1 - diag[k] mu_i - sum_j Q_ij mu_j over the j of the tiles
 * (I, J) kept under the threshold tau (J == I, or tmax > tau), as the
 * tile-sparse matrix defines it.  O(nrows n m). */
int orc_rows_tile_sparse(const double* X, const double* y, long n, long m, double gamma, double lam, double C,
                         int diag_rule, double delta, long block, double tau, const long* rows, long nrows,
                         const double* mu, double* tmax_rows, double* R, double* diag, double* r)
{
    if (n < 1 || m < 1 || block < 1 || !(gamma > 0) || !(C > 0)) return ORC_EINVAL;
    const long Nt = (n + block - 1) / block;
    for (long k = 0; k < nrows; ++k) {
        const long i = rows[k];
        if (i < 0 || i >= n) return ORC_EINVAL;
        const long I = i / block, a1 = (I + 1) * block < n ? (I + 1) * block : n;
        double* tm = tmax_rows + k * Nt;
        /* tile maxima of block row I (those of the previous row when it has the same block) */
        const int same = k > 0 && rows[k - 1] / block == I;
#pragma omp parallel for schedule(dynamic, 4)
        for (long J = 0; J < Nt; ++J) {
            if (same) { tm[J] = tm[J - Nt]; continue; }
            const long b1 = (J + 1) * block < n ? (J + 1) * block : n;
            double v = 0.0;
            for (long a = I * block; a < a1; ++a)
                for (long bb = J * block; bb < b1; ++bb) {
                    if (a == bb) continue;
                    const double q = fabs(orc_q_offdiag(X + a * m, X + bb * m, y[a], y[bb], m, gamma, lam));
                    if (q > v) v = q;
                }
            tm[J] = v;
        }
        /* whole-row sum, diagonal, kept-tile residual */
        double s_abs = 0.0, s_mu = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s_abs, s_mu)
        for (long j = 0; j < n; ++j) {
            if (j == i) continue;
            const double q = orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam);
            s_abs += fabs(q);
            const long J = j / block;
            if (J == I || tm[J] > tau) s_mu += q * mu[j];
        }
        R[k] = s_abs;
        diag[k] = orc_q_diag(s_abs, lam, C, diag_rule, delta);
        r[k] = 1.0 - diag[k] * mu[i] - s_mu;
    }
    return ORC_OK;
}

/* r = b - Q mu, returns ||r||_inf.  The paper's Step 3 tests the messages for
 * convergence without naming a norm; the reading used throughout is the
 * infinity norm of the linear-system residual of the current means. */
static double residual(const double* Q, const double* b, const double* mu, long n, double* r)
{
    double rmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : rmax)
    for (long i = 0; i < n; ++i) {
        double s = b[i];
        for (long j = 0; j < n; ++j) s -= Q[i * n + j] * mu[j];
        if (r) r[i] = s;
        double a = fabs(s);
        if (a > rmax || a != a) rmax = (a != a) ? INFINITY : a;
    }
    return rmax;
}

/*
 * Algorithm 2 (broadcast GaBP, Section 4), synchronous schedule, written in
 * information form.  For every ordered pair the message i->j carries a
 * precision P_ij and a mean mu_ij; here H_ij = P_ij mu_ij is stored instead of
 * mu_ij, which is the same message and never divides by Q_ij.
 *
 *   Step 1 (init):  P_ii = Q_ii, mu_ii = b_i / Q_ii, all messages 0.
 *   Step 2:         Ptilde_i = P_ii + sum_k P_ki,
 *                   htilde_i = P_ii mu_ii + sum_k H_ki   (= b_i + sum_k H_ki),
 *                   mutilde_i = htilde_i / Ptilde_i;
 *                   P_ij <- -Q_ij^2 / (Ptilde_i - P_ji),
 *                   mu_ij <- (Ptilde_i mutilde_i - P_ji mu_ji) / Q_ij, i.e.
 *                   H_ij <- -Q_ij (htilde_i - H_ji) / (Ptilde_i - P_ji).
 *   Step 3:         stop once ||b - Q mutilde||_inf < tol.
 *   Steps 4-5:      mu_i = mutilde_i is the solution.
 *
 * Counting: t = number of synchronous message updates done.  For t = 0, 1, ..
 * the aggregates and r(t) are formed; the loop stops at the first t with
 * ||r(t)||_inf < tol (kstar = t) or at t = iters (kstar = iters); otherwise
 * all messages are updated from the aggregates of t.
 *
 * State layout: Pin[i*n + k] = P_ki, Hin[i*n + k] = H_ki (messages INTO node
 * i), so an aggregate is a row sum.  Callers may pass Pin/Hin (n*n doubles)
 * to read the final messages back, else they are allocated here.
 * Outputs: mu (n), Pt (n, may be NULL), kstar, rinf = ||r(kstar)||_inf,
 * rhist[t] = ||r(t)||_inf for t = 0..kstar (may be NULL; iters+1 entries).
 */
int orc_gabp_info(const double* Q, const double* b, long n, int iters, double tol,
                  double* mu, double* Pt_out, int* kstar, double* rinf,
                  double* rhist, double* Pin_io, double* Hin_io)
{
    if (n < 1 || iters < 0) return ORC_EINVAL;
    size_t nn = (size_t)n * (size_t)n;
    double* Pin = Pin_io ? Pin_io : (double*)malloc(nn * sizeof(double));
    double* Hin = Hin_io ? Hin_io : (double*)malloc(nn * sizeof(double));
    double* Pt = (double*)malloc((size_t)n * sizeof(double));
    double* ht = (double*)malloc((size_t)n * sizeof(double));
    int rc = ORC_OK;
    if (!Pin || !Hin || !Pt || !ht) { rc = ORC_ENOMEM; goto done; }
    memset(Pin, 0, nn * sizeof(double));
    memset(Hin, 0, nn * sizeof(double));

    for (int t = 0;; ++t) {
        /* Step 2, broadcast aggregates. */
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) {
            double P = Q[i * n + i], h = b[i];
            for (long k = 0; k < n; ++k) {
                if (k == i) continue;
                P += Pin[i * n + k];
                h += Hin[i * n + k];
            }
            Pt[i] = P;
            ht[i] = h;
            mu[i] = h / P;
        }
        /* Step 3, convergence check on the residual of the means. */
        double rn = residual(Q, b, mu, n, NULL);
        if (rhist) rhist[t] = rn;
        if (rn < tol || t == iters) {
            *kstar = t;
            *rinf = rn;
            break;
        }
        /* Step 2, message update: every unordered pair {i<j} from the old
         * messages of that pair and the aggregates of this round. */
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
        for (long i = 0; i < n; ++i) {
            for (long j = i + 1; j < n; ++j) {
                double q = Q[i * n + j];
                double P_ij = Pin[j * n + i], P_ji = Pin[i * n + j];
                double H_ij = Hin[j * n + i], H_ji = Hin[i * n + j];
                double di = Pt[i] - P_ji;   /* cavity precision P_{i\j} */
                double dj = Pt[j] - P_ij;   /* cavity precision P_{j\i} */
                if (!(di > 0.0) || !(dj > 0.0) || !isfinite(di) || !isfinite(dj)) bad = 1;
                Pin[j * n + i] = -q * q / di;
                Hin[j * n + i] = -q * (ht[i] - H_ji) / di;
                Pin[i * n + j] = -q * q / dj;
                Hin[i * n + j] = -q * (ht[j] - H_ij) / dj;
            }
        }
        if (bad) { rc = ORC_ENUMERIC; *kstar = t; *rinf = rn; break; }
    }
    if (Pt_out) memcpy(Pt_out, Pt, (size_t)n * sizeof(double));
done:
    if (!Pin_io) free(Pin);
    if (!Hin_io) free(Hin);
    free(Pt);
    free(ht);
    return rc;
}

/*
 * Stage boundaries of the block Gauss-Seidel schedule below: nodes form
 * blocks of `block` consecutive indices (Nt blocks); B[0] = 0, B[S] = Nt and
 * B[s] is the smallest b with S * b (b + 1) / 2 >= s * Nt (Nt + 1) / 2, so
 * that the stages hold about equal numbers of block pairs (J, I <= J).
 */
void orc_stage_bounds(long Nt, int S, long* B)
{
    const long tot = Nt * (Nt + 1) / 2;
    B[0] = 0;
    for (int s = 1; s < S; ++s) {
        long b = B[s - 1];
        while (b < Nt && (long)S * (b * (b + 1) / 2) < (long)s * tot) ++b;
        B[s] = b;
    }
    B[S] = Nt;
}

/*
 * Algorithm 2 under a block Gauss-Seidel schedule.  Section 3.2 shows that
 * GaBP also converges when messages are not all updated together, and the
 * paper names asynchronous schedules as the faster ones.  Here one round still
 * updates every pair exactly once, in S stages: with node blocks as in
 * orc_stage_bounds, the pair {i < j} is updated in the stage whose range
 * [B[s], B[s+1]) holds the block of j.  A stage updates its pairs from the
 * current aggregates (Step 2, information form as in orc_gabp_info), and the
 * aggregates are formed again from all messages before the next stage, so
 * later stages see the messages of earlier ones.  The residual test of Step 3
 * is taken at the start of every round, on the aggregates of all messages.
 * S = 1 is the synchronous schedule of orc_gabp_info.  Arguments and outputs
 * as for orc_gabp_info.
 */
int orc_gabp_staged(const double* Q, const double* b, long n, int iters, double tol, int S, long block,
                    double* mu, double* Pt_out, int* kstar, double* rinf, double* rhist,
                    double* Pin_io, double* Hin_io)
{
    if (n < 1 || iters < 0 || S < 1 || block < 1) return ORC_EINVAL;
    const long Nt = (n + block - 1) / block;
    size_t nn = (size_t)n * (size_t)n;
    double* Pin = Pin_io ? Pin_io : (double*)malloc(nn * sizeof(double));
    double* Hin = Hin_io ? Hin_io : (double*)malloc(nn * sizeof(double));
    double* Pt = (double*)malloc((size_t)n * sizeof(double));
    double* ht = (double*)malloc((size_t)n * sizeof(double));
    long* B = (long*)malloc((size_t)(S + 1) * sizeof(long));
    int rc = ORC_OK;
    if (!Pin || !Hin || !Pt || !ht || !B) { rc = ORC_ENOMEM; goto done; }
    memset(Pin, 0, nn * sizeof(double));
    memset(Hin, 0, nn * sizeof(double));
    orc_stage_bounds(Nt, S, B);

    for (int t = 0;; ++t) {
        /* aggregates of all messages (Step 2) and the residual test (Step 3) */
        for (long i = 0; i < n; ++i) {
            double P = Q[i * n + i], h = b[i];
            for (long k = 0; k < n; ++k) {
                if (k == i) continue;
                P += Pin[i * n + k];
                h += Hin[i * n + k];
            }
            Pt[i] = P;
            ht[i] = h;
            mu[i] = h / P;
        }
        double rn = residual(Q, b, mu, n, NULL);
        if (rhist) rhist[t] = rn;
        if (rn < tol || t == iters) {
            *kstar = t;
            *rinf = rn;
            break;
        }
        int bad = 0;
        for (int s = 0; s < S; ++s) {
            const long j0 = B[s] * block, j1 = B[s + 1] * block < n ? B[s + 1] * block : n;
            /* the pairs {i < j} with j in this stage's blocks */
            for (long j = j0; j < j1; ++j) {
                for (long i = 0; i < j; ++i) {
                    double q = Q[i * n + j];
                    double P_ij = Pin[j * n + i], P_ji = Pin[i * n + j];
                    double H_ij = Hin[j * n + i], H_ji = Hin[i * n + j];
                    double di = Pt[i] - P_ji;
                    double dj = Pt[j] - P_ij;
                    if (!(di > 0.0) || !(dj > 0.0) || !isfinite(di) || !isfinite(dj)) bad = 1;
                    Pin[j * n + i] = -q * q / di;
                    Hin[j * n + i] = -q * (ht[i] - H_ji) / di;
                    Pin[i * n + j] = -q * q / dj;
                    Hin[i * n + j] = -q * (ht[j] - H_ij) / dj;
                }
            }
            /* aggregates again, for the next stage */
            for (long i = 0; i < n; ++i) {
                double P = Q[i * n + i], h = b[i];
                for (long k = 0; k < n; ++k) {
                    if (k == i) continue;
                    P += Pin[i * n + k];
                    h += Hin[i * n + k];
                }
                Pt[i] = P;
                ht[i] = h;
            }
        }
        if (bad) { rc = ORC_ENUMERIC; *kstar = t; *rinf = rn; break; }
    }
    if (Pt_out) memcpy(Pt_out, Pt, (size_t)n * sizeof(double));
done:
    if (!Pin_io) free(Pin);
    if (!Hin_io) free(Hin);
    free(Pt);
    free(ht);
    free(B);
    return rc;
}

/*
 * Algorithm 2 exactly as printed, with the message means mu_ij as state:
 *   mu_ij <- (Ptilde_i mutilde_i - P_ji mu_ji) / Q_ij.
 * Only pairs with Q_ij != 0 are neighbours (Step 1).  Runs `iters` updates
 * and returns the means and precisions formed from the final messages.
 */
int orc_gabp_literal(const double* Q, const double* b, long n, int iters,
                     double* mu, double* Pt_out)
{
    size_t nn = (size_t)n * (size_t)n;
    double* Pin = (double*)calloc(nn, sizeof(double));   /* Pin[i*n+k] = P_ki */
    double* Min = (double*)calloc(nn, sizeof(double));   /* Min[i*n+k] = mu_ki */
    double* Pt = (double*)malloc((size_t)n * sizeof(double));
    double* mt = (double*)malloc((size_t)n * sizeof(double));
    int rc = ORC_OK;
    if (!Pin || !Min || !Pt || !mt) { rc = ORC_ENOMEM; goto done; }
    for (int t = 0;; ++t) {
        for (long i = 0; i < n; ++i) {
            double Pii = Q[i * n + i], muii = b[i] / Pii;
            double P = Pii, s = Pii * muii;
            for (long k = 0; k < n; ++k) {
                if (k == i || Q[k * n + i] == 0.0) continue;
                P += Pin[i * n + k];
                s += Pin[i * n + k] * Min[i * n + k];
            }
            Pt[i] = P;
            mt[i] = s / P;
        }
        if (t == iters) break;
        for (long i = 0; i < n; ++i) {
            for (long j = i + 1; j < n; ++j) {
                double q = Q[i * n + j];
                if (q == 0.0) continue;
                double P_ij = Pin[j * n + i], P_ji = Pin[i * n + j];
                double m_ij = Min[j * n + i], m_ji = Min[i * n + j];
                double di = Pt[i] - P_ji, dj = Pt[j] - P_ij;
                if (!(di > 0.0) || !(dj > 0.0)) rc = ORC_ENUMERIC;
                Pin[j * n + i] = -q * q / di;
                Min[j * n + i] = (Pt[i] * mt[i] - P_ji * m_ji) / q;
                Pin[i * n + j] = -q * q / dj;
                Min[i * n + j] = (Pt[j] * mt[j] - P_ij * m_ij) / q;
            }
        }
    }
    memcpy(mu, mt, (size_t)n * sizeof(double));
    if (Pt_out) memcpy(Pt_out, Pt, (size_t)n * sizeof(double));
done:
    free(Pin); free(Min); free(Pt); free(mt);
    return rc;
}

/*
 * Algorithm 1 (pairwise GaBP, Section 2), synchronous: every message i->j is
 * formed from the explicit exclusion sums over N(i) \ j of the previous
 * round's messages,
 *   P_ij  = -Q_ij^2 / (P_ii + sum_{k in N(i)\j} P_ki),
 *   mu_ij = (P_ii mu_ii + sum_{k in N(i)\j} P_ki mu_ki) / Q_ij,
 * and Step 4 infers mu_i from all incoming messages.  O(n^3) per round: only
 * for small n.
 */
int orc_gabp_alg1(const double* Q, const double* b, long n, int iters,
                  double* mu, double* Pt_out)
{
    size_t nn = (size_t)n * (size_t)n;
    double* P = (double*)calloc(nn, sizeof(double));     /* P[k*n+i] = P_ki */
    double* M = (double*)calloc(nn, sizeof(double));     /* M[k*n+i] = mu_ki */
    double* P2 = (double*)calloc(nn, sizeof(double));
    double* M2 = (double*)calloc(nn, sizeof(double));
    int rc = ORC_OK;
    if (!P || !M || !P2 || !M2) { rc = ORC_ENOMEM; goto done; }
    for (int t = 0; t < iters; ++t) {
        for (long i = 0; i < n; ++i) {
            double Pii = Q[i * n + i], muii = b[i] / Pii;
            for (long j = 0; j < n; ++j) {
                if (j == i || Q[i * n + j] == 0.0) continue;
                double Ps = Pii, ms = Pii * muii;
                for (long k = 0; k < n; ++k) {
                    if (k == i || k == j || Q[k * n + i] == 0.0) continue;
                    Ps += P[k * n + i];
                    ms += P[k * n + i] * M[k * n + i];
                }
                if (!(Ps > 0.0)) rc = ORC_ENUMERIC;
                double q = Q[i * n + j];
                P2[i * n + j] = -q * q / Ps;
                M2[i * n + j] = ms / q;
            }
        }
        double* tp = P; P = P2; P2 = tp;
        double* tm = M; M = M2; M2 = tm;
    }
    for (long i = 0; i < n; ++i) {
        double Pii = Q[i * n + i], muii = b[i] / Pii;
        double Ps = Pii, ms = Pii * muii;
        for (long k = 0; k < n; ++k) {
            if (k == i || Q[k * n + i] == 0.0) continue;
            Ps += P[k * n + i];
            ms += P[k * n + i] * M[k * n + i];
        }
        mu[i] = ms / Ps;
        if (Pt_out) Pt_out[i] = Ps;
    }
done:
    free(P); free(M); free(P2); free(M2);
    return rc;
}

/* One pair's synchronous information-form update (the inner step of
 * orc_gabp_info), exposed so that a caller holding a solver's state for a few
 * sampled pairs can recompute them one by one.
 * in: q = Q_ij, Pt_i, ht_i, Pt_j, ht_j, msg = {P_ij, P_ji, H_ij, H_ji}
 * out: the new {P_ij, P_ji, H_ij, H_ji}. */
void orc_pair_update(double q, double Pt_i, double ht_i, double Pt_j, double ht_j,
                     const double* msg, double* out)
{
    double di = Pt_i - msg[1], dj = Pt_j - msg[0];
    out[0] = -q * q / di;
    out[1] = -q * q / dj;
    out[2] = -q * (ht_i - msg[3]) / di;
    out[3] = -q * (ht_j - msg[2]) / dj;
}

/* Fixed point of GaBP: the mean of N(Q^-1 b, Q^-1) (Section 2), by an FP64
 * Cholesky factorisation Q = L L^T and two triangular solves. */
int orc_cholesky_solve(const double* Q, const double* b, long n, double* x)
{
    double* L = (double*)calloc((size_t)n * (size_t)n, sizeof(double));
    if (!L) return ORC_ENOMEM;
    for (long j = 0; j < n; ++j) {
        double s = Q[j * n + j];
        for (long k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) { free(L); return ORC_ENUMERIC; }
        L[j * n + j] = sqrt(s);
        for (long i = j + 1; i < n; ++i) {
            double v = Q[i * n + j];
            for (long k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = v / L[j * n + j];
        }
    }
    for (long i = 0; i < n; ++i) {          /* L z = b */
        double s = b[i];
        for (long k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (long i = n - 1; i >= 0; --i) {     /* L^T x = z */
        double s = x[i];
        for (long k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
    free(L);
    return ORC_OK;
}

/* Row i of the SVM matrix, formed on the fly from X (the diagonal by the same
 * rule as orc_build_q).  O(n m) per row, O(n) memory. */
void orc_q_row(const double* X, const double* y, long n, long m, double gamma,
               double lam, double C, int diag_rule, double delta, long i, double* row)
{
    double R = 0.0;
    for (long j = 0; j < n; ++j) {
        if (j == i) continue;
        row[j] = orc_q_offdiag(X + i * m, X + j * m, y[i], y[j], m, gamma, lam);
        R += fabs(row[j]);
    }
    row[i] = orc_q_diag(R, lam, C, diag_rule, delta);
}

/* Matrix-free FP64 conjugate gradients on Q alpha = b, with Q's rows formed on
 * the fly (orc_q_row), for sizes whose dense Q does not fit in host memory.
 * Stops when ||b - Q x||_2 <= rtol ||b||_2 or after maxit iterations; returns
 * the iteration count in *its. */
int orc_cg_rbf(const double* X, const double* y, long n, long m, double gamma,
               double lam, double C, int diag_rule, double delta, const double* b,
               double rtol, int maxit, double* x, int* its)
{
    double* r = (double*)malloc((size_t)n * sizeof(double));
    double* p = (double*)malloc((size_t)n * sizeof(double));
    double* Ap = (double*)malloc((size_t)n * sizeof(double));
    if (!r || !p || !Ap) { free(r); free(p); free(Ap); return ORC_ENOMEM; }
    double bn = 0.0;
    for (long i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; bn += b[i] * b[i]; }
    double rr = bn;
    int k = 0;
    for (; k < maxit && sqrt(rr) > rtol * sqrt(bn); ++k) {
#pragma omp parallel
        {
            double* row = (double*)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(static)
            for (long i = 0; i < n; ++i) {
                orc_q_row(X, y, n, m, gamma, lam, C, diag_rule, delta, i, row);
                double s = 0.0;
                for (long j = 0; j < n; ++j) s += row[j] * p[j];
                Ap[i] = s;
            }
            free(row);
        }
        double pAp = 0.0;
        for (long i = 0; i < n; ++i) pAp += p[i] * Ap[i];
        double a = rr / pAp, rr2 = 0.0;
        for (long i = 0; i < n; ++i) { x[i] += a * p[i]; r[i] -= a * Ap[i]; rr2 += r[i] * r[i]; }
        double beta = rr2 / rr;
        rr = rr2;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    *its = k;
    free(r); free(p); free(Ap);
    return ORC_OK;
}

/* Dual objective L_D(h) = sum_i h_i - 1/2 h' Q h (Section 1.1, dual). */
double orc_dual_objective(const double* Q, const double* h, long n)
{
    double quad = 0.0, lin = 0.0;
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (long j = 0; j < n; ++j) s += Q[i * n + j] * h[j];
        quad += h[i] * s;
        lin += h[i];
    }
    return lin - 0.5 * quad;
}

/* Decision values f(x) = sum_i h_i y_i K'(x_i, x) (Section 1.1), with the bias
 * carried by the lambda^2 term of K' (Section 3), for t test rows Xt. */
int orc_decision(const double* X, const double* y, const double* h, long n, long m,
                 const double* Xt, long t, double gamma, double lam, double* f)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < t; ++s) {
        double acc = 0.0;
        for (long i = 0; i < n; ++i)
            acc += h[i] * y[i] * (rbf(X + i * m, Xt + s * m, m, gamma) + lam * lam);
        f[s] = acc;
    }
    return ORC_OK;
}

/* Box-constrained dual without the equality constraint,
 *   min 1/2 a'Qa - 1'a  subject to 0 <= a_i <= C,
 * by brute force over the 3^n active sets (each index at 0, at C or free):
 * for each set solve the free block, keep the candidates that satisfy every
 * KKT condition, return the one with the lowest objective.  n <= 12. */
static int small_solve(double* A, double* rhs, int k)
{
    /* Gaussian elimination with partial pivoting, k <= 12, in place. */
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[r * k + c]) > fabs(A[p * k + c])) p = r;
        if (A[p * k + c] == 0.0) return 1;
        if (p != c) {
            for (int q = 0; q < k; ++q) { double t = A[c * k + q]; A[c * k + q] = A[p * k + q]; A[p * k + q] = t; }
            double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
        }
        for (int r = c + 1; r < k; ++r) {
            double f = A[r * k + c] / A[c * k + c];
            for (int q = c; q < k; ++q) A[r * k + q] -= f * A[c * k + q];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int r = k - 1; r >= 0; --r) {
        double s = rhs[r];
        for (int q = r + 1; q < k; ++q) s -= A[r * k + q] * rhs[q];
        rhs[r] = s / A[r * k + r];
    }
    return 0;
}

int orc_boxqp_bruteforce(const double* Q, long n, double C, double kkt_tol,
                         double* alpha, int* n_kkt)
{
    if (n < 1 || n > 12) return ORC_EINVAL;
    long total = 1;
    for (long i = 0; i < n; ++i) total *= 3;
    double best = INFINITY;
    int found = 0;
    double a[12], g[12], A[144], rhs[12];
    int st[12], fidx[12];
    for (long code = 0; code < total; ++code) {
        long c = code;
        int k = 0;
        for (long i = 0; i < n; ++i) { st[i] = (int)(c % 3); c /= 3; if (st[i] == 2) fidx[k++] = (int)i; }
        for (long i = 0; i < n; ++i) a[i] = st[i] == 1 ? C : 0.0;
        if (k > 0) {
            for (int r = 0; r < k; ++r) {
                long i = fidx[r];
                double s = 1.0;
                for (long j = 0; j < n; ++j) if (st[j] == 1) s -= Q[i * n + j] * C;
                rhs[r] = s;
                for (int q = 0; q < k; ++q) A[r * k + q] = Q[i * n + fidx[q]];
            }
            if (small_solve(A, rhs, k)) continue;
            for (int r = 0; r < k; ++r) a[fidx[r]] = rhs[r];
        }
        int ok = 1;
        for (long i = 0; i < n && ok; ++i) {
            double s = -1.0;
            for (long j = 0; j < n; ++j) s += Q[i * n + j] * a[j];
            g[i] = s;
            if (st[i] == 2 && (a[i] < -kkt_tol || a[i] > C + kkt_tol)) ok = 0;
            if (st[i] == 0 && g[i] < -kkt_tol) ok = 0;
            if (st[i] == 1 && g[i] > kkt_tol) ok = 0;
        }
        if (!ok) continue;
        /* 1/2 a'Qa - 1'a = 1/2 a'(Qa - 1) - 1/2 1'a, with g = Qa - 1 */
        double obj = 0.0;
        for (long i = 0; i < n; ++i) obj += 0.5 * a[i] * g[i] - 0.5 * a[i];
        ++found;
        if (obj < best) { best = obj; memcpy(alpha, a, (size_t)n * sizeof(double)); }
    }
    *n_kkt = found;
    return found ? ORC_OK : ORC_ENUMERIC;
}
