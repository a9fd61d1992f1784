/*
 * sap_oracle.c -- plain, slow FP64 CPU oracle for the Secant-Avoidance
 * Projection (SAP) algorithm of Kvinge, Farnell, Kirby and Peterson,
 * "A GPU-Oriented Algorithm Design for Secant-Based Dimensionality Reduction"
 * (arXiv:1807.03425).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness bar for the CUDA
 * library; it shares no code, header, table or helper with it.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * The product path never calls it.
 *
 * Notation (the paper's letters are remapped so that N counts points):
 *   X  N x n, row-major, point x_i = X[i*n .. i*n+n-1]          (Sec. IV)
 *   U  n x k, column-major, column c = U[c*n .. c*n+n-1]; the paper's P^(i)
 *   pair (i,j) with i<j, index p(i,j) = i*N - i(i+1)/2 + (j-i-1)
 *   unit secant s = (x_i - x_j)/||x_i - x_j||                   (Sec. IV)
 *   ratio r_ij = ||U^T s||, the projected length of the unit secant
 *
 * Everything is FP64.  Inputs given in FP32/BF16 are widened exactly by the
 * caller.  Loops are plain; OpenMP only splits the outer row loop, and every
 * reduction is finished serially in row order so results do not depend on the
 * thread count.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - "distinct points" (Sec. II): a pair with x_i == x_j is excluded.
 *  - noisy-data variant (Sec. VII): a secant is discarded when its length is
 *    "less than" the threshold; decided as d^2 < eps^2 in FP64, so d == eps
 *    is kept.
 *  - ties in the argmin step of Algorithm 1: smallest pair index; ties in
 *    the pivot (argmax) step: smallest column index.  If all <p_l, s> are zero, t = 1 (Sec. IV).
 *  - update (Algorithm 1, Sec. IV): literal reading, the direction
 *    (1-a) P P^T s + a (s - P P^T s) with unnormalised terms; an alternative
 *    "angle" reading blends the two unit vectors instead.
 *  - if P P^T s == 0 the first MGS vector is zero: it is skipped, so
 *    p_2..p_m are the remaining columns orthonormalised on their own.
 *  - the loop-counter update printed in Algorithm 1 as "i+1 <- i" is read
 *    as i <- i+1.
 *  - after the update one more MGS pass re-orthonormalises the basis (a no-op
 *    in exact arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MODE_LITERAL 0
#define ORC_MODE_ANGLE 1

int64_t orc_pair_index(int64_t i, int64_t j, int64_t N)
{
    return i * N - i * (i + 1) / 2 + (j - i - 1);
}

/* Squared length of x_i - x_j, from explicit FP64 differences. */
static double secant_len2(const double *X, int n, int64_t i, int64_t j)
{
    double d2 = 0.0;
    for (int l = 0; l < n; ++l) {
        double D = X[i * n + l] - X[j * n + l];
        d2 += D * D;
    }
    return d2;
}

/* Is the pair kept?  Distinct points only (Sec. II) and, for the noisy-data
 * variant, length not less than eps (Sec. VII). */
static int pair_kept(double d2, double eps)
{
    if (d2 == 0.0) return 0;
    if (eps > 0.0 && d2 < eps * eps) return 0;
    return 1;
}

/* Projected length ||U^T s|| of the unit secant of pair (i,j) (Sec. IV:
 * "the l2-norms of all secants under the current projection").  Returns -1
 * for an excluded pair. */
double orc_ratio(const double *X, int64_t N, int n, const double *U, int k,
                 int64_t i, int64_t j, double eps)
{
    (void)N;
    double d2 = secant_len2(X, n, i, j);
    if (!pair_kept(d2, eps)) return -1.0;
    double d = sqrt(d2);
    double acc = 0.0;
    for (int c = 0; c < k; ++c) {
        double z = 0.0;
        for (int l = 0; l < n; ++l) {
            double s_l = (X[i * n + l] - X[j * n + l]) / d;
            z += U[(int64_t)c * n + l] * s_l;
        }
        acc += z * z;
    }
    return sqrt(acc);
}

/* All P ratios in pair-index order (excluded pairs get -1).  For small N. */
void orc_all_ratios(const double *X, int64_t N, int n, const double *U, int k,
                    double eps, double *out)
{
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j)
            out[orc_pair_index(i, j, N)] = orc_ratio(X, N, n, U, k, i, j, eps);
}

/*
 * Algorithm 1, argmin step: the secant with the smallest projected length.
 * Outputs the argmin pair (ties -> smallest pair index), its ratio, the
 * second-smallest ratio over all kept pairs (the runner-up, equal to the min
 * on a tie) and the number of excluded pairs.  Returns 0, or -1 when every
 * pair is excluded.
 */
int orc_min_secant(const double *X, int64_t N, int n, const double *U, int k,
                   double eps, int64_t *i_out, int64_t *j_out, double *r_out,
                   double *r2_out, int64_t *n_excluded)
{
    double *best = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *second = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int64_t *bestj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t *excl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double b = INFINITY, s2 = INFINITY;
        int64_t bj = -1, ex = 0;
        for (int64_t j = i + 1; j < N; ++j) {
            double r = orc_ratio(X, N, n, U, k, i, j, eps);
            if (r < 0.0) { ++ex; continue; }
            if (r < b) { s2 = b; b = r; bj = j; }
            else if (r < s2) { s2 = r; }
        }
        best[i] = b; second[i] = s2; bestj[i] = bj; excl[i] = ex;
    }

    /* global minimum; rows are visited in increasing i and each row's best
     * is its smallest j, so a strict "<" keeps the smallest pair index */
    double gb = INFINITY;
    int64_t gi = -1, gj = -1, gex = 0;
    for (int64_t i = 0; i < N; ++i) {
        gex += excl[i];
        if (bestj[i] >= 0 && best[i] < gb) { gb = best[i]; gi = i; gj = bestj[i]; }
    }
    /* runner-up: the second value of the winning row, or another row's best */
    double gs = gi >= 0 ? second[gi] : INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (i != gi) gs = fmin(gs, best[i]);
    free(best); free(second); free(bestj); free(excl);
    if (n_excluded) *n_excluded = gex;
    if (gi < 0) return -1;
    *i_out = gi; *j_out = gj; *r_out = gb;
    if (r2_out) *r2_out = gs;
    return 0;
}

static double dot(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += a[l] * b[l];
    return s;
}

/* One modified Gram-Schmidt sweep over m vectors of length n stored one after
 * another in V (vector a at V + a*n), in place.  A vector whose norm is
 * exactly zero is marked dead (flag 0) and skipped by later projections. */
static void mgs(double *V, int m, int n, int *alive)
{
    for (int a = 0; a < m; ++a) {
        double *w = V + (int64_t)a * n;
        for (int b = 0; b < a; ++b) {
            if (!alive[b]) continue;
            const double *q = V + (int64_t)b * n;
            double h = dot(q, w, n);
            for (int l = 0; l < n; ++l) w[l] -= h * q[l];
        }
        double nrm = sqrt(dot(w, w, n));
        if (nrm == 0.0) { alive[a] = 0; continue; }
        alive[a] = 1;
        for (int l = 0; l < n; ++l) w[l] /= nrm;
    }
}

/*
 * Algorithm 1, update steps (prose in Sec. IV): rotate the basis towards the unit
 * secant s.  U and Unew are n x k column-major; they may not alias.
 * Writes the pivot column t (0-based) to *t_out when non-null.
 */
void orc_update_with_secant(const double *s, const double *U, int n, int k,
                            double alpha, int mode, double *Unew, int *t_out)
{
    double *c = (double *)malloc(sizeof(double) * (size_t)k);
    double *v = (double *)calloc((size_t)n, sizeof(double));
    double *L = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k);
    int *alive = (int *)malloc(sizeof(int) * (size_t)k);

    /* <p_l, s> for every column, and the projection P P^T s in R^n */
    for (int l = 0; l < k; ++l) c[l] = dot(U + (int64_t)l * n, s, n);
    for (int l = 0; l < k; ++l)
        for (int q = 0; q < n; ++q) v[q] += c[l] * U[(int64_t)l * n + q];

    /* pivot step: the column with the largest |<p_l, s>| (first on ties); if all
     * are zero, the first column */
    int t = 0;
    double cmax = fabs(c[0]);
    for (int l = 1; l < k; ++l)
        if (fabs(c[l]) > cmax) { cmax = fabs(c[l]); t = l; }
    if (t_out) *t_out = t;

    /* Gram-Schmidt step: MGS on the ordered list P P^T s, p_1..p_{t-1}, p_{t+1}..p_m */
    memcpy(L, v, sizeof(double) * (size_t)n);
    int a = 1;
    for (int l = 0; l < k; ++l) {
        if (l == t) continue;
        memcpy(L + (int64_t)a * n, U + (int64_t)l * n, sizeof(double) * (size_t)n);
        ++a;
    }
    mgs(L, k, n, alive);

    /* rotation step: new first column along (1-a) P P^T s + a (s - P P^T s) */
    double *dir = (double *)malloc(sizeof(double) * (size_t)n);
    if (mode == ORC_MODE_ANGLE) {
        double nv = sqrt(dot(v, v, n));
        double ne2 = 0.0;
        for (int q = 0; q < n; ++q) { double e = s[q] - v[q]; ne2 += e * e; }
        double ne = sqrt(ne2);
        for (int q = 0; q < n; ++q) {
            double vh = nv > 0.0 ? v[q] / nv : 0.0;
            double eh = ne > 0.0 ? (s[q] - v[q]) / ne : 0.0;
            dir[q] = (1.0 - alpha) * vh + alpha * eh;
        }
    } else {
        for (int q = 0; q < n; ++q)
            dir[q] = (1.0 - alpha) * v[q] + alpha * (s[q] - v[q]);
    }
    double nd = sqrt(dot(dir, dir, n));
    if (nd > 0.0) {
        for (int q = 0; q < n; ++q) Unew[q] = dir[q] / nd;
    } else if (alive[0]) {
        /* alpha = 1 with s already in the span: keep the normalised P P^T s */
        memcpy(Unew, L, sizeof(double) * (size_t)n);
    } else {
        memcpy(Unew, s, sizeof(double) * (size_t)n);
    }
    for (int l = 1; l < k; ++l)
        memcpy(Unew + (int64_t)l * n, L + (int64_t)l * n, sizeof(double) * (size_t)n);

    /* re-orthonormalisation: one more MGS pass over the new basis */
    mgs(Unew, k, n, alive);

    free(c); free(v); free(L); free(alive); free(dir);
}

/* The unit secant of pair (i,j), s = (x_i - x_j)/||x_i - x_j|| (Sec. IV). */
void orc_unit_secant(const double *X, int n, int64_t i, int64_t j, double *s)
{
    double d = sqrt(secant_len2(X, n, i, j));
    for (int l = 0; l < n; ++l) s[l] = (X[i * n + l] - X[j * n + l]) / d;
}

void orc_update(const double *X, int64_t N, int n, const double *U, int k,
                int64_t i, int64_t j, double alpha, int mode, double *Unew,
                int *t_out)
{
    (void)N;
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    orc_unit_secant(X, n, i, j, s);
    orc_update_with_secant(s, U, n, k, alpha, mode, Unew, t_out);
    free(s);
}

/*
 * Algorithm 1, main loop: T iterations from U0.  Each iteration evaluates the
 * current basis (argmin step) and updates it (pivot, MGS, rotation).  hist[0..T] holds the
 * min ratio of U_0..U_T (T+1 evaluations); argmin[2*it], argmin[2*it+1] the
 * pair found at evaluation it.  U_out receives U_T.  Returns 0, or -1 when
 * every pair is excluded.
 */
int orc_run(const double *X, int64_t N, int n, const double *U0, int k,
            double alpha, int T, double eps, int mode, double *U_out,
            double *hist, int64_t *argmin)
{
    size_t ub = sizeof(double) * (size_t)n * (size_t)k;
    double *U = (double *)malloc(ub);
    double *Un = (double *)malloc(ub);
    memcpy(U, U0, ub);
    int rc = 0;
    for (int it = 0; it <= T; ++it) {
        int64_t i, j;
        double r;
        if (orc_min_secant(X, N, n, U, k, eps, &i, &j, &r, NULL, NULL) != 0) {
            rc = -1;
            break;
        }
        if (hist) hist[it] = r;
        if (argmin) { argmin[2 * it] = i; argmin[2 * it + 1] = j; }
        if (it == T) break;
        orc_update(X, N, n, U, k, i, j, alpha, mode, Un, NULL);
        double *tmp = U; U = Un; Un = tmp;
    }
    memcpy(U_out, U, ub);
    free(U); free(Un);
    return rc;
}

/*
 * Dimension estimation (Sec. VI-A): run SAP for every target dimension
 * k = 1..kmax, starting from the first k columns of U0full (n x kmax,
 * column-major), and report the min ratio of the final basis for each k.
 * k_out = smallest k whose ratio exceeds threshold, or -1.
 */
int orc_estimate_dim(const double *X, int64_t N, int n, const double *U0full,
                     int kmax, int T, double alpha, double eps, int mode,
                     double threshold, double *ratios, int *k_out)
{
    double *Ut = (double *)malloc(sizeof(double) * (size_t)n * (size_t)kmax);
    double *hist = (double *)malloc(sizeof(double) * (size_t)(T + 1));
    *k_out = -1;
    int rc = 0;
    for (int k = 1; k <= kmax; ++k) {
        if (orc_run(X, N, n, U0full, k, alpha, T, eps, mode, Ut, hist, NULL) != 0) {
            rc = -1;
            break;
        }
        ratios[k - 1] = hist[T];
        if (*k_out < 0 && hist[T] > threshold) *k_out = k;
    }
    free(Ut); free(hist);
    return rc;
}

/*
 * Soft-min objective L(U) = -tau * log sum_{i<j} exp(-r_ij / tau) over kept
 * pairs, evaluated with the minimum ratio m as shift:
 *   L = m - tau * log sum exp(-(r_ij - m)/tau),
 * and its gradient dL/dU (n x k, column-major)
 *   G = sum_{i<j} pi_ij * (x_i - x_j) (U^T (x_i - x_j))^T / (d_ij^2 r_ij),
 *   pi_ij = exp(-(r_ij - L)/tau)   (the softmax weights, summing to 1).
 * A pair with r_ij == 0 contributes no gradient (the norm is not
 * differentiable there).  Returns 0, or -1 when every pair is excluded.
 */
int orc_softmin(const double *X, int64_t N, int n, const double *U, int k,
                double tau, double eps, double *L_out, double *G)
{
    /* pass 1: minimum ratio */
    double *rowmin = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double b = INFINITY;
        for (int64_t j = i + 1; j < N; ++j) {
            double r = orc_ratio(X, N, n, U, k, i, j, eps);
            if (r >= 0.0 && r < b) b = r;
        }
        rowmin[i] = b;
    }
    double m = INFINITY;
    for (int64_t i = 0; i < N; ++i) m = fmin(m, rowmin[i]);
    free(rowmin);
    if (!(m < INFINITY)) return -1;

    /* pass 2: shifted sum of exponentials */
    double *rowsum = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int64_t j = i + 1; j < N; ++j) {
            double r = orc_ratio(X, N, n, U, k, i, j, eps);
            if (r >= 0.0) acc += exp(-(r - m) / tau);
        }
        rowsum[i] = acc;
    }
    double S = 0.0;
    for (int64_t i = 0; i < N; ++i) S += rowsum[i];
    free(rowsum);
    double L = m - tau * log(S);
    *L_out = L;
    if (!G) return 0;

    /* pass 3: gradient, one n x k partial per row, summed in row order */
    size_t gsz = (size_t)n * (size_t)k;
    double *Gp = (double *)calloc((size_t)N * gsz, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double *g = Gp + (size_t)i * gsz;
        double *D = (double *)malloc(sizeof(double) * (size_t)n);
        double *z = (double *)malloc(sizeof(double) * (size_t)k);
        for (int64_t j = i + 1; j < N; ++j) {
            double d2 = secant_len2(X, n, i, j);
            if (!pair_kept(d2, eps)) continue;
            for (int l = 0; l < n; ++l) D[l] = X[i * n + l] - X[j * n + l];
            double zz = 0.0;
            for (int c = 0; c < k; ++c) {
                z[c] = dot(U + (int64_t)c * n, D, n);
                zz += z[c] * z[c];
            }
            double r = sqrt(zz / d2);
            if (r == 0.0) continue;
            double coef = exp(-(r - L) / tau) / (d2 * r);
            for (int c = 0; c < k; ++c)
                for (int l = 0; l < n; ++l)
                    g[(size_t)c * n + l] += coef * D[l] * z[c];
        }
        free(D); free(z);
    }
    memset(G, 0, sizeof(double) * gsz);
    for (int64_t i = 0; i < N; ++i)
        for (size_t q = 0; q < gsz; ++q) G[q] += Gp[(size_t)i * gsz + q];
    free(Gp);
    return 0;
}

/*
 * Secant Gram matrix for the PCA initialisation of Algorithm 1 (Sec. IV: the
 * first basis is made of the top k left singular vectors of the n x p matrix
 * S whose columns are the unit secants).  C = S S^T = sum over kept pairs of
 * s s^T, s = (x_i - x_j)/||x_i - x_j||, written out pair by pair (n x n,
 * row-major, symmetric).  Rows of C are summed per thread over i and then in
 * a fixed order.  Returns the number of kept pairs, or -1 if none.
 */
int64_t orc_secant_gram(const double *X, int64_t N, int n, double eps, double *C)
{
    const size_t nn = (size_t)n * n;
    memset(C, 0, sizeof(double) * nn);
    int64_t kept = 0;
    double *Cp = (double *)calloc((size_t)N * nn, sizeof(double));
    int64_t *kp = (int64_t *)calloc((size_t)N, sizeof(int64_t));
#pragma omp parallel
    {
        double *s = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < N; ++i) {
            double *Ci = Cp + (size_t)i * nn;
            for (int64_t j = i + 1; j < N; ++j) {
                const double d2 = secant_len2(X, n, i, j);
                if (!pair_kept(d2, eps)) continue;
                orc_unit_secant(X, n, i, j, s);
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) Ci[(size_t)a * n + b] += s[a] * s[b];
                kp[i] += 1;
            }
        }
        free(s);
    }
    for (int64_t i = 0; i < N; ++i) {
        for (size_t q = 0; q < nn; ++q) C[q] += Cp[(size_t)i * nn + q];
        kept += kp[i];
    }
    free(Cp);
    free(kp);
    return kept > 0 ? kept : -1;
}

/* Number of threads OpenMP will use (reported beside CPU timings). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
