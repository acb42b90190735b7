/*
 * FP64 CPU oracle for the exact nearest-neighbour DTW retrieval cascade of
 * D. Lemire, "Faster Retrieval with a Two-Pass Dynamic-Time-Warping Lower
 * Bound" (arXiv:0811.3301).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Conventions.
 *  - Series are fp32 arrays as the CUDA path receives them; every value is
 *    widened exactly to double on read and all arithmetic is double.
 *  - Indices are 0-based here; the paper's are 1-based (Sec. 2).
 *  - p is 1 or 2 for the retrieval measure (any integer p >= 1 works for the
 *    bounds and DTW); p == 0 selects p = infinity for the DTW recursion only
 *    (Sec. 4), used by the appendix checks.
 *  - w >= n - 1 means no locality constraint (Sec. 4); negative w is invalid.
 *  - "pow" functions return the p-th power (the sum of |.|^p); callers take
 *    the p-th root where the paper's quantity carries it.
 *
 * Parity pins for every function are in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* |a - b|^p for integer p >= 1 (Sec. 2, the l_p norm). */
static double abs_pow(double a, double b, int p)
{
    double d = fabs(a - b);
    if (p == 1)
        return d;
    if (p == 2)
        return d * d;
    return pow(d, (double)p);
}

static int64_t clamp_w(int64_t n, int64_t w)
{
    return w > n ? n : w;
}

/*
 * Warping envelope, Sec. 5 definition:
 *   U(y)_i = max { y_k : |k - i| <= w },  L(y)_i = min { y_k : |k - i| <= w },
 * with k restricted to the series (1..n in the paper).  Computed by the
 * naive window scan, not by the streaming Algorithm 1 of Sec. 6 (whose
 * printed form emits each output one step early).
 */
void oracle_envelope_d(const double *y, int64_t n, int64_t w, double *U, double *L)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo = i - w < 0 ? 0 : i - w;
        int64_t hi = i + w > n - 1 ? n - 1 : i + w;
        double u = y[lo], l = y[lo];
        for (int64_t k = lo; k <= hi; ++k) {
            if (y[k] > u)
                u = y[k];
            if (y[k] < l)
                l = y[k];
        }
        U[i] = u;
        L[i] = l;
    }
}

void oracle_envelope(const float *y, int64_t n, int64_t w, double *U, double *L)
{
    double *yd = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        yd[i] = (double)y[i];
    oracle_envelope_d(yd, n, w, U, L);
    free(yd);
}

/*
 * Projection of x on the envelope (U, L), Eq. (1) of Sec. 7:
 *   H_i = U_i if x_i >= U_i;  L_i if x_i <= L_i;  x_i otherwise.
 */
void oracle_projection(const double *x, const double *U, const double *L, int64_t n, double *H)
{
    for (int64_t i = 0; i < n; ++i) {
        if (x[i] >= U[i])
            H[i] = U[i];
        else if (x[i] <= L[i])
            H[i] = L[i];
        else
            H[i] = x[i];
    }
}

/*
 * LB_Keogh_p(x, y)^p = || x - H(x, y) ||_p^p  (Sec. 7), given the envelope
 * U = U(y), L = L(y).  For p = 1 this is the sum accumulated in Algorithm 2.
 */
double oracle_lb_keogh_pow_d(const double *x, const double *U, const double *L, int64_t n, int p)
{
    double *H = (double *)malloc((size_t)n * sizeof(double));
    oracle_projection(x, U, L, n, H);
    double beta = 0.0;
    for (int64_t i = 0; i < n; ++i)
        beta += abs_pow(x[i], H[i], p);
    free(H);
    return beta;
}

double oracle_lb_keogh_pow(const float *x, const double *U, const double *L, int64_t n, int p)
{
    double *xd = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        xd[i] = (double)x[i];
    double r = oracle_lb_keogh_pow_d(xd, U, L, n, p);
    free(xd);
    return r;
}

/*
 * The second term of LB_Improved (Sec. 8): LB_Keogh_p(y, H(x, y))^p, the
 * distance from y to the envelope, with the same w, of the projection
 * H(x, y) of x onto the envelope U = U(y), L = L(y) (Eq. 1).
 */
double oracle_lb_improved_second_pow(const float *x, const float *y, const double *U, const double *L,
                                     int64_t n, int64_t w, int p)
{
    w = clamp_w(n, w);
    double *xd = (double *)malloc((size_t)n * sizeof(double));
    double *yd = (double *)malloc((size_t)n * sizeof(double));
    double *H = (double *)malloc((size_t)n * sizeof(double));
    double *UH = (double *)malloc((size_t)n * sizeof(double));
    double *LH = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        xd[i] = (double)x[i];
        yd[i] = (double)y[i];
    }
    oracle_projection(xd, U, L, n, H);
    oracle_envelope_d(H, n, w, UH, LH);
    double r = oracle_lb_keogh_pow_d(yd, UH, LH, n, p);
    free(xd);
    free(yd);
    free(H);
    free(UH);
    free(LH);
    return r;
}

/*
 * LB_Improved_p(x, y)^p = LB_Keogh_p(x, y)^p + LB_Keogh_p(y, H(x, y))^p
 * (Sec. 8), U, L the envelope of y.  If first_pass is non-null it receives
 * the first term, LB_Keogh_p(x, y)^p.
 */
double oracle_lb_improved_pow(const float *x, const float *y, const double *U, const double *L,
                              int64_t n, int64_t w, int p, double *first_pass)
{
    double first = oracle_lb_keogh_pow(x, U, L, n, p);
    if (first_pass)
        *first_pass = first;
    return first + oracle_lb_improved_second_pow(x, y, U, L, n, w, p);
}

/*
 * Monotonic, band-constrained DTW_p by the suffix recursion of Sec. 4:
 *   q_{i,j} = 0                     if both suffixes are empty,
 *           = inf                   if exactly one is empty, or |i - j| > w,
 *           = |x_i - y_j|^p + min(q_{i+1,j}, q_{i,j+1}, q_{i+1,j+1})  otherwise,
 * and DTW_p(x, y)^p = q_{1,1}.  For p == 0 (p = infinity) the cell value is
 * max(|x_i - y_j|, min(...)) and the result is DTW_inf itself.
 *
 * Rows i = n .. 1 are evaluated in turn, keeping the rows i (cur) and i + 1
 * (nxt) as arrays indexed j = 1 .. n + 1 (slot n + 1 is the empty suffix of
 * y).  Only the band j in [i - w, i + w] is computed; the slots the
 * recursion reads just outside the band are set to inf explicitly.
 * Returns DTW_p^p (or DTW_inf).
 */
double oracle_dtw_pow(const float *x, const float *y, int64_t n, int64_t w, int p)
{
    w = clamp_w(n, w);
    double *bufa = (double *)malloc((size_t)(n + 2) * sizeof(double));
    double *bufb = (double *)malloc((size_t)(n + 2) * sizeof(double));
    double *nxt = bufa, *cur = bufb;
    for (int64_t j = 0; j <= n + 1; ++j) {
        bufa[j] = INFINITY;
        bufb[j] = INFINITY;
    }
    /* row n + 1 (x suffix empty): 0 at j = n + 1, inf elsewhere */
    nxt[n + 1] = 0.0;
    for (int64_t i = n; i >= 1; --i) {
        int64_t jlo = i - w < 1 ? 1 : i - w;
        int64_t jhi = i + w > n ? n : i + w;
        /* q_{i, jhi+1}: out of band, or the empty y suffix (j = n + 1) */
        cur[jhi + 1] = INFINITY;
        for (int64_t j = jhi; j >= jlo; --j) {
            double a = nxt[j], b = cur[j + 1], c = nxt[j + 1];
            double m = a < b ? a : b;
            m = m < c ? m : c;
            double xi = (double)x[i - 1], yj = (double)y[j - 1];
            if (p == 0) {
                double d = fabs(xi - yj);
                cur[j] = d > m ? d : m;
            } else {
                cur[j] = abs_pow(xi, yj, p) + m;
            }
        }
        /* q_{i, jlo-1} is out of band for row i; row i - 1 reads it */
        if (jlo - 1 >= 1)
            cur[jlo - 1] = INFINITY;
        double *t = nxt;
        nxt = cur;
        cur = t;
    }
    double r = nxt[1];
    free(bufa);
    free(bufb);
    return r;
}

/*
 * Piecewise-sum bound of Sec. 9.  P_d(x) = (sum_{i in C_j} x_i)_j over the
 * cover C_j = [1 + (j-1) floor(n/d), j floor(n/d)] for j < d and
 * C_d = [1 + (d-1) floor(n/d), n].  With D_j = d(P_d(x)_j, [P_d(L)_j, P_d(U)_j])
 * (U = U(y), L = L(y)):
 *   p = 1: sum_j D_j  (the paper's bound, <= LB_Keogh_1(x, y));
 *   p = 2: sum_j D_j^2 / max_j |C_j|  (reading for p = 2: D_j is at most the
 *          sum of the LB_Keogh terms over C_j, so D_j^2 / |C_j| is at most
 *          their sum of squares by Cauchy-Schwarz; the common denominator
 *          max_j |C_j| only weakens it).
 * Returns the p-th power of the bound.  Requires 1 <= d <= n.
 */
double oracle_lb_piecewise_pow(const float *x, const double *U, const double *L, int64_t n, int64_t d, int p)
{
    const int64_t s = n / d;
    const int64_t smax = n - (d - 1) * s; /* the last part takes the rest */
    double total = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        const int64_t lo = j * s;
        const int64_t hi = (j == d - 1) ? n : (j + 1) * s;
        double px = 0.0, pu = 0.0, pl = 0.0;
        for (int64_t i = lo; i < hi; ++i) {
            px += (double)x[i];
            pu += U[i];
            pl += L[i];
        }
        double dj = 0.0;
        if (px > pu)
            dj = px - pu;
        else if (px < pl)
            dj = pl - px;
        total += (p == 1) ? dj : dj * dj;
    }
    return (p == 1) ? total : total / (double)smax;
}

/* ---------------------------------------------------------------------- */
/* k nearest neighbours                                                    */
/* ---------------------------------------------------------------------- */

/* (d, idx) lexicographic order: the distance, then the lower index. */
static int before(double d, int64_t idx, double e, int64_t jdx)
{
    return d < e || (d == e && idx < jdx);
}

/* Insert (d, idx) into the sorted list (kd, ki) of length k if it belongs. */
static void topk_insert(double *kd, int64_t *ki, int k, double d, int64_t idx)
{
    if (!before(d, idx, kd[k - 1], ki[k - 1]))
        return;
    int pos = k - 1;
    while (pos > 0 && before(d, idx, kd[pos - 1], ki[pos - 1])) {
        kd[pos] = kd[pos - 1];
        ki[pos] = ki[pos - 1];
        --pos;
    }
    kd[pos] = d;
    ki[pos] = idx;
}

static void topk_init(double *kd, int64_t *ki, int k)
{
    for (int j = 0; j < k; ++j) {
        kd[j] = INFINITY;
        ki[j] = -1;
    }
}

static double root_p(double v, int p)
{
    if (p == 1 || p == 0)
        return v;
    if (p == 2)
        return sqrt(v);
    return pow(v, 1.0 / (double)p);
}

/*
 * The exact k-NN result by its definition: DTW_p of the query y against every
 * candidate, the k smallest by (distance, index).  Outputs DTW_p (root
 * taken); missing entries (k > N) are idx -1, distance +inf.
 */
void oracle_knn_bruteforce(const float *db, int64_t N, const float *y, int64_t n, int64_t w,
                           int p, int k, int64_t *out_idx, double *out_dist)
{
    double *kd = (double *)malloc((size_t)k * sizeof(double));
    int64_t *ki = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    topk_init(kd, ki, k);
    for (int64_t c = 0; c < N; ++c) {
        double t = oracle_dtw_pow(db + c * n, y, n, w, p);
        topk_insert(kd, ki, k, t, c);
    }
    for (int j = 0; j < k; ++j) {
        out_idx[j] = ki[j];
        out_dist[j] = isinf(kd[j]) ? INFINITY : root_p(kd[j], p);
    }
    free(kd);
    free(ki);
}

/*
 * Exact k-NN by one pass over the candidates in index order with lower-bound
 * pruning: the scans of Algorithm 2 (mode 0) and Algorithm 3 (mode 1) of
 * Sec. 7 and 8, generalised from 1-NN to k-NN.  Let b be the k-th smallest
 * DTW_p^p among the candidates evaluated so far (+inf until there are k).
 * Since LB_Keogh_p^p <= LB_Improved_p^p <= DTW_p^p (Sec. 7, Sec. 8), a
 * candidate with a bound >= b cannot displace any of the current k (on a
 * tie the lower index, already held, wins), so its DTW is not needed.  Mode
 * 0 tests LB_Keogh alone; mode 1 tests LB_Keogh and, if that passes,
 * LB_Improved = LB_Keogh + the second term.  Bounds and b are compared in
 * power space.
 *
 * stats (nullable) receives: [0] candidates, [1] discarded by LB_Keogh,
 * [2] discarded by LB_Improved, [3] full DTW computed.
 */
void oracle_knn_cascade(const float *db, int64_t N, const float *y, int64_t n, int64_t w, int p,
                        int k, int mode, int64_t *out_idx, double *out_dist, int64_t *stats)
{
    w = clamp_w(n, w);
    double *U = (double *)malloc((size_t)n * sizeof(double));
    double *L = (double *)malloc((size_t)n * sizeof(double));
    double *kd = (double *)malloc((size_t)k * sizeof(double));
    int64_t *ki = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int64_t st[4] = {0, 0, 0, 0};

    oracle_envelope(y, n, w, U, L); /* the query's envelope, once */
    topk_init(kd, ki, k);
    for (int64_t c = 0; c < N; ++c) {
        const float *x = db + c * n;
        const double b = kd[k - 1];
        st[0] += 1;
        double bound = oracle_lb_keogh_pow(x, U, L, n, p);
        if (!(bound < b)) {
            st[1] += 1;
            continue;
        }
        if (mode == 1) {
            bound += oracle_lb_improved_second_pow(x, y, U, L, n, w, p);
            if (!(bound < b)) {
                st[2] += 1;
                continue;
            }
        }
        st[3] += 1;
        topk_insert(kd, ki, k, oracle_dtw_pow(x, y, n, w, p), c);
    }
    for (int j = 0; j < k; ++j) {
        out_idx[j] = ki[j];
        out_dist[j] = isinf(kd[j]) ? INFINITY : root_p(kd[j], p);
    }
    if (stats)
        memcpy(stats, st, sizeof(st));
    free(U);
    free(L);
    free(kd);
    free(ki);
}
