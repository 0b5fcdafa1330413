/*
 * FP64 oracle for the exact k-NN / eps-NN scan under banded DTW and the
 * dog-keeper distance DK (Bachmann & Freytag, "An Analytical Approach to
 * Improving Time Warping on Multidimensional Time Series").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code with the
 * CUDA path.  Everything is plain, slow and written to be checked by eye
 * against the paper: double precision, no blocking, no fusion, no reordering.
 *
 * Conventions (0-based indices; the paper is 1-based):
 *   - a series of length n in d dimensions is n*d doubles, point-major;
 *   - point cost for DTW is the squared Euclidean distance (Section 2.1,
 *     the DTW recursion uses d(s,t)^2); DTW returns the path SUM (no root);
 *   - point cost for DK is the Euclidean distance (Section 2.1, DK recursion);
 *   - Sakoe-Chiba band (Section 2.2): cell (i,j) is allowed iff |i-j| <= r,
 *     r = floor(band * max(m,n)), band >= 1 means unconstrained;
 *   - an unreachable end cell (|m-n| > r) or an empty series gives +inf, as
 *     the recursion's base case does for an empty series (Section 2.1).
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against brute-force path enumeration, closed forms, the paper's inequalities
 * (Eq. 1 and the GDK upper-bound property of Section 4.1) and SciPy's
 * sliding-window filters.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF (1.0 / 0.0)

enum { ORC_DTW = 0, ORC_DK = 1 };

/* ----------------------------------------------------------------------- */
/* point costs (Section 3: d(s_i,t_j) = ||s_i - t_j||_2)                     */

static double sqdist(const double *a, const double *b, int d)
{
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double diff = a[k] - b[k];
        acc += diff * diff;
    }
    return acc;
}

static double eucl(const double *a, const double *b, int d)
{
    return sqrt(sqdist(a, b, d));
}

static int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }

/* Band radius from a fraction of the longer length (Section 2.2 gives the
 * band only as a width; the fraction-of-length reading is ours). */
int64_t orc_band_radius(int64_t m, int64_t n, double band)
{
    int64_t L = m > n ? m : n;
    if (band >= 1.0)
        return L;
    return (int64_t)floor(band * (double)L);
}

/* ----------------------------------------------------------------------- */
/* DTW and DK by the quadratic dynamic program (Section 2.1, last paragraph):
 * fill the warping matrix cell by cell, each cell combining its own cost with
 * the best of its left, lower and lower-left neighbours.                    */

double orc_dtw(const double *s, int64_t m, const double *t, int64_t n, int d, int64_t r)
{
    if (m <= 0 || n <= 0 || iabs64(m - n) > r)
        return ORC_INF;
    double *prev = malloc(sizeof(double) * (size_t)n);
    double *cur = malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        prev[j] = ORC_INF;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (iabs64(i - j) > r) {
                cur[j] = ORC_INF;
                continue;
            }
            double c = sqdist(s + i * d, t + j * d, d);
            double best;
            if (i == 0 && j == 0) {
                best = 0.0;
            } else {
                double left = j > 0 ? cur[j - 1] : ORC_INF;
                double low = i > 0 ? prev[j] : ORC_INF;
                double diag = (i > 0 && j > 0) ? prev[j - 1] : ORC_INF;
                best = fmin(fmin(left, low), diag);
            }
            cur[j] = c + best;
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    double res = prev[n - 1];
    free(prev);
    free(cur);
    return res;
}

double orc_dk(const double *s, int64_t m, const double *t, int64_t n, int d, int64_t r)
{
    if (m <= 0 || n <= 0 || iabs64(m - n) > r)
        return ORC_INF;
    double *prev = malloc(sizeof(double) * (size_t)n);
    double *cur = malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        prev[j] = ORC_INF;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (iabs64(i - j) > r) {
                cur[j] = ORC_INF;
                continue;
            }
            double c = eucl(s + i * d, t + j * d, d);
            if (i == 0 && j == 0) {
                cur[j] = c;
                continue;
            }
            double left = j > 0 ? cur[j - 1] : ORC_INF;
            double low = i > 0 ? prev[j] : ORC_INF;
            double diag = (i > 0 && j > 0) ? prev[j - 1] : ORC_INF;
            cur[j] = fmax(c, fmin(fmin(left, low), diag));
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    double res = prev[n - 1];
    free(prev);
    free(cur);
    return res;
}

double orc_distance(int kind, const double *s, int64_t m, const double *t, int64_t n,
                    int d, int64_t r)
{
    return kind == ORC_DK ? orc_dk(s, m, t, n, d, r) : orc_dtw(s, m, t, n, d, r);
}

/* ----------------------------------------------------------------------- */
/* Envelope (Section 2.3; per dimension in Section 3): for i in [0, len),
 *   l_{i,j} = min { t_{p,j} : |p - i| <= r, 0 <= p < n },  u likewise with max.
 * Positions whose window is empty get l = +inf, u = -inf.                   */

void orc_envelope(const double *t, int64_t n, int d, int64_t r, int64_t len,
                  double *l, double *u)
{
    for (int64_t i = 0; i < len; ++i) {
        for (int j = 0; j < d; ++j) {
            double lo = ORC_INF, hi = -ORC_INF;
            int64_t p0 = i - r < 0 ? 0 : i - r;
            int64_t p1 = i + r > n - 1 ? n - 1 : i + r;
            for (int64_t p = p0; p <= p1; ++p) {
                double v = t[p * d + j];
                if (v < lo)
                    lo = v;
                if (v > hi)
                    hi = v;
            }
            l[i * d + j] = lo;
            u[i * d + j] = hi;
        }
    }
}

/* Distance of a scalar to an interval (Section 2.3). */
static double dist_interval(double x, double lo, double hi)
{
    if (x < lo)
        return lo - x;
    if (x > hi)
        return x - hi;
    return 0.0;
}

/* LB_Keogh for 1-D series (Section 2.3): sum_i d(s_i, [l_i, u_i])^2 with the
 * envelope of T.  s and t are 1-D arrays. */
double orc_lb_keogh_1d(const double *s, int64_t m, const double *t, int64_t n, int64_t r)
{
    double *l = malloc(sizeof(double) * (size_t)m);
    double *u = malloc(sizeof(double) * (size_t)m);
    orc_envelope(t, n, 1, r, m, l, u);
    double acc = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        if (l[i] > u[i]) { /* empty window: no coupling possible */
            acc = ORC_INF;
            break;
        }
        double e = dist_interval(s[i], l[i], u[i]);
        acc += e * e;
    }
    free(l);
    free(u);
    return acc;
}

/* LB_Box (Section 3, Eq. 1): sum_i d(s_i, B_i)^2, B_i the bounding box of
 * T's points within the band around i.  form 0: the sum (bounds DTW);
 * form 1: max_i d(s_i, B_i)^2 (bounds DK^2: every s_i is coupled to a point of
 * its box, so the largest box distance cannot exceed the max along the path). */
double orc_lb_box(const double *s, int64_t m, const double *t, int64_t n, int d, int64_t r,
                  int form)
{
    double *l = malloc(sizeof(double) * (size_t)(m * d));
    double *u = malloc(sizeof(double) * (size_t)(m * d));
    orc_envelope(t, n, d, r, m, l, u);
    double acc = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double box = 0.0;
        for (int j = 0; j < d; ++j) {
            if (l[i * d + j] > u[i * d + j]) {
                box = ORC_INF;
                break;
            }
            double e = dist_interval(s[i * d + j], l[i * d + j], u[i * d + j]);
            box += e * e;
        }
        if (form == 0)
            acc += box;
        else if (box > acc)
            acc = box;
    }
    free(l);
    free(u);
    return acc;
}

/* LB_Box over segment boxes (the coarse first stage of the cascade; Eq. 1 of
 * Section 3 applied to coarsened boxes).  The points of s are grouped into
 * segments of W consecutive points (a partial last segment is left out); the
 * box of segment g is the smallest box holding the envelope boxes B_i of t
 * (window |p - i| <= r) of its points, and the bound is
 *   form 0: sum_g W * ||mean_g(s) - clamp(mean_g(s), box_g)||^2
 *   form 1: max_g     ||mean_g(s) - clamp(mean_g(s), box_g)||^2.
 * An empty window (no point of t within r) makes the pair infeasible: +inf. */
double orc_lb_seg(const double *s, int64_t m, const double *t, int64_t n, int d, int64_t r,
                  int64_t W, int form)
{
    double *l = malloc(sizeof(double) * (size_t)(m * d));
    double *u = malloc(sizeof(double) * (size_t)(m * d));
    orc_envelope(t, n, d, r, m, l, u);
    double acc = 0.0;
    for (int64_t g = 0; g + W <= m; g += W) {
        double box = 0.0;
        for (int j = 0; j < d; ++j) {
            double lo = ORC_INF, hi = -ORC_INF, mean = 0.0;
            for (int64_t i = g; i < g + W; ++i) {
                if (l[i * d + j] < lo)
                    lo = l[i * d + j];
                if (u[i * d + j] > hi)
                    hi = u[i * d + j];
                mean += s[i * d + j];
            }
            mean /= (double)W;
            if (lo > hi) {
                box = ORC_INF;
                break;
            }
            double e = dist_interval(mean, lo, hi);
            box += e * e;
        }
        if (form == 0)
            acc += (double)W * box;
        else if (box > acc)
            acc = box;
    }
    free(l);
    free(u);
    return acc;
}

/* LB_Sigma-min (Section 3): sum_i min_{|l|<=r} d(s_i, t_{i+l})^2. */
double orc_lb_sigma_min(const double *s, int64_t m, const double *t, int64_t n, int d,
                        int64_t r)
{
    double acc = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double best = ORC_INF;
        for (int64_t p = i - r; p <= i + r; ++p) {
            if (p < 0 || p >= n)
                continue;
            double c = sqdist(s + i * d, t + p * d, d);
            if (c < best)
                best = c;
        }
        acc += best;
    }
    return acc;
}

/* ----------------------------------------------------------------------- */
/* Greedy dog-keeper (Section 4.1, Algorithm 1).  From (0,0) step to the
 * cheapest of (i+1,j), (i+1,j+1), (i,j+1) (first minimum in that order);
 * undefined or out-of-band cells cost +inf.  The walk continues until it
 * reaches (m-1,n-1) (our reading of the loop condition).  form 0 keeps the
 * max of the Euclidean costs along the path (GDK, an upper bound of DK);
 * form 1 keeps the sum of the squared costs along the same path (an upper
 * bound of DTW: it is the cost of one admissible warping path).  Returns as
 * soon as the running value exceeds eps. */
double orc_greedy(const double *s, int64_t m, const double *t, int64_t n, int d, int64_t r,
                  double eps, int form)
{
    if (m <= 0 || n <= 0 || iabs64(m - n) > r)
        return ORC_INF;
    int64_t i = 0, j = 0;
    double g = form == 0 ? eucl(s, t, d) : sqdist(s, t, d);
    if (g > eps)
        return g;
    while (!(i == m - 1 && j == n - 1)) {
        double c[3];
        int64_t ni[3] = {i + 1, i + 1, i};
        int64_t nj[3] = {j, j + 1, j + 1};
        for (int a = 0; a < 3; ++a) {
            if (ni[a] >= m || nj[a] >= n || iabs64(ni[a] - nj[a]) > r)
                c[a] = ORC_INF;
            else
                c[a] = eucl(s + ni[a] * d, t + nj[a] * d, d);
        }
        int best = 0;
        for (int a = 1; a < 3; ++a)
            if (c[a] < c[best])
                best = a;
        i = ni[best];
        j = nj[best];
        if (form == 0)
            g = fmax(g, c[best]);
        else
            g += sqdist(s + i * d, t + j * d, d);
        if (g > eps)
            return g;
    }
    return g;
}

/* ----------------------------------------------------------------------- */
/* Sparse dog-keeper, whole-sequence match (Section 4.2, Algorithm 3 with
 * SUB = false).  Sweeps the columns of T; I holds the rows to visit in the
 * current column, J the rows for the next one; only cells whose cost is at
 * most eps are evaluated.  Readings: the start cell (0,0) has no predecessor
 * (its value is its own cost); out-of-band cells are treated like cells above
 * eps; an empty I means DK > eps and is reported as +inf instead of the
 * listing's eps sentinel.  Returns DK when DK <= eps, +inf otherwise.
 * If cells != NULL it receives the number of evaluated cells. */
double orc_sparse_dk(const double *s, int64_t m, const double *t, int64_t n, int d,
                     int64_t r, double eps, int64_t *cells)
{
    if (cells)
        *cells = 0;
    if (m <= 0 || n <= 0 || iabs64(m - n) > r)
        return ORC_INF;
    /* rows are 1..m; index 0 is the virtual row below the matrix */
    double *D = malloc(sizeof(double) * (size_t)(m + 2));
    double *E = malloc(sizeof(double) * (size_t)(m + 2));
    char *I = calloc((size_t)(m + 2), 1);
    char *J = calloc((size_t)(m + 2), 1);
    for (int64_t i = 0; i < m + 2; ++i)
        D[i] = E[i] = ORC_INF;
    I[1] = 1;
    int64_t evaluated = 0;
    double result = ORC_INF;
    for (int64_t k = 1; k <= n; ++k) {
        for (int64_t i = 1; i <= m; ++i) { /* I may grow upward while we sweep */
            if (!I[i])
                continue;
            double c = (iabs64(i - k) <= r) ? eucl(s + (i - 1) * d, t + (k - 1) * d, d)
                                            : ORC_INF;
            if (iabs64(i - k) <= r)
                ++evaluated;
            if (c <= eps) {
                double pred = (i == 1 && k == 1) ? 0.0 : fmin(fmin(D[i - 1], E[i]), E[i - 1]);
                D[i] = fmax(c, pred);
                if (i + 1 <= m)
                    I[i + 1] = 1;
                J[i] = 1;
                if (i + 1 <= m)
                    J[i + 1] = 1;
            } else {
                I[i] = 0;
            }
        }
        if (k == n) {
            result = D[m];
            break;
        }
        for (int64_t i = 0; i < m + 2; ++i)
            E[i] = D[i];
        for (int64_t i = 0; i < m + 2; ++i)
            D[i] = ORC_INF; /* reset D */
        int any = 0;
        for (int64_t i = 0; i < m + 2; ++i) {
            I[i] = J[i];
            J[i] = 0;
            any |= I[i];
        }
        if (!any) {
            result = ORC_INF;
            break;
        }
    }
    free(D);
    free(E);
    free(I);
    free(J);
    if (cells)
        *cells = evaluated;
    return result <= eps ? result : ORC_INF;
}

/* ----------------------------------------------------------------------- */
/* Subsequence search (Section 4.1 Algorithm 2, Section 4.2 Algorithm 3 with  */
/* SUB = true): the query S (m points) against every subsequence T[a..b] of a */
/* long series T (n points), no band.                                         */

/* Plain definition by the free-start, free-end dynamic program: row 0 of
 * every column starts a match (its value is its own cost), rows above follow
 * the DTW or DK recursion of Section 2.1, and the result is the minimum of the
 * last row over all columns, i.e. min over a <= b of DTW(S, T[a..b]) (sum of
 * squared costs) or DK(S, T[a..b]) (max of Euclidean costs).  *end receives
 * the smallest end column b of a minimum. */
double orc_sub_distance(int kind, const double *s, int64_t m, const double *t, int64_t n, int d,
                        int64_t *end)
{
    if (end)
        *end = -1;
    if (m <= 0 || n <= 0)
        return ORC_INF;
    double *prev = malloc(sizeof(double) * (size_t)m); /* column k-1 */
    double *cur = malloc(sizeof(double) * (size_t)m);  /* column k   */
    for (int64_t i = 0; i < m; ++i)
        prev[i] = ORC_INF;
    double best = ORC_INF;
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = 0; i < m; ++i) {
            const double c = kind == ORC_DTW ? sqdist(s + i * d, t + k * d, d)
                                             : eucl(s + i * d, t + k * d, d);
            double pred;
            if (i == 0)
                pred = 0.0; /* a match may start in any column */
            else
                pred = fmin(fmin(cur[i - 1], prev[i]), prev[i - 1]);
            cur[i] = kind == ORC_DTW ? c + pred : fmax(c, pred);
        }
        if (cur[m - 1] < best) {
            best = cur[m - 1];
            if (end)
                *end = k;
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    free(prev);
    free(cur);
    return best;
}

/* The k best end columns of subsequence search (the free-start recursion of
 * orc_sub_distance): every column b of T ends a best match of value D(m, b),
 * the minimum over all starts a <= b; the k smallest (value, b) pairs, in
 * that order (equal values: the smaller b first), are written to val / end
 * (padded with +inf / -1).  Returns how many were written. */
int64_t orc_sub_ends(int kind, const double *s, int64_t m, const double *t, int64_t n, int d,
                     int64_t k, double *val, int64_t *end)
{
    for (int64_t j = 0; j < k; ++j) {
        val[j] = ORC_INF;
        end[j] = -1;
    }
    if (m <= 0 || n <= 0 || k <= 0)
        return 0;
    double *prev = malloc(sizeof(double) * (size_t)m);
    double *cur = malloc(sizeof(double) * (size_t)m);
    for (int64_t i = 0; i < m; ++i)
        prev[i] = ORC_INF;
    int64_t cnt = 0;
    for (int64_t b = 0; b < n; ++b) {
        for (int64_t i = 0; i < m; ++i) {
            const double c = kind == ORC_DTW ? sqdist(s + i * d, t + b * d, d)
                                             : eucl(s + i * d, t + b * d, d);
            const double pred = i == 0 ? 0.0 : fmin(fmin(cur[i - 1], prev[i]), prev[i - 1]);
            cur[i] = kind == ORC_DTW ? c + pred : fmax(c, pred);
        }
        /* insert (cur[m-1], b) into the sorted list; b grows, so it goes after
         * every equal value */
        const double v = cur[m - 1];
        if (cnt < k || v < val[k - 1]) {
            int64_t p = cnt < k ? cnt : k - 1;
            while (p > 0 && val[p - 1] > v) {
                val[p] = val[p - 1];
                end[p] = end[p - 1];
                --p;
            }
            val[p] = v;
            end[p] = b;
            if (cnt < k)
                ++cnt;
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    free(prev);
    free(cur);
    return cnt;
}

/* Sparse dog-keeper distance for subsequence search (Algorithm 3 with
 * SUB = true): the column sweep of orc_sparse_dk without a band, where row 1
 * joins the rows to visit in every column (a match may start anywhere) and
 * the last row of every column is a candidate end.  Readings: d starts at
 * +inf once, before the sweep (the listing resets it inside the column
 * loop, which would keep only the last column's value, against the text's
 * "each position as possible end"); a row-1 cell takes its own cost, like
 * the whole-match start cell.  Returns the minimum when it is <= eps, +inf
 * otherwise; *end as in orc_sub_distance; *cells counts evaluated cells. */
double orc_sub_sparse_dk(const double *s, int64_t m, const double *t, int64_t n, int d,
                         double eps, int64_t *end, int64_t *cells)
{
    if (end)
        *end = -1;
    if (cells)
        *cells = 0;
    if (m <= 0 || n <= 0)
        return ORC_INF;
    double *D = malloc(sizeof(double) * (size_t)(m + 2));
    double *E = malloc(sizeof(double) * (size_t)(m + 2));
    char *I = calloc((size_t)(m + 2), 1);
    char *J = calloc((size_t)(m + 2), 1);
    for (int64_t i = 0; i < m + 2; ++i)
        D[i] = E[i] = ORC_INF;
    I[1] = 1;
    double best = ORC_INF;
    int64_t evaluated = 0;
    for (int64_t k = 1; k <= n; ++k) {
        for (int64_t i = 1; i <= m; ++i) { /* I may grow upward while we sweep */
            if (!I[i])
                continue;
            const double c = eucl(s + (i - 1) * d, t + (k - 1) * d, d);
            ++evaluated;
            if (c <= eps) {
                const double pred = i == 1 ? 0.0 : fmin(fmin(D[i - 1], E[i]), E[i - 1]);
                D[i] = fmax(c, pred);
                if (i + 1 <= m)
                    I[i + 1] = 1;
                J[i] = 1;
                if (i + 1 <= m)
                    J[i + 1] = 1;
            } else {
                I[i] = 0;
            }
        }
        if (D[m] < best) {
            best = D[m];
            if (end)
                *end = k - 1;
        }
        for (int64_t i = 0; i < m + 2; ++i)
            E[i] = D[i];
        for (int64_t i = 0; i < m + 2; ++i)
            D[i] = ORC_INF;
        for (int64_t i = 0; i < m + 2; ++i) {
            I[i] = J[i];
            J[i] = 0;
        }
        I[1] = 1; /* SUB: every column may start a match */
    }
    free(D);
    free(E);
    free(I);
    free(J);
    if (cells)
        *cells = evaluated;
    if (!(best <= eps)) {
        if (end)
            *end = -1;
        return ORC_INF;
    }
    return best;
}

/* Greedy dog-keeper for subsequence search (Algorithm 2): start at row 0 in
 * the column of T closest to s_0 (the first such column), walk to the
 * cheapest of (i+1, j), (i+1, j+1), (i, j+1) (the first in this order on
 * ties; a column beyond T costs +inf) until the last row is reached, and
 * return the largest cost met (early exit once it exceeds eps).  An upper
 * bound of the subsequence DK: the walk is one admissible path.  *end: the
 * column where the walk reached the last row. */
double orc_sub_gdk(const double *s, int64_t m, const double *t, int64_t n, int d, double eps,
                   int64_t *end)
{
    if (end)
        *end = -1;
    if (m <= 0 || n <= 0)
        return ORC_INF;
    int64_t i = 0, j = 0;
    double g = ORC_INF;
    for (int64_t k = 0; k < n; ++k) {
        const double c = eucl(s, t + k * d, d);
        if (c < g) {
            g = c;
            j = k;
        }
    }
    if (g > eps)
        return g;
    while (i != m - 1) {
        const double c_up = eucl(s + (i + 1) * d, t + j * d, d);
        const double c_diag = j + 1 < n ? eucl(s + (i + 1) * d, t + (j + 1) * d, d) : ORC_INF;
        const double c_right = j + 1 < n ? eucl(s + i * d, t + (j + 1) * d, d) : ORC_INF;
        double c = c_up;
        int64_t ni = i + 1, nj = j;
        if (c_diag < c) {
            c = c_diag;
            ni = i + 1;
            nj = j + 1;
        }
        if (c_right < c) {
            c = c_right;
            ni = i;
            nj = j + 1;
        }
        i = ni;
        j = nj;
        g = fmax(g, c);
        if (g > eps)
            return g;
    }
    if (end)
        *end = j;
    return g;
}

/* DTW with early abandoning (Section 4, first paragraph): the minimum of a
 * row of the warping matrix bounds the final value from below, so stop as
 * soon as it exceeds eps.  Returns DTW when DTW <= eps, +inf otherwise. */
double orc_dtw_abandon(const double *s, int64_t m, const double *t, int64_t n, int d,
                       int64_t r, double eps, int64_t *cells)
{
    if (cells)
        *cells = 0;
    if (m <= 0 || n <= 0 || iabs64(m - n) > r)
        return ORC_INF;
    double *prev = malloc(sizeof(double) * (size_t)n);
    double *cur = malloc(sizeof(double) * (size_t)n);
    int64_t evaluated = 0;
    for (int64_t j = 0; j < n; ++j)
        prev[j] = ORC_INF;
    double res = ORC_INF;
    for (int64_t i = 0; i < m; ++i) {
        double rowmin = ORC_INF;
        for (int64_t j = 0; j < n; ++j) {
            if (iabs64(i - j) > r) {
                cur[j] = ORC_INF;
                continue;
            }
            ++evaluated;
            double c = sqdist(s + i * d, t + j * d, d);
            double best;
            if (i == 0 && j == 0) {
                best = 0.0;
            } else {
                double left = j > 0 ? cur[j - 1] : ORC_INF;
                double low = i > 0 ? prev[j] : ORC_INF;
                double diag = (i > 0 && j > 0) ? prev[j - 1] : ORC_INF;
                best = fmin(fmin(left, low), diag);
            }
            cur[j] = c + best;
            if (cur[j] < rowmin)
                rowmin = cur[j];
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
        if (rowmin > eps)
            goto done;
    }
    res = prev[n - 1];
done:
    free(prev);
    free(cur);
    if (cells)
        *cells = evaluated;
    return res <= eps ? res : ORC_INF;
}

/* ----------------------------------------------------------------------- */
/* Nearest-neighbour queries (Section 1: k-NN returns the k most similar
 * series, eps-NN all series within distance eps).  Ties are ordered by id. */

typedef struct {
    double dist;
    int64_t id;
} orc_hit;

static int hit_cmp(const void *a, const void *b)
{
    const orc_hit *x = a, *y = b;
    if (x->dist < y->dist)
        return -1;
    if (x->dist > y->dist)
        return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int hit_less(double d1, int64_t i1, double d2, int64_t i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

typedef struct {
    const double *db;
    const int64_t *db_off;
    int64_t N;
    const double *q;
    const int64_t *q_off;
    int64_t nq;
    int d;
    double band;
    int kind;
    int64_t k;
    double eps;
    int64_t cap;
    int method;
    int64_t *out_ids;
    double *out_dist;
    int64_t *out_counts;
    int64_t *stats; /* per query: [lb_pruned, dp_calls, dp_abandoned, cells, ub_calls] */
    int64_t next;
    pthread_mutex_t lock;
} orc_job;

/* Plain definition: every distance, then sort by (distance, id). */
static void query_brute(orc_job *J, int64_t qi)
{
    const double *q = J->q + J->q_off[qi] * J->d;
    int64_t m = J->q_off[qi + 1] - J->q_off[qi];
    orc_hit *h = malloc(sizeof(orc_hit) * (size_t)(J->N > 0 ? J->N : 1));
    int64_t cnt = 0;
    for (int64_t c = 0; c < J->N; ++c) {
        const double *x = J->db + J->db_off[c] * J->d;
        int64_t n = J->db_off[c + 1] - J->db_off[c];
        int64_t r = orc_band_radius(m, n, J->band);
        double dist = orc_distance(J->kind, q, m, x, n, J->d, r);
        if (J->k == 0 && !(dist <= J->eps))
            continue;
        h[cnt].dist = dist;
        h[cnt].id = c;
        ++cnt;
    }
    qsort(h, (size_t)cnt, sizeof(orc_hit), hit_cmp);
    if (J->k > 0) {
        for (int64_t a = 0; a < J->k; ++a) {
            int ok = a < cnt && isfinite(h[a].dist);
            J->out_ids[qi * J->k + a] = ok ? h[a].id : -1;
            J->out_dist[qi * J->k + a] = ok ? h[a].dist : ORC_INF;
        }
    } else {
        J->out_counts[qi] = cnt;
        for (int64_t a = 0; a < J->cap; ++a) {
            int ok = a < cnt;
            J->out_ids[qi * J->cap + a] = ok ? h[a].id : -1;
            J->out_dist[qi * J->cap + a] = ok ? h[a].dist : ORC_INF;
        }
    }
    free(h);
}

/* The paper's method in FP64, as a sequential scan in database order.
 *   DTW: LB_Box (sum form) pruning and DTW with early abandoning against the
 *        k-th best distance found so far (Sections 2.3, 3 and 4).
 *   DK:  GDK pre-pass over all series for the k smallest upper bounds
 *        (Section 4.3; k=1 is the paper's "lowest upper bound"), then the
 *        scan with the max-form LB_Box pruning and the sparse DK of
 *        Algorithm 3 thresholded at the current k-th best.
 * Pruning uses strict ">" so that an equal distance with a smaller id is
 * still examined.  For eps-NN the threshold is eps throughout. */
static void query_method(orc_job *J, int64_t qi)
{
    const int d = J->d;
    const double *q = J->q + J->q_off[qi] * d;
    int64_t m = J->q_off[qi + 1] - J->q_off[qi];
    int64_t kk = J->k > 0 ? J->k : 0;
    orc_hit *top = malloc(sizeof(orc_hit) * (size_t)(kk > 0 ? kk : 1));
    int64_t ntop = 0;
    orc_hit *all = NULL;
    int64_t nall = 0;
    if (kk == 0)
        all = malloc(sizeof(orc_hit) * (size_t)(J->N > 0 ? J->N : 1));
    int64_t st[5] = {0, 0, 0, 0, 0};
    double ub = ORC_INF; /* k-th smallest upper bound (DK k-NN only) */

    if (J->kind == ORC_DK && kk > 0) {
        double *ubs = malloc(sizeof(double) * (size_t)kk);
        int64_t nub = 0;
        for (int64_t c = 0; c < J->N; ++c) {
            const double *x = J->db + J->db_off[c] * d;
            int64_t n = J->db_off[c + 1] - J->db_off[c];
            int64_t r = orc_band_radius(m, n, J->band);
            double eps = nub < kk ? ORC_INF : ubs[kk - 1];
            double g = orc_greedy(q, m, x, n, d, r, eps, 0);
            ++st[4];
            if (!(g <= eps) || !isfinite(g))
                continue;
            /* insert g into the sorted list of the kk smallest */
            int64_t pos = nub < kk ? nub : kk - 1;
            while (pos > 0 && ubs[pos - 1] > g) {
                ubs[pos] = ubs[pos - 1];
                --pos;
            }
            ubs[pos] = g;
            if (nub < kk)
                ++nub;
        }
        if (nub == kk)
            ub = ubs[kk - 1];
        free(ubs);
    }

    for (int64_t c = 0; c < J->N; ++c) {
        const double *x = J->db + J->db_off[c] * d;
        int64_t n = J->db_off[c + 1] - J->db_off[c];
        int64_t r = orc_band_radius(m, n, J->band);
        double thr;
        if (kk == 0)
            thr = J->eps;
        else
            thr = ntop < kk ? ub : fmin(ub, top[kk - 1].dist);
        if (J->kind == ORC_DTW) {
            double lb = orc_lb_box(x, n, q, m, d, r, 0);
            if (lb > thr) {
                ++st[0];
                continue;
            }
            int64_t cells = 0;
            ++st[1];
            double dist = orc_dtw_abandon(q, m, x, n, d, r, thr, &cells);
            st[3] += cells;
            if (!isfinite(dist)) {
                ++st[2];
                continue;
            }
            if (kk == 0) {
                all[nall].dist = dist;
                all[nall].id = c;
                ++nall;
                continue;
            }
            if (ntop == kk && !hit_less(dist, c, top[kk - 1].dist, top[kk - 1].id))
                continue;
            int64_t pos = ntop < kk ? ntop : kk - 1;
            while (pos > 0 && hit_less(dist, c, top[pos - 1].dist, top[pos - 1].id)) {
                top[pos] = top[pos - 1];
                --pos;
            }
            top[pos].dist = dist;
            top[pos].id = c;
            if (ntop < kk)
                ++ntop;
        } else {
            double lbsq = orc_lb_box(x, n, q, m, d, r, 1);
            if (sqrt(lbsq) > thr) {
                ++st[0];
                continue;
            }
            int64_t cells = 0;
            ++st[1];
            double dist = orc_sparse_dk(q, m, x, n, d, r, thr, &cells);
            st[3] += cells;
            if (!isfinite(dist)) {
                ++st[2];
                continue;
            }
            if (kk == 0) {
                all[nall].dist = dist;
                all[nall].id = c;
                ++nall;
                continue;
            }
            if (ntop == kk && !hit_less(dist, c, top[kk - 1].dist, top[kk - 1].id))
                continue;
            int64_t pos = ntop < kk ? ntop : kk - 1;
            while (pos > 0 && hit_less(dist, c, top[pos - 1].dist, top[pos - 1].id)) {
                top[pos] = top[pos - 1];
                --pos;
            }
            top[pos].dist = dist;
            top[pos].id = c;
            if (ntop < kk)
                ++ntop;
        }
    }
    if (kk > 0) {
        for (int64_t a = 0; a < kk; ++a) {
            J->out_ids[qi * kk + a] = a < ntop ? top[a].id : -1;
            J->out_dist[qi * kk + a] = a < ntop ? top[a].dist : ORC_INF;
        }
    } else {
        qsort(all, (size_t)nall, sizeof(orc_hit), hit_cmp);
        J->out_counts[qi] = nall;
        for (int64_t a = 0; a < J->cap; ++a) {
            J->out_ids[qi * J->cap + a] = a < nall ? all[a].id : -1;
            J->out_dist[qi * J->cap + a] = a < nall ? all[a].dist : ORC_INF;
        }
        free(all);
    }
    if (J->stats)
        memcpy(J->stats + qi * 5, st, sizeof(st));
    free(top);
}

static void *worker(void *arg)
{
    orc_job *J = arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t qi = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (qi >= J->nq)
            break;
        if (J->method)
            query_method(J, qi);
        else
            query_brute(J, qi);
    }
    return NULL;
}

/* Exact k-NN (k > 0) or eps-NN (k == 0) for a batch of queries.
 * db/db_off: N series (point offsets, N+1 entries); q/q_off likewise.
 * k-NN outputs are [nq][k] (id -1 / +inf padding); eps-NN outputs are
 * [nq][cap] plus the true count per query.  method=0: plain definition;
 * method=1: the paper's pruned scan.  stats (nullable): [nq][5]. */
int orc_knn(const double *db, const int64_t *db_off, int64_t N, const double *q,
            const int64_t *q_off, int64_t nq, int d, double band, int kind, int64_t k,
            double eps, int64_t cap, int method, int nthreads, int64_t *out_ids,
            double *out_dist, int64_t *out_counts, int64_t *stats)
{
    orc_job J = {db, db_off, N, q, q_off, nq, d, band, kind, k, eps, cap, method,
                 out_ids, out_dist, out_counts, stats, 0, PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1)
        nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int a = 0; a < nthreads; ++a)
        pthread_create(&th[a], NULL, worker, &J);
    for (int a = 0; a < nthreads; ++a)
        pthread_join(th[a], NULL);
    free(th);
    return 0;
}

/* Distances for an explicit list of pairs (a_i, b_i), in parallel. */
typedef struct {
    const double *a, *b;
    const int64_t *a_off, *b_off;
    const int64_t *pa, *pb;
    int64_t n;
    int d;
    double band;
    int kind;
    double *out;
    int64_t next;
    pthread_mutex_t lock;
} orc_pairs;

static void *pair_worker(void *arg)
{
    orc_pairs *P = arg;
    for (;;) {
        pthread_mutex_lock(&P->lock);
        int64_t s = P->next;
        P->next += 64;
        pthread_mutex_unlock(&P->lock);
        if (s >= P->n)
            break;
        int64_t e = s + 64 < P->n ? s + 64 : P->n;
        for (int64_t i = s; i < e; ++i) {
            int64_t ia = P->pa[i], ib = P->pb[i];
            int64_t m = P->a_off[ia + 1] - P->a_off[ia];
            int64_t n = P->b_off[ib + 1] - P->b_off[ib];
            int64_t r = orc_band_radius(m, n, P->band);
            P->out[i] = orc_distance(P->kind, P->a + P->a_off[ia] * P->d, m,
                                     P->b + P->b_off[ib] * P->d, n, P->d, r);
        }
    }
    return NULL;
}

int orc_pairwise(const double *a, const int64_t *a_off, const double *b, const int64_t *b_off,
                 const int64_t *pa, const int64_t *pb, int64_t n_pairs, int d, double band,
                 int kind, int nthreads, double *out)
{
    orc_pairs P = {a, b, a_off, b_off, pa, pb, n_pairs, d, band, kind, out, 0,
                   PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1)
        nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int i = 0; i < nthreads; ++i)
        pthread_create(&th[i], NULL, pair_worker, &P);
    for (int i = 0; i < nthreads; ++i)
        pthread_join(th[i], NULL);
    free(th);
    return 0;
}
