/*
 * Plain FP64 CPU oracle for Adaptive Inverse Distance Weighting (AIDW).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct statement of what the
 * GPU library computes. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it; the product path never does. It shares no code,
 * header, table or constant with the CUDA implementation.
 *
 * Source: G. Mei, L. Xu, N. Xu, "Accelerating Adaptive IDW Interpolation Algorithm on a
 * Single GPU" (arXiv 1511.02186).
 *   Sec. 2.1, Eq. 1      standard IDW weighting, w_i = d(x, x_i)^-alpha, over all n points
 *   Sec. 2.2, Step 1     Eq. 2 (expected NN distance), Eq. 3 (observed mean kNN distance),
 *                        Eq. 4 (NN statistic R)
 *   Sec. 2.2, Step 2     Eq. 5 (fuzzy membership mu_R)
 *   Sec. 2.2, Step 3     Eq. 6 (triangular mapping of mu_R to alpha over five levels)
 *   Sec. 3.1.2           the k-nearest-neighbour procedure (sort the first k distances, then
 *                        for each further point replace the k-th if strictly closer and let
 *                        it sink into place)
 *   Sec. 3.2.1           both phases visit every data point
 *
 * Notation follows the paper's Sec. 2: n data points (x_i, y_i, z_i), m query
 * ("interpolated") points, k neighbours, study area A, levels alpha_1..alpha_5,
 * membership bounds R_min, R_max.
 *
 * Readings where the paper is silent or inconsistent:
 *   - Sec. 3 swaps the letters n and m; here n always counts data points (as in Eq. 2).
 *   - Eq. 5 is used literally, with pi / R_max (not pi / (R_max - R_min)).
 *   - Ties in the kNN go to the lower data index (the strict "<" of Sec. 3.1.2 in scan
 *     order); r_obs does not depend on this choice.
 *   - A query that coincides exactly with one or more data points (d = 0, where Eq. 1 is
 *     undefined) returns the mean z of those points, the limit of Eq. 1 as the query
 *     approaches them.
 *
 * Arithmetic: every distance is d2 = dx*dx + dy*dy evaluated in IEEE double with no fused
 * multiply-add (build with -ffp-contract=off), d = sqrt(d2), weights use pow(), and both
 * weighted sums use Neumaier's compensated summation so that the oracle's own rounding
 * error stays near one ulp of the result's condition number.
 *
 * Parity pins for every function here live in the "not gpu" oracle tests: closed forms of
 * Eq. 2/5/6, brute-force and literal-procedure kNN, the Clark-Evans statistic, and the
 * invariants of the weighted mean.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* Eq. 2: expected nearest-neighbour distance of a random pattern of n points on area A. */
double aidw_oracle_r_exp(int64_t n, double area)
{
    double density = (double)n / area;
    return 1.0 / (2.0 * sqrt(density));
}

/* Eq. 5: fuzzy membership of the NN statistic R, bounded to [0, 1]. */
double aidw_oracle_mu(double R, double r_min, double r_max)
{
    if (R <= r_min)
        return 0.0;
    if (R >= r_max)
        return 1.0;
    return 0.5 - 0.5 * cos((M_PI / r_max) * (R - r_min));
}

/* Eq. 6: triangular membership mapping mu_R to alpha, case by case as printed. */
double aidw_oracle_alpha(double mu, const double a[5])
{
    const double a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3], a5 = a[4];
    if (mu <= 0.1)
        return a1;
    if (mu <= 0.3)
        return a1 * (1.0 - 5.0 * (mu - 0.1)) + 5.0 * a2 * (mu - 0.1);
    if (mu <= 0.5)
        return 5.0 * a3 * (mu - 0.3) + a2 * (1.0 - 5.0 * (mu - 0.3));
    if (mu <= 0.7)
        return a3 * (1.0 - 5.0 * (mu - 0.5)) + 5.0 * a4 * (mu - 0.5);
    if (mu <= 0.9)
        return 5.0 * a5 * (mu - 0.7) + a4 * (1.0 - 5.0 * (mu - 0.7));
    return a5;
}

/* Squared Euclidean distance, two products and one sum, each rounded (no FMA). */
static double dist2(double qx, double qy, double x, double y)
{
    double dx = qx - x;
    double dy = qy - y;
    return dx * dx + dy * dy;
}

/*
 * Sec. 3.1.2: the k nearest data points of one query.
 * Step 1 computes the first k distances, Step 2 sorts them ascending, Step 3 visits the
 * remaining points: a point strictly closer than the current k-th replaces it and sinks
 * toward the front past every strictly larger distance. Scanning in index order with strict
 * comparisons yields the k smallest (d2, index) pairs in lexicographic order.
 * Outputs idx[0..k) and d2[0..k), ascending.
 */
static void knn_one(const double *x, const double *y, int64_t n, double qx, double qy,
                    int k, int64_t *idx, double *d2)
{
    /* Steps 1 and 2: first k distances, insertion-sorted (stable: equal keep index order). */
    for (int j = 0; j < k; ++j) {
        double v = dist2(qx, qy, x[j], y[j]);
        int p = j;
        while (p > 0 && v < d2[p - 1]) {
            d2[p] = d2[p - 1];
            idx[p] = idx[p - 1];
            --p;
        }
        d2[p] = v;
        idx[p] = j;
    }
    /* Step 3: every remaining point. */
    for (int64_t i = k; i < n; ++i) {
        double v = dist2(qx, qy, x[i], y[i]);
        if (!(v < d2[k - 1]))
            continue;
        int p = k - 1;
        while (p > 0 && v < d2[p - 1]) {
            d2[p] = d2[p - 1];
            idx[p] = idx[p - 1];
            --p;
        }
        d2[p] = v;
        idx[p] = i;
    }
}

/* Neumaier's variant of Kahan summation: sum += v with the lost low part kept in *c. */
static void neumaier_add(double *sum, double *c, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v))
        *c += (*sum - t) + v;
    else
        *c += (v - t) + *sum;
    *sum = t;
}

typedef struct {
    const double *x, *y, *z;
    int64_t n;
    double r_exp;
    const double *qx, *qy;
    int64_t q_begin, q_end;
    int k;
    const double *levels;
    double r_min, r_max;
    int fixed_alpha; /* nonzero: standard IDW with alpha = levels[0], no kNN (Eq. 1 alone) */
    double *out_z, *out_alpha, *out_R, *out_scale;
    int64_t *out_knn;
    int status;
} work_t;

static void *interpolate_range(void *arg)
{
    work_t *w = (work_t *)arg;
    int k = w->k;
    int64_t *idx = NULL;
    double *d2 = NULL;
    if (!w->fixed_alpha) {
        idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        d2 = (double *)malloc(sizeof(double) * (size_t)k);
        if (!idx || !d2) {
            free(idx);
            free(d2);
            w->status = ORC_ENOMEM;
            return NULL;
        }
    }
    for (int64_t q = w->q_begin; q < w->q_end; ++q) {
        double qx = w->qx[q], qy = w->qy[q];
        double alpha, R = NAN;
        if (w->fixed_alpha) {
            alpha = w->levels[0];
        } else {
            /* Phase 1 (Sec. 2.2): kNN, Eq. 3, Eq. 4, Eq. 5, Eq. 6. */
            knn_one(w->x, w->y, w->n, qx, qy, k, idx, d2);
            double s = 0.0;
            for (int j = 0; j < k; ++j)
                s += sqrt(d2[j]);
            double r_obs = s / (double)k;          /* Eq. 3 */
            R = r_obs / w->r_exp;                  /* Eq. 4 */
            double mu = aidw_oracle_mu(R, w->r_min, w->r_max); /* Eq. 5 */
            alpha = aidw_oracle_alpha(mu, w->levels);          /* Eq. 6 */
            if (w->out_knn)
                memcpy(w->out_knn + q * k, idx, sizeof(int64_t) * (size_t)k);
        }
        /* Phase 2 (Eq. 1): weighted average over all n data points. Exactly coincident
         * points (d2 == 0) are counted apart; if there are any, they decide the value. */
        double sw = 0.0, cw = 0.0, swz = 0.0, cwz = 0.0, swa = 0.0, cwa = 0.0;
        double sz0 = 0.0, cz0 = 0.0, sa0 = 0.0, ca0 = 0.0;
        int64_t n0 = 0;
        for (int64_t i = 0; i < w->n; ++i) {
            double dd = dist2(qx, qy, w->x[i], w->y[i]);
            if (dd == 0.0) {
                ++n0;
                neumaier_add(&sz0, &cz0, w->z[i]);
                neumaier_add(&sa0, &ca0, fabs(w->z[i]));
                continue;
            }
            double wi = pow(sqrt(dd), -alpha);
            neumaier_add(&sw, &cw, wi);
            neumaier_add(&swz, &cwz, wi * w->z[i]);
            neumaier_add(&swa, &cwa, wi * fabs(w->z[i]));
        }
        double Z, scale;
        if (n0 > 0) {
            Z = (sz0 + cz0) / (double)n0;
            scale = (sa0 + ca0) / (double)n0;
        } else {
            double W = sw + cw;
            Z = (swz + cwz) / W;
            scale = (swa + cwa) / W;
        }
        w->out_z[q] = Z;
        if (w->out_alpha)
            w->out_alpha[q] = alpha;
        if (w->out_R)
            w->out_R[q] = R;
        if (w->out_scale)
            w->out_scale[q] = scale;
    }
    free(idx);
    free(d2);
    w->status = ORC_OK;
    return NULL;
}

static int run_threads(work_t *proto, int64_t m, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    if ((int64_t)nthreads > m)
        nthreads = (int)(m > 0 ? m : 1);
    work_t *ws = (work_t *)calloc((size_t)nthreads, sizeof(work_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) {
        free(ws);
        free(th);
        return ORC_ENOMEM;
    }
    int64_t per = m / nthreads, rem = m % nthreads, b = 0;
    for (int t = 0; t < nthreads; ++t) {
        ws[t] = *proto;
        ws[t].q_begin = b;
        b += per + (t < rem ? 1 : 0);
        ws[t].q_end = b;
        ws[t].status = ORC_EINVAL;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, interpolate_range, &ws[t]) != 0)
            ws[t].status = ORC_ENOMEM, th[t] = 0;
    interpolate_range(&ws[0]);
    int status = ws[0].status;
    for (int t = 1; t < nthreads; ++t) {
        if (th[t])
            pthread_join(th[t], NULL);
        else
            interpolate_range(&ws[t]);
        if (ws[t].status != ORC_OK)
            status = ws[t].status;
    }
    free(ws);
    free(th);
    return status;
}

/*
 * AIDW for m queries (Sec. 2.2 phases 1 and 2). Outputs: out_z[m]; optional out_alpha[m],
 * out_R[m] (NN statistic), out_knn[m*k] (ascending by distance), out_scale[m] =
 * sum(w|z|)/sum(w), the condition scale of the weighted mean used as an error denominator.
 */
int aidw_oracle_interpolate(const double *x, const double *y, const double *z, int64_t n,
                            double area, const double *qx, const double *qy, int64_t m, int k,
                            const double levels[5], double r_min, double r_max, double *out_z,
                            double *out_alpha, double *out_R, int64_t *out_knn,
                            double *out_scale, int nthreads)
{
    if (n < 1 || m < 0 || k < 1 || (int64_t)k > n || !(area > 0.0) || !(r_max > r_min))
        return ORC_EINVAL;
    if (m == 0)
        return ORC_OK;
    work_t p;
    memset(&p, 0, sizeof p);
    p.x = x, p.y = y, p.z = z, p.n = n;
    p.r_exp = aidw_oracle_r_exp(n, area);
    p.qx = qx, p.qy = qy, p.k = k, p.levels = levels;
    p.r_min = r_min, p.r_max = r_max;
    p.out_z = out_z, p.out_alpha = out_alpha, p.out_R = out_R, p.out_knn = out_knn;
    p.out_scale = out_scale;
    return run_threads(&p, m, nthreads);
}

/* Standard IDW of Eq. 1 with a user constant alpha over all n points (Sec. 2.1). */
int aidw_oracle_idw(const double *x, const double *y, const double *z, int64_t n,
                    const double *qx, const double *qy, int64_t m, double alpha, double *out_z,
                    double *out_scale, int nthreads)
{
    if (n < 1 || m < 0)
        return ORC_EINVAL;
    if (m == 0)
        return ORC_OK;
    double lv[5] = {alpha, alpha, alpha, alpha, alpha};
    work_t p;
    memset(&p, 0, sizeof p);
    p.x = x, p.y = y, p.z = z, p.n = n, p.qx = qx, p.qy = qy, p.k = 1;
    p.levels = lv, p.fixed_alpha = 1, p.out_z = out_z, p.out_scale = out_scale;
    return run_threads(&p, m, nthreads);
}

/* Sec. 3.1.2 kNN alone, for m queries: idx[m*k], d2[m*k], ascending. */
int aidw_oracle_knn(const double *x, const double *y, int64_t n, const double *qx,
                    const double *qy, int64_t m, int k, int64_t *idx, double *d2)
{
    if (n < 1 || m < 0 || k < 1 || (int64_t)k > n)
        return ORC_EINVAL;
    for (int64_t q = 0; q < m; ++q)
        knn_one(x, y, n, qx[q], qy[q], k, idx + q * k, d2 + q * k);
    return ORC_OK;
}
