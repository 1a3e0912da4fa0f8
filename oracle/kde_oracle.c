/*
 * FP64 CPU oracle for exact Gaussian kernel density estimation.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path calls, links or
 * loads this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code, header or constant with the CUDA path.
 *
 * What it computes is the plain definition (Sec. 3 "Kernel Density Estimation"):
 *     K(q) = sum_{i=1..n} k(||q - x_i||),   k(x) = exp(-a x^2)   (Gaussian kernel, Sec. 3)
 * evaluated the "naive" way the paper describes as exact (Sec. 3, O(dmn); Sec. 6.1
 * "Naive": the kernel with every data point). The 1/n factor of the paper's
 * definition is left to the caller (the library returns the unnormalised sum; the
 * reading is recorded in the design notes).
 *
 * Arithmetic, per query j (fixed order, independent of the thread count):
 *     s = 0; for i = 0..n-1: d2 = sum_{k=0..d-1} (q_jk - x_ik)^2  (direct differences)
 *                           s += exp(-a * d2)                   (libm exp)
 * Threads split the queries into contiguous blocks; each query is summed by one thread.
 *
 * Also, from the same section: the exponential kernel k(r) = exp(-a r) and the logistic
 * kernel k(r) = 4 / (2 + exp(a r) + exp(-a r)) (Sec. 3 writes the logistic one without a
 * bandwidth; its argument is read as a r, so a = 1 is the paper's k), with r = sqrt(d2);
 * and the subset sum over a per-query list of (index, weight) pairs,
 *     out_j = sum_{p = off[j] .. off[j+1]-1} w_p k(||q_j - x_{idx[p]}||),
 * the estimator that random sampling (weight n/s) and the CKNS scheme (weights 2^i on
 * the hashed candidates) evaluate (Sec. 3.1), summed in list order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    const double *X, *Q, *W;
    int64_t n, m, d, q0, q1;
    double a;
    int self_skip;        /* exclude i == j (query j is data point j) */
    double *out, *logk, *d2min, *kappa;
    int kind;             /* 0 Gaussian, 1 exponential, 2 logistic */
    const int64_t *off, *idx; /* subset lists (CSR): query j owns entries off[j] .. off[j+1]-1 */
} job_t;

/* The kernel function of the distance r = sqrt(d2) (Sec. 3). */
static double kern(int kind, double a, double d2) {
    if (kind == 0) return exp(-a * d2);
    double x = a * sqrt(d2);
    if (kind == 1) return exp(-x);
    return 4.0 / (2.0 + exp(x) + exp(-x));
}

static double sqdist(const double *q, const double *x, int64_t d) {
    double s = 0.0;
    for (int64_t k = 0; k < d; ++k) {
        double t = q[k] - x[k];
        s += t * t;
    }
    return s;
}

/* K(q_j) = sum_i w_i exp(-a ||q_j - x_i||^2), w_i = 1 when W is NULL. */
static void *run_sum(void *p) {
    job_t *J = (job_t *)p;
    for (int64_t j = J->q0; j < J->q1; ++j) {
        const double *q = J->Q + j * J->d;
        double s = 0.0;
        for (int64_t i = 0; i < J->n; ++i) {
            if (J->self_skip && i == j) continue;
            double e = kern(J->kind, J->a, sqdist(q, J->X + i * J->d, J->d));
            s += J->W ? J->W[i] * e : e;
        }
        J->out[j] = s;
    }
    return NULL;
}

/* Log-domain evaluation for cases where every term underflows double:
 *   d2min = min_i d2_i,  s' = sum_i exp(-a (d2_i - d2min)),  log K = -a d2min + log s'.
 * Also the exponent's condition number kappa = sum_i a d2_i w_i / sum_i w_i with
 * w_i = exp(-a (d2_i - d2min)): the relative error of K caused by a relative
 * perturbation eps of every squared distance is kappa * eps to first order. */
static void *run_log(void *p) {
    job_t *J = (job_t *)p;
    for (int64_t j = J->q0; j < J->q1; ++j) {
        const double *q = J->Q + j * J->d;
        double mn = INFINITY;
        for (int64_t i = 0; i < J->n; ++i) {
            double t = sqdist(q, J->X + i * J->d, J->d);
            if (t < mn) mn = t;
        }
        double s = 0.0, sk = 0.0;
        for (int64_t i = 0; i < J->n; ++i) {
            double t = sqdist(q, J->X + i * J->d, J->d);
            double w = exp(-J->a * (t - mn));
            s += w;
            sk += J->a * t * w;
        }
        J->logk[j] = -J->a * mn + log(s);
        J->d2min[j] = mn;
        J->kappa[j] = sk / s;
    }
    return NULL;
}

/* Subset sums over each query's own list of (index, weight) pairs, in list order. */
static void *run_subset(void *p) {
    job_t *J = (job_t *)p;
    for (int64_t j = J->q0; j < J->q1; ++j) {
        const double *q = J->Q + j * J->d;
        double s = 0.0;
        for (int64_t e = J->off[j]; e < J->off[j + 1]; ++e) {
            double k = kern(J->kind, J->a, sqdist(q, J->X + J->idx[e] * J->d, J->d));
            s += J->W ? J->W[e] * k : k;
        }
        J->out[j] = s;
    }
    return NULL;
}

static int launch(job_t base, int threads, void *(*fn)(void *)) {
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    if ((int64_t)threads > base.m) threads = (int)(base.m > 0 ? base.m : 1);
    pthread_t tid[1024];
    job_t jobs[1024];
    for (int t = 0; t < threads; ++t) {
        jobs[t] = base;
        jobs[t].q0 = base.m * t / threads;
        jobs[t].q1 = base.m * (t + 1) / threads;
    }
    int started = 0;
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, fn, &jobs[t]) != 0) break;
        started = t;
    }
    fn(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    for (int t = started + 1; t < threads; ++t) fn(&jobs[t]); /* threads that failed to start */
    return 0;
}

int oracle_kde(const double *X, int64_t n, const double *Q, int64_t m, int64_t d, double a,
               double *out, int threads) {
    if (n < 0 || m < 0 || d < 1 || !out) return -1;
    job_t b = {X, Q, NULL, n, m, d, 0, m, a, 0, out, NULL, NULL, NULL};
    return launch(b, threads, run_sum);
}

/* Weighted sum: sum_i w_i exp(-a ||q - x_i||^2). */
int oracle_kde_weighted(const double *X, const double *W, int64_t n, const double *Q, int64_t m,
                        int64_t d, double a, double *out, int threads) {
    if (n < 0 || m < 0 || d < 1 || !out || !W) return -1;
    job_t b = {X, Q, W, n, m, d, 0, m, a, 0, out, NULL, NULL, NULL};
    return launch(b, threads, run_sum);
}

/* Self-KDE (degree of every data point in the fully connected similarity graph,
 * Sec. 4): deg(i) = sum_{j != i} exp(-a ||x_i - x_j||^2). */
int oracle_kde_self(const double *X, int64_t n, int64_t d, double a, double *out, int threads) {
    if (n < 0 || d < 1 || !out) return -1;
    job_t b = {X, X, NULL, n, n, d, 0, n, a, 1, out, NULL, NULL, NULL};
    return launch(b, threads, run_sum);
}

/* K(q_j) = sum_i k(||q_j - x_i||) for kernel kind 0 (Gaussian), 1 (exponential) or
 * 2 (logistic). */
int oracle_kde_kernel(int kind, const double *X, int64_t n, const double *Q, int64_t m, int64_t d,
                      double a, double *out, int threads) {
    if (n < 0 || m < 0 || d < 1 || !out || kind < 0 || kind > 2) return -1;
    job_t b = {X, Q, NULL, n, m, d, 0, m, a, 0, out, NULL, NULL, NULL, kind, NULL, NULL};
    return launch(b, threads, run_sum);
}

/* Subset sums (see the header): off has m + 1 non-decreasing entries starting at 0, idx
 * and W (NULL: all weights 1) have off[m] entries. Returns -2 if an index is outside
 * [0, n). */
int oracle_kde_subset(int kind, const double *X, int64_t n, const double *Q, int64_t m, int64_t d,
                      double a, const int64_t *off, const int64_t *idx, const double *W, double *out,
                      int threads) {
    if (n < 0 || m < 0 || d < 1 || !out || !off || kind < 0 || kind > 2 || off[0] != 0) return -1;
    for (int64_t j = 0; j < m; ++j)
        if (off[j + 1] < off[j]) return -1;
    for (int64_t e = 0; e < off[m]; ++e)
        if (idx[e] < 0 || idx[e] >= n) return -2;
    job_t b = {X, Q, W, n, m, d, 0, m, a, 0, out, NULL, NULL, NULL, kind, off, idx};
    return launch(b, threads, run_subset);
}

int oracle_kde_log(const double *X, int64_t n, const double *Q, int64_t m, int64_t d, double a,
                   double *logk, double *d2min, double *kappa, int threads) {
    if (n < 1 || m < 0 || d < 1 || !logk || !d2min || !kappa) return -1;
    job_t b = {X, Q, NULL, n, m, d, 0, m, a, 0, NULL, logk, d2min, kappa};
    return launch(b, threads, run_log);
}
