/*
 * CPU oracle for exact k-nearest-neighbour search — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product (the CUDA library) never calls it.
 *
 * What it computes is the plain definition of the problem the paper's kd-tree
 * and BDL-tree answer exactly (Section 5, "Data-Parallel k-NN", and Appendix
 * A.1.3): for each query point q and the live data points p_t,
 *
 *     D(q, t) = sum_c (q_c - p_{t,c})^2          (evaluated in float64),
 *
 * and the answer is the k smallest (D, id_t) pairs in lexicographic order, i.e.
 * ties on D are broken by the smaller point id.  When fewer than k live points
 * exist, the remaining slots are padded with id -1 and distance +inf.
 *
 * No tree, no pruning, no blocking: every query is compared with every live
 * point, and the k best are kept in a sorted list by insertion.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    double d;
    int64_t id;
} cand;

static int cand_less(cand a, cand b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

/* The k smallest (D, id) pairs for one query, by exhaustive comparison. */
static void knn_one(const float *data, int64_t n, const float *q, int dim, int k,
                    const uint8_t *live, const int64_t *ids, cand *best,
                    int64_t *out_idx, double *out_dist) {
    int cnt = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (live && !live[t]) continue;
        double D = 0.0;
        for (int c = 0; c < dim; ++c) {
            double diff = (double)q[c] - (double)data[t * (int64_t)dim + c];
            D += diff * diff;
        }
        cand x = {D, ids ? ids[t] : t};
        if (cnt < k) {
            int j = cnt++;
            while (j > 0 && cand_less(x, best[j - 1])) { best[j] = best[j - 1]; --j; }
            best[j] = x;
        } else if (cand_less(x, best[k - 1])) {
            int j = k - 1;
            while (j > 0 && cand_less(x, best[j - 1])) { best[j] = best[j - 1]; --j; }
            best[j] = x;
        }
    }
    for (int j = 0; j < k; ++j) {
        if (j < cnt) { out_idx[j] = best[j].id; out_dist[j] = best[j].d; }
        else { out_idx[j] = -1; out_dist[j] = INFINITY; }
    }
}

typedef struct {
    const float *data; int64_t n; const float *queries; int64_t q0, q1;
    int dim, k; const uint8_t *live; const int64_t *ids;
    int64_t *out_idx; double *out_dist;
} job;

static void *run_job(void *arg) {
    job *j = (job *)arg;
    cand *best = (cand *)malloc(sizeof(cand) * (size_t)(j->k > 0 ? j->k : 1));
    for (int64_t i = j->q0; i < j->q1; ++i)
        knn_one(j->data, j->n, j->queries + i * (int64_t)j->dim, j->dim, j->k, j->live, j->ids,
                best, j->out_idx + i * (int64_t)j->k, j->out_dist + i * (int64_t)j->k);
    free(best);
    return NULL;
}

/* Number of host threads used when nthreads <= 0. */
int oracle_default_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/*
 * Exact k-NN by brute force.
 *   data     n*dim float32, row-major     queries  m*dim float32, row-major
 *   live     n bytes (nonzero = live) or NULL (all live)
 *   ids      n int64 point ids or NULL (id = row index)
 *   out_idx  m*k int64, out_dist m*k float64 (squared Euclidean distance)
 *   nthreads threads over queries (<= 0: all online cores).  The result does not
 *            depend on it.
 * Returns 0, or -1 on invalid arguments.
 */
int oracle_knn_f64(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                   const uint8_t *live, const int64_t *ids, int64_t *out_idx, double *out_dist,
                   int nthreads) {
    if (n < 0 || m < 0 || dim < 1 || k < 1) return -1;
    if (m == 0) return 0;
    if (nthreads <= 0) nthreads = oracle_default_threads();
    if (nthreads > m) nthreads = (int)m;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    job *jobs = (job *)malloc(sizeof(job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        job j = {data, n, queries, m * t / nthreads, m * (t + 1) / nthreads, dim, k, live, ids,
                 out_idx, out_dist};
        jobs[t] = j;
        pthread_create(&th[t], NULL, run_job, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return 0;
}
