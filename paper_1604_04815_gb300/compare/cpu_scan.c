/* cpu_scan.c -- a comparator for the benchmark, not part of the scan
 * library: a multi-threaded inclusive scan on the host cores, the
 * counterpart of the paper's comparison with a parallel CPU library (TBB on
 * 16 cores, Section 5.3).  Reduce-then-scan over contiguous chunks, one per
 * thread: each thread folds its chunk, the chunk totals are scanned in
 * order, and each thread scans its chunk again from its offset -- the input
 * is read twice and the output written once.  Built into its own shared
 * library (libcpuscan.so); liblscan.so does not link or call it.  The
 * oracle stays the plain sequential loop of oracle/. */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

/* op: 0 add, 1 max; dtype: 0 int32 (add wraps modulo 2^32), 1 fp32 */
typedef struct {
    int op, dtype;
    const void *x;
    void *y;
    int64_t lo, hi;  /* [lo, hi) */
    double total;    /* fp32 chunk total (pass 1) */
    int64_t itotal;  /* int32 chunk total as int64 (add: mod 2^32) */
    double off;      /* carry-in of the chunk (pass 2) */
    int64_t ioff;
    int has_off;
    int pass;
} job;

static int32_t wrap_add(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a + (uint32_t)b);
}

static void *run(void *arg) {
    job *j = (job *)arg;
    if (j->dtype == 0) {
        const int32_t *x = (const int32_t *)j->x;
        int32_t *y = (int32_t *)j->y;
        if (j->pass == 1) {
            int32_t acc = j->op == 0 ? 0 : INT32_MIN;
            for (int64_t i = j->lo; i < j->hi; ++i)
                acc = j->op == 0 ? wrap_add(acc, x[i]) : (x[i] > acc ? x[i] : acc);
            j->itotal = acc;
        } else {
            int32_t acc = j->has_off ? (int32_t)j->ioff : (j->op == 0 ? 0 : INT32_MIN);
            for (int64_t i = j->lo; i < j->hi; ++i) {
                acc = j->op == 0 ? wrap_add(acc, x[i]) : (x[i] > acc ? x[i] : acc);
                y[i] = acc;
            }
        }
    } else {
        const float *x = (const float *)j->x;
        float *y = (float *)j->y;
        if (j->pass == 1) {
            float acc = j->op == 0 ? 0.0f : -INFINITY;
            for (int64_t i = j->lo; i < j->hi; ++i)
                acc = j->op == 0 ? acc + x[i] : (x[i] > acc ? x[i] : acc);
            j->total = acc;
        } else {
            float acc = j->has_off ? (float)j->off : (j->op == 0 ? 0.0f : -INFINITY);
            for (int64_t i = j->lo; i < j->hi; ++i) {
                acc = j->op == 0 ? acc + x[i] : (x[i] > acc ? x[i] : acc);
                y[i] = acc;
            }
        }
    }
    return NULL;
}

/* Inclusive scan of n elements of x (host memory) into y with `threads`
 * threads (1 .. 256).  Returns 0, or -1 on bad arguments or a thread that
 * could not start. */
int cpuscan_inclusive(int op, int dtype, const void *x, void *y, int64_t n, int threads) {
    if ((op != 0 && op != 1) || (dtype != 0 && dtype != 1) || n < 0 || threads < 1 ||
        threads > 256 || (n > 0 && (x == NULL || y == NULL)))
        return -1;
    if (n == 0) return 0;
    if ((int64_t)threads > n) threads = (int)n;
    job *jobs = (job *)calloc((size_t)threads, sizeof(job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -1;
    }
    const int64_t per = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        jobs[t].op = op;
        jobs[t].dtype = dtype;
        jobs[t].x = x;
        jobs[t].y = y;
        jobs[t].lo = (int64_t)t * per < n ? (int64_t)t * per : n;
        jobs[t].hi = (int64_t)(t + 1) * per < n ? (int64_t)(t + 1) * per : n;
    }
    int rc = 0;
    for (int pass = 1; pass <= 2 && rc == 0; ++pass) {
        if (pass == 2) {
            /* carry-ins: the chunk totals folded in chunk order */
            for (int t = 1; t < threads; ++t) {
                jobs[t].has_off = 1;
                if (dtype == 0) {
                    const int32_t prev = jobs[t - 1].has_off ? (int32_t)jobs[t - 1].ioff
                                                              : (op == 0 ? 0 : INT32_MIN);
                    const int32_t tot = (int32_t)jobs[t - 1].itotal;
                    jobs[t].ioff = op == 0 ? wrap_add(prev, tot) : (tot > prev ? tot : prev);
                } else {
                    const float prev = jobs[t - 1].has_off ? (float)jobs[t - 1].off
                                                           : (op == 0 ? 0.0f : -INFINITY);
                    const float tot = (float)jobs[t - 1].total;
                    jobs[t].off = op == 0 ? prev + tot : (tot > prev ? tot : prev);
                }
            }
        }
        int started = 0;
        for (int t = 0; t < threads; ++t) {
            jobs[t].pass = pass;
            if (pthread_create(&tid[t], NULL, run, &jobs[t]) != 0) {
                rc = -1;
                break;
            }
            ++started;
        }
        for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    }
    free(jobs);
    free(tid);
    return rc;
}
