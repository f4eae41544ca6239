/* All-core build of the oracle's monotone chain -- TEST AND BASELINE
 * INFRASTRUCTURE ONLY (the CPU-baseline leg of bench.py and its tests).
 *
 * The oracle source is included unchanged.  This file adds one driver,
 * qho_hull2d_parallel: the oracle's hull of T contiguous chunks of the input
 * in T threads, then the oracle's hull once more over the union of the chunk
 * hulls.  The result is the single-thread result:
 *   - a vertex of the hull of the whole set is a vertex of the hull of every
 *     subset holding it, so the union of the chunk hulls holds every vertex;
 *   - among points with equal coordinates the oracle keeps the lowest index;
 *     the lowest-index copy of a vertex is the lowest in its own chunk, and
 *     the union is handed to the second pass in increasing input index, so the
 *     second pass keeps that copy too;
 *   - both passes start at the lexicographically smallest point and run CCW.
 * A non-finite coordinate makes a chunk, and so the call, return
 * QHO_ERR_NONFINITE, as the single-thread call does.
 */
#include "qh_oracle.c"

#include <pthread.h>

typedef struct {
    const float *xy;
    int64_t off, n, cnt;
    int32_t *out;
    int st;
    int started; /* written by the calling thread only */
} qhop_chunk_t;

static void *qhop_run(void *arg)
{
    qhop_chunk_t *c = (qhop_chunk_t *)arg;
    c->st = qho_hull2d(c->xy + 2 * c->off, c->n, c->out, &c->cnt, 0);
    return NULL;
}

static int qhop_cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Convex hull of n points with `threads` threads; out must hold n entries. */
int qho_hull2d_parallel(const float *xy, int64_t n, int32_t *out, int64_t *out_count, int threads)
{
    qhop_chunk_t *c;
    pthread_t *th;
    int32_t *part, *idx, *cout;
    float *cxy;
    int64_t total, k, m, ccnt = 0;
    int t, T = threads, st = QHO_OK;
    if (n < 0 || !out_count || (n > 0 && (!xy || !out)) || n > INT32_MAX)
        return QHO_ERR_INVALID_ARG;
    if (T > 256)
        T = 256;
    if (T < 2 || n < (int64_t)T * 4096)
        return qho_hull2d(xy, n, out, out_count, 0);
    *out_count = 0;
    c = (qhop_chunk_t *)calloc((size_t)T, sizeof(*c));
    th = (pthread_t *)calloc((size_t)T, sizeof(*th));
    part = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!c || !th || !part) {
        free(c);
        free(th);
        free(part);
        return QHO_ERR_OOM;
    }
    for (t = 0; t < T; t++) {
        c[t].xy = xy;
        c[t].off = n * t / T;
        c[t].n = n * (t + 1) / T - c[t].off;
        c[t].out = part + c[t].off; /* a chunk's hull has at most its own points */
    }
    for (t = 1; t < T; t++)
        c[t].started = pthread_create(&th[t], NULL, qhop_run, &c[t]) == 0;
    qhop_run(&c[0]);
    for (t = 1; t < T; t++) {
        if (c[t].started)
            pthread_join(th[t], NULL);
        else
            qhop_run(&c[t]); /* no thread could be started: run the chunk here */
    }
    total = 0;
    for (t = 0; t < T; t++) {
        if (c[t].st != QHO_OK && st == QHO_OK)
            st = c[t].st;
        total += c[t].cnt > 0 ? c[t].cnt : 0;
    }
    if (st != QHO_OK) {
        free(c);
        free(th);
        free(part);
        return st;
    }
    idx = (int32_t *)malloc((size_t)total * sizeof(int32_t));
    cxy = (float *)malloc((size_t)total * 2 * sizeof(float));
    cout = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!idx || !cxy || !cout) {
        free(idx);
        free(cxy);
        free(cout);
        free(c);
        free(th);
        free(part);
        return QHO_ERR_OOM;
    }
    m = 0;
    for (t = 0; t < T; t++)
        for (k = 0; k < c[t].cnt; k++)
            idx[m++] = (int32_t)(c[t].off + part[c[t].off + k]);
    qsort(idx, (size_t)m, sizeof(int32_t), qhop_cmp_i32);
    for (k = 0; k < m; k++) {
        cxy[2 * k] = xy[2 * (int64_t)idx[k]];
        cxy[2 * k + 1] = xy[2 * (int64_t)idx[k] + 1];
    }
    st = qho_hull2d(cxy, m, cout, &ccnt, 0);
    if (st == QHO_OK) {
        for (k = 0; k < ccnt; k++)
            out[k] = idx[cout[k]];
        *out_count = ccnt;
    }
    free(idx);
    free(cxy);
    free(cout);
    free(c);
    free(th);
    free(part);
    return st;
}
