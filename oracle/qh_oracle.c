/*
 * CPU oracle for the 2D convex hull (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this file's library.  The CUDA path never calls it and shares no code with it.
 *
 * What it computes (problem statement, Sec. 1 of Zhang, Mei, Xu, Zhao,
 * "A Novel Implementation of QuickHull Algorithm on the GPU"): the convex
 * polygon enclosing all planar input points, reported as the indices of its
 * strictly convex vertices in counter-clockwise order, starting at the
 * lexicographically smallest (x, then y) point.  Points on a hull edge are not
 * vertices.  Points with identical coordinates are represented by the lowest
 * input index.  Coordinates compare by value (-0 == +0).
 *
 * Two independent routes to that result:
 *
 *  qho_hull2d     Andrew's monotone chain (named in Sec. 1 and Sec. 3): sort
 *                 by (x, y, index), drop coordinate duplicates, build the
 *                 lower and upper chains popping while the turn is not
 *                 strictly counter-clockwise.
 *
 *  qho_quickhull  the generation-synchronous QuickHull rounds of Sec. 3-4.4:
 *                 initial split (chord A->B, or the quadrilateral of the four
 *                 extreme points of Sec. 4.2), then per generation: farthest
 *                 point of every segment (Sec. 4.4.1), new heads (Sec. 4.4.2),
 *                 discard of points not strictly right of A->C or C->B
 *                 (Sec. 4.4.3), regrouping into the new segments (Sec. 4.4.4).
 *                 It also reports the number of live points after each
 *                 generation, which pins the method's internal state.
 *
 * Every geometric decision is exact.  orient(a,b,c) = (bx-ax)(cy-ay) -
 * (by-ay)(cx-ax) is expanded into six products of input floats; each product is
 * exact in double.  A double-precision sum with a static bound decides the sign
 * when it can; otherwise the six products are summed exactly in a 640-bit
 * two's-complement fixed-point accumulator (every float is m * 2^e with an
 * integer |m| < 2^24, so every product is an integer below 2^48 times a power
 * of two between 2^-344 and 2^208).  The farthest-point comparison uses the
 * same machinery on eight products.
 *
 * Readings of points the paper leaves open (all also listed in the design notes):
 *  - farthest-point ties: larger distance, then lexicographically smaller
 *    (x, y), then lower index;
 *  - extreme points: A = lexicographic minimum of (x, y), B = maximum; the
 *    quadrilateral adds Bot = minimum of (y, x) and Top = maximum of (y, x),
 *    each skipped when it coincides with A or B; every tie goes to the lower
 *    index;
 *  - a point exactly on a dividing line is discarded (strictly-right test).
 *
 * QHO_MUTATION (compile-time, default 0) plants a known mistake; the test
 * suite builds such variants on the CPU to show that its pins catch them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef QHO_MUTATION
#define QHO_MUTATION 0
#endif

enum {
    QHO_OK = 0,
    QHO_ERR_INVALID_ARG = 1,
    QHO_ERR_NONFINITE = 2,
    QHO_ERR_OOM = 4,
    QHO_ERR_INTERNAL = 7
};

/* ------------------------------------------------------------------------- */
/* Exact sums of products of floats                                           */
/* ------------------------------------------------------------------------- */

#define ACC_LIMBS 10   /* 640 bits */
#define ACC_BIAS 352   /* bit 0 of the accumulator weighs 2^-352 */

typedef struct {
    uint64_t w[ACC_LIMBS];
} acc_t;

/* x = m * 2^e with m an integer, |m| < 2^24 (exact for every finite float). */
static void split_float(float x, int64_t *m, int *e)
{
    int ex = 0;
    float f = frexpf(x, &ex); /* x = f * 2^ex, 0.5 <= |f| < 1, or f == 0 */
    *m = (int64_t)ldexpf(f, 24);
    *e = ex - 24;
}

/* a += m * 2^e, with |m| < 2^62 and e + ACC_BIAS in [0, 575]. */
static void acc_add(acc_t *a, int64_t m, int e)
{
    uint64_t part[ACC_LIMBS];
    uint64_t mag;
    int sh, li, off, i;
    if (m == 0)
        return;
    mag = (uint64_t)(m < 0 ? -m : m);
    sh = e + ACC_BIAS;
    li = sh >> 6;
    off = sh & 63;
    memset(part, 0, sizeof(part));
    part[li] = mag << off;
    if (off != 0 && li + 1 < ACC_LIMBS)
        part[li + 1] = mag >> (64 - off);
    if (m > 0) {
        uint64_t carry = 0;
        for (i = 0; i < ACC_LIMBS; i++) {
            uint64_t s = a->w[i] + part[i];
            uint64_t c1 = s < part[i];
            uint64_t s2 = s + carry;
            uint64_t c2 = s2 < s;
            a->w[i] = s2;
            carry = c1 | c2;
        }
    } else {
        uint64_t borrow = 0;
        for (i = 0; i < ACC_LIMBS; i++) {
            uint64_t d = a->w[i] - part[i];
            uint64_t b1 = a->w[i] < part[i];
            uint64_t d2 = d - borrow;
            uint64_t b2 = d < borrow;
            a->w[i] = d2;
            borrow = b1 | b2;
        }
    }
}

static int acc_sign(const acc_t *a)
{
    int i;
    if (a->w[ACC_LIMBS - 1] >> 63)
        return -1;
    for (i = 0; i < ACC_LIMBS; i++)
        if (a->w[i] != 0)
            return 1;
    return 0;
}

/* a += s * x * y exactly (s = +1 or -1). */
static void acc_add_product(acc_t *a, float x, float y, int s)
{
    int64_t mx, my;
    int ex, ey;
    split_float(x, &mx, &ex);
    split_float(y, &my, &ey);
    acc_add(a, (int64_t)s * mx * my, ex + ey);
}

/* The sign of sum_k s_k * x_k * y_k: a double filter, then the exact sum. */
static int sign_of_products(int k, const float *x, const float *y, const int *s, int always_exact)
{
    int i;
    if (!always_exact) {
        double sum = 0.0, mag = 0.0;
        for (i = 0; i < k; i++) {
            double p = (double)x[i] * (double)y[i]; /* exact: 24 x 24 bits */
            if (s[i] < 0)
                p = -p;
            sum += p;
            mag += fabs(p);
        }
        /* Recursive summation of k <= 8 exact terms errs by at most
         * (k-1) 2^-53 (1 + small) * mag; 2^-40 * mag leaves a wide margin. */
#if QHO_MUTATION == 5
        if (sum != 0.0)
#else
        if (fabs(sum) > mag * 0x1p-40)
#endif
            return sum > 0.0 ? 1 : -1;
    }
    {
        acc_t a;
        memset(&a, 0, sizeof(a));
        for (i = 0; i < k; i++)
            acc_add_product(&a, x[i], y[i], s[i]);
        return acc_sign(&a);
    }
}

/* sign of orient(a, b, c) = (bx-ax)(cy-ay) - (by-ay)(cx-ax)
 *   = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx. */
static int orient_sign(float ax, float ay, float bx, float by, float cx, float cy, int always_exact)
{
    float x[6] = {bx, bx, ax, by, by, ay};
    float y[6] = {cy, ay, cy, cx, ax, cx};
#if QHO_MUTATION == 2
    int s[6] = {+1, -1, -1, -1, -1, +1};
#else
    int s[6] = {+1, -1, -1, -1, +1, +1};
#endif
    return sign_of_products(6, x, y, s, always_exact);
}

/* Distance of P beyond the directed chord u->v is dist(P) = -orient(u, v, P),
 * positive for points strictly to the right.  Returns sign(dist(P) - dist(Q)):
 *   dist(P) - dist(Q) = -(vx-ux)(Py-Qy) + (vy-uy)(Px-Qx)
 *     = -vx*Py + vx*Qy + ux*Py - ux*Qy + vy*Px - vy*Qx - uy*Px + uy*Qx. */
static int dist_cmp(float ux, float uy, float vx, float vy, float px, float py, float qx, float qy,
                    int always_exact)
{
    float x[8] = {vx, vx, ux, ux, vy, vy, uy, uy};
    float y[8] = {py, qy, py, qy, px, qx, px, qx};
    int s[8] = {-1, +1, +1, -1, +1, -1, -1, +1};
    return sign_of_products(8, x, y, s, always_exact);
}

/* Exported wrappers so the tests can pin the predicates themselves. */
int qho_orient_sign(float ax, float ay, float bx, float by, float cx, float cy, int always_exact)
{
    return orient_sign(ax, ay, bx, by, cx, cy, always_exact);
}

int qho_dist_cmp(float ux, float uy, float vx, float vy, float px, float py, float qx, float qy,
                 int always_exact)
{
    return dist_cmp(ux, uy, vx, vy, px, py, qx, qy, always_exact);
}

/* ------------------------------------------------------------------------- */
/* Monotone chain                                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    float x, y;
    int32_t i;
} pt_t;

static int cmp_pt(const void *pa, const void *pb)
{
    const pt_t *a = (const pt_t *)pa, *b = (const pt_t *)pb;
    if (a->x < b->x) return -1;
    if (a->x > b->x) return 1;
#if QHO_MUTATION == 4
    if (a->y > b->y) return -1;
    if (a->y < b->y) return 1;
#else
    if (a->y < b->y) return -1;
    if (a->y > b->y) return 1;
#endif
    return (a->i > b->i) - (a->i < b->i);
}

static int all_finite(const float *xy, int64_t n)
{
    int64_t k;
    for (k = 0; k < 2 * n; k++)
        if (!isfinite(xy[k]))
            return 0;
    return 1;
}

static int turn_pops(const pt_t *a, const pt_t *b, const pt_t *c, int always_exact)
{
    int s = orient_sign(a->x, a->y, b->x, b->y, c->x, c->y, always_exact);
#if QHO_MUTATION == 1
    return s < 0;  /* keeps collinear boundary points */
#else
    return s <= 0;
#endif
}

/* Convex hull of n points xy[2k], xy[2k+1]; out must hold n entries. */
int qho_hull2d(const float *xy, int64_t n, int32_t *out, int64_t *out_count, int always_exact)
{
    pt_t *p;
    int64_t *h;
    int64_t m, k, t, i;
    if (n < 0 || !out_count || (n > 0 && (!xy || !out)) || n > INT32_MAX)
        return QHO_ERR_INVALID_ARG;
    *out_count = 0;
    if (n == 0)
        return QHO_OK;
    if (!all_finite(xy, n))
        return QHO_ERR_NONFINITE;
    p = (pt_t *)malloc((size_t)n * sizeof(pt_t));
    if (!p)
        return QHO_ERR_OOM;
    for (i = 0; i < n; i++) {
        p[i].x = xy[2 * i];
        p[i].y = xy[2 * i + 1];
        p[i].i = (int32_t)i;
    }
    qsort(p, (size_t)n, sizeof(pt_t), cmp_pt);
    /* drop coordinate duplicates, keeping the lowest index (first after the sort) */
    m = 0;
    for (i = 0; i < n; i++) {
        if (m == 0 || p[i].x != p[m - 1].x || p[i].y != p[m - 1].y) {
            p[m++] = p[i];
        }
#if QHO_MUTATION == 3
        else {
            p[m - 1] = p[i]; /* keeps the highest index instead */
        }
#endif
    }
    if (m == 1) {
        out[0] = p[0].i;
        *out_count = 1;
        free(p);
        return QHO_OK;
    }
    h = (int64_t *)malloc((size_t)(2 * m) * sizeof(int64_t));
    if (!h) {
        free(p);
        return QHO_ERR_OOM;
    }
    k = 0;
    for (i = 0; i < m; i++) { /* lower chain, left to right */
        while (k >= 2 && turn_pops(&p[h[k - 2]], &p[h[k - 1]], &p[i], always_exact))
            k--;
        h[k++] = i;
    }
    t = k + 1;
    for (i = m - 2; i >= 0; i--) { /* upper chain, right to left */
        while (k >= t && turn_pops(&p[h[k - 2]], &p[h[k - 1]], &p[i], always_exact))
            k--;
        h[k++] = i;
    }
    /* the last entry repeats the first point; a correct chain holds at most m
     * distinct vertices */
    if (k - 1 > m) {
        free(h);
        free(p);
        return QHO_ERR_INTERNAL;
    }
    for (i = 0; i < k - 1; i++)
        out[i] = p[h[i]].i;
    *out_count = k - 1;
    free(h);
    free(p);
    return QHO_OK;
}

/* Batched: set s occupies xy[offsets[s] .. offsets[s+1]); its hull (indices
 * local to the set) goes to out + offsets[s], its vertex count to counts[s]
 * (or -status when the set is rejected).  Returns the first error seen. */
int qho_hull2d_batched(const float *xy, const int64_t *offsets, int32_t num_sets, int32_t *out,
                       int32_t *counts, int always_exact)
{
    int32_t s;
    int first = QHO_OK;
    if (num_sets < 0 || (num_sets > 0 && (!offsets || !counts)))
        return QHO_ERR_INVALID_ARG;
    for (s = 0; s < num_sets; s++) {
        int64_t a = offsets[s], b = offsets[s + 1], c = 0;
        int st;
        if (b < a)
            return QHO_ERR_INVALID_ARG;
        st = qho_hull2d(xy + 2 * a, b - a, out + a, &c, always_exact);
        counts[s] = st == QHO_OK ? (int32_t)c : -st;
        if (st != QHO_OK && first == QHO_OK)
            first = st;
    }
    return first;
}

/* ------------------------------------------------------------------------- */
/* Generation-synchronous QuickHull (Sec. 3 and 4 of the paper)               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t head;  /* input index of the segment's first (head) point */
    int64_t begin; /* its points occupy pts[begin .. begin + count) */
    int64_t count;
} seg_t;

#define PX(i) (xy[2 * (int64_t)(i)])
#define PY(i) (xy[2 * (int64_t)(i) + 1])

/* Lexicographic order of (a0, a1, index): < 0 when point i precedes point j. */
static int lex_cmp(float ai0, float ai1, int32_t i, float aj0, float aj1, int32_t j)
{
    if (ai0 != aj0) return ai0 < aj0 ? -1 : 1;
    if (ai1 != aj1) return ai1 < aj1 ? -1 : 1;
    return (i > j) - (i < j);
}

/* Is P (index p) a better farthest point than Q for chord h->e? */
static int farther(const float *xy, int32_t h, int32_t e, int32_t p, int32_t q)
{
    int s = dist_cmp(PX(h), PY(h), PX(e), PY(e), PX(p), PY(p), PX(q), PY(q), 0);
    if (s != 0)
        return s > 0;
    if (PX(p) != PX(q)) return PX(p) < PX(q);
    if (PY(p) != PY(q)) return PY(p) < PY(q);
#if QHO_MUTATION == 6
    return p > q;
#else
    return p < q;
#endif
}

static int strictly_right(const float *xy, int32_t u, int32_t v, int32_t p)
{
    return orient_sign(PX(u), PY(u), PX(v), PY(v), PX(p), PY(p), 0) < 0;
}

/*
 * mode 0: initial chord A->B, B->A (the paper's Mode 2);
 * mode 1: initial quadrilateral A->Bot->B->Top (the paper's Mode 1 pre-step).
 * live[g] receives the number of points held by segments after generation g
 * (generation 0 is the initial split), for g < max_gen; *n_gen receives the
 * number of generations run (also beyond max_gen).
 */
int qho_quickhull(const float *xy, int64_t n, int mode, int32_t *out, int64_t *out_count,
                  int64_t *live, int max_gen, int *n_gen)
{
    int32_t a = 0, b = 0, bot = 0, top = 0, poly[4];
    int npoly = 0, gen = 0;
    int64_t i, nseg, nseg2, pos, total;
    int32_t *cur, *nxt;
    seg_t *seg, *seg2;
    if (n < 0 || !out_count || !n_gen || (n > 0 && (!xy || !out)) || n > INT32_MAX ||
        (max_gen > 0 && !live))
        return QHO_ERR_INVALID_ARG;
    *out_count = 0;
    *n_gen = 0;
    if (n == 0)
        return QHO_OK;
    if (!all_finite(xy, n))
        return QHO_ERR_NONFINITE;

    /* Sec. 4.2: extreme points (ties to the lower index) */
    for (i = 1; i < n; i++) {
        int32_t k = (int32_t)i;
        if (lex_cmp(PX(k), PY(k), k, PX(a), PY(a), a) < 0) a = k;
        if (lex_cmp(PX(k), PY(k), -k, PX(b), PY(b), -b) > 0) b = k;
        if (lex_cmp(PY(k), PX(k), k, PY(bot), PX(bot), bot) < 0) bot = k;
        if (lex_cmp(PY(k), PX(k), -k, PY(top), PX(top), -top) > 0) top = k;
    }
    if (PX(a) == PX(b) && PY(a) == PY(b)) {
        out[0] = a;
        *out_count = 1;
        return QHO_OK;
    }
    poly[npoly++] = a;
    if (mode == 1 && !(PX(bot) == PX(a) && PY(bot) == PY(a)) && !(PX(bot) == PX(b) && PY(bot) == PY(b)))
        poly[npoly++] = bot;
    poly[npoly++] = b;
    if (mode == 1 && !(PX(top) == PX(a) && PY(top) == PY(a)) && !(PX(top) == PX(b) && PY(top) == PY(b)))
        poly[npoly++] = top;

    cur = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    nxt = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    seg = (seg_t *)malloc((size_t)(n + 4) * sizeof(seg_t));
    seg2 = (seg_t *)malloc((size_t)(n + 4) * sizeof(seg_t));
    if (!cur || !nxt || !seg || !seg2) {
        free(cur); free(nxt); free(seg); free(seg2);
        return QHO_ERR_OOM;
    }

    /* Sec. 4.3 / 4.2: the first split; a point joins the first polygon edge it
     * lies strictly right of, and is discarded when there is none.  The owner
     * of point p is kept in nxt[p] (-1: discarded) before the regrouping. */
    for (i = 0; i < n; i++) {
        int32_t p = (int32_t)i;
        int k;
        nxt[i] = -1;
        for (k = 0; k < npoly; k++) {
            if (strictly_right(xy, poly[k], poly[(k + 1) % npoly], p)) {
                nxt[i] = k;
                break;
            }
        }
    }
    pos = 0;
    for (int k = 0; k < npoly; k++) {
        seg[k].head = poly[k];
        seg[k].begin = pos;
        for (i = 0; i < n; i++)
            if (nxt[i] == k)
                cur[pos++] = (int32_t)i;
        seg[k].count = pos - seg[k].begin;
    }
    nseg = npoly;
    if (max_gen > 0)
        live[0] = pos;
    gen = 1;

    /* Sec. 4.4: rounds until no segment holds points */
    for (;;) {
        total = 0;
        for (i = 0; i < nseg; i++)
            total += seg[i].count;
        if (total == 0)
            break;
        nseg2 = 0;
        pos = 0;
        for (i = 0; i < nseg; i++) {
            int32_t h = seg[i].head, e = seg[(i + 1) % nseg].head, c;
            int64_t j, b0, b1;
            /* a correct run has at most one segment per distinct vertex */
            if (nseg2 + 2 > n + 4) {
                free(cur); free(nxt); free(seg); free(seg2);
                return QHO_ERR_INTERNAL;
            }
            if (seg[i].count == 0) {
                seg2[nseg2].head = h;
                seg2[nseg2].begin = pos;
                seg2[nseg2].count = 0;
                nseg2++;
                continue;
            }
            /* Sec. 4.4.1: the farthest point of the segment from its chord */
            c = cur[seg[i].begin];
            for (j = 1; j < seg[i].count; j++) {
                int32_t p = cur[seg[i].begin + j];
                if (farther(xy, h, e, p, c))
                    c = p;
            }
            /* Sec. 4.4.3: keep points strictly right of h->c or of c->e */
            b0 = pos;
            for (j = 0; j < seg[i].count; j++) {
                int32_t p = cur[seg[i].begin + j];
                if (strictly_right(xy, h, c, p))
                    nxt[pos++] = p;
            }
            b1 = pos;
            for (j = 0; j < seg[i].count; j++) {
                int32_t p = cur[seg[i].begin + j];
                if (!strictly_right(xy, h, c, p) && strictly_right(xy, c, e, p))
                    nxt[pos++] = p;
            }
            /* Sec. 4.4.2 / 4.4.4: c becomes the head of the second new segment */
            seg2[nseg2].head = h;
            seg2[nseg2].begin = b0;
            seg2[nseg2].count = b1 - b0;
            nseg2++;
            seg2[nseg2].head = c;
            seg2[nseg2].begin = b1;
            seg2[nseg2].count = pos - b1;
            nseg2++;
        }
        if (gen < max_gen)
            live[gen] = pos;
        gen++;
        {
            int32_t *t = cur; cur = nxt; nxt = t;
        }
        {
            seg_t *t = seg; seg = seg2; seg2 = t;
        }
        nseg = nseg2;
    }
    for (i = 0; i < nseg; i++)
        out[i] = seg[i].head;
    *out_count = nseg;
    *n_gen = gen;
    free(cur); free(nxt); free(seg); free(seg2);
    return QHO_OK;
}
