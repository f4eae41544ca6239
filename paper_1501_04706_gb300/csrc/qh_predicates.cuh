// Exact geometric predicates for the hull kernels (host + device).
//
// orient(u, v, p) = (vx-ux)(py-uy) - (vy-uy)(px-ux): > 0 when p is left of the
// directed line u->v.  A point is outside a CCW hull edge u->v when it is
// strictly right (orient < 0), the "right side of the directed line AC and CB"
// test of Sec. 4.4.3.  Its distance beyond the edge is dist(p) = -orient(u,v,p);
// the paper's distance (Sec. 4.4.1) differs from it by the positive factor
// 1/|uv|, so the farthest point is the same and no division is needed.
//
// Fast path (the "filter"): the difference form evaluated in P = float or
// double with round-to-nearest and no fused multiply-add.  Error analysis (our
// derivation): with unit roundoff u, the two rounded differences feeding each
// product, the two products and the final subtraction give
//     |det - D| <= (4u + O(u^2)) (|l| + |r|),
// l and r being the two rounded products.  We use 5u * fl(|l| + |r|), which
// covers the O(u^2) terms and the rounding of the bound itself.  In FP32 the
// bound gets an absolute floor of 2^-140: a product that underflowed is off by
// at most 2^-150 and a subnormal difference is exact, so below |l| + |r| =
// 2^-96 the floor covers every error and above it the slack u (|l| + |r|)
// does.  A sum |l| + |r| that overflowed (or is NaN: inf * 0) marks the value
// unusable and the point goes to the exact path.  In FP64 the products of
// float differences neither underflow nor overflow.
//
// Exact path: every float x float product is exact in FP64; the sign of a sum of
// such products is the sign of the top non-zero component of the nonoverlapping
// expansion built with Knuth's TwoSum by Shewchuk's GROW-EXPANSION (Shewchuk,
// "Adaptive precision floating-point arithmetic and fast robust geometric
// predicates", 1997).  orient needs 6 products, the farthest-point comparison 8.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define QH_HD __host__ __device__ __forceinline__
// The exact fallback is rare: kept out of line so its registers do not burden the fast path.
#define QH_HD_COLD static __host__ __device__ __noinline__
#else
#define QH_HD inline
#define QH_HD_COLD static inline
#endif

namespace qh {

// ---------------------------------------------------------------------------
// Rounding-explicit arithmetic: intrinsics on the device (never contracted into
// FMA); plain operators on the host, where the library is compiled with
// -ffp-contract=off.
// ---------------------------------------------------------------------------
QH_HD float radd(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
QH_HD float rsub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
QH_HD float rmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
QH_HD double radd(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
QH_HD double rsub(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
QH_HD double rmul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
// a - b rounded toward -inf / a + b rounded toward +inf.
QH_HD float sub_down(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rd(a, b);
#else
    return std::nextafter(a - b, -INFINITY);
#endif
}
QH_HD float add_up(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_ru(a, b);
#else
    return std::nextafter(a + b, INFINITY);
#endif
}
QH_HD double sub_down(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rd(a, b);
#else
    return std::nextafter(a - b, -INFINITY);
#endif
}
QH_HD double add_up(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_ru(a, b);
#else
    return std::nextafter(a + b, INFINITY);
#endif
}

template <typename P> struct Lim;
template <> struct Lim<float> {
    static QH_HD float errc() { return 5.0f * 0x1p-24f; }
    static QH_HD float efloor() { return 0x1p-140f; }
    static QH_HD float smax() { return FLT_MAX; }
};
template <> struct Lim<double> {
    static QH_HD double errc() { return 5.0 * 0x1p-53; }
    static QH_HD double efloor() { return 0.0; }
    static QH_HD double smax() { return DBL_MAX; }
};

QH_HD float rmax(float a, float b) { return a > b ? a : b; }
QH_HD double rmax(double a, double b) { return a > b ? a : b; }

// A directed edge u->v with its rounded direction, the constants every
// orientation test against it reuses.
template <typename P> struct Edge {
    float ux, uy;
    P ex, ey;
};

template <typename P> QH_HD Edge<P> make_edge(float ux, float uy, float vx, float vy) {
    Edge<P> e;
    e.ux = ux;
    e.uy = uy;
    e.ex = rsub(P(vx), P(ux));
    e.ey = rsub(P(vy), P(uy));
    return e;
}

// Filtered orientation of p against edge e: det ~ orient(u, v, p), |det - D| <= err
// when ok is true.
template <typename P> struct Approx {
    P det, err;
    bool ok;
};

template <typename P> QH_HD Approx<P> orient_approx(const Edge<P> &e, float px, float py) {
    P a = rsub(P(py), P(e.uy));
    P b = rsub(P(px), P(e.ux));
    P l = rmul(e.ex, a);
    P r = rmul(e.ey, b);
    Approx<P> o;
    o.det = rsub(l, r);
    P s = radd(l < P(0) ? -l : l, r < P(0) ? -r : r);
    o.err = rmax(rmul(s, Lim<P>::errc()), Lim<P>::efloor());
    o.ok = s <= Lim<P>::smax();
    return o;
}

// --------------------------- exact fallback --------------------------------
QH_HD void two_sum(double a, double b, double &s, double &e) {
    s = radd(a, b);
    double bb = rsub(s, a);
    e = radd(rsub(a, rsub(s, bb)), rsub(b, bb));
}

// Sign of t[0] + ... + t[n-1] (each an exact double), n <= 8.
QH_HD int expansion_sign(const double *t, int n) {
    double h[8];
    int m = 0;
    for (int i = 0; i < n; i++) {
        double q = t[i];
        for (int j = 0; j < m; j++) {
            double s, err;
            two_sum(q, h[j], s, err);
            h[j] = err;
            q = s;
        }
        h[m++] = q;
    }
    for (int j = m - 1; j >= 0; j--)
        if (h[j] != 0.0)
            return h[j] > 0.0 ? 1 : -1;
    return 0;
}

QH_HD double xp(float a, float b) { return rmul(double(a), double(b)); }

// orient(a,b,c) = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx, exactly.
QH_HD_COLD int orient_exact(float ax, float ay, float bx, float by, float cx, float cy) {
    double t[6] = {xp(bx, cy), -xp(bx, ay), -xp(ax, cy), -xp(by, cx), xp(by, ax), xp(ay, cx)};
    return expansion_sign(t, 6);
}

// sign(dist(p) - dist(q)) for the chord u->v, dist(x) = -orient(u, v, x):
//   -(vx-ux)(py-qy) + (vy-uy)(px-qx), expanded into eight exact products.
QH_HD_COLD int dist_cmp_exact(float ux, float uy, float vx, float vy, float px, float py, float qx, float qy) {
    double t[8] = {-xp(vx, py), xp(vx, qy), xp(ux, py), -xp(ux, qy),
                   xp(vy, px), -xp(vy, qx), -xp(uy, px), xp(uy, qx)};
    return expansion_sign(t, 8);
}

// Decided sign of orient(u, v, p) given its filtered value; *exact_used counts fallbacks.
template <typename P>
QH_HD int orient_sign(const Edge<P> &e, float vx, float vy, float px, float py, const Approx<P> &o, int &exact_used) {
    if (o.ok) {
        if (o.det > o.err) return 1;
        if (-o.det > o.err) return -1;
    }
    exact_used++;
    return orient_exact(e.ux, e.uy, vx, vy, px, py);
}

// Distance interval [lo, hi] of a point beyond edge u->v from its filtered orientation.
template <typename P> struct DistIv {
    P lo, hi;
};
template <typename P> QH_HD DistIv<P> dist_interval(const Approx<P> &o) {
    DistIv<P> d;
    if (o.ok) {
        d.lo = sub_down(-o.det, o.err);
        d.hi = add_up(-o.det, o.err);
    } else {
        d.lo = -INFINITY;
        d.hi = INFINITY;
    }
    return d;
}

// Total order of farthest-point candidates of one chord u->v: larger distance,
// then lexicographically smaller (x, y), then lower index.  On equal distance
// the tied points lie on one line parallel to the chord; the lexicographic
// minimum of a collinear set is an end point, hence a strict hull vertex.
template <typename P>
QH_HD bool farther(const Edge<P> &e, float vx, float vy, float ax, float ay, int ai, DistIv<P> da,
                   float bx, float by, int bi, DistIv<P> db, int &exact_used) {
    if (bi < 0) return ai >= 0;
    if (ai < 0) return false;
    if (da.lo > db.hi) return true;
    if (db.lo > da.hi) return false;
    if (!(ax == bx && ay == by)) {
        exact_used++;
        int s = dist_cmp_exact(e.ux, e.uy, vx, vy, ax, ay, bx, by);
        if (s != 0) return s > 0;
        if (ax != bx) return ax < bx;
        return ay < by;
    }
    return ai < bi;
}

// Lexicographic orders used by the extreme-point search (Sec. 4.2).  Ties in
// coordinates go to the lower index.
QH_HD bool lex_less(float ax, float ay, int ai, float bx, float by, int bi) {  // min (x, y, idx)
    if (bi < 0) return ai >= 0;
    if (ai < 0) return false;
    if (ax != bx) return ax < bx;
    if (ay != by) return ay < by;
    return ai < bi;
}
QH_HD bool lex_greater(float ax, float ay, int ai, float bx, float by, int bi) {  // max (x, y), min idx
    if (bi < 0) return ai >= 0;
    if (ai < 0) return false;
    if (ax != bx) return ax > bx;
    if (ay != by) return ay > by;
    return ai < bi;
}

}  // namespace qh
