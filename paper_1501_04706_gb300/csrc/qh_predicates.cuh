// Exact geometric predicates for the hull kernels (host + device).
//
// orient(u, v, p) = (vx-ux)(py-uy) - (vy-uy)(px-ux): > 0 when p is left of the
// directed line u->v.  A point is outside a CCW hull edge u->v when it is
// strictly right of it (orient < 0): the side test of Sec. 4.4.3 against the
// two new edges h->c and c->e.  Its distance beyond the edge is dist(p) = -orient(u,v,p);
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
// Exact path: the sign of a sum of products of floats is the sign of the top
// non-zero component of the nonoverlapping expansion built with Knuth's TwoSum
// by Shewchuk's GROW-EXPANSION (Shewchuk, "Adaptive precision floating-point
// arithmetic and fast robust geometric predicates", 1997).  orient needs 6
// products, the farthest-point comparison 8.  The expansion is built in FP32:
// each product ab is the exact sum of p = fl(ab) and the FMA residue
// fl(ab - p) when every factor is zero or has magnitude in [2^-51, 2^61]: then
// ab is an integer multiple of 2^-148 and |ab - p| is at most 2^23 such units,
// so the residue is representable, and |ab| < 2^122, so no partial sum of up to
// 16 terms overflows (TwoSum is exact without overflow, subnormal sums
// included).  Inputs outside that range take the same expansion in FP64, where
// every float x float product is exact; FP64 runs at a small fraction of the
// FP32 rate on the GPU, so it is kept for those inputs only.
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
QH_HD float add_down(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rd(a, b);
#else
    return std::nextafter(a + b, -INFINITY);
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
QH_HD float rfma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

QH_HD double rfma(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
// a * b rounded toward +inf.
QH_HD float mul_up(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_ru(a, b);
#else
    return std::nextafter(a * b, INFINITY);
#endif
}
QH_HD double mul_up(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_ru(a, b);
#else
    return std::nextafter(a * b, INFINITY);
#endif
}

template <typename T> QH_HD void two_sum(T a, T b, T &s, T &e) {
    s = radd(a, b);
    const T bb = rsub(s, a);
    e = radd(rsub(a, rsub(s, bb)), rsub(b, bb));
}

// Sign of t[0] + ... + t[N-1] (each an exact value of type T) by
// GROW-EXPANSION; kept as loops (the code is cold: its size costs more than
// its speed).
template <typename T, int N> QH_HD int expansion_sign(const T (&t)[N]) {
    T h[N];
#pragma unroll 1
    for (int i = 0; i < N; i++) {
        T q = t[i];
#pragma unroll 1
        for (int j = 0; j < i; j++) {
            T s, err;
            two_sum(q, h[j], s, err);
            h[j] = err;
            q = s;
        }
        h[i] = q;
    }
#pragma unroll 1
    for (int j = N - 1; j >= 0; j--)  // the top non-zero component decides
        if (h[j] != T(0)) return h[j] > T(0) ? 1 : -1;
    return 0;
}

QH_HD float fabs_f(float x) { return x < 0.f ? -x : x; }

// Sign of p[0] + ... + p[N-1] (exact floats).  A VecSum pass (TwoSum along the
// vector: p[i], p[i-1] <- sum, error) leaves the exact total unchanged and
// moves its rounded value to p[N-1]; the sign is that of p[N-1] as soon as
// |p[N-1]| exceeds the sum of the other magnitudes (accumulated rounding
// upward, an upper bound), and 0 when that bound and p[N-1] are both zero.
// Cases still open after a few passes take GROW-EXPANSION.
template <int N> QH_HD int sum_sign_f32(float (&p)[N]) {
#pragma unroll 1
    for (int pass = 0; pass < 4; pass++) {
#pragma unroll
        for (int i = 1; i < N; i++) {
            float s, e;
            two_sum(p[i], p[i - 1], s, e);
            p[i] = s;
            p[i - 1] = e;
        }
        float rest = 0.f;
#pragma unroll
        for (int i = 0; i < N - 1; i++) rest = add_up(rest, fabs_f(p[i]));
        const float top = p[N - 1];
        if (fabs_f(top) > rest) return top > 0.f ? 1 : -1;
        if (rest == 0.f) return 0;
    }
    return expansion_sign(p);
}

QH_HD bool f32_exact_range(float x) {
    const float a = x < 0.f ? -x : x;
    return a == 0.f || (a >= 0x1p-51f && a <= 0x1p61f);
}

QH_HD double xp(float a, float b) { return rmul(double(a), double(b)); }

// Every factor zero or in [2^-51, 2^61]: the products' FP32 expansion is exact.
template <int N> QH_HD bool factors_in_f32_range(const float (&a)[N], const float (&b)[N]) {
    bool in = true;
#pragma unroll
    for (int k = 0; k < N; k++) in = in && f32_exact_range(a[k]) && f32_exact_range(b[k]);
    return in;
}

// sign(sum of s_k a_k b_k), s_k = +-1, exactly (FP32 expansion when in range).
template <int N>
QH_HD int product_sum_sign(const float (&a)[N], const float (&b)[N], const int (&sg)[N]) {
    if (factors_in_f32_range(a, b)) {
        float t[2 * N];
#pragma unroll
        for (int k = 0; k < N; k++) {
            const float x = sg[k] > 0 ? a[k] : -a[k];
            const float p = rmul(x, b[k]);
            t[2 * k] = rfma(x, b[k], -p);
            t[2 * k + 1] = p;
        }
        return sum_sign_f32(t);
    }
    double t[N];
#pragma unroll
    for (int k = 0; k < N; k++) t[k] = sg[k] > 0 ? xp(a[k], b[k]) : -xp(a[k], b[k]);
    return expansion_sign(t);
}

// sign((a1 - a0)(b1 - b0) - (c1 - c0)(d1 - d0)) for floats, decided in FP64
// where that is certain (*decided = false otherwise).  Used before the FP64
// expansion only (factors outside the FP32 range): GB300's FP64 rate is a
// small fraction of its FP32 rate, so in range the FP32 expansion is faster.  A difference of two
// floats is exact in FP64 unless their exponents lie far apart; TwoSum's error
// term (exact in round-to-nearest) tells which.  With exact differences, each
// product is exact when its FMA residue is zero (float differences are
// multiples of 2^-149, so products cannot underflow, and they cannot overflow);
// then the sign is the comparison of the two products.  Otherwise l - r is
// within 2u (|l| + |r|) of the exact value (u = 2^-53), and a bound of 4u,
// which also covers the rounding of the bound, decides all but near-zero cases.
QH_HD int diff_products_sign64(float a1, float a0, float b1, float b0, float c1, float c0, float d1, float d0,
                               bool &decided) {
    double x[4], e[4];
    const float hi[4] = {a1, b1, c1, d1}, lo[4] = {a0, b0, c0, d0};
    bool exactDiff = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        two_sum(double(hi[k]), -double(lo[k]), x[k], e[k]);
        exactDiff = exactDiff && e[k] == 0.0;
    }
    decided = false;
    if (!exactDiff) return 0;
    const double l = rmul(x[0], x[1]), r = rmul(x[2], x[3]);
    if (rfma(x[0], x[1], -l) == 0.0 && rfma(x[2], x[3], -r) == 0.0) {
        decided = true;
        return (l > r) - (l < r);
    }
    const double det = rsub(l, r);
    const double err = rmul(radd(l < 0.0 ? -l : l, r < 0.0 ? -r : r), 4.0 * 0x1p-53);
    if (det > err || -det > err) {
        decided = true;
        return det > 0.0 ? 1 : -1;
    }
    return 0;
}

// The same in FP32 when every difference is exact (TwoSum error zero; always
// so for coordinates within a factor of two of each other) and zero or in
// [2^-51, 2^61]: each product is then exactly the sum of its rounded value and
// its FMA residue (as in the expansions below), so the sign is that of a
// four-term sum -- the nearly collinear triples of nearby points the filter
// leaves open cost a few TwoSums instead of a twelve-term expansion.
QH_HD int diff_products_sign32(float a1, float a0, float b1, float b0, float c1, float c0, float d1, float d0,
                               bool &decided) {
    float x[4];
    const float hi[4] = {a1, b1, c1, d1}, lo[4] = {a0, b0, c0, d0};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float e;
        two_sum(hi[k], -lo[k], x[k], e);
        ok = ok && e == 0.f && f32_exact_range(x[k]);
    }
    decided = ok;
    if (!ok) return 0;
    const float l = rmul(x[0], x[1]), r = rmul(x[2], x[3]);
    float t[4] = {rfma(x[0], x[1], -l), -rfma(x[2], x[3], -r), l, -r};
    return sum_sign_f32(t);
}

// The value (a1 - a0)(b1 - b0) - (c1 - c0)(d1 - d0) in compensated FP32 with a
// certified bound, between the filter and the expansions.  Each difference is
// split exactly by TwoSum into a high and a low part, so the value is exactly
//   m1 + [m0 + p0 - q0 + ah bl + al bh - ch dl - cl dh + al bl - cl dl],
// where p1 + p0 = ah bh and q1 + q0 = ch dh (FMA residues) and m1 + m0 =
// p1 - q1 (TwoSum).  The bracket's nine terms are summed in round-to-nearest;
// six of them are rounded products.  Its error is at most 8u (summation) + u
// (products) times the sum of the magnitudes, plus 2^-150 for each product or
// residue that underflows; 10u times the upward-rounded magnitude sum plus
// 2^-144 bounds it (u = 2^-24).  The sign is decided when the directed-rounded
// interval around m1 + bracket excludes zero; exact zeros and non-finite
// intermediates stay undecided.
QH_HD int diff_products_sign_comp(float a1, float a0, float b1, float b0, float c1, float c0, float d1, float d0,
                                  bool &decided) {
    float ah, al, bh, bl, ch, cl, dh, dl;
    two_sum(a1, -a0, ah, al);
    two_sum(b1, -b0, bh, bl);
    two_sum(c1, -c0, ch, cl);
    two_sum(d1, -d0, dh, dl);
    const float p1 = rmul(ah, bh), p0 = rfma(ah, bh, -p1);
    const float q1 = rmul(ch, dh), q0 = rfma(ch, dh, -q1);
    float m1, m0;
    two_sum(p1, -q1, m1, m0);
    const float t[9] = {m0, p0, -q0, rmul(ah, bl), rmul(al, bh), -rmul(ch, dl), -rmul(cl, dh), rmul(al, bl),
                        -rmul(cl, dl)};
    float sum = 0.f, mag = 0.f;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        sum = radd(sum, t[k]);
        mag = add_up(mag, fabs_f(t[k]));
    }
    decided = false;
    const float err = add_up(mul_up(mag, 10.f * 0x1p-24f), 0x1p-144f);
    if (!(fabs_f(m1) <= FLT_MAX && fabs_f(sum) <= FLT_MAX && err <= FLT_MAX)) return 0;
    if (sub_down(add_down(m1, sum), err) > 0.f) {
        decided = true;
        return 1;
    }
    if (add_up(add_up(m1, sum), err) < 0.f) {
        decided = true;
        return -1;
    }
    return 0;
}

// orient(a,b,c) = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx, exactly.
QH_HD_COLD int orient_exact(float ax, float ay, float bx, float by, float cx, float cy) {
    const float fa[6] = {bx, bx, ax, by, by, ay};
    const float fb[6] = {cy, ay, cy, cx, ax, cx};
    const int sg[6] = {1, -1, -1, -1, 1, 1};
    bool decided;
    const int sc = diff_products_sign_comp(bx, ax, cy, ay, by, ay, cx, ax, decided);
    if (decided) return sc;
    if (!factors_in_f32_range(fa, fb)) {
        const int s64 = diff_products_sign64(bx, ax, cy, ay, by, ay, cx, ax, decided);
        if (decided) return s64;
    } else {
        const int s32 = diff_products_sign32(bx, ax, cy, ay, by, ay, cx, ax, decided);
        if (decided) return s32;
    }
    return product_sum_sign(fa, fb, sg);
}

// sign(dist(p) - dist(q)) for the chord u->v, dist(x) = -orient(u, v, x):
//   -(vx-ux)(py-qy) + (vy-uy)(px-qx), expanded into eight exact products.
QH_HD_COLD int dist_cmp_exact(float ux, float uy, float vx, float vy, float px, float py, float qx, float qy) {
    const float fa[8] = {vx, vx, ux, ux, vy, vy, uy, uy};
    const float fb[8] = {py, qy, py, qy, px, qx, px, qx};
    const int sg[8] = {-1, 1, 1, -1, 1, -1, -1, 1};
    bool decided;  // the same value as (vy-uy)(px-qx) - (vx-ux)(py-qy)
    const int sc = diff_products_sign_comp(vy, uy, px, qx, vx, ux, py, qy, decided);
    if (decided) return sc;
    if (!factors_in_f32_range(fa, fb)) {
        const int s64 = diff_products_sign64(vy, uy, px, qx, vx, ux, py, qy, decided);
        if (decided) return s64;
    } else {
        const int s32 = diff_products_sign32(vy, uy, px, qx, vx, ux, py, qy, decided);
        if (decided) return s32;
    }
    return product_sum_sign(fa, fb, sg);
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
