// The x-sorted form of the rounds (Sec. 3, Sec. 4.2-4.4), the paper's own
// arrangement: after the first split the points are sorted by x, so that the
// lower subset (ascending x) followed by the upper subset (descending x) lists
// the points in the order of one polygon that starts at A.  Every round keeps
// that order: a segment is the run of points between two consecutive heads,
// its farthest point C becomes a head in place, and a stable compaction drops
// the points that are not strictly right of their new chord.
//
// Why one orientation test per point suffices (the positional split): inside a
// segment h -> e of a chain, every point lies strictly right of the chord and
// between h and e in the chain's x order.  A point before C (x not past x_C)
// that lies strictly right of C -> e would be farther from the chord than C,
// and so would a point after C that lies strictly right of h -> C; points at
// x_C other than C lie on the inner side of both new chords.  So a point
// before C can only survive as a point of h -> C and a point after C only as a
// point of C -> e, exactly the classes of the two-test rule, and the children
// stay contiguous in x order.  This holds for any order of points with equal
// x, so the sort key is x alone (the chain's direction folded in).
//
// Kernels, all 256 threads per CTA:
//   sx_extremes  A, B, Bot, Top (Sec. 4.2) with the lowest index on ties; the
//                last CTA merges the partials and forms the initial polygon.
//   sx_split     first split (Sec. 4.2 / 4.3): each point joins the first
//                polygon edge it lies strictly right of; lower-chain items go
//                to the front of the key buffer, upper-chain items to its back.
//   sx_hist / sx_scan_rows / sx_scan_bins / sx_radix_move
//                LSD radix sort, 4 passes of 8-bit digits of the x key, each
//                chain a separate range (bins = chain x digit); stable per pass.
//   sx_gather    coordinates and indices in sorted order; head positions.
//   rounds: sx_far (farthest point per segment, exact), sx_count (survivor
//                counts per tile; the last CTA scans them), sx_move (stable
//                compaction through shared memory; the last CTA commits the
//                round).  The host enqueues rounds in batches and reads the
//                end flag between batches.
//   sx_emit      the heads, which are the hull in CCW order from A.
#include <cuda_runtime.h>

#include "../../include/qh.h"
#include "qh_sorted.cuh"

namespace qh {
namespace sx {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ Cand shfl_down_cand(const Cand &c, int off) {
    Cand o;
    o.x = __shfl_down_sync(FULL, c.x, off);
    o.y = __shfl_down_sync(FULL, c.y, off);
    o.idx = __shfl_down_sync(FULL, c.idx, off);
    o.pad = 0;
    return o;
}

__device__ __forceinline__ void ext_init(Ext4 &e) {
    const Cand none = {0.f, 0.f, -1, 0};
    e.a = e.b = e.bot = e.top = none;
    e.nonfinite = 0;
}

__device__ __forceinline__ void ext_add(Ext4 &e, const Cand &c) {
    if (c.idx < 0) return;
    if (lex_less(c.x, c.y, c.idx, e.a.x, e.a.y, e.a.idx)) e.a = c;
    if (lex_greater(c.x, c.y, c.idx, e.b.x, e.b.y, e.b.idx)) e.b = c;
    if (lex_less(c.y, c.x, c.idx, e.bot.y, e.bot.x, e.bot.idx)) e.bot = c;
    if (lex_greater(c.y, c.x, c.idx, e.top.y, e.top.x, e.top.idx)) e.top = c;
}

__device__ __forceinline__ void ext_merge(Ext4 &e, const Ext4 &o) {
    ext_add(e, o.a);
    ext_add(e, o.b);
    ext_add(e, o.bot);
    ext_add(e, o.top);
    e.nonfinite |= o.nonfinite;
}

// Block-wide merge; the result is valid in thread 0.  Ends with no barrier.
__device__ Ext4 block_reduce_ext(Ext4 e, Ext4 *sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 1
    for (int off = 16; off > 0; off >>= 1) {
        Ext4 o;
        o.a = shfl_down_cand(e.a, off);
        o.b = shfl_down_cand(e.b, off);
        o.bot = shfl_down_cand(e.bot, off);
        o.top = shfl_down_cand(e.top, off);
        o.nonfinite = __shfl_down_sync(FULL, e.nonfinite, off);
        ext_merge(e, o);
    }
    if (lane == 0) sm[w] = e;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < SNW; k++) ext_merge(e, sm[k]);
    return e;
}

__device__ __forceinline__ Ext4 load_ext_cg(const Ext4 *p) {
    union {
        int4 v[5];
        Ext4 e;
    } u;
    const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
    for (int k = 0; k < 5; k++) u.v[k] = __ldcg(q + k);
    return u.e;
}

__device__ __forceinline__ bool same_xy(const Cand &a, const Cand &b) { return a.x == b.x && a.y == b.y; }

// Sort key of an x coordinate: -0 and +0 coincide; unsigned order is float order.
__device__ __forceinline__ unsigned xkey(float x) {
    unsigned b = __float_as_uint(x);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ----------------------------------------------------------------------------
// extreme points and the initial polygon
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(SNT) sx_extremes(const float2 *__restrict__ pts, int n, int mode, Ext4 *part,
                                                   SxState *st) {
    __shared__ Ext4 sm[SNW];
    __shared__ bool last;
    Ext4 e;
    ext_init(e);
    const int stride = gridDim.x * SNT;
    for (int i0 = blockIdx.x * SNT + threadIdx.x; i0 < n; i0 += 4 * stride) {
        float2 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = i0 + u * stride < n ? pts[i0 + u * stride] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = i0 + u * stride;
            if (i >= n) continue;
            if (!isfinite(q[u].x) || !isfinite(q[u].y)) {
                e.nonfinite = 1;
                continue;
            }
            const Cand c = {q[u].x, q[u].y, i, 0};
            ext_add(e, c);
        }
    }
    e = block_reduce_ext(e, sm);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = e;
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Ext4 f;
    ext_init(f);
    for (int k = threadIdx.x; k < (int)gridDim.x; k += SNT) ext_merge(f, load_ext_cg(part + k));
    f = block_reduce_ext(f, sm);
    if (threadIdx.x != 0) return;
    st->ticket = 0;
    if (f.nonfinite || f.a.idx < 0) {
        st->nonfinite = f.nonfinite;
        st->K = 0;
        return;
    }
    if (same_xy(f.a, f.b)) {  // every point coincides
        st->poly[0] = f.a;
        st->K = 1;
        return;
    }
    int k = 0;
    st->poly[k++] = f.a;
    if (mode == 0 && !same_xy(f.bot, f.a) && !same_xy(f.bot, f.b)) st->poly[k++] = f.bot;
    st->iB = k;
    st->poly[k++] = f.b;
    if (mode == 0 && !same_xy(f.top, f.a) && !same_xy(f.top, f.b)) st->poly[k++] = f.top;
    st->K = k;
}

// ----------------------------------------------------------------------------
// first split: items (x key, index | head rank) of both chains
// ----------------------------------------------------------------------------
template <typename P>
__global__ void __launch_bounds__(SNT) sx_split(const float2 *__restrict__ pts, int n, unsigned *key, unsigned *val,
                                                SxState *st, Ctl *ctl) {
    __shared__ Edge<P> ed[4];
    __shared__ float vend[4][2];
    __shared__ int pidx[4];
    __shared__ long long scr[SNW + 1];
    __shared__ unsigned base[2];
    __shared__ unsigned sk[STILE], sv[STILE];  // the tile's items: chain 0 first, then chain 1
    const int K = st->K;
    if (K < 2) return;
    if (threadIdx.x < K) {
        const Cand u = st->poly[threadIdx.x], v = st->poly[(threadIdx.x + 1) % K];
        ed[threadIdx.x] = make_edge<P>(u.x, u.y, v.x, v.y);
        vend[threadIdx.x][0] = v.x;
        vend[threadIdx.x][1] = v.y;
        pidx[threadIdx.x] = u.idx;
    }
    __syncthreads();
    const int iB = st->iB;
    int ex = 0;
    unsigned live = 0;
    const int tiles = (n + STILE - 1) / STILE;
    // One tile of STILE points per step (point tile*STILE + j*SNT + thread): the
    // survivors of both chains are counted over the tile first, so that each
    // chain's cursor takes one atomic per tile.
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        unsigned k[SIPT], v[SIPT];
        unsigned in0 = 0u, in1 = 0u;  // bit j: item j joins chain 0 / chain 1
#pragma unroll
        for (int j = 0; j < SIPT; j++) {
            const int i = tile * STILE + j * SNT + threadIdx.x;
            k[j] = 0u;
            v[j] = 0u;
            if (i >= n) continue;
            const float2 q = pts[i];
            int head = -1;
            for (int t = 0; t < K; t++)
                if (pidx[t] == i) head = t;
            int seg = -1;
            if (head < 0) {
                for (int t = 0; t < K; t++) {
                    const Approx<P> o = orient_approx(ed[t], q.x, q.y);
                    if (orient_sign(ed[t], vend[t][0], vend[t][1], q.x, q.y, o, ex) < 0) {
                        seg = t;
                        break;
                    }
                }
            }
            const int which = head >= 0 ? head : seg;
            if (which < 0) continue;
            const bool upper = which >= iB;  // edges and vertices before B: lower chain
            k[j] = xkey(q.x);
            if (upper) k[j] = ~k[j];         // the upper chain runs in descending x
            v[j] = (unsigned)i;
            if (head >= 0)
                v[j] |= HEAD_BIT | ((unsigned)head << 29);
            else
                live++;
            if (upper)
                in1 |= 1u << j;
            else
                in0 |= 1u << j;
        }
        const long long packed = ((long long)__popc(in0) << 32) | (long long)__popc(in1);
        long long tot;
        const long long pre = block_excl_scan<long long, SNT>(packed, scr, tot);
        if (threadIdx.x == 0) {
            const unsigned t0 = (unsigned)(tot >> 32), t1 = (unsigned)(tot & 0xffffffffll);
            base[0] = t0 ? atomicAdd(&st->c0, t0) : 0u;
            base[1] = t1 ? atomicAdd(&st->c1, t1) : 0u;
        }
        const int t0 = (int)(tot >> 32), t1 = (int)(tot & 0xffffffffll);
        int q0 = (int)(pre >> 32), q1 = t0 + (int)(pre & 0xffffffffll);
#pragma unroll
        for (int j = 0; j < SIPT; j++) {
            if ((in0 >> j) & 1u) {
                sk[q0] = k[j];
                sv[q0] = v[j];
                q0++;
            } else if ((in1 >> j) & 1u) {
                sk[q1] = k[j];
                sv[q1] = v[j];
                q1++;
            }
        }
        __syncthreads();
        const unsigned b0 = base[0], b1 = base[1];
        for (int q = threadIdx.x; q < t0 + t1; q += SNT) {
            const unsigned dst = q < t0 ? b0 + (unsigned)q : (unsigned)n - 1u - (b1 + (unsigned)(q - t0));
            key[dst] = sk[q];
            val[dst] = sv[q];
        }
        __syncthreads();  // sk, sv and base[] are rewritten by the next tile
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        live += __shfl_down_sync(FULL, live, off);
        ex += __shfl_down_sync(FULL, ex, off);
    }
    if (lane == 0) {
        if (live) atomicAdd((unsigned long long *)&ctl->live[0], (unsigned long long)live);
        if (ex) atomicAdd(&ctl->exactOrient, (unsigned long long)ex);
    }
}

// ----------------------------------------------------------------------------
// radix sort of the items by x key, the two chains kept apart
// ----------------------------------------------------------------------------
// Item v of the sorted range [0, T): the first pass reads the split's layout
// (lower chain at [0, c0), upper chain at [n - c1, n)), later passes a dense one.
__device__ __forceinline__ int item_src(int v, int c0, int gap) { return v < c0 ? v : v + gap; }

__global__ void __launch_bounds__(SNT) sx_hist(const unsigned *__restrict__ key, int shift, int first, int n,
                                               const SxState *st, int *hist) {
    __shared__ int h[BINS];
    const int c0 = (int)st->c0, T = c0 + (int)st->c1;
    const int tiles = (T + STILE - 1) / STILE, tile = blockIdx.x;
    if (tile >= tiles) return;
    const int gap = first ? n - T : 0;
    for (int b = threadIdx.x; b < BINS; b += SNT) h[b] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = tile * STILE + warp * 32 * SIPT;
#pragma unroll 4
    for (int j = 0; j < SIPT; j++) {
        const int v = base + j * 32 + lane;
        int bin = -1;
        if (v < T) bin = (v < c0 ? 0 : 256) + (int)((__ldg(key + item_src(v, c0, gap)) >> shift) & 255u);
        const unsigned mt = __match_any_sync(FULL, bin);
        if (bin >= 0 && lane == __ffs(mt) - 1) atomicAdd(&h[bin], __popc(mt));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < BINS; b += SNT) hist[(long long)b * tiles + tile] = h[b];
}

// One CTA per bin: exclusive scan of the bin's per-tile counts, in place.
__global__ void __launch_bounds__(SNT) sx_scan_rows(int *hist, int *rowTot, const SxState *st) {
    __shared__ int scr[SNW + 1];
    const int T = (int)st->c0 + (int)st->c1, tiles = (T + STILE - 1) / STILE;
    int *row = hist + (long long)blockIdx.x * tiles;
    const int per = (tiles + SNT - 1) / SNT;
    const int lo = min(threadIdx.x * per, tiles), hi = min(lo + per, tiles);
    int sum = 0;
    for (int k = lo; k < hi; k++) sum += row[k];
    int tot;
    int run = block_excl_scan<int, SNT>(sum, scr, tot);
    for (int k = lo; k < hi; k++) {
        const int c = row[k];
        row[k] = run;
        run += c;
    }
    if (threadIdx.x == 0) rowTot[blockIdx.x] = tot;
}

// One CTA of BINS threads: exclusive scan of the bin totals.
__global__ void __launch_bounds__(BINS) sx_scan_bins(const int *rowTot, int *binBase) {
    __shared__ int scr[BINS / 32 + 1];
    int tot;
    const int r = block_excl_scan<int, BINS>(rowTot[threadIdx.x], scr, tot);
    binBase[threadIdx.x] = r;
}

// Stable scatter of one pass: warp w of a tile owns items [w*512, w*512+512)
// in rows of 32, so per-warp counters taken row by row rank the items in
// their original order; a scan over the warps per bin joins them.  The tile is
// then laid out in shared memory in bin order, and consecutive threads write
// consecutive addresses of each bin's run.
__global__ void __launch_bounds__(SNT) sx_radix_move(const unsigned *__restrict__ kin, const unsigned *__restrict__ vin,
                                                     unsigned *kout, unsigned *vout, int shift, int first, int n,
                                                     const SxState *st, const int *__restrict__ hist,
                                                     const int *__restrict__ binBase) {
    __shared__ union {
        int wc[SNW][BINS];  // per-warp counts, then their exclusive prefix over the warps
        struct {
            unsigned k[STILE], v[STILE];
            unsigned short bin[STILE];
        } stg;              // the tile in bin order
    } u;
    __shared__ int off[BINS];  // global start of the tile's run of each bin
    __shared__ int tbs[BINS];  // tile-local start of each bin
    __shared__ int scr[SNW + 1];
    const int c0 = (int)st->c0, T = c0 + (int)st->c1;
    const int tiles = (T + STILE - 1) / STILE, tile = blockIdx.x;
    if (tile >= tiles) return;
    const int gap = first ? n - T : 0;
    for (int b = threadIdx.x; b < BINS; b += SNT) {
        off[b] = binBase[b] + hist[(long long)b * tiles + tile];
#pragma unroll
        for (int w = 0; w < SNW; w++) u.wc[w][b] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = tile * STILE + warp * 32 * SIPT;
    const unsigned lt = lanemask_lt();
    unsigned kr[SIPT], vr[SIPT];
    int rk[SIPT];
#pragma unroll
    for (int j = 0; j < SIPT; j++) {
        const int v = base + j * 32 + lane;
        int bin = -1;
        kr[j] = 0u;
        vr[j] = 0u;
        if (v < T) {
            const int src = item_src(v, c0, gap);
            kr[j] = __ldg(kin + src);
            vr[j] = __ldg(vin + src);
            bin = (v < c0 ? 0 : 256) + (int)((kr[j] >> shift) & 255u);
        }
        const unsigned mt = __match_any_sync(FULL, bin);
        int r = 0;
        if (bin >= 0) r = u.wc[warp][bin] + __popc(mt & lt);
        __syncwarp();
        if (bin >= 0 && lane == __ffs(mt) - 1) u.wc[warp][bin] += __popc(mt);
        __syncwarp();
        rk[j] = r;
    }
    __syncthreads();
    // per bin: exclusive prefix over the warps, and the tile's count of the bin
    int cnt2 = 0;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int b = 2 * threadIdx.x + q;
        int run = 0;
#pragma unroll
        for (int w = 0; w < SNW; w++) {
            const int c = u.wc[w][b];
            u.wc[w][b] = run;
            run += c;
        }
        tbs[b] = run;
        cnt2 += run;
    }
    int tot;
    const int pre = block_excl_scan<int, SNT>(cnt2, scr, tot);
    {
        const int b = 2 * threadIdx.x, c = tbs[b];
        tbs[b] = pre;
        tbs[b + 1] = pre + c;
    }
    __syncthreads();
    int lp[SIPT];
#pragma unroll
    for (int j = 0; j < SIPT; j++) {
        const int v = base + j * 32 + lane;
        lp[j] = -1;
        if (v < T) {
            const int bin = (v < c0 ? 0 : 256) + (int)((kr[j] >> shift) & 255u);
            lp[j] = tbs[bin] + u.wc[warp][bin] + rk[j];
        }
    }
    __syncthreads();  // the counts are read; the staging area overwrites them
#pragma unroll
    for (int j = 0; j < SIPT; j++) {
        const int v = base + j * 32 + lane;
        if (lp[j] >= 0 && lp[j] < STILE) {
            u.stg.k[lp[j]] = kr[j];
            u.stg.v[lp[j]] = vr[j];
            u.stg.bin[lp[j]] = (unsigned short)((v < c0 ? 0 : 256) + (int)((kr[j] >> shift) & 255u));
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < tot; q += SNT) {
        const int bin = u.stg.bin[q];
        const int dst = off[bin] + (q - tbs[bin]);
        if (dst >= 0 && dst < T) {  // always, when the counts of sx_hist hold
            kout[dst] = u.stg.k[q];
            vout[dst] = u.stg.v[q];
        }
    }
}

// Sorted items -> polygon arrays of the first round, head positions, and the copy of A at T.
__global__ void __launch_bounds__(SNT) sx_gather(const float2 *__restrict__ pts, int n, const unsigned *__restrict__ val,
                                                 SxBufs b, SxState *st, const Ctl *ctl) {
    const int K = st->K;
    if (K < 2) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 1;
        return;
    }
    const int T = (int)st->c0 + (int)st->c1;
    for (int v = blockIdx.x * SNT + threadIdx.x; v < T; v += gridDim.x * SNT) {
        const unsigned u = __ldg(val + v);
        const int idx = (int)(u & IDX_MASK);
        if (idx >= n) continue;  // never, when the sort is a permutation
        const float2 q = pts[idx];
        b.X[0][v] = q.x;
        b.Y[0][v] = q.y;
        b.I[0][v] = idx;
        if (u & HEAD_BIT) {
            const int j = (int)((u >> 29) & 3u);
            b.hp[0][j] = v;
            b.best[0][j] = -1;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const Cand A = st->poly[0];
        b.X[0][T] = A.x;
        b.Y[0][T] = A.y;
        b.I[0][T] = A.idx;
        b.hp[0][K] = T;
        st->m = T;
        st->S = K;
        st->cur = 0;
        st->gen = 1;
        st->liveLast = ctl->live[0];
        st->done = ctl->live[0] == 0;
    }
}

// ----------------------------------------------------------------------------
// rounds
// ----------------------------------------------------------------------------
// Segment of position p: the last head at or before p (hp ascending, hp[0] = 0, hp[S] = m > p).
__device__ __forceinline__ int seg_of(const int *__restrict__ hp, int S, int p) {
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(hp + mid) <= p)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_items(const float *__restrict__ X, const float *__restrict__ Y, int p0,
                                           float (&x)[SIPT], float (&y)[SIPT]) {
    const float4 *x4 = reinterpret_cast<const float4 *>(X + p0);
    const float4 *y4 = reinterpret_cast<const float4 *>(Y + p0);
#pragma unroll
    for (int k = 0; k < SIPT / 4; k++) {
        const float4 a = __ldg(x4 + k), c = __ldg(y4 + k);
        x[4 * k] = a.x;
        x[4 * k + 1] = a.y;
        x[4 * k + 2] = a.z;
        x[4 * k + 3] = a.w;
        y[4 * k] = c.x;
        y[4 * k + 1] = c.y;
        y[4 * k + 2] = c.z;
        y[4 * k + 3] = c.w;
    }
}

// A farthest-point candidate: coordinates, position and distance interval.
template <typename P> struct SC {
    float x, y;
    int pos;  // -1: none
    P lo, hi;
};

template <typename P> __device__ __forceinline__ SC<P> make_sc(const Edge<P> &e, float x, float y, int pos) {
    SC<P> c;
    c.x = x;
    c.y = y;
    c.pos = pos;
    const DistIv<P> d = dist_interval(orient_approx(e, x, y));
    c.lo = d.lo;
    c.hi = d.hi;
    return c;
}

// Is a farther from the chord u -> v than b?  The total order of the farthest
// point (Sec. 4.4.1): larger distance, then lexicographically smaller (x, y),
// then lower input index.
template <typename P>
__device__ __forceinline__ bool sx_farther(const Edge<P> &e, float vx, float vy, const SC<P> &a, const SC<P> &b,
                           const int *__restrict__ I, int &ex) {
    if (b.pos < 0) return a.pos >= 0;
    if (a.pos < 0) return false;
    if (a.lo > b.hi) return true;
    if (b.lo > a.hi) return false;
    if (!(a.x == b.x && a.y == b.y)) {
        ex++;
        const int s = dist_cmp_exact(e.ux, e.uy, vx, vy, a.x, a.y, b.x, b.y);
        if (s != 0) return s > 0;
        if (a.x != b.x) return a.x < b.x;
        return a.y < b.y;
    }
    return __ldg(I + a.pos) < __ldg(I + b.pos);
}

// Offer a candidate as the farthest point of segment s: a compare-and-swap
// loop on the segment's position word.  The word only ever moves to a farther
// point in a strict total order, so the loop ends.
template <typename P>
__device__ __forceinline__ void sx_offer(int *best, int s, const SC<P> &c, const Edge<P> &e, float vx, float vy,
                         const float *__restrict__ X, const float *__restrict__ Y, const int *__restrict__ I, int &ex) {
    int cur = __ldcg(best + s);
    for (;;) {
        if (cur >= 0) {
            const SC<P> o = make_sc(e, __ldg(X + cur), __ldg(Y + cur), cur);
            if (!sx_farther(e, vx, vy, c, o, I, ex)) return;
        }
        const int prev = atomicCAS(best + s, cur, c.pos);
        if (prev == cur) return;
        cur = prev;
    }
}

template <typename P>
__global__ void __launch_bounds__(SNT, 2) sx_far(SxBufs b, SxState *st, Ctl *ctl) {
    if (st->done) return;
    const int m = st->m, S = st->S, cur = st->cur;
    const float *__restrict__ X = b.X[cur];
    const float *__restrict__ Y = b.Y[cur];
    const int *__restrict__ I = b.I[cur];
    const int *__restrict__ hp = b.hp[cur];
    int *best = b.best[cur];
    const int tiles = (m + STILE - 1) / STILE;
    const int lane = threadIdx.x & 31;
    int ex = 0;
    unsigned bad = 0u;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int p0 = tile * STILE + threadIdx.x * SIPT;
        int rs = -1;
        SC<P> bc;
        bc.pos = -1;
        bc.x = bc.y = 0.f;
        bc.lo = bc.hi = P(0);
        Edge<P> ed = make_edge<P>(0.f, 0.f, 0.f, 0.f);
        float vx = 0.f, vy = 0.f;
        if (p0 < m) {
            float x[SIPT], y[SIPT];
            load_items(X, Y, p0, x, y);
            int s = seg_of(hp, S, p0);
            int h = __ldg(hp + s), e = __ldg(hp + s + 1);
#pragma unroll
            for (int j = 0; j < SIPT; j++) {
                const int p = p0 + j;
                if (p >= m) continue;  // (not break: the loop stays unrolled and x, y in registers)
                if (p >= e) {
                    do {
                        s++;
                        e = __ldg(hp + s + 1);
                    } while (e <= p && s + 1 < S);
                    h = __ldg(hp + s);
                }
                // heads ascend from 0 to m, so h <= p < e <= m; anything else is a broken state
                if (!(h >= 0 && h <= p && p < e && e <= m)) {
                    bad = 1u;
                    continue;
                }
                if (p == h) continue;
                if (s != rs) {
                    if (bc.pos >= 0) sx_offer(best, rs, bc, ed, vx, vy, X, Y, I, ex);
                    rs = s;
                    vx = __ldg(X + e);
                    vy = __ldg(Y + e);
                    ed = make_edge<P>(__ldg(X + h), __ldg(Y + h), vx, vy);
                    bc.pos = -1;
                }
                const SC<P> c = make_sc(ed, x[j], y[j], p);
                if (sx_farther(ed, vx, vy, c, bc, I, ex)) bc = c;
            }
        }
        // The common case of a big segment: the whole warp ends in one run,
        // which it reduces before a single offer.
        const int rs0 = __shfl_sync(FULL, rs, 0);
        if (__all_sync(FULL, rs == rs0)) {
            if (rs0 >= 0) {
#pragma unroll 1
                for (int off = 16; off > 0; off >>= 1) {
                    SC<P> o;
                    o.x = __shfl_down_sync(FULL, bc.x, off);
                    o.y = __shfl_down_sync(FULL, bc.y, off);
                    o.pos = __shfl_down_sync(FULL, bc.pos, off);
                    o.lo = __shfl_down_sync(FULL, bc.lo, off);
                    o.hi = __shfl_down_sync(FULL, bc.hi, off);
                    if (lane + off < 32 && sx_farther(ed, vx, vy, o, bc, I, ex)) bc = o;
                }
                if (lane == 0 && bc.pos >= 0) sx_offer(best, rs0, bc, ed, vx, vy, X, Y, I, ex);
            }
        } else if (bc.pos >= 0) {
            sx_offer(best, rs, bc, ed, vx, vy, X, Y, I, ex);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ex += __shfl_down_sync(FULL, ex, off);
    if (lane == 0 && ex) atomicAdd(&ctl->exactCmp, (unsigned long long)ex);
    if (bad) atomicOr(&ctl->err, E_INTERNAL);
}

// Segment context of the classification: head h, end e, farthest point c and the two new chords.
template <typename P> struct SegCtx {
    int s, h, e, c;
    Edge<P> L, R;  // h -> C, C -> e
    float cx, cy, ex, ey;
};

template <typename P>
__device__ __forceinline__ void seg_load(SegCtx<P> &g, const float *__restrict__ X, const float *__restrict__ Y,
                                         const int *__restrict__ hp, const int *__restrict__ best, int m) {
    g.h = __ldg(hp + g.s);
    g.e = __ldg(hp + g.s + 1);
    g.c = __ldg(best + g.s);
    if (g.c >= 0 && g.h >= 0 && g.h < g.c && g.c < g.e && g.e <= m) {  // (the caller flags anything else)
        const float hx = __ldg(X + g.h), hy = __ldg(Y + g.h);
        g.cx = __ldg(X + g.c);
        g.cy = __ldg(Y + g.c);
        g.ex = __ldg(X + g.e);
        g.ey = __ldg(Y + g.e);
        g.L = make_edge<P>(hx, hy, g.cx, g.cy);
        g.R = make_edge<P>(g.cx, g.cy, g.ex, g.ey);
    }
}

// Survivors of the thread's items p0 .. p0 + SIPT - 1: bit j of keep is set
// when item j stays (a head, a new head, or a point strictly right of its new
// chord), bit j of head when it is a head after the round.
template <typename P>
__device__ __forceinline__ void classify(const float *__restrict__ X, const float *__restrict__ Y,
                                         const int *__restrict__ hp, const int *__restrict__ best, int m, int S,
                                         int p0, const float (&x)[SIPT], const float (&y)[SIPT], unsigned &keep,
                                         unsigned &head, int &ex, unsigned &bad) {
    keep = 0u;
    head = 0u;
    SegCtx<P> g;
    g.s = seg_of(hp, S, p0);
    seg_load(g, X, Y, hp, best, m);
#pragma unroll
    for (int j = 0; j < SIPT; j++) {
        const int p = p0 + j;
        if (p >= m) continue;
        if (p >= g.e) {
            do {
                g.s++;
            } while (__ldg(hp + g.s + 1) <= p && g.s + 1 < S);
            seg_load(g, X, Y, hp, best, m);
        }
        if (!(g.h >= 0 && g.h <= p && p < g.e && g.e <= m && g.c < g.e && (g.c < 0 || g.c > g.h))) {
            bad = 1u;  // heads ascend from 0 to m and a farthest point lies inside its segment
            continue;
        }
        if (p == g.h || p == g.c) {
            keep |= 1u << j;
            head |= 1u << j;
            continue;
        }
        if (g.c < 0) {  // a segment holding a point always has a farthest point
            bad = 1u;
            continue;
        }
        const bool left = p < g.c;
        Edge<P> E;  // selected field by field, so that both chords stay in registers
        E.ux = left ? g.L.ux : g.R.ux;
        E.uy = left ? g.L.uy : g.R.uy;
        E.ex = left ? g.L.ex : g.R.ex;
        E.ey = left ? g.L.ey : g.R.ey;
        const float vx = left ? g.cx : g.ex, vy = left ? g.cy : g.ey;
        if (orient_sign(E, vx, vy, x[j], y[j], orient_approx(E, x[j], y[j]), ex) < 0) keep |= 1u << j;
    }
}

template <typename P>
__global__ void __launch_bounds__(SNT, 2) sx_count(SxBufs b, SxState *st, Ctl *ctl) {
    __shared__ long long scr[SNW + 1];
    __shared__ bool last;
    if (st->done) return;
    const int m = st->m, S = st->S, cur = st->cur;
    const float *__restrict__ X = b.X[cur];
    const float *__restrict__ Y = b.Y[cur];
    const int *__restrict__ hp = b.hp[cur];
    const int *__restrict__ best = b.best[cur];
    const int tiles = (m + STILE - 1) / STILE;
    long long liveBlk = 0;
    int ex = 0;
    unsigned bad = 0u;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int p0 = tile * STILE + threadIdx.x * SIPT;
        unsigned keep = 0u, head = 0u;
        if (p0 < m) {
            float x[SIPT], y[SIPT];
            load_items(X, Y, p0, x, y);
            classify<P>(X, Y, hp, best, m, S, p0, x, y, keep, head, ex, bad);
        }
        const long long packed = ((long long)__popc(keep) << 32) | (long long)__popc(head);
        long long tot;
        block_excl_scan<long long, SNT>(packed, scr, tot);
        if (threadIdx.x == 0) {
            const int kept = (int)(tot >> 32), heads = (int)(tot & 0xffffffffll);
            b.tcnt[tile] = make_int2(kept, heads);
            liveBlk += kept - heads;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ex += __shfl_down_sync(FULL, ex, off);
    if ((threadIdx.x & 31) == 0 && ex) atomicAdd(&ctl->exactOrient, (unsigned long long)ex);
    if (bad) atomicOr(&ctl->err, E_INTERNAL);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (liveBlk) atomicAdd((unsigned long long *)&st->liveNew, (unsigned long long)liveBlk);
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last CTA: exclusive offsets of the tiles, in place, and the totals
    const int per = (tiles + SNT - 1) / SNT;
    const int lo = min((int)threadIdx.x * per, tiles), hi = min(lo + per, tiles);
    long long sum = 0;
    for (int k = lo; k < hi; k++) {
        const int2 c = __ldcg(b.tcnt + k);
        sum += ((long long)c.x << 32) | (long long)c.y;
    }
    long long tot;
    long long run = block_excl_scan<long long, SNT>(sum, scr, tot);
    for (int k = lo; k < hi; k++) {
        const int2 c = __ldcg(b.tcnt + k);
        b.tcnt[k] = make_int2((int)(run >> 32), (int)(run & 0xffffffffll));
        run += ((long long)c.x << 32) | (long long)c.y;
    }
    if (threadIdx.x == 0) {
        st->mNew = (int)(tot >> 32);
        st->SNew = (int)(tot & 0xffffffffll);
        st->ticket = 0;
    }
}

constexpr size_t MOVE_SMEM = (size_t)STILE * (sizeof(float2) + sizeof(int));

template <typename P>
__global__ void __launch_bounds__(SNT, 2) sx_move(SxBufs b, SxState *st, Ctl *ctl) {
    extern __shared__ float4 dyn[];
    float2 *sxy = reinterpret_cast<float2 *>(dyn);
    int *si = reinterpret_cast<int *>(sxy + STILE);
    __shared__ long long scr[SNW + 1];
    __shared__ bool last;
    if (st->done) return;
    const int m = st->m, S = st->S, cur = st->cur, nc = cur ^ 1;
    const float *__restrict__ X = b.X[cur];
    const float *__restrict__ Y = b.Y[cur];
    const int *__restrict__ I = b.I[cur];
    const int *__restrict__ hp = b.hp[cur];
    const int *__restrict__ best = b.best[cur];
    float *Xn = b.X[nc], *Yn = b.Y[nc];
    int *In = b.I[nc], *hpn = b.hp[nc], *bestn = b.best[nc];
    const int tiles = (m + STILE - 1) / STILE;
    int ex = 0;
    unsigned bad = 0u;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int p0 = tile * STILE + threadIdx.x * SIPT;
        unsigned keep = 0u, head = 0u;
        float x[SIPT], y[SIPT];
        if (p0 < m) {
            load_items(X, Y, p0, x, y);
            classify<P>(X, Y, hp, best, m, S, p0, x, y, keep, head, ex, bad);
        }
        const long long packed = ((long long)__popc(keep) << 32) | (long long)__popc(head);
        long long tot;
        const long long pre = block_excl_scan<long long, SNT>(packed, scr, tot);
        const int2 to = __ldg(b.tcnt + tile);
        if (keep) {
            int k = (int)(pre >> 32), hk = (int)(pre & 0xffffffffll);
            const int4 *i4 = reinterpret_cast<const int4 *>(I + p0);
#pragma unroll
            for (int q = 0; q < SIPT / 4; q++) {
                const int4 iv = __ldg(i4 + q);
                const int idx[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int j = 4 * q + r;
                    if ((keep >> j) & 1u) {
                        sxy[k] = make_float2(x[j], y[j]);
                        si[k] = idx[r];
                        if (((head >> j) & 1u) && to.y + hk < m) {  // (always: heads <= survivors <= m)
                            hpn[to.y + hk] = to.x + k;
                            bestn[to.y + hk] = -1;
                            hk++;
                        }
                        k++;
                    }
                }
            }
        }
        __syncthreads();
        const int kT = (int)(tot >> 32);
        for (int q = threadIdx.x; q < kT && to.x + q < m; q += SNT) {  // (survivors <= m)
            const float2 c = sxy[q];
            Xn[to.x + q] = c.x;
            Yn[to.x + q] = c.y;
            In[to.x + q] = si[q];
        }
        __syncthreads();
    }
    if (bad) atomicOr(&ctl->err, E_INTERNAL);
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    // the last CTA commits the round: the copy of A after the new polygon,
    // the statistics, and the end flag
    const int mN = st->mNew, SN = st->SNew;
    const long long L = st->liveNew;
    // never: survivors <= m, heads <= survivors, and every round turns at
    // least one point of each non-empty segment into a head
    if (mN > m || SN > mN || L >= st->liveLast) {
        atomicOr(&ctl->err, E_INTERNAL);
        st->done = 1;
        return;
    }
    const Cand A = st->poly[0];
    Xn[mN] = A.x;
    Yn[mN] = A.y;
    In[mN] = A.idx;
    hpn[SN] = mN;
    const int g = st->gen;
    ctl->live[g < MAX_GEN ? g : MAX_GEN - 1] += L;
    ctl->rounds += 1;
    st->gen = g + 1;
    st->cur = nc;
    st->m = mN;
    st->S = SN;
    st->liveNew = 0;
    st->liveLast = L;
    if (L == 0) st->done = 1;
    st->ticket = 0;
}

__global__ void __launch_bounds__(SNT) sx_emit(SxBufs b, const SxState *st, const Ctl *ctl, int *out, int *count) {
    const int gt = blockIdx.x * SNT + threadIdx.x;
    if (st->nonfinite) {
        if (gt == 0) *count = -QH_ERR_NONFINITE;
        return;
    }
    if (ctl->err) {
        if (gt == 0) *count = -QH_ERR_INTERNAL;
        return;
    }
    if (st->K == 1) {
        if (gt == 0) {
            out[0] = st->poly[0].idx;
            *count = 1;
        }
        return;
    }
    if (st->K < 2 || !st->done) {
        if (gt == 0) *count = -QH_ERR_INTERNAL;
        return;
    }
    const int m = st->m;
    const int *I = b.I[st->cur];
    for (int v = gt; v < m; v += gridDim.x * SNT) out[v] = I[v];
    if (gt == 0) *count = m;
}

template <typename P> void launch_round(const SortedWs &w, Ctl *ctl, int grid, cudaStream_t s) {
    sx_far<P><<<grid, SNT, 0, s>>>(w.b, w.st, ctl);
    sx_count<P><<<grid, SNT, 0, s>>>(w.b, w.st, ctl);
    sx_move<P><<<grid, SNT, MOVE_SMEM, s>>>(w.b, w.st, ctl);
}

int status_of(cudaError_t e) { return e == cudaErrorMemoryAllocation ? QH_ERR_OOM : QH_ERR_CUDA; }

}  // namespace

cudaError_t sorted_alloc(SortedWs &w, long long cap) {
    const long long tiles = (cap + STILE - 1) / STILE;
    const size_t padded = (size_t)(cap + STILE + 16);
    const size_t plain = (size_t)(cap + 16);
    cudaError_t e = cudaSuccess;
#define SX_ALLOC(ptr, bytes)                                    \
    do {                                                        \
        e = cudaMalloc((void **)&(ptr), (bytes));               \
        if (e != cudaSuccess) return e;                         \
    } while (0)
    for (int k = 0; k < 2; k++) {
        SX_ALLOC(w.key[k], sizeof(unsigned) * plain);
        SX_ALLOC(w.val[k], sizeof(unsigned) * plain);
        SX_ALLOC(w.b.X[k], sizeof(float) * padded);
        SX_ALLOC(w.b.Y[k], sizeof(float) * padded);
        SX_ALLOC(w.b.I[k], sizeof(int) * padded);
        SX_ALLOC(w.b.hp[k], sizeof(int) * plain);
        SX_ALLOC(w.b.best[k], sizeof(int) * plain);
    }
    SX_ALLOC(w.b.tcnt, sizeof(int2) * (size_t)(tiles + 16));
    SX_ALLOC(w.hist, sizeof(int) * (size_t)(BINS * tiles + 16));
    SX_ALLOC(w.rowTot, sizeof(int) * BINS);
    SX_ALLOC(w.binBase, sizeof(int) * BINS);
    SX_ALLOC(w.part, sizeof(Ext4) * MAX_PARTIALS);
    SX_ALLOC(w.st, sizeof(SxState));
#undef SX_ALLOC
    e = cudaMallocHost((void **)&w.hDone, sizeof(int));
    if (e != cudaSuccess) return e;
    w.cap = cap;
    return cudaSuccess;
}

void sorted_free(SortedWs &w) {
    for (int k = 0; k < 2; k++) {
        cudaFree(w.key[k]);
        cudaFree(w.val[k]);
        cudaFree(w.b.X[k]);
        cudaFree(w.b.Y[k]);
        cudaFree(w.b.I[k]);
        cudaFree(w.b.hp[k]);
        cudaFree(w.b.best[k]);
    }
    cudaFree(w.b.tcnt);
    cudaFree(w.hist);
    cudaFree(w.rowTot);
    cudaFree(w.binBase);
    cudaFree(w.part);
    cudaFree(w.st);
    if (w.hDone) cudaFreeHost(w.hDone);
    w = SortedWs();
}

int sorted_run(SortedWs &w, const float2 *pts, int n, int mode, int prec, int *outIdx, int *outCount, Ctl *ctl,
               int numSMs, cudaStream_t s, cudaEvent_t *ev) {
    if (n < 1 || n > w.cap) return QH_ERR_INVALID_ARG;
    cudaError_t e = cudaMemsetAsync(w.st, 0, sizeof(SxState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess && prec)
        e = cudaFuncSetAttribute(sx_move<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MOVE_SMEM);
    else if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sx_move<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MOVE_SMEM);
    if (e != cudaSuccess) return status_of(e);
    if (ev) cudaEventRecord(ev[0], s);
    int extGrid = (n + SNT * 8 - 1) / (SNT * 8);
    if (extGrid > MAX_PARTIALS) extGrid = MAX_PARTIALS;
    sx_extremes<<<extGrid, SNT, 0, s>>>(pts, n, mode, w.part, w.st);
    const int grid = numSMs * 4;
    if (prec)
        sx_split<double><<<grid, SNT, 0, s>>>(pts, n, w.key[0], w.val[0], w.st, ctl);
    else
        sx_split<float><<<grid, SNT, 0, s>>>(pts, n, w.key[0], w.val[0], w.st, ctl);
    if (ev) cudaEventRecord(ev[1], s);
    const int sortTiles = (n + STILE - 1) / STILE;
    for (int pass = 0; pass < 4; pass++) {
        const int src = pass & 1, dst = src ^ 1;
        sx_hist<<<sortTiles, SNT, 0, s>>>(w.key[src], 8 * pass, pass == 0, n, w.st, w.hist);
        sx_scan_rows<<<BINS, SNT, 0, s>>>(w.hist, w.rowTot, w.st);
        sx_scan_bins<<<1, BINS, 0, s>>>(w.rowTot, w.binBase);
        sx_radix_move<<<sortTiles, SNT, 0, s>>>(w.key[src], w.val[src], w.key[dst], w.val[dst], 8 * pass,
                                                pass == 0, n, w.st, w.hist, w.binBase);
    }
    sx_gather<<<grid, SNT, 0, s>>>(pts, n, w.val[0], w.b, w.st, ctl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return status_of(e);
    if (ev) cudaEventRecord(ev[2], s);
    // Every productive round turns at least one point into a head, so a set
    // of n points needs at most n rounds; the bound only guards the loop.
    const int roundGrid = numSMs * 2;
    for (long long rounds = 0;; rounds += ROUND_BATCH) {
        if (rounds > (long long)n + ROUND_BATCH) return QH_ERR_INTERNAL;
        for (int r = 0; r < ROUND_BATCH; r++) {
            if (prec)
                launch_round<double>(w, ctl, roundGrid, s);
            else
                launch_round<float>(w, ctl, roundGrid, s);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.hDone, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return status_of(e);
        if (*w.hDone) break;
    }
    if (ev) cudaEventRecord(ev[3], s);
    sx_emit<<<grid, SNT, 0, s>>>(w.b, w.st, ctl, outIdx, outCount);
    if (ev) cudaEventRecord(ev[4], s);
    e = cudaGetLastError();
    return e == cudaSuccess ? QH_OK : status_of(e);
}

}  // namespace sx
}  // namespace qh
