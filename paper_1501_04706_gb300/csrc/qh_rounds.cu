// Grid-wide part of segmented QuickHull: one cooperative, persistent launch.
//
// Phases (separated by bounded grid barriers):
//   prep       CTA 0 classifies the sets: empty, small (<= FIN_MAX points, left
//              to the block finisher) or big (tiled here).
//   extremes   per big set, the four extreme points of Sec. 4.2 (lexicographic
//              min/max of (x, y) and of (y, x), ties to the lower index).  Each
//              CTA streams a contiguous chunk of tiles and keeps running
//              extremes; the CTA that completes a set merges its partials.
//   round 0    the initial split (Sec. 4.2-4.3): each point joins the first
//              edge of the initial polygon it lies strictly right of (the
//              quadrilateral A->Bot->B->Top, or the chord A->B / B->A), and is
//              discarded otherwise.  Survivors are compacted and every new
//              segment's farthest point is found in the same pass.
//   round r    for every big segment (h, e) with farthest point c: keep the
//              points strictly right of h->c or of c->e (Sec. 4.4.3), compact
//              them into the two child segments (h, c), (c, e) (Sec. 4.4.2/4.4.4)
//              and find each child's farthest point (Sec. 4.4.1) in the same
//              pass; then the last CTA builds the next level of segments.
//
// Memory pipeline: every CTA owns a ring of NS shared-memory stages filled by
// TMA bulk copies (cp.async.bulk + mbarrier).  Thread 0 resolves the segment
// descriptors of tile k + NS and starts its copies while the CTA works on tile
// k, so HBM latency and descriptor lookups overlap the per-tile work.
//
// Compaction is a single pass.  Segments are contiguous ranges of a live
// buffer and a child never leaves its parent's range: the first child grows
// upward from the parent's start, the second downward from its end.  Every
// tile reserves its output range in each child with one atomic add on the
// child's cursor, so no tile ever waits for another (a tile-ordered scan would
// chain the ~600 tiles a persistent grid has in flight; the order of points
// inside a segment is irrelevant to the method).  The farthest point of each
// child is exact: each tile stores its own exact best per child, and the last
// tile of a parent (per-parent tile counter) merges the parent's tile bests.
// Segments with at most `cut` points (cut >= TILE) leave the grid-wide rounds
// for the block finisher, so a tile of a round spans at most two segments.
#include "qh_internal.cuh"

namespace qh {

constexpr int NS = 3;          // pipeline stages per CTA
constexpr int DB = 16;         // tile descriptors resolved per batch (one thread per tile)
constexpr int CAND_CAP = 128;  // farthest-point candidates kept per tile before the fallback

// Items of one segment inside a tile: physical range [q0, q0 + c) of the
// source buffer, first tile-local item vofs; [a0, a1) / [b0, b1) are the
// 16-byte aligned interiors copied by TMA to stage offsets sx / si (the
// ragged ends, at most one point on each side, are read directly).
struct PartGeo {
    long long q0, a0, a1, b0, b1;
    int c, vofs, sx, si;
};

struct TileRec {
    long long t;
    int np, nItems, valid, inst;
    unsigned bytes;  // TMA bytes of the tile
    int srcBuf;      // live buffer read by a round tile
    // round 0 / extremes: the set
    long long lt, setOff, setN, tile0;
    int tiles, K, iB, hasBox;
    float box[4];
    Cand poly[4];
    // rounds: the (at most two) parent segments
    int node[2], count[2];
    long long vstart[2], pstart[2];
    Cand nh[2], ne[2], nc[2];
    PartGeo g[2];
};

struct StageBuf {
    float2 xy[TILE];
    int id[TILE];
};

template <typename P> struct RoundSmem {
    unsigned long long mbar[NS];
    TileRec desc[2][DB];  // descriptors of the CTA's tiles, double-buffered by batch
    // tile working set
    Edge<P> edge[5];   // per slot; edge[4]: the chord A->B of the initial split
    float vend[5][2];
    int kflag;
    unsigned long long warpTot[IPT * NWARP];
    unsigned long long tileTot;
    unsigned maxLo[4];
    int ncand;
    Cand best[4];
    Cand fin[4];
    int base[4];   // this tile's first output rank in each slot's child
    int fflag[2];  // this tile is the last of part A / part B's parent
    long long scanTmp[NWARP + 1];
    Ext wext[NWARP];
    Cand wbest[NWARP][4];
    Cand cand[CAND_CAP];
    unsigned char cslot[CAND_CAP];
    alignas(128) StageBuf stage[NS];
};

// --------------------------------------------------------------------------
// TMA / mbarrier helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// 1-D bulk copy global -> shared, completing on mbarrier b (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Bounded wait for stage s; false (error bit set) when it never completes.
template <typename P> __device__ __forceinline__ bool pipe_wait(const Params &p, RoundSmem<P> &sm, int s, unsigned par) {
    unsigned it = 0;
    while (!mbar_try_wait(&sm.mbar[s], par)) {
        if (++it > SPIN_LIMIT) {
            set_err(p.ctl, E_TIMEOUT);
            return false;
        }
    }
    return true;
}

// xyPhase / idPhase: element offset of the array base from a 16-byte boundary
// (0/1 float2, 0..3 int), so that the copied interior is 16-byte aligned in memory.
__device__ __forceinline__ void part_geo(PartGeo &g, long long q0, int c, int vofs, bool withId, int &sx, int &si,
                                         unsigned &bytes, int xyPhase, int idPhase) {
    g.q0 = q0;
    g.c = c;
    g.vofs = vofs;
    const long long end = q0 + c;
    long long a0 = q0 + ((q0 + xyPhase) & 1), a1 = end - ((end + xyPhase) & 1);
    if (a1 < a0) a1 = a0;
    g.a0 = a0;
    g.a1 = a1;
    g.sx = sx;
    sx += (int)(a1 - a0);
    bytes += (unsigned)(a1 - a0) * 8u;
    if (withId) {
        long long b0 = q0 + ((4 - ((q0 + idPhase) & 3)) & 3), b1 = end - ((end + idPhase) & 3);
        if (b1 < b0) b1 = b0;
        g.b0 = b0;
        g.b1 = b1;
        g.si = si;
        si += (int)(b1 - b0);
        bytes += (unsigned)(b1 - b0) * 4u;
    } else {
        g.b0 = g.b1 = 0;
        g.si = 0;
    }
}

__device__ __forceinline__ int part_of(const TileRec &R, int i) { return (R.np == 2 && i >= R.g[1].vofs) ? 1 : 0; }

__device__ __forceinline__ float2 fetch_xy(const TileRec &R, const StageBuf &S, int i, const float2 *gxy,
                                           bool readOnly) {
    const PartGeo &g = R.g[part_of(R, i)];
    const long long q = g.q0 + (i - g.vofs);
    if (q >= g.a0 && q < g.a1) return S.xy[g.sx + (int)(q - g.a0)];
    return readOnly ? __ldg(&gxy[q]) : __ldcg(&gxy[q]);
}
__device__ __forceinline__ int fetch_id(const TileRec &R, const StageBuf &S, int i, const int *gid) {
    const PartGeo &g = R.g[part_of(R, i)];
    const long long q = g.q0 + (i - g.vofs);
    if (q >= g.b0 && q < g.b1) return S.id[g.si + (int)(q - g.b0)];
    return __ldcg(&gid[q]);
}

// --------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ long long upper_bound_ll(const long long *a, long long n, long long key) {
    // first i in [0, n) with a[i] > key (a non-decreasing), read through L2
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (__ldcg(a + mid) <= key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int src) {
    Cand o;
    o.x = __shfl_sync(0xffffffffu, c.x, src);
    o.y = __shfl_sync(0xffffffffu, c.y, src);
    o.idx = __shfl_sync(0xffffffffu, c.idx, src);
    o.pad = 0;
    return o;
}

__device__ __forceinline__ void ext_merge(Ext &a, const Ext &b) {
    if (lex_less(b.a.x, b.a.y, b.a.idx, a.a.x, a.a.y, a.a.idx)) a.a = b.a;
    if (lex_greater(b.b.x, b.b.y, b.b.idx, a.b.x, a.b.y, a.b.idx)) a.b = b.b;
    if (lex_less(b.bot.y, b.bot.x, b.bot.idx, a.bot.y, a.bot.x, a.bot.idx)) a.bot = b.bot;
    if (lex_greater(b.top.y, b.top.x, b.top.idx, a.top.y, a.top.x, a.top.idx)) a.top = b.top;
    a.nonfinite |= b.nonfinite;
}

__device__ __forceinline__ Ext ext_empty() {
    Ext e;
    e.a = e.b = e.bot = e.top = no_cand();
    e.nonfinite = 0;
    e.pad[0] = e.pad[1] = e.pad[2] = 0;
    return e;
}

__device__ __forceinline__ Ext warp_ext_reduce(Ext e) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        Ext o;
        o.a = shfl_cand(e.a, (threadIdx.x & 31) ^ d);
        o.b = shfl_cand(e.b, (threadIdx.x & 31) ^ d);
        o.bot = shfl_cand(e.bot, (threadIdx.x & 31) ^ d);
        o.top = shfl_cand(e.top, (threadIdx.x & 31) ^ d);
        o.nonfinite = __shfl_xor_sync(0xffffffffu, e.nonfinite, d);
        ext_merge(e, o);
    }
    return e;
}

__device__ __forceinline__ void st_ext(Ext *p, const Ext &e) {
    stcg_cand(&p->a, e.a);
    stcg_cand(&p->b, e.b);
    stcg_cand(&p->bot, e.bot);
    stcg_cand(&p->top, e.top);
    __stcg(&p->nonfinite, e.nonfinite);
}
__device__ __forceinline__ Ext ld_ext(const Ext *p) {
    Ext e;
    e.a = ldcg_cand(&p->a);
    e.b = ldcg_cand(&p->b);
    e.bot = ldcg_cand(&p->bot);
    e.top = ldcg_cand(&p->top);
    e.nonfinite = __ldcg(&p->nonfinite);
    return e;
}

__device__ __forceinline__ bool same_xy(const Cand &a, const Cand &b) { return a.x == b.x && a.y == b.y; }

// Returns true in every thread of the CTA that finished this phase last.
__device__ __forceinline__ bool last_cta(Ctl *ctl, unsigned &donePhase, int *flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        donePhase++;
        unsigned d = atomicAdd(&ctl->done, 1u);
        *flag = (d == donePhase * gridDim.x - 1u);
        __threadfence();
    }
    __syncthreads();
    return *flag != 0;
}

// --------------------------------------------------------------------------
// per-tile ranks and farthest points
// --------------------------------------------------------------------------
// slot[k] in {-1, 0..3} for the item of row k; rank[k] receives its exclusive
// rank among the tile's items of the same slot, in tile order; tot[] the totals.
template <typename P>
__device__ __forceinline__ void tile_ranks(const int (&slot)[IPT], int (&rank)[IPT], unsigned (&tot)[4],
                                           RoundSmem<P> &sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        unsigned long long packed = 0ull;
        int r = 0;
#pragma unroll
        for (int s = 0; s < 4; s++) {
            unsigned b = __ballot_sync(0xffffffffu, slot[k] == s);
            if (slot[k] == s) r = __popc(b & lt);
            packed |= (unsigned long long)__popc(b) << (16 * s);
        }
        rank[k] = r;
        if (lane == 0) sm.warpTot[k * NWARP + w] = packed;
    }
    __syncthreads();
    if (w == 0) {
        constexpr int E = IPT * NWARP;
        constexpr int PER = E / 32;
        unsigned long long v[PER], s = 0ull;
#pragma unroll
        for (int i = 0; i < PER; i++) {
            v[i] = sm.warpTot[lane * PER + i];
            s += v[i];
        }
        unsigned long long inc = warp_incl_scan(s);
        unsigned long long ex = inc - s;
#pragma unroll
        for (int i = 0; i < PER; i++) {
            sm.warpTot[lane * PER + i] = ex;
            ex += v[i];
        }
        if (lane == 31) sm.tileTot = inc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < IPT; k++)
        if (slot[k] >= 0) rank[k] += (int)((sm.warpTot[k * NWARP + w] >> (16 * slot[k])) & 0xffffull);
#pragma unroll
    for (int s = 0; s < 4; s++) tot[s] = (unsigned)((sm.tileTot >> (16 * s)) & 0xffffull);
}

// Merge candidate b into a for the chord of slot s (exact order).
template <typename P>
__device__ __forceinline__ void cand_merge(Cand &a, const Cand &b, int s, const RoundSmem<P> &sm, int &exact_c) {
    if (b.idx < 0) return;
    if (a.idx < 0) {
        a = b;
        return;
    }
    const Edge<P> &e = sm.edge[s];
    const DistIv<P> da = dist_interval(orient_approx(e, a.x, a.y));
    const DistIv<P> db = dist_interval(orient_approx(e, b.x, b.y));
    if (farther(e, sm.vend[s][0], sm.vend[s][1], b.x, b.y, b.idx, db, a.x, a.y, a.idx, da, exact_c)) a = b;
}

// Farthest point of each slot within the tile, exactly: the largest lower
// bound per slot, then every item whose upper bound reaches it is a candidate,
// and thread s picks the best candidate of slot s with the exact order.  When
// more than CAND_CAP items are candidates (massive exact ties), every thread
// reduces its own candidates and the warps combine them with the exact order.
template <typename P>
__device__ __forceinline__ void tile_farthest(const int (&slot)[IPT], const float (&x)[IPT], const float (&y)[IPT],
                                              const int (&idx)[IPT], const P (&lo)[IPT], const P (&hi)[IPT],
                                              RoundSmem<P> &sm, int &exact_c) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < 4) sm.maxLo[threadIdx.x] = 0u;
    if (threadIdx.x == 0) sm.ncand = 0;
    __syncthreads();
    unsigned mk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < IPT; k++) {
#pragma unroll
        for (int s = 0; s < 4; s++)
            if (slot[k] == s) mk[s] = max(mk[s], max(pkey(lo[k]), 1u));
    }
#pragma unroll
    for (int s = 0; s < 4; s++) {
        unsigned v = __reduce_max_sync(0xffffffffu, mk[s]);
        if (lane == 0 && v != 0u) atomicMax(&sm.maxLo[s], v);
    }
    __syncthreads();
    bool cand[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        cand[k] = false;
        if (slot[k] >= 0) {
            const P thr = (P)fkey_inv(sm.maxLo[slot[k]]);
            if (hi[k] >= thr) {
                cand[k] = true;
                int j = atomicAdd(&sm.ncand, 1);
                if (j < CAND_CAP) {
                    sm.cand[j] = mk_cand(x[k], y[k], idx[k]);
                    sm.cslot[j] = (unsigned char)slot[k];
                }
            }
        }
    }
    __syncthreads();
    const int nc = sm.ncand;
    if (nc <= CAND_CAP) {
        if (threadIdx.x < 4) {
            const int s = threadIdx.x;
            Cand b = no_cand();
            for (int j = 0; j < nc; j++)
                if (sm.cslot[j] == s) cand_merge(b, sm.cand[j], s, sm, exact_c);
            sm.best[s] = b;
        }
    } else {
#pragma unroll 1
        for (int s = 0; s < 4; s++) {
            Cand b = no_cand();
#pragma unroll
            for (int k = 0; k < IPT; k++)
                if (cand[k] && slot[k] == s) cand_merge(b, mk_cand(x[k], y[k], idx[k]), s, sm, exact_c);
            for (int d = 16; d >= 1; d >>= 1) cand_merge(b, shfl_cand(b, lane ^ d), s, sm, exact_c);
            if (lane == 0) sm.wbest[w][s] = b;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            const int s = threadIdx.x;
            Cand b = no_cand();
            for (int j = 0; j < NWARP; j++) cand_merge(b, sm.wbest[j][s], s, sm, exact_c);
            sm.best[s] = b;
        }
    }
    __syncthreads();
}

// Classify a point against an edge: returns true when strictly right, with the
// distance interval beyond the edge.
template <typename P>
__device__ __forceinline__ bool right_of(const Edge<P> &e, float vx, float vy, float px, float py, P &lo, P &hi,
                                         int &exact_o) {
    Approx<P> o = orient_approx(e, px, py);
    int s = orient_sign(e, vx, vy, px, py, o, exact_o);
    if (s < 0) {
        DistIv<P> d = dist_interval(o);
        lo = d.lo;
        hi = d.hi;
        return true;
    }
    return false;
}

// --------------------------------------------------------------------------
// per-tile farthest points and their merge per parent
// --------------------------------------------------------------------------
// Thread of warp 1: the tile's own farthest points, read by the parent's last tile.
__device__ __forceinline__ void store_tile_bests(const Params &p, long long t, const Cand (&b)[4]) {
    for (int s = 0; s < 4; s++) stcg_cand(&p.tbest[4 * t + s], b[s]);
}

// Exact farthest point of each of the nslot children of a parent whose points
// span tiles [ta, tb]: merge of the per-tile bests (tile ta reads its slots
// from slotBase0, the others from 0) with the chords sm.edge[edgeOff ..
// edgeOff + nslot).  Whole CTA; result in sm.fin.
template <typename P>
__device__ __noinline__ void merge_parent_bests(const Params &p, RoundSmem<P> &sm, long long ta, long long tb, int slotBase0,
                                   int nslot, int edgeOff, int &exact_c) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Cand b[4] = {no_cand(), no_cand(), no_cand(), no_cand()};
    for (long long u = ta + threadIdx.x; u <= tb; u += NT) {
        const int base = (u == ta) ? slotBase0 : 0;
        for (int s = 0; s < nslot; s++)
            cand_merge(b[s], ldcg_cand(&p.tbest[4 * u + base + s]), edgeOff + s, sm, exact_c);
    }
    for (int s = 0; s < nslot; s++) {
        for (int d = 16; d >= 1; d >>= 1) cand_merge(b[s], shfl_cand(b[s], lane ^ d), edgeOff + s, sm, exact_c);
        if (lane == 0) sm.wbest[w][s] = b[s];
    }
    __syncthreads();
    if (threadIdx.x < nslot) {
        Cand r = no_cand();
        for (int k = 0; k < NWARP; k++) cand_merge(r, sm.wbest[k][threadIdx.x], edgeOff + threadIdx.x, sm, exact_c);
        sm.fin[threadIdx.x] = r;
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// prep: classify sets (CTA 0)
// --------------------------------------------------------------------------
template <typename P> __device__ __noinline__ void prep(const Params &p, RoundSmem<P> &sm) {
    long long *scr = sm.scanTmp;
    long long carryBig = 0, carrySmall = 0, carryTiles = 0, bigPts = 0, smallPts = 0;
    for (int base = 0; base < p.numSets; base += NT) {
        const int i = base + threadIdx.x;
        long long off = 0, n = 0;
        int kind = I_EMPTY;
        if (i < p.numSets) {
            if (p.offsets) {
                off = p.offsets[i];
                n = p.offsets[i + 1] - off;
            } else {
                off = 0;
                n = p.nSingle;
            }
            if (off < 0 || n < 0 || off + n > p.ncap) {
                set_err(p.ctl, E_ARG);
                n = 0;
            }
            kind = n == 0 ? I_EMPTY : (n <= FIN_MAX ? I_SMALL : I_BIG);
        }
        const long long tiles = kind == I_BIG ? (n + TILE - 1) / TILE : 0;
        // packed scan: big count (bits 0..19), small count (20..39), tiles (40..63) would
        // overflow for large batches, so scan the three quantities separately.
        long long tb, ts, tt;
        long long xb = block_excl_scan<long long, NT>(kind == I_BIG ? 1 : 0, scr, tb);
        long long xs = block_excl_scan<long long, NT>(kind == I_SMALL ? 1 : 0, scr, ts);
        long long xt = block_excl_scan<long long, NT>(tiles, scr, tt);
        long long tbp, tsp;
        block_excl_scan<long long, NT>(kind == I_BIG ? n : 0, scr, tbp);
        block_excl_scan<long long, NT>(kind == I_SMALL ? n : 0, scr, tsp);
        bigPts += tbp;
        smallPts += tsp;
        if (i < p.numSets) {
            Inst &I = p.inst[i];
            I.off = off;
            I.n = n;
            I.kind = kind;
            I.K = 0;
            I.tiles = (int)tiles;
            I.tile0 = carryTiles + xt;
            I.level0 = -1;
            I.done = 0u;
            I.done0 = 0u;
            for (int k = 0; k < 4; k++) I.chCount[k] = 0;
            if (kind == I_BIG) {
                p.bigInst[carryBig + xb] = i;
                p.bigTilePrefix[carryBig + xb] = carryTiles + xt;
            } else if (kind == I_SMALL) {
                p.smallInst[carrySmall + xs] = i;
            } else {
                p.outCounts[i] = 0;
            }
        }
        carryBig += tb;
        carrySmall += ts;
        carryTiles += tt;
    }
    if (threadIdx.x == 0) {
        p.bigTilePrefix[carryBig] = carryTiles;
        if (carryTiles > p.maxTiles) set_err(p.ctl, E_CAPACITY);
        p.ctl->nBig = (int)carryBig;
        p.ctl->nSmallInst = (int)carrySmall;
        p.ctl->bigTiles = carryTiles;
        p.ctl->bigPoints = bigPts;
        p.ctl->smallPoints = smallPts;
        p.ctl->S = 0;
        p.ctl->L = 0;
        p.ctl->tiles = 0;
        p.ctl->nNodes = 0;
        p.ctl->nLevels = 0;
        p.ctl->nSmall = 0;
    }
    __threadfence();
}

// --------------------------------------------------------------------------
// tile descriptors: resolved in batches, one thread per tile, so the lookups
// (binary searches, segment records) of DB tiles overlap; thread 0 then only
// copies a descriptor and starts its TMA copies.
// --------------------------------------------------------------------------
__device__ void resolve_set_tile(const Params &p, TileRec &R, long long t, bool withPoly) {
    const int nBig = __ldcg(&p.ctl->nBig);
    const long long j = upper_bound_ll(p.bigTilePrefix, nBig + 1, t) - 1;
    const int i = __ldcg(&p.bigInst[j]);
    const Inst *I = &p.inst[i];
    R.t = t;
    R.inst = i;
    R.np = 1;
    R.valid = 1;
    R.srcBuf = 0;
    R.lt = t - __ldcg(&p.bigTilePrefix[j]);
    R.setOff = __ldcg(&I->off);
    R.setN = __ldcg(&I->n);
    R.tile0 = __ldcg(&I->tile0);
    R.tiles = __ldcg(&I->tiles);
    R.K = 0;
    R.iB = 1;
    R.hasBox = 0;
    if (withPoly) {
        R.K = __ldcg(&I->K);
        R.iB = __ldcg(&I->iB);
        R.hasBox = __ldcg(&I->hasBox);
        for (int k = 0; k < 4; k++) {
            R.poly[k] = ldcg_cand(&I->poly[k]);
            R.box[k] = __ldcg(&I->box[k]);
        }
    }
    const long long first = R.lt * TILE;
    const int c = (int)min((long long)TILE, R.setN - first);
    R.nItems = c;
    int sx = 0, si = 0;
    unsigned bytes = 0u;
    part_geo(R.g[0], R.setOff + first, c, 0, false, sx, si, bytes, (int)((reinterpret_cast<uintptr_t>(p.pts) >> 3) & 1),
             0);
    if (withPoly && R.K == 0) bytes = 0u;  // no segments: the tile is skipped
    R.bytes = bytes;
}

__device__ void resolve_round_tile(const Params &p, TileRec &R, long long t, int S, long long L, int cur, int src) {
    const long long v0 = t * TILE, v1 = min(v0 + (long long)TILE, L);
    const long long *vs = p.vstart[cur];
    const int *bl = p.bigList[cur];
    const long long sA = upper_bound_ll(vs, (long long)S + 1, v0) - 1;
    R.t = t;
    R.nItems = (int)(v1 - v0);
    R.valid = 1;
    R.srcBuf = src;
    int np = 1;
    R.node[0] = __ldcg(&bl[sA]);
    R.vstart[0] = __ldcg(&vs[sA]);
    if (sA + 1 < S) {
        const long long vb = __ldcg(&vs[sA + 1]);
        if (vb < v1) {
            np = 2;
            R.node[1] = __ldcg(&bl[sA + 1]);
            R.vstart[1] = vb;
        }
    }
    R.np = np;
    int sx = 0, si = 0;
    unsigned bytes = 0u;
    for (int part = 0; part < np; part++) {
        const Node *N = &p.nodes[R.node[part]];
        R.pstart[part] = __ldcg(&N->pstart);
        R.count[part] = __ldcg(&N->count);
        R.nh[part] = ldcg_cand(&N->h);
        R.ne[part] = ldcg_cand(&N->e);
        R.nc[part] = ldcg_cand(&N->c);
        const long long fv = part ? R.vstart[1] : v0;
        const long long lv = (part == 0 && np == 2) ? R.vstart[1] : v1;
        const long long q0 = R.pstart[part] + (fv - R.vstart[part]);
        const int c = (int)(lv - fv);
        if (c < 0 || q0 < 0 || q0 + c > 2 * p.ncap) {  // guard: never copy outside the live buffer
            set_err(p.ctl, E_INTERNAL);
            R.valid = 0;
        }
        part_geo(R.g[part], q0, c, (int)(fv - v0), true, sx, si, bytes,
                 (int)((reinterpret_cast<uintptr_t>(p.xy[src]) >> 3) & 1),
                 (int)((reinterpret_cast<uintptr_t>(p.id[src]) >> 2) & 3));
    }
    R.bytes = R.valid ? bytes : 0u;
}

// Thread 0: start the copies of tile descriptor R into stage s.
template <typename P>
__device__ void issue_desc(const Params &p, RoundSmem<P> &sm, int s, const TileRec &R, bool set) {
    mbar_expect_tx(&sm.mbar[s], R.bytes);
    if (R.bytes == 0u) return;
    if (set) {
        bulk_g2s(&sm.stage[s].xy[0], p.pts + R.g[0].a0, R.bytes, &sm.mbar[s]);
        return;
    }
    const float2 *gxy = p.xy[R.srcBuf];
    const int *gid = p.id[R.srcBuf];
    for (int part = 0; part < R.np; part++) {
        const PartGeo &g = R.g[part];
        if (g.a1 > g.a0) bulk_g2s(&sm.stage[s].xy[g.sx], gxy + g.a0, (unsigned)(g.a1 - g.a0) * 8u, &sm.mbar[s]);
        if (g.b1 > g.b0) bulk_g2s(&sm.stage[s].id[g.si], gid + g.b0, (unsigned)(g.b1 - g.b0) * 4u, &sm.mbar[s]);
    }
}

// Descriptor of the CTA's k-th tile of the current sequence.
template <typename P> __device__ __forceinline__ TileRec &desc_of(RoundSmem<P> &sm, long long k) {
    return sm.desc[(k / DB) & 1][k % DB];
}

// All threads: resolve the descriptors of the CTA's tiles k0 .. k0+DB-1.
struct TileSeq {
    long long first, step, cnt;
    int kind;  // 0: set tiles (extremes), 1: set tiles with polygon (round 0), 2: round tiles
    int S, cur, src;
    long long L;
};
template <typename P> __device__ void resolve_batch(const Params &p, RoundSmem<P> &sm, const TileSeq &q, long long k0) {
    __syncthreads();
    const long long j = threadIdx.x;
    if (j < DB && k0 + j < q.cnt) {
        const long long t = q.first + (k0 + j) * q.step;
        if (q.kind == 2)
            resolve_round_tile(p, desc_of(sm, k0 + j), t, q.S, q.L, q.cur, q.src);
        else
            resolve_set_tile(p, desc_of(sm, k0 + j), t, q.kind == 1);
    }
    __syncthreads();
}

// Start the pipeline: first batch of descriptors, then the first NS tiles.
// The global data a phase copies with TMA was written by ordinary stores of
// earlier phases (ordered by the grid barrier); one proxy fence per phase by
// the issuing thread orders them before the async copies.  Stage reuse needs
// none: the CTA barrier after the consumers' reads precedes every refill.
template <typename P>
__device__ void pipe_start(const Params &p, RoundSmem<P> &sm, const TileSeq &q, unsigned long long &gI) {
    if (q.cnt <= 0) return;
    if (threadIdx.x == 0) fence_proxy_async();
    resolve_batch(p, sm, q, 0);
    for (long long j = 0; j < min(q.cnt, (long long)NS); j++) {
        if (threadIdx.x == 0) issue_desc(p, sm, (int)(gI % NS), desc_of(sm, j), q.kind != 2);
        gI++;
    }
}

// After tile k's points are in registers (and a barrier): refill its stage with tile k + NS.
template <typename P>
__device__ void pipe_refill(const Params &p, RoundSmem<P> &sm, const TileSeq &q, long long k, int s,
                            unsigned long long &gI) {
    const long long nk = k + NS;
    if (nk >= q.cnt) return;
    if (nk % DB == 0) resolve_batch(p, sm, q, nk);
    if (threadIdx.x == 0) issue_desc(p, sm, s, desc_of(sm, nk), q.kind != 2);
    gI++;
}

// Wait for every copy still in flight (used on the error path before leaving).
template <typename P>
__device__ void pipe_drain(const Params &p, RoundSmem<P> &sm, unsigned long long gI, unsigned long long gC) {
    for (unsigned long long q = gC; q < gI; q++) {
        unsigned it = 0;
        while (!mbar_try_wait(&sm.mbar[q % NS], (unsigned)((q / NS) & 1ull)))
            if (++it > SPIN_LIMIT) break;
    }
}

// --------------------------------------------------------------------------
// extremes (Sec. 4.2)
// --------------------------------------------------------------------------
// An axis-aligned box inside the closed initial polygon (K >= 3 vertices, CCW):
// points in the closed box are never strictly right of an edge, so the
// initial split can drop them with four comparisons.  Candidate: half-way
// between the centroid and the four extreme points; every corner is verified
// with the exact orientation test (shrunk towards the centroid on failure).
__device__ __noinline__ int inner_box(const Cand (&poly)[4], int K, const Ext &a, float (&box)[4]) {
    float cx = 0.f, cy = 0.f;
    for (int k = 0; k < K; k++) {
        cx += poly[k].x;
        cy += poly[k].y;
    }
    cx /= (float)K;
    cy /= (float)K;
    float hx0 = 0.5f * (a.a.x - cx), hx1 = 0.5f * (a.b.x - cx);
    float hy0 = 0.5f * (a.bot.y - cy), hy1 = 0.5f * (a.top.y - cy);
    for (int tries = 0; tries < 4; tries++) {
        const float bx[4] = {cx + hx0, cx + hx1, cy + hy0, cy + hy1};
        bool ok = isfinite(bx[0]) && isfinite(bx[1]) && isfinite(bx[2]) && isfinite(bx[3]) && bx[0] <= bx[1] &&
                  bx[2] <= bx[3];
        for (int c = 0; c < 4 && ok; c++) {
            const float px = (c & 1) ? bx[1] : bx[0], py = (c & 2) ? bx[3] : bx[2];
            for (int k = 0; k < K && ok; k++) {
                const Cand &u = poly[k], &v = poly[(k + 1) % K];
                if (orient_exact(u.x, u.y, v.x, v.y, px, py) < 0) ok = false;
            }
        }
        if (ok) {
            for (int k = 0; k < 4; k++) box[k] = bx[k];
            return 1;
        }
        hx0 *= 0.5f;
        hx1 *= 0.5f;
        hy0 *= 0.5f;
        hy1 *= 0.5f;
    }
    return 0;
}

// Reduce this CTA's running extremes of set i, store them as the partial of
// the CTA's first tile of that set, and let the CTA that completes the set's
// tiles merge all partials into the initial polygon.
template <typename P>
__device__ __noinline__ void ext_flush(const Params &p, RoundSmem<P> &sm, Ext e, int i, long long segFirst, int segTiles) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    e = warp_ext_reduce(e);
    __syncthreads();
    if (lane == 0) sm.wext[w] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext r = sm.wext[0];
        for (int k = 1; k < NWARP; k++) ext_merge(r, sm.wext[k]);
        st_ext(&p.text[segFirst], r);
        __threadfence();
        const unsigned prev = atomicAdd(&p.inst[i].done, (unsigned)segTiles);
        sm.kflag = (prev + (unsigned)segTiles == (unsigned)__ldcg(&p.inst[i].tiles));
        __threadfence();
    }
    __syncthreads();
    if (!sm.kflag) return;
    const Inst *I = &p.inst[i];
    const long long tile0 = __ldcg(&I->tile0);
    const long long tiles = __ldcg(&I->tiles);
    const long long T = __ldcg(&p.ctl->bigTiles), G = gridDim.x;
    Ext r = ext_empty();
    if (threadIdx.x == 0) ext_merge(r, ld_ext(&p.text[tile0]));
    for (long long b = threadIdx.x; b < G; b += NT) {
        const long long c = b * T / G;  // chunk starts inside the set hold partials too
        if (c > tile0 && c < tile0 + tiles) ext_merge(r, ld_ext(&p.text[c]));
    }
    r = warp_ext_reduce(r);
    __syncthreads();
    if (lane == 0) sm.wext[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext a = sm.wext[0];
        for (int k = 1; k < NWARP; k++) ext_merge(a, sm.wext[k]);
        Inst &W = p.inst[i];
        int K = 0, iB = 1, hasBox = 0;
        Cand poly[4];
        float box[4] = {0.f, 0.f, 0.f, 0.f};
        int kind = I_BIG;
        if (a.nonfinite) {
            kind = I_NONFINITE;
        } else if (same_xy(a.a, a.b)) {
            kind = I_DEGEN;
            poly[0] = a.a;
        } else {
            const bool quad = (p.mode == 0);
            poly[K++] = a.a;
            if (quad && !same_xy(a.bot, a.a) && !same_xy(a.bot, a.b)) poly[K++] = a.bot;
            iB = K;
            poly[K++] = a.b;
            if (quad && !same_xy(a.top, a.a) && !same_xy(a.top, a.b)) poly[K++] = a.top;
            if (K >= 3) hasBox = inner_box(poly, K, a, box);
        }
        W.kind = kind;
        W.K = K;
        W.iB = iB;
        W.hasBox = hasBox;
        for (int k = 0; k < 4; k++) W.box[k] = box[k];
        for (int k = 0; k < 4; k++) W.poly[k] = (k < K || (kind == I_DEGEN && k == 0)) ? poly[k] : no_cand();
        __threadfence();
    }
    __syncthreads();
}

template <typename P>
__device__ __noinline__ bool phase_extremes(const Params &p, RoundSmem<P> &sm, unsigned long long &gI, unsigned long long &gC) {
    const long long T = __ldcg(&p.ctl->bigTiles), G = gridDim.x;
    const long long cb = (long long)blockIdx.x * T / G, ce = ((long long)blockIdx.x + 1) * T / G;
    const long long cnt = ce - cb;
    TileSeq q;
    q.first = cb;
    q.step = 1;
    q.cnt = cnt;
    q.kind = 0;
    q.S = q.cur = q.src = 0;
    q.L = 0;
    pipe_start(p, sm, q, gI);
    Ext acc = ext_empty();
    int accInst = -1, segTiles = 0;
    long long segFirst = 0;
    QH_PROF_DECL;
    for (long long k = 0; k < cnt; k++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain(p, sm, gI, gC);
            return false;
        }
        QH_PROF(0);
        const TileRec &R = desc_of(sm, k);
        const int inst = R.inst;
        if (inst != accInst) {
            if (accInst >= 0) ext_flush(p, sm, acc, accInst, segFirst, segTiles);
            acc = ext_empty();
            accInst = inst;
            segFirst = R.t;
            segTiles = 0;
        }
        const int nItems = R.nItems;
        const long long base = R.lt * TILE;
#pragma unroll
        for (int kk = 0; kk < IPT; kk++) {
            const int i = kk * NT + threadIdx.x;
            if (i < nItems) {
                const float2 q = fetch_xy(R, sm.stage[s], i, p.pts, true);
                if (!isfinite(q.x) || !isfinite(q.y)) {
                    acc.nonfinite = 1;
                } else {
                    const int id = (int)(base + i);
                    if (lex_less(q.x, q.y, id, acc.a.x, acc.a.y, acc.a.idx)) acc.a = mk_cand(q.x, q.y, id);
                    if (lex_greater(q.x, q.y, id, acc.b.x, acc.b.y, acc.b.idx)) acc.b = mk_cand(q.x, q.y, id);
                    if (lex_less(q.y, q.x, id, acc.bot.y, acc.bot.x, acc.bot.idx)) acc.bot = mk_cand(q.x, q.y, id);
                    if (lex_greater(q.y, q.x, id, acc.top.y, acc.top.x, acc.top.idx)) acc.top = mk_cand(q.x, q.y, id);
                }
            }
        }
        segTiles++;
        QH_PROF(1);
        __syncthreads();
        QH_PROF(2);
        pipe_refill(p, sm, q, k, s, gI);
        QH_PROF(3);
    }
    if (accInst >= 0) ext_flush(p, sm, acc, accInst, segFirst, segTiles);
    QH_PROF(4);
    QH_PROF_FLUSH_AT(p.ctl, 8);
    return true;
}

// --------------------------------------------------------------------------
// round 0: the initial split
// --------------------------------------------------------------------------
template <typename P>
__device__ __noinline__ bool phase_round0(const Params &p, RoundSmem<P> &sm, unsigned long long &gI, unsigned long long &gC,
                             int &exact_o, int &exact_c, long long &survivors) {
    const long long T = __ldcg(&p.ctl->bigTiles);
    const long long first = blockIdx.x, step = gridDim.x;
    const long long cnt = first < T ? (T - 1 - first) / step + 1 : 0;
    TileSeq q;
    q.first = first;
    q.step = step;
    q.cnt = cnt;
    q.kind = 1;
    q.S = q.cur = q.src = 0;
    q.L = 0;
    pipe_start(p, sm, q, gI);
    QH_PROF_DECL;
    for (long long kt = 0; kt < cnt; kt++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        QH_PROF(7);
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain(p, sm, gI, gC);
            return false;
        }
        QH_PROF(0);
        const TileRec &R = desc_of(sm, kt);
        const int K = R.K;
        float x[IPT], y[IPT];
        int idx[IPT], slot[IPT], rank[IPT];
        P lo[IPT], hi[IPT];
        const int nItems = R.nItems;
        const long long base = R.lt * TILE;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int i = k * NT + threadIdx.x;
            slot[k] = -1;
            lo[k] = hi[k] = P(0);
            x[k] = y[k] = 0.f;
            idx[k] = (int)(base + i);
            if (K > 0 && i < nItems) {
                const float2 q = fetch_xy(R, sm.stage[s], i, p.pts, true);
                x[k] = q.x;
                y[k] = q.y;
            }
        }
        if (threadIdx.x < K) {
            const Cand u = R.poly[threadIdx.x], v = R.poly[(threadIdx.x + 1) % K];
            sm.edge[threadIdx.x] = make_edge<P>(u.x, u.y, v.x, v.y);
            sm.vend[threadIdx.x][0] = v.x;
            sm.vend[threadIdx.x][1] = v.y;
        } else if (threadIdx.x == 32 && K > 0) {
            const Cand u = R.poly[0], v = R.poly[R.iB];
            sm.edge[4] = make_edge<P>(u.x, u.y, v.x, v.y);
            sm.vend[4][0] = v.x;
            sm.vend[4][1] = v.y;
        }
        __syncthreads();
        pipe_refill(p, sm, q, kt, s, gI);
        QH_PROF(1);
        if (K == 0) continue;  // degenerate or rejected set: no segments
        const TileRec &C = R;
        // A point lies strictly outside at most one edge of the initial polygon.
        // Its side of the chord A->B tells which chain (A..B below, B..A above)
        // can hold that edge; on the chord (or in the inner box) it is inside.
        const int iB = C.iB, hasBox = C.hasBox;
        const float bx0 = C.box[0], bx1 = C.box[1], by0 = C.box[2], by1 = C.box[3];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int i = k * NT + threadIdx.x;
            if (i >= nItems) continue;
            const float px = x[k], py = y[k];
            if (hasBox && px >= bx0 && px <= bx1 && py >= by0 && py <= by1) continue;
            const Edge<P> &ch = sm.edge[4];
            const Approx<P> o = orient_approx(ch, px, py);
            const int sg = orient_sign(ch, sm.vend[4][0], sm.vend[4][1], px, py, o, exact_o);
            if (sg == 0) continue;
            const int e0 = sg < 0 ? 0 : iB, e1 = sg < 0 ? iB : K;
            if (e1 - e0 == 1) {  // the chain is the chord itself: A->B below, B->A above
                const DistIv<P> d = dist_interval(o);
                slot[k] = e0;
                if (sg < 0) {
                    lo[k] = d.lo;
                    hi[k] = d.hi;
                } else {  // distance right of B->A is +orient(A, B, P)
                    lo[k] = -d.hi;
                    hi[k] = -d.lo;
                }
                continue;
            }
            for (int e = e0; e < e1; e++) {
                if (right_of(sm.edge[e], sm.vend[e][0], sm.vend[e][1], px, py, lo[k], hi[k], exact_o)) {
                    slot[k] = e;
                    break;
                }
            }
        }
        QH_PROF(2);
        unsigned tot[4];
        tile_ranks(slot, rank, tot, sm);
        QH_PROF(3);
        tile_farthest(slot, x, y, idx, lo, hi, sm, exact_c);
        QH_PROF(4);

        const long long t = C.t;
        Inst *W = &p.inst[C.inst];
        if (threadIdx.x < K)  // reserve this tile's range in each initial segment
            sm.base[threadIdx.x] = tot[threadIdx.x] ? atomicAdd(&W->chCount[threadIdx.x], (int)tot[threadIdx.x]) : 0;
        if (threadIdx.x == 32) {
            store_tile_bests(p, t, sm.best);
            __threadfence();
            sm.fflag[0] = atomicAdd(&W->done0, 1u) == (unsigned)C.tiles - 1u;
        }
        __syncthreads();
        QH_PROF(5);
        const long long off = C.setOff, n = C.setN;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int q = slot[k];
            if (q < 0) continue;
            const long long b = (q < 2 ? 0ll : p.ncap) + off;
            const long long rr = (long long)sm.base[q] + rank[k];
            const long long pos = (q & 1) ? b + n - 1 - rr : b + rr;
            if (pos < b || pos >= b + n) {  // guard: never write outside the set's range
                set_err(p.ctl, E_INTERNAL);
                continue;
            }
            __stcg(&p.xy[0][pos], make_float2(x[k], y[k]));
            __stcg(&p.id[0][pos], idx[k]);
        }
        if (sm.fflag[0]) {  // last tile of the set: farthest point of every initial segment
            __threadfence();
            merge_parent_bests(p, sm, C.tile0, C.tile0 + C.tiles - 1, 0, K, 0, exact_c);
            if (threadIdx.x < K) stcg_cand(&W->chC[threadIdx.x], sm.fin[threadIdx.x]);
        }
        if (threadIdx.x == 0) survivors += (long long)tot[0] + tot[1] + tot[2] + tot[3];
        QH_PROF(6);
    }
    QH_PROF_FLUSH(p.ctl);
    return true;
}

// --------------------------------------------------------------------------
// round r >= 1
// --------------------------------------------------------------------------
template <typename P>
__device__ __noinline__ bool phase_round(const Params &p, RoundSmem<P> &sm, unsigned long long &gI, unsigned long long &gC, int r,
                            int S, long long L, int cur, int &exact_o, int &exact_c, long long &survivors) {
    const int src = (r - 1) & 1, dst = r & 1;
    const long long T = (L + TILE - 1) / TILE;
    const long long first = blockIdx.x, step = gridDim.x;
    const long long cnt = first < T ? (T - 1 - first) / step + 1 : 0;
    TileSeq q;
    q.first = first;
    q.step = step;
    q.cnt = cnt;
    q.kind = 2;
    q.S = S;
    q.cur = cur;
    q.src = src;
    q.L = L;
    pipe_start(p, sm, q, gI);
    for (long long kt = 0; kt < cnt; kt++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain(p, sm, gI, gC);
            return false;
        }
        const TileRec &R = desc_of(sm, kt);
        const int valid = R.valid, np = R.np, nItems = R.nItems;
        float x[IPT], y[IPT];
        int idx[IPT], slot[IPT], rank[IPT];
        P lo[IPT], hi[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int i = k * NT + threadIdx.x;
            slot[k] = -1;
            lo[k] = hi[k] = P(0);
            x[k] = y[k] = 0.f;
            idx[k] = -1;
            if (valid && i < nItems) {
                const float2 q = fetch_xy(R, sm.stage[s], i, p.xy[src], false);
                x[k] = q.x;
                y[k] = q.y;
                idx[k] = fetch_id(R, sm.stage[s], i, p.id[src]);
            }
        }
        if (threadIdx.x < 2 * np) {
            const int part = threadIdx.x >> 1, which = threadIdx.x & 1;
            const Cand u = which ? R.nc[part] : R.nh[part];
            const Cand v = which ? R.ne[part] : R.nc[part];
            sm.edge[threadIdx.x] = make_edge<P>(u.x, u.y, v.x, v.y);
            sm.vend[threadIdx.x][0] = v.x;
            sm.vend[threadIdx.x][1] = v.y;
        }
        __syncthreads();
        pipe_refill(p, sm, q, kt, s, gI);
        if (!valid) continue;
        const TileRec &C = R;
        const long long vB = np == 2 ? (long long)C.g[1].vofs : (long long)TILE;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int i = k * NT + threadIdx.x;
            if (i < nItems) {
                const int s0 = (i >= vB) ? 2 : 0;
                if (right_of(sm.edge[s0], sm.vend[s0][0], sm.vend[s0][1], x[k], y[k], lo[k], hi[k], exact_o))
                    slot[k] = s0;
                else if (right_of(sm.edge[s0 + 1], sm.vend[s0 + 1][0], sm.vend[s0 + 1][1], x[k], y[k], lo[k], hi[k],
                                  exact_o))
                    slot[k] = s0 + 1;
            }
        }
        unsigned tot[4];
        tile_ranks(slot, rank, tot, sm);
        tile_farthest(slot, x, y, idx, lo, hi, sm, exact_c);

        const long long t = C.t;
        if (threadIdx.x < 2 * np) {  // reserve this tile's range in each child
            const int q = threadIdx.x;
            Node *N = &p.nodes[C.node[q >> 1]];
            sm.base[q] = tot[q] ? atomicAdd(&N->chCount[q & 1], (int)tot[q]) : 0;
        }
        if (threadIdx.x == 32) {
            store_tile_bests(p, t, sm.best);
            __threadfence();
            for (int part = 0; part < 2; part++) {
                int last = 0;
                if (part < np) {
                    const long long vs = C.vstart[part], cn = C.count[part];
                    const unsigned nt = (unsigned)((vs + cn - 1) / TILE - vs / TILE + 1);
                    last = atomicAdd(&p.nodes[C.node[part]].tdone, 1u) == nt - 1u;
                }
                sm.fflag[part] = last;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const int q = slot[k];
            if (q < 0) continue;
            const int part = q >> 1;
            const long long ps = C.pstart[part], cn = C.count[part];
            const long long rr = (long long)sm.base[q] + rank[k];
            const long long pos = (q & 1) ? ps + cn - 1 - rr : ps + rr;
            if (pos < ps || pos >= ps + cn || pos >= 2 * p.ncap) {
                set_err(p.ctl, E_INTERNAL);  // guard: a child never leaves its parent's range
                continue;
            }
            __stcg(&p.xy[dst][pos], make_float2(x[k], y[k]));
            __stcg(&p.id[dst][pos], idx[k]);
        }
        for (int part = 0; part < np; part++) {
            if (!sm.fflag[part]) continue;  // this tile closes the parent: farthest points of its children
            __threadfence();
            const long long vs = C.vstart[part], cn = C.count[part];
            const long long ta = vs / TILE, tb = (vs + cn - 1) / TILE;
            merge_parent_bests(p, sm, ta, tb, (vs % TILE) != 0 ? 2 : 0, 2, 2 * part, exact_c);
            if (threadIdx.x < 2) stcg_cand(&p.nodes[C.node[part]].chC[threadIdx.x], sm.fin[threadIdx.x]);
        }
        if (threadIdx.x == 0) survivors += (long long)tot[0] + tot[1] + tot[2] + tot[3];
    }
    return true;
}

// --------------------------------------------------------------------------
// level construction (last CTA of a round)
// --------------------------------------------------------------------------
// List the big nodes of [first, first + count) for the next round (exclusive
// prefix of their sizes), queue the small ones for the block finisher.
template <typename P>
__device__ void build_biglist(const Params &p, RoundSmem<P> &sm, int first, int count, int dstBuf) {
    long long *scr = sm.scanTmp;
    const int per = (count + NT - 1) / NT;
    const int b = min(count, threadIdx.x * per), e = min(count, b + per);
    long long nb = 0, np = 0;
    for (int k = b; k < e; k++) {
        const Node *N = &p.nodes[first + k];
        if (__ldcg(&N->kind) == K_BIG) {
            nb++;
            np += __ldcg(&N->count);
        }
    }
    long long totB, totP;
    long long xb = block_excl_scan<long long, NT>(nb, scr, totB);
    long long xp = block_excl_scan<long long, NT>(np, scr, totP);
    if (totB > p.maxBig) {
        if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
        return;
    }
    int *bl = p.bigList[dstBuf];
    long long *vs = p.vstart[dstBuf];
    for (int k = b; k < e; k++) {
        const int q = first + k;
        const Node *N = &p.nodes[q];
        const int kind = __ldcg(&N->kind);
        if (kind == K_BIG) {
            __stcg(&bl[xb], q);
            __stcg(&vs[xb], xp);
            xb++;
            xp += __ldcg(&N->count);
        } else if (kind == K_SMALL) {
            int j = atomicAdd(&p.ctl->nSmall, 1);
            __stcg(&p.smallQ[j], q);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __stcg(&vs[totB], totP);
        p.ctl->S = (int)totB;
        p.ctl->L = totP;
        p.ctl->tiles = (totP + TILE - 1) / TILE;
        p.ctl->cur = dstBuf;
    }
    __threadfence();
    __syncthreads();
}

__device__ __forceinline__ int node_kind(int count, int cut) {
    return count == 0 ? K_LEAF : (count <= cut ? K_SMALL : K_BIG);
}

template <typename P> __device__ __noinline__ void build_level0(const Params &p, RoundSmem<P> &sm) {
    long long *scr = sm.scanTmp;
    const int nBig = __ldcg(&p.ctl->nBig);
    long long carry = 0;
    for (int base = 0; base < nBig; base += NT) {
        const int j = base + threadIdx.x;
        int K = 0, i = -1;
        if (j < nBig) {
            i = __ldcg(&p.bigInst[j]);
            K = __ldcg(&p.inst[i].K);
        }
        long long tot;
        long long x = block_excl_scan<long long, NT>(K, scr, tot);
        if (carry + tot > p.maxNodes) {
            if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
            return;
        }
        if (j < nBig) {
            Inst *I = &p.inst[i];
            const int q0 = (int)(carry + x);
            __stcg(&I->level0, q0);
            const long long off = __ldcg(&I->off), n = __ldcg(&I->n);
            for (int k = 0; k < K; k++) {
                Node *N = &p.nodes[q0 + k];
                const int cnt = __ldcg(&I->chCount[k]);
                stcg_cand(&N->h, ldcg_cand(&I->poly[k]));
                stcg_cand(&N->e, ldcg_cand(&I->poly[(k + 1) % K]));
                stcg_cand(&N->c, ldcg_cand(&I->chC[k]));
                __stcg(&N->count, cnt);
                __stcg(&N->kind, node_kind(cnt, p.cut));
                __stcg(&N->pstart, (k < 2 ? 0ll : p.ncap) + off + ((k & 1) ? n - cnt : 0ll));
                __stcg(&N->buf, 0);
                __stcg(&N->inst, i);
                __stcg(&N->level, 0);
                __stcg(&N->child, -1);
                __stcg(&N->inner, 0);
                __stcg(&N->chCount[0], 0);
                __stcg(&N->chCount[1], 0);
                __stcg(&N->tdone, 0u);
            }
        }
        carry += tot;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctl->nNodes = (int)carry;
        p.ctl->nLevels = 1;
        p.ctl->levelBase[0] = 0;
        p.ctl->levelBase[1] = (int)carry;
    }
    build_biglist(p, sm, 0, (int)carry, 0);
}

template <typename P> __device__ __noinline__ void build_level(const Params &p, RoundSmem<P> &sm, int r) {
    const int S = __ldcg(&p.ctl->S);
    const int cur = __ldcg(&p.ctl->cur);
    const int base = __ldcg(&p.ctl->nNodes);
    if (base + 2ll * S > p.maxNodes || r + 1 > MAX_LEVELS) {
        if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
        return;
    }
    const int *bl = p.bigList[cur];
    for (int j = threadIdx.x; j < S; j += NT) {
        const int q = __ldcg(&bl[j]);
        Node *Q = &p.nodes[q];
        const Cand h = ldcg_cand(&Q->h), e = ldcg_cand(&Q->e), c = ldcg_cand(&Q->c);
        const long long ps = __ldcg(&Q->pstart);
        const int cnt = __ldcg(&Q->count), buf = __ldcg(&Q->buf), inst = __ldcg(&Q->inst);
        __stcg(&Q->child, base + 2 * j);
        for (int w = 0; w < 2; w++) {
            Node *N = &p.nodes[base + 2 * j + w];
            const int cc = __ldcg(&Q->chCount[w]);
            stcg_cand(&N->h, w ? c : h);
            stcg_cand(&N->e, w ? e : c);
            stcg_cand(&N->c, ldcg_cand(&Q->chC[w]));
            __stcg(&N->count, cc);
            __stcg(&N->kind, node_kind(cc, p.cut));
            __stcg(&N->pstart, w ? ps + cnt - cc : ps);
            __stcg(&N->buf, buf ^ 1);
            __stcg(&N->inst, inst);
            __stcg(&N->level, r);
            __stcg(&N->child, -1);
            __stcg(&N->inner, 0);
            __stcg(&N->chCount[0], 0);
            __stcg(&N->chCount[1], 0);
            __stcg(&N->tdone, 0u);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctl->nNodes = base + 2 * S;
        p.ctl->nLevels = r + 1;
        p.ctl->levelBase[r + 1] = base + 2 * S;
        p.ctl->rounds = r;
    }
    build_biglist(p, sm, base, 2 * S, cur ^ 1);
}

// --------------------------------------------------------------------------
// the kernel
// --------------------------------------------------------------------------
template <typename P> __global__ void __launch_bounds__(NT, MINB) rounds_kernel(Params p) {
    extern __shared__ __align__(128) unsigned char rounds_smem_raw[];
    RoundSmem<P> &sm = *reinterpret_cast<RoundSmem<P> *>(rounds_smem_raw);
    unsigned phase = 0, donePhase = 0;
    int exact_o = 0, exact_c = 0;
    long long surv = 0;
    unsigned long long gI = 0, gC = 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) mbar_init(&sm.mbar[s], 1u);
        fence_mbar_init();
    }
    __syncthreads();
    stamp(p.ctl, 0);
    if (blockIdx.x == 0) prep(p, sm);
    if (!grid_sync(p.ctl, phase)) goto out;
    stamp(p.ctl, 1);

    phase_extremes(p, sm, gI, gC);
    if (!grid_sync(p.ctl, phase)) goto out;
    stamp(p.ctl, 2);

    phase_round0(p, sm, gI, gC, exact_o, exact_c, surv);
    if (threadIdx.x == 0 && surv) {
        atomicAdd((unsigned long long *)&p.ctl->live[0], (unsigned long long)surv);
        atomicAdd((unsigned long long *)&p.ctl->gridWritten, (unsigned long long)surv);
    }
    surv = 0;
    if (last_cta(p.ctl, donePhase, &sm.kflag)) build_level0(p, sm);
    if (!grid_sync(p.ctl, phase)) goto out;
    stamp(p.ctl, 3);

    for (int r = 1;; r++) {
        const int S = __ldcg(&p.ctl->S);
        if (S == 0) break;
        const long long L = __ldcg(&p.ctl->L);
        const int cur = __ldcg(&p.ctl->cur);
        if ((L + TILE - 1) / TILE > p.maxTiles) {
            if (blockIdx.x == 0 && threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
            break;
        }
        phase_round(p, sm, gI, gC, r, S, L, cur, exact_o, exact_c, surv);
        if (threadIdx.x == 0 && surv) {
            atomicAdd((unsigned long long *)&p.ctl->live[min(r, MAX_GEN - 1)], (unsigned long long)surv);
            atomicAdd((unsigned long long *)&p.ctl->gridWritten, (unsigned long long)surv);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->gridRead += L;
        surv = 0;
        if (last_cta(p.ctl, donePhase, &sm.kflag)) build_level(p, sm, r);
        if (!grid_sync(p.ctl, phase)) goto out;
        stamp(p.ctl, 3 + r);
    }
out:
    {
        // statistics: exact-fallback counts
        __syncthreads();
        unsigned long long eo = (unsigned long long)exact_o, ec = (unsigned long long)exact_c;
        for (int d = 16; d >= 1; d >>= 1) {
            eo += __shfl_xor_sync(0xffffffffu, eo, d);
            ec += __shfl_xor_sync(0xffffffffu, ec, d);
        }
        if ((threadIdx.x & 31) == 0) {
            if (eo) atomicAdd(&p.ctl->exactOrient, eo);
            if (ec) atomicAdd(&p.ctl->exactCmp, ec);
        }
    }
}

template <typename P> static cudaError_t set_rounds_smem() {
    return cudaFuncSetAttribute(rounds_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(RoundSmem<P>));
}

cudaError_t launch_rounds(const Params &p, int prec, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    cudaError_t e;
    if (prec) {
        e = set_rounds_smem<double>();
        if (e != cudaSuccess) return e;
        return cudaLaunchCooperativeKernel((void *)rounds_kernel<double>, dim3(grid), dim3(NT), args,
                                           sizeof(RoundSmem<double>), s);
    }
    e = set_rounds_smem<float>();
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((void *)rounds_kernel<float>, dim3(grid), dim3(NT), args,
                                       sizeof(RoundSmem<float>), s);
}

int rounds_max_ctas_per_sm(int prec) {
    int b = 0;
    if (prec) {
        if (set_rounds_smem<double>() != cudaSuccess) return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rounds_kernel<double>, NT, sizeof(RoundSmem<double>));
    } else {
        if (set_rounds_smem<float>() != cudaSuccess) return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rounds_kernel<float>, NT, sizeof(RoundSmem<float>));
    }
    return b;
}

}  // namespace qh
