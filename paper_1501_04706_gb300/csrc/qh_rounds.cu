// Grid-wide part of segmented QuickHull: one cooperative, persistent launch.
//
// Phases (separated by bounded grid barriers):
//   prep       CTA 0 classifies the sets: empty, small (<= FIN_MAX points, left
//              to the block finisher) or big (tiled here), and sizes the tiles.
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
//              pass.  The last CTA to reach the grid barrier that ends the
//              round (its leader) builds the next level of segments and the
//              lists for the next round and the finisher, then releases the
//              others.  The rounds end when no big segment is left, at any
//              depth: the segment tree keeps every level.
//
// Memory pipeline: every CTA owns a ring of NS shared-memory stages filled by
// TMA bulk copies (cp.async.bulk + mbarrier).  Thread 0 resolves the segment
// descriptors of tile k + NS and starts its copies while the CTA works on tile
// k, so HBM latency and descriptor lookups overlap the per-tile work.  Short
// rounds (and a single small set) use smaller tiles, so they spread over more
// CTAs.
//
// Compaction is a single pass.  Segments are contiguous ranges of a live
// buffer and a child never leaves its parent's range: the first child grows
// upward from the parent's start, the second downward from its end.  Every
// tile reserves its output range in each child with one atomic add on the
// child's cursor, so no tile ever waits for another (a tile-ordered scan would
// chain the ~600 tiles a persistent grid has in flight; the order of points
// inside a segment is irrelevant to the method).  The farthest point of each
// child is exact: every CTA works on a contiguous chunk of tiles, keeps the
// exact best of each child over its run of tiles of one parent and publishes
// it once, as a record in the run's first tile; the CTA whose publication
// completes the parent's tile count merges the parent's records (they sit at
// the parent's first tile and at the chunk starts inside its range).
// Segments with at most `cut` points (cut >= TILE) leave the grid-wide rounds
// for the block finisher, so a tile of a round spans at most two segments.
#include "qh_internal.cuh"

#ifndef QH_VARIANT_NS
#define QH_VARIANT_NS v256
#endif

namespace qh {
namespace QH_VARIANT_NS {

constexpr int NS = 2;          // pipeline stages per CTA
constexpr int DB = NT >= 256 ? 8 : 4;  // tile descriptors resolved per batch (one thread per tile)
constexpr int CLS_NONE = 15;
#ifndef QH_UNROLL
#define QH_UNROLL 4
#endif
constexpr int UNROLL_ITEMS = QH_UNROLL;  // items of a thread handled per iteration of the per-tile loops
constexpr int CQ = NT >= 256 ? 16 : 12;  // farthest-point candidates kept per slot before the fallback

// Items of one segment inside a tile: physical range [q0, q0 + c) of the
// source buffer, first tile-local item vofs.  The copies take the 16-byte
// blocks that hold the range: na points from a0 to stage offset sx and nb ids
// from b0 to stage offset si, so item i of the part sits at stage xy[i + dx]
// and id[i + di].  A 16-byte aligned block holding a byte of a valid element
// lies inside one memory page, so the rounded-out copy reads mapped memory
// only; the elements it adds at either end are never used.
struct PartGeo {
    long long q0, a0, b0;
    int c, vofs, na, nb, sx, si, dx, di;
};

struct TileRec {
    long long t;
    int np, nItems, valid, inst;
    unsigned bytes;  // TMA bytes of the tile
    int srcBuf;      // live buffer read by a round tile
    // round 0 / extremes: the set
    long long lt, setOff, setN, tile0;
    int tiles, K, iB;
    Cand poly[4];
    // rounds: the (at most two) parent segments
    int node[2], count[2];
    long long vstart[2], pstart[2];
    Cand nh[2], ne[2], nc[2];
    PartGeo g[2];
};

constexpr int STAGE_PAD = 16;  // room for the rounded-out ends of two parts
// The set of the last resolved set tile (descriptor batches of the extreme-point
// pass and the initial split): consecutive tiles mostly belong to one set.
struct SetCache {
    long long tile0, setOff, setN;
    int tiles, inst, K, iB, valid, pad;
    Cand poly[4];
};

struct StageBuf {
    float2 xy[TILE + STAGE_PAD];
    int id[TILE + STAGE_PAD];
};

// A farthest-point candidate with its distance interval beyond the slot's
// edge, computed once: most comparisons are then two float comparisons.
template <typename P> struct ICand {
    Cand c;
    P lo, hi;
};

// The CTA's running farthest-point candidates for the parent it is working on
// (a run of consecutive tiles of one parent: a set in the initial split, a
// segment in the rounds).
template <typename P> struct RunAcc {
    int node;          // parent (set index in the initial split, node index in the rounds); -1: none
    int nslot;         // child slots of the parent
    int tiles;         // tiles merged into this run
    int total;         // tiles of the parent
    int slotBase;      // record slots of this run: tbest[4 * first + slotBase + s]
    int slotBase0;     // record slot base of the parent's first run
    int edgeOff;       // the parent's edges in the working set: edge[edgeOff + s]
    int pad;
    long long first;   // tile holding this run's record
    long long ta, tb;  // first and last tile of the parent
    ICand<P> best[4];
};

template <typename P> struct RoundSmem {
    unsigned long long mbar[NS];
    RunAcc<P> run;
    SetCache setc;
    TileRec desc[2][DB];  // descriptors of the CTA's tiles, double-buffered by batch
    // tile working set
    Edge<P> edge[4];   // per slot: the edge a point of the slot lies strictly right of
    float vend[4][2];
    int kflag;
    unsigned warpCnt[NWARP][4];  // pass 1: points per warp and slot
    int warpOff[NWARP][4];       // their offsets inside the tile's reservation
    int tot[4];                  // points per slot in the tile
    unsigned maxLo[4];
    unsigned tk[4];  // extremes: keys of the tile's min x, max x, min y, max y
    int nq[4];      // candidates per slot
    int candOver;   // a slot's candidate list overflowed
    ICand<P> best[4];
    Cand fin[4];
    int base[4];   // this tile's first output rank in each slot's child
    int fflag[2];  // this tile is the last of part A / part B's parent
    long long scanTmp[NWARP + 1];
    Ext wext[NWARP];
    alignas(16) ICand<P> wbest[NWARP][4];  // per-warp bests; the level build's scan scratch between rounds
    unsigned mthr[4];  // parent merge: largest lower-bound key per child
    ICand<P> candq[4][CQ];
    unsigned clsPack[2][NT];     // 4-bit slot of every item of the tile (CLS_NONE: discarded)
    alignas(128) StageBuf stage[NS];
};

// The CTA's working set.  Functions that are not inlined take it from the
// symbol rather than through a reference, so that its accesses stay
// shared-memory loads and stores instead of generic ones.
extern __shared__ __align__(128) unsigned char rounds_smem_raw[];
template <typename P> __device__ __forceinline__ RoundSmem<P> &round_smem() {
    return *reinterpret_cast<RoundSmem<P> *>(rounds_smem_raw);
}

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
// L2 policy of the tile copies: every tile is read once per pass, so its lines
// go first and the round outputs, tables and code stay in L2.
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 1-D bulk copy global -> shared, completing on mbarrier b (16-byte aligned, size % 16 == 0),
// with L2 cache policy pol.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b,
                                         unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b)), "l"(pol)
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
// (0/1 float2, 0..3 int), so that every copy starts and ends on a 16-byte
// boundary in memory.
__device__ __forceinline__ void part_geo(PartGeo &g, long long q0, int c, int vofs, bool withId, int &sx, int &si,
                                         unsigned &bytes, int xyPhase, int idPhase) {
    g.q0 = q0;
    g.c = c;
    g.vofs = vofs;
    g.a0 = g.b0 = q0;
    g.na = g.nb = 0;
    g.sx = sx;
    g.si = si;
    g.dx = sx - vofs;
    g.di = si - vofs;
    if (c <= 0) return;
    const long long end = q0 + c;
    const long long a0 = q0 - ((q0 + xyPhase) & 1), a1 = end + ((end + xyPhase) & 1);
    g.a0 = a0;
    g.na = (int)(a1 - a0);
    g.dx = sx + (int)(q0 - a0) - vofs;
    sx += g.na;
    bytes += (unsigned)g.na * 8u;
    if (withId) {
        const long long b0 = q0 - ((q0 + idPhase) & 3), b1 = end + ((4 - ((end + idPhase) & 3)) & 3);
        g.b0 = b0;
        g.nb = (int)(b1 - b0);
        g.di = si + (int)(q0 - b0) - vofs;
        si += g.nb;
        bytes += (unsigned)g.nb * 4u;
    }
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

// --------------------------------------------------------------------------
// farthest-point candidates
// --------------------------------------------------------------------------

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

template <typename P> __device__ __forceinline__ ICand<P> no_icand() {
    ICand<P> r;
    r.c = no_cand();
    r.lo = r.hi = P(0);
    return r;
}

// Candidate c with its interval beyond the edge of slot s.
template <typename P> __device__ __forceinline__ ICand<P> icand_of(const RoundSmem<P> &sm, int s, const Cand &c) {
    ICand<P> r;
    r.c = c;
    const DistIv<P> d = dist_interval(orient_approx(sm.edge[s], c.x, c.y));
    r.lo = d.lo;
    r.hi = d.hi;
    return r;
}

// a <- the farther of a and b beyond the edge of slot s (exact order).
template <typename P>
__device__ __forceinline__ void imerge(ICand<P> &a, const ICand<P> &b, int s, const RoundSmem<P> &sm, int &exact_c) {
    if (b.c.idx < 0) return;
    DistIv<P> da, db;
    da.lo = a.lo;
    da.hi = a.hi;
    db.lo = b.lo;
    db.hi = b.hi;
    if (a.c.idx < 0 ||
        farther(sm.edge[s], sm.vend[s][0], sm.vend[s][1], b.c.x, b.c.y, b.c.idx, db, a.c.x, a.c.y, a.c.idx, da, exact_c))
        a = b;
}

template <typename P> __device__ __forceinline__ ICand<P> shfl_icand(const ICand<P> &a, int src) {
    ICand<P> r;
    r.c = shfl_cand(a.c, src);
    r.lo = __shfl_sync(0xffffffffu, a.lo, src);
    r.hi = __shfl_sync(0xffffffffu, a.hi, src);
    return r;
}

// --------------------------------------------------------------------------
// farthest points per parent: runs of tiles and their merge
// --------------------------------------------------------------------------
// Every CTA works on a contiguous chunk of tiles, so a parent (a set in the
// initial split, a segment in the rounds) is split between CTAs only at chunk
// starts.  A CTA keeps the exact best candidate of every child over its run of
// tiles of one parent and publishes it once, as a record in the run's first
// tile; the publication that completes the parent's tile count merges the
// parent's records.

// Chunk of tiles of CTA b: [floor(b T / G), floor((b + 1) T / G)).
__device__ __forceinline__ long long chunk_start(long long b, long long T, long long G) { return b * T / G; }
// The same in 32-bit arithmetic (a 64-bit division is a long dependent chain)
// when b * T fits: narrow = G * T < 2^32.
__device__ __forceinline__ long long chunk_start_n(long long b, long long T, long long G, bool narrow) {
    return narrow ? (long long)((unsigned)b * (unsigned)T / (unsigned)G) : b * T / G;
}
// Records of a parent a thread keeps in registers while merging (one per CTA
// of the largest grid of the variant, NT per pass).
constexpr int MREC = (152 * MINB + NT - 1) / NT;
// The chunk holding tile t: the largest b with chunk_start(b) <= t.
__device__ __forceinline__ long long chunk_of(long long t, long long T, long long G) {
    return min(((t + 1) * G + T - 1) / T - 1, G - 1);
}

// Farthest point of every child of a parent spanning tiles [ta, tb] -> sm.fin.
// The parent's runs start at ta (record slots slotBase0..) and at every chunk
// start inside (ta, tb] (slots 0..), each holding the exact best of its tiles.
// All records are read at once (every load of a thread in flight together) and
// their bound keys kept in registers; only those whose upper bound reaches the
// child's largest lower bound can be its farthest point, and only these are
// read again and compared (exactly) by one thread per child.
template <typename P>
__device__ __noinline__ void merge_runs(const Params &p, long long ta, long long tb, int slotBase0, int nslot,
                                        int edgeOff, long long T, int &exact_c) {
    RoundSmem<P> &sm = round_smem<P>();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long G = gridDim.x;
    const long long c0 = chunk_of(ta, T, G), c1 = chunk_of(tb, T, G);
    const long long nrec = 1 + (c1 - c0);  // record 0 at ta, then the chunks c0 + 1 .. c1
    if (threadIdx.x < 4) {
        sm.mthr[threadIdx.x] = 0u;
        sm.nq[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) sm.candOver = 0;
    __syncthreads();
    const bool narrow = (unsigned long long)G * (unsigned long long)(T + 1) < (1ull << 32);
    // record r: its tile (-1: none) and record slot base
    auto rec_tile = [&](long long r, int &base) -> long long {
        base = 0;
        if (r == 0) {
            base = slotBase0;
            return ta;
        }
        const long long st = chunk_start_n(c0 + r, T, G, narrow);
        return (st > ta && st < chunk_start_n(c0 + r + 1, T, G, narrow)) ? st : -1;  // a non-empty chunk inside
    };
    auto offer = [&](int q, const ICand<P> &ic) {
        const int j = atomicAdd(&sm.nq[q], 1);
        if (j < CQ)
            sm.candq[q][j] = ic;
        else
            sm.candOver = 1;
    };
    // pass 1: records threadIdx.x + k NT (k < MREC) with their keys kept; any
    // further records (larger grids) are read again in pass 2
    unsigned mlo[4] = {0u, 0u, 0u, 0u};
    unsigned khi[MREC][4];
    long long rtile[MREC];
    int rbase[MREC];
#pragma unroll
    for (int k = 0; k < MREC; k++) {
        const long long r = threadIdx.x + (long long)k * NT;
        rtile[k] = r < nrec ? rec_tile(r, rbase[k]) : -1;
        Cand c[4];
#pragma unroll
        for (int q = 0; q < 4; q++)
            c[q] = (rtile[k] >= 0 && q < nslot) ? ldcg_cand(&p.tbest[4 * rtile[k] + rbase[k] + q]) : no_cand();
#pragma unroll
        for (int q = 0; q < 4; q++) {
            khi[k][q] = 0u;
            if (c[q].idx >= 0) {
                const ICand<P> ic = icand_of(sm, edgeOff + q, c[q]);
                mlo[q] = max(mlo[q], max(pkey(ic.lo), 1u));
                khi[k][q] = max(pkey_up(ic.hi), 1u);
            }
        }
    }
    for (long long r = threadIdx.x + (long long)MREC * NT; r < nrec; r += NT) {
        int base;
        const long long tile = rec_tile(r, base);
        if (tile < 0) continue;
        for (int q = 0; q < nslot; q++) {
            const ICand<P> ic = icand_of(sm, edgeOff + q, ldcg_cand(&p.tbest[4 * tile + base + q]));
            if (ic.c.idx >= 0) mlo[q] = max(mlo[q], max(pkey(ic.lo), 1u));
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const unsigned v = __reduce_max_sync(0xffffffffu, mlo[q]);
        if (lane == 0 && v) atomicMax(&sm.mthr[q], v);
    }
    __syncthreads();
    // pass 2: the candidates among the kept records are read again (rare)
#pragma unroll
    for (int k = 0; k < MREC; k++) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (khi[k][q] != 0u && khi[k][q] >= sm.mthr[q])
                offer(q, icand_of(sm, edgeOff + q, ldcg_cand(&p.tbest[4 * rtile[k] + rbase[k] + q])));
        }
    }
    for (long long r = threadIdx.x + (long long)MREC * NT; r < nrec; r += NT) {
        int base;
        const long long tile = rec_tile(r, base);
        if (tile < 0) continue;
        for (int q = 0; q < nslot; q++) {
            const ICand<P> ic = icand_of(sm, edgeOff + q, ldcg_cand(&p.tbest[4 * tile + base + q]));
            if (ic.c.idx >= 0 && pkey_up(ic.hi) >= sm.mthr[q]) offer(q, ic);
        }
    }
    __syncthreads();
    if (!sm.candOver) {
        if (threadIdx.x < nslot) {
            const int q = threadIdx.x, n = sm.nq[q];
            ICand<P> b = no_icand<P>();
            for (int j = 0; j < n; j++) imerge(b, sm.candq[q][j], edgeOff + q, sm, exact_c);
            sm.fin[q] = b.c;
        }
    } else {  // massive exact ties: every slot at once, each reduced by its own group of warps
        const int wps = NWARP / nslot;  // nslot is 2..4 and NWARP >= 4
        const int q = w / wps, sub = w - q * wps;
        if (q < nslot) {
            ICand<P> b = no_icand<P>();
#pragma unroll 1
            for (long long r = (long long)sub * 32 + lane; r < nrec; r += (long long)wps * 32) {
                int base;
                const long long tile = rec_tile(r, base);
                if (tile >= 0) imerge(b, icand_of(sm, edgeOff + q, ldcg_cand(&p.tbest[4 * tile + base + q])), edgeOff + q, sm, exact_c);
            }
#pragma unroll 1
            for (int d = 16; d >= 1; d >>= 1) imerge(b, shfl_icand(b, lane ^ d), edgeOff + q, sm, exact_c);
            if (lane == 0) sm.wbest[w][0] = b;
        }
        __syncthreads();
        if (threadIdx.x < nslot) {
            ICand<P> b = no_icand<P>();
            for (int k = 0; k < wps; k++) imerge(b, sm.wbest[threadIdx.x * wps + k][0], edgeOff + threadIdx.x, sm, exact_c);
            sm.fin[threadIdx.x] = b.c;
        }
    }
    __syncthreads();
    if (threadIdx.x < 4) sm.nq[threadIdx.x] = 0;
    if (threadIdx.x == 0) sm.candOver = 0;
    __syncthreads();
}

// Publish the CTA's run (record + tile count on the parent's counter); the
// publication that completes the parent's tiles merges all its runs and stores
// the children's farthest points.  kind 1: a set of the initial split; 2: a
// segment of the rounds.  Uniform over the CTA.
template <typename P>
__device__ __noinline__ void flush_run(const Params &p, int kind, long long T, int &exact_c) {
    RoundSmem<P> &sm = round_smem<P>();
    RunAcc<P> &ra = sm.run;
    const int nslot = ra.nslot;
    if (threadIdx.x == 32) {
        for (int s = 0; s < nslot; s++) stcg_cand(&p.tbest[4 * ra.first + ra.slotBase + s], ra.best[s].c);
        unsigned *cnt = kind == 1 ? &p.inst[ra.node].done0 : &p.nodes[ra.node].tdone;
        // release: this run's record; acquire: the records of the runs counted before
        const unsigned old = atom_add_acq_rel(cnt, (unsigned)ra.tiles);
        sm.fflag[0] = old + (unsigned)ra.tiles == (unsigned)ra.total;
    }
    __syncthreads();
    if (sm.fflag[0]) {
        merge_runs<P>(p, ra.ta, ra.tb, ra.slotBase0, nslot, ra.edgeOff, T, exact_c);
        if (threadIdx.x < nslot) {
            Cand *dstC = kind == 1 ? &p.inst[ra.node].chC[threadIdx.x] : &p.nodes[ra.node].chC[threadIdx.x];
            stcg_cand(dstC, sm.fin[threadIdx.x]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ra.node = -1;
    __syncthreads();
}

// Start a run of parent `node` at tile t (thread 0 sets the fields; the caller
// synchronises before they are read).
template <typename P>
__device__ __forceinline__ void run_start(RunAcc<P> &ra, int node, int nslot, long long t, int slotBase, int edgeOff,
                                          long long ta, long long tb, int slotBase0) {
    if (threadIdx.x < 4) ra.best[threadIdx.x] = no_icand<P>();
    if (threadIdx.x == 0) {
        ra.node = node;
        ra.nslot = nslot;
        ra.tiles = 0;
        ra.total = (int)(tb - ta + 1);
        ra.slotBase = slotBase;
        ra.slotBase0 = slotBase0;
        ra.edgeOff = edgeOff;
        ra.first = t;
        ra.ta = ta;
        ra.tb = tb;
    }
}

// --------------------------------------------------------------------------
// prep: classify sets (CTA 0)
// --------------------------------------------------------------------------
// Five exclusive prefix sums over the CTA in one pass (three barriers instead
// of three per sum); totals in tot.
__device__ __forceinline__ void block_excl_scan5(long long (&v)[5], long long (&tot)[5],
                                                 long long (*scr)[NWARP + 1]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc[5];
#pragma unroll
    for (int c = 0; c < 5; c++) inc[c] = warp_incl_scan(v[c]);
    if (lane == 31) {
#pragma unroll
        for (int c = 0; c < 5; c++) scr[c][w] = inc[c];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int c = 0; c < 5; c++) {
            const long long x = lane < NWARP ? scr[c][lane] : 0ll;
            const long long xi = warp_incl_scan(x);
            if (lane < NWARP) scr[c][lane] = xi - x;
            if (lane == NWARP - 1) scr[c][NWARP] = xi;
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 5; c++) {
        v[c] = scr[c][w] + inc[c] - v[c];
        tot[c] = scr[c][NWARP];
    }
    __syncthreads();
}

// The scratch of the five-way scan: the warp-best array, idle outside the tile loops.
template <typename P> __device__ __forceinline__ long long (*scan5_scratch())[NWARP + 1] {
    RoundSmem<P> &sm = round_smem<P>();
    static_assert(sizeof(sm.wbest) >= sizeof(long long[5][NWARP + 1]), "scan scratch fits the warp bests");
    return reinterpret_cast<long long(*)[NWARP + 1]>(&sm.wbest[0][0]);
}

// Points per tile of the extreme-point pass and the initial split: a single
// set small enough for the grid spreads over more CTAs with smaller tiles
// (halved down to TILE_MIN while every CTA still gets at most one); a batch
// keeps the full tile.
__device__ __forceinline__ int set_tile_points(const Params &p) {
    int ts = TILE;
    if (p.numSets == 1 && !p.offsets) {
        const long long n = p.nSingle;
        while (ts > TILE_MIN && (n + ts / 2 - 1) / (ts / 2) <= (long long)gridDim.x) ts /= 2;
    }
    return ts;
}

template <typename P> __device__ __noinline__ void prep(const Params &p) {
    long long carryBig = 0, carrySmall = 0, carryTiles = 0, bigPts = 0, smallPts = 0;
    const int ts = set_tile_points(p);
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
        const long long tiles = kind == I_BIG ? (n + ts - 1) / ts : 0;
        // big sets, small sets, tiles, big-set points, small-set points: one five-way scan
        long long v[5] = {kind == I_BIG ? 1 : 0, kind == I_SMALL ? 1 : 0, tiles, kind == I_BIG ? n : 0,
                          kind == I_SMALL ? n : 0};
        long long tot[5];
        block_excl_scan5(v, tot, scan5_scratch<P>());
        const long long xb = v[0], xs = v[1], xt = v[2];
        const long long tb = tot[0], tsm = tot[1], tt = tot[2];
        bigPts += tot[3];
        smallPts += tot[4];
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
        carrySmall += tsm;
        carryTiles += tt;
    }
    if (threadIdx.x == 0) {
        p.bigTilePrefix[carryBig] = carryTiles;
        if (carryTiles > p.maxTiles) set_err(p.ctl, E_CAPACITY);
        p.ctl->nBig = (int)carryBig;
        p.ctl->nSmallInst = (int)carrySmall;
        p.ctl->setTile = ts;
        p.ctl->bigTiles = carryTiles;
        p.ctl->bigPoints = bigPts;
        p.ctl->smallPoints = smallPts;
        p.ctl->S = 0;
        p.ctl->L = 0;
        p.ctl->tiles = 0;
        p.ctl->nNodes = 0;
        p.ctl->nLevels = 0;
        p.ctl->nSmall = 0;
        p.ctl->nPack = 0;
        p.ctl->packW = 0;
    }
}

// --------------------------------------------------------------------------
// tile descriptors: resolved in batches, one thread per tile, so the lookups
// (binary searches, segment records) of DB tiles overlap; thread 0 then only
// copies a descriptor and starts its TMA copies.
// --------------------------------------------------------------------------
__device__ void resolve_set_tile(const Params &p, TileRec &R, long long t, bool withPoly, const SetCache &sc,
                                 int ts) {
    R.t = t;
    R.np = 1;
    R.valid = 1;
    R.srcBuf = 0;
    R.K = 0;
    R.iB = 1;
    if (sc.valid && t >= sc.tile0 && t < sc.tile0 + sc.tiles) {  // the cached set: no lookups
        R.inst = sc.inst;
        R.setOff = sc.setOff;
        R.setN = sc.setN;
        R.tile0 = sc.tile0;
        R.tiles = sc.tiles;
        if (withPoly) {
            R.K = sc.K;
            R.iB = sc.iB;
            for (int k = 0; k < 4; k++) R.poly[k] = sc.poly[k];
        }
    } else {
        const int nBig = __ldcg(&p.ctl->nBig);
        const long long j = upper_bound_ll(p.bigTilePrefix, nBig + 1, t) - 1;
        const int i = __ldcg(&p.bigInst[j]);
        const Inst *I = &p.inst[i];
        R.inst = i;
        R.setOff = __ldcg(&I->off);
        R.setN = __ldcg(&I->n);
        R.tile0 = __ldcg(&I->tile0);
        R.tiles = __ldcg(&I->tiles);
        if (withPoly) {
            R.K = __ldcg(&I->K);
            R.iB = __ldcg(&I->iB);
            for (int k = 0; k < 4; k++) R.poly[k] = ldcg_cand(&I->poly[k]);
        }
    }
    R.lt = t - R.tile0;
    const long long first = R.lt * ts;
    const int c = (int)min((long long)ts, R.setN - first);
    R.nItems = c;
    int sx = 0, si = 0;
    unsigned bytes = 0u;
    part_geo(R.g[0], R.setOff + first, c, 0, false, sx, si, bytes, (int)((reinterpret_cast<uintptr_t>(p.pts) >> 3) & 1),
             0);
    if (withPoly && R.K == 0) bytes = 0u;  // no segments: the tile is skipped
    R.bytes = bytes;
}

__device__ void resolve_round_tile(const Params &p, TileRec &R, long long t, int S, long long L, int cur, int src,
                                   int ts) {
    const long long v0 = t * ts, v1 = min(v0 + (long long)ts, L);
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
    {  // no second part unless set below: an empty one at the stage start
        PartGeo &g1 = R.g[1];
        g1.q0 = g1.a0 = g1.b0 = 0;
        g1.c = g1.na = g1.nb = g1.sx = g1.si = g1.dx = g1.di = 0;
        g1.vofs = TILE;
    }
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
__device__ void issue_desc(const Params &p, int s, const TileRec &R, bool set) {
    RoundSmem<P> &sm = round_smem<P>();
    mbar_expect_tx(&sm.mbar[s], R.bytes);
    if (R.bytes == 0u) return;
    const unsigned long long pol = l2_evict_first();
    if (set) {
        const PartGeo &g = R.g[0];
        bulk_g2s(&sm.stage[s].xy[g.sx], p.pts + g.a0, (unsigned)g.na * 8u, &sm.mbar[s], pol);
        return;
    }
    const float2 *gxy = p.xy[R.srcBuf];
    const int *gid = p.id[R.srcBuf];
    for (int part = 0; part < R.np; part++) {
        const PartGeo &g = R.g[part];
        if (g.na > 0) bulk_g2s(&sm.stage[s].xy[g.sx], gxy + g.a0, (unsigned)g.na * 8u, &sm.mbar[s], pol);
        if (g.nb > 0) bulk_g2s(&sm.stage[s].id[g.si], gid + g.b0, (unsigned)g.nb * 4u, &sm.mbar[s], pol);
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
    int ts;    // round tiles: points per tile
    long long L;
};
template <typename P> __device__ void resolve_batch(const Params &p, const TileSeq &q, long long k0) {
    RoundSmem<P> &sm = round_smem<P>();
    __syncthreads();
    const long long j = threadIdx.x;
    if (j < DB && k0 + j < q.cnt) {
        const long long t = q.first + (k0 + j) * q.step;
        if (q.kind == 2)
            resolve_round_tile(p, desc_of(sm, k0 + j), t, q.S, q.L, q.cur, q.src, q.ts);
        else
            resolve_set_tile(p, desc_of(sm, k0 + j), t, q.kind == 1, sm.setc, q.ts);
    }
    __syncthreads();
    if (q.kind != 2 && threadIdx.x == 0) {  // cache the set of the batch's last tile
        const long long last = min(q.cnt, k0 + DB) - 1;
        if (last >= k0) {
            const TileRec &R = desc_of(sm, last);
            SetCache &c = sm.setc;
            c.tile0 = R.tile0;
            c.setOff = R.setOff;
            c.setN = R.setN;
            c.tiles = R.tiles;
            c.inst = R.inst;
            c.K = R.K;
            c.iB = R.iB;
            for (int k = 0; k < 4; k++) c.poly[k] = R.poly[k];
            c.valid = 1;
        }
    }
}

// Start the pipeline: first batch of descriptors, then the first NS tiles.
// The global data a phase copies with TMA was written by ordinary stores of
// earlier phases (ordered by the grid barrier); one proxy fence per phase by
// the issuing thread orders them before the async copies.  Stage reuse needs
// none: the CTA barrier after the consumers' reads precedes every refill.
template <typename P>
__device__ void pipe_start(const Params &p, const TileSeq &q, unsigned long long &gI) {
    RoundSmem<P> &sm = round_smem<P>();
    if (q.cnt <= 0) return;
    if (threadIdx.x == 0) {
        fence_proxy_async();
        sm.setc.valid = 0;  // sets change between phases (the polygon appears after the extreme points)
    }
    resolve_batch<P>(p, q, 0);
    for (long long j = 0; j < min(q.cnt, (long long)NS); j++) {
        if (threadIdx.x == 0) issue_desc<P>(p, (int)(gI % NS), desc_of(sm, j), q.kind != 2);
        gI++;
    }
}

// After tile k's points are in registers (and a barrier): refill its stage with tile k + NS.
template <typename P>
__device__ void pipe_refill(const Params &p, const TileSeq &q, long long k, int s,
                            unsigned long long &gI) {
    RoundSmem<P> &sm = round_smem<P>();
    const long long nk = k + NS;
    if (nk >= q.cnt) return;
    if (nk % DB == 0) resolve_batch<P>(p, q, nk);
    if (threadIdx.x == 0) issue_desc<P>(p, s, desc_of(sm, nk), q.kind != 2);
    gI++;
}


// Wait for every copy still in flight (used on the error path before leaving).
template <typename P>
__device__ void pipe_drain(const Params &p, unsigned long long gI, unsigned long long gC) {
    RoundSmem<P> &sm = round_smem<P>();
    for (unsigned long long q = gC; q < gI; q++) {
        unsigned it = 0;
        while (!mbar_try_wait(&sm.mbar[q % NS], (unsigned)((q / NS) & 1ull)))
            if (++it > SPIN_LIMIT) break;
    }
}

// --------------------------------------------------------------------------
// extremes (Sec. 4.2)
// --------------------------------------------------------------------------

// Reduce this CTA's running extremes of set i, store them as the partial of
// the CTA's first tile of that set, and let the CTA that completes the set's
// tiles merge all partials into the initial polygon.
template <typename P>
__device__ __noinline__ void ext_flush(const Params &p, Ext e, int i, long long segFirst, int segTiles) {
    RoundSmem<P> &sm = round_smem<P>();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    e = warp_ext_reduce(e);
    __syncthreads();
    if (lane == 0) sm.wext[w] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext r = sm.wext[0];
        for (int k = 1; k < NWARP; k++) ext_merge(r, sm.wext[k]);
        st_ext(&p.text[segFirst], r);
        // release: this CTA's partial; acquire: the partials counted before
        const unsigned prev = atom_add_acq_rel(&p.inst[i].done, (unsigned)segTiles);
        sm.kflag = (prev + (unsigned)segTiles == (unsigned)__ldcg(&p.inst[i].tiles));
    }
    __syncthreads();
    if (!sm.kflag) {
        return;
    }
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
        int K = 0, iB = 1;
        Cand poly[4];
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
        }
        W.kind = kind;
        W.K = K;
        W.iB = iB;
        for (int k = 0; k < 4; k++) W.poly[k] = (k < K || (kind == I_DEGEN && k == 0)) ? poly[k] : no_cand();
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// two-pass tile engine (initial split and grid-wide rounds)
// --------------------------------------------------------------------------
// Thread t owns items j * NT + t (j < IPT) of the tile, all read from the TMA
// stage.  Pass 1 classifies them, keeps their slots packed in two registers
// (4 bits per item), counts the points of every slot per thread (8-bit
// fields) and keeps, per slot, the largest lower distance bound.  One
// reservation per (tile, slot) on the child's cursor then gives every warp its
// output range; while its round trip is in flight the items whose upper bound
// reaches their slot's largest lower bound are offered as farthest-point
// candidates.  Pass 2 writes the survivors (ranks from warp ballots, so stores
// are coalesced) while one thread per slot resolves the slot's candidates.

// Record the slot c (CLS_NONE: discarded) of item j with the keys of its
// distance bounds.
__device__ __forceinline__ void note_item(int j, int c, unsigned klo, unsigned khi, unsigned &cp0, unsigned &cp1,
                                          unsigned &cnt, unsigned (&mlo)[4], unsigned &mhi) {
    const unsigned v = (unsigned)c << (4 * (j & 7));
    cp0 |= j < 8 ? v : 0u;
    cp1 |= j < 8 ? 0u : v;
    cnt += c < 4 ? 1u << (8 * c) : 0u;
#pragma unroll
    for (int q = 0; q < 4; q++) mlo[q] = c == q ? max(mlo[q], klo) : mlo[q];
    mhi = c < 4 ? max(mhi, khi) : mhi;
}

// The same for an item j known only at run time whose slot was CLS_NONE.
__device__ __forceinline__ void renote_item(int j, int c, unsigned klo, unsigned khi, unsigned &cp0, unsigned &cp1,
                                            unsigned &cnt, unsigned (&mlo)[4], unsigned &mhi) {
    const unsigned sh = 4u * (unsigned)(j & 7);
    const unsigned m = ~(15u << sh) | ((unsigned)c << sh);
    if (j < 8)
        cp0 &= m;
    else
        cp1 &= m;
    if (c != CLS_NONE) {
        cnt += 1u << (8 * c);
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (c == q) mlo[q] = max(mlo[q], klo);
        mhi = max(mhi, khi);
    }
}

// Items j >= jn of every thread are outside a short tile: their slot nibbles
// read as CLS_NONE.
__device__ __forceinline__ void mark_unused_items(int jn, unsigned &cp0, unsigned &cp1) {
    if (jn >= IPT) return;
    cp0 |= jn >= 8 ? 0u : (0xffffffffu << (4 * jn));
    if (IPT > 8) cp1 |= jn <= 8 ? 0xffffffffu : (jn >= 16 ? 0u : (0xffffffffu << (4 * (jn - 8))));
}

// The item groups of a tile that hold points (the same in the whole CTA): a
// short tile's loops stop after them.
__device__ __forceinline__ int item_groups_end(int nItems) {
    return min(IPT, ((nItems + NT - 1) / NT + UNROLL_ITEMS - 1) / UNROLL_ITEMS * UNROLL_ITEMS);
}

// Bit k of the result: nibble k of w equals q (an exact zero-nibble test:
// adding 7 to the low three bits of a nibble never carries out of it).
__device__ __forceinline__ unsigned nibbles_equal(unsigned w, unsigned q) {
    const unsigned x = w ^ (0x11111111u * q);
    unsigned t = (~(((x & 0x77777777u) + 0x77777777u) | x) & 0x88888888u) >> 3;  // bit 4k
    t = (t | (t >> 3)) & 0x03030303u;
    t = (t | (t >> 6)) & 0x000f000fu;
    return (t | (t >> 12)) & 0xffu;
}

// Items (bit j < IPT) of this thread whose slot is in the set fl.  The nibbles
// of items beyond IPT are never written (zero), so they are masked off.
__device__ __forceinline__ unsigned items_in_slots(unsigned fl, unsigned cp0, unsigned cp1) {
    unsigned m = 0u;
#pragma unroll
    for (int q = 0; q < 4; q++)
        if ((fl >> q) & 1u) m |= nibbles_equal(cp0, q) | (nibbles_equal(cp1, q) << 8);
    return m & ((1u << IPT) - 1u);
}

__device__ __forceinline__ int item_cls(int j, unsigned cp0, unsigned cp1) {
    return (int)(((j < 8 ? cp0 : cp1) >> (4 * (j & 7))) & 15u);
}

// Filter decisions of one orientation: certainly strictly right / certainly left.
template <typename P> struct Side {
    bool r, l;
};
template <typename P> __device__ __forceinline__ Side<P> side_of(const Approx<P> &o) {
    Side<P> d;
    d.r = o.ok && o.det < -o.err;
    d.l = o.ok && o.det > o.err;
    return d;
}

// Classification against two candidate edges e0, e1 of which a point can be
// strictly right of at most one (the first and second child of a segment in
// the rounds; the lower- and upper-chain edge of the initial polygon in the
// split).  Filter only: the slot (CLS_NONE when right of neither) with its
// distance bounds; unsure when a decision needs the exact predicate.
template <typename P>
__device__ __forceinline__ int classify_fast(const RoundSmem<P> &sm, int e0, int e1, float px, float py, P &lo, P &hi,
                                             bool &unsure) {
    const Approx<P> oa = orient_approx(sm.edge[e0], px, py);
    const Approx<P> ob = orient_approx(sm.edge[e1], px, py);
    const Side<P> a = side_of(oa), b = side_of(ob);
    const DistIv<P> d = dist_interval(a.r ? oa : ob);
    lo = d.lo;
    hi = d.hi;
    unsure = !(a.r | b.r) & (!a.l | !b.l);
    return unsure ? CLS_NONE : (a.r ? e0 : (b.r ? e1 : CLS_NONE));
}

// The same with exact decisions (the filter's undecided cases).
template <typename P>
__device__ __noinline__ int classify_exact(int e0, int e1, float px, float py, P &lo, P &hi, int &exact_o) {
    const RoundSmem<P> &sm = round_smem<P>();
    lo = hi = P(0);
    if (right_of(sm.edge[e0], sm.vend[e0][0], sm.vend[e0][1], px, py, lo, hi, exact_o)) return e0;
    if (right_of(sm.edge[e1], sm.vend[e1][0], sm.vend[e1][1], px, py, lo, hi, exact_o)) return e1;
    return CLS_NONE;
}

// Initial split: the only edges of the CCW polygon A, [Bot,] B, [Top] a point
// can be strictly right of.  Below the chord the point is right of A->Bot only
// if x < Bot.x and of Bot->B only if x > Bot.x (Bot has the least y); above
// it, of B->Top only if x > Top.x and of Top->A only if x < Top.x (Top has the
// greatest y).  A chain without its middle vertex is the chord itself.  So the
// lower-chain candidate is edge 0 or 1 and the upper-chain candidate edge iB
// or iB + 1, chosen by exact comparisons of x; a point is right of at most one
// of the two.
__device__ __forceinline__ void split_edges(float px, bool hasBot, float botx, bool hasTop, float topx, int iB,
                                            int &e0, int &e1) {
    e0 = (hasBot & !(px < botx)) ? 1 : 0;
    e1 = (hasTop & !(px > topx)) ? iB + 1 : iB;
}

// Warp totals of pass 1 -> sm.warpCnt, sm.maxLo; the packed slots -> sm.clsPack.
template <typename P>
__device__ __forceinline__ void pass1_commit(RoundSmem<P> &sm, unsigned cp0, unsigned cp1, unsigned cnt,
                                             const unsigned (&mlo)[4]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sm.clsPack[0][threadIdx.x] = cp0;
    sm.clsPack[1][threadIdx.x] = cp1;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const unsigned wc = __reduce_add_sync(0xffffffffu, (cnt >> (8 * q)) & 0xffu);
        const unsigned v = __reduce_max_sync(0xffffffffu, mlo[q]);
        if (lane == 0) {
            sm.warpCnt[w][q] = wc;
            if (v) atomicMax(&sm.maxLo[q], v);
        }
    }
}


// Pass-2 rank of an item of slot c among its slot's points: the warp's running
// rank plus the lane rank.
__device__ __forceinline__ int slot_rank(int c, int (&wr)[4], unsigned lt) {
    int rank = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const unsigned b = __ballot_sync(0xffffffffu, c == q);
        rank = c == q ? wr[q] + __popc(b & lt) : rank;
        wr[q] += __popc(b);
    }
    return rank;
}

// Candidate for the farthest point of slot c (pass 2): the key of its upper
// bound reaches the slot's largest lower-bound key thr.
template <typename P>
__device__ __forceinline__ void offer_candidate(RoundSmem<P> &sm, int c, unsigned thr, float px, float py, int idx) {
    const DistIv<P> d = dist_interval(orient_approx(sm.edge[c], px, py));
    if (pkey_up(d.hi) >= thr) {
        const int j = atomicAdd(&sm.nq[c], 1);
        if (j < CQ) {
            ICand<P> ic;
            ic.c = mk_cand(px, py, idx);
            ic.lo = d.lo;
            ic.hi = d.hi;
            sm.candq[c][j] = ic;
        } else {
            sm.candOver = 1;
        }
    }
}

// Slots in which this thread may hold an item whose upper-bound key reaches the
// slot's threshold (bit q for slot q): it holds items of the slot and the
// largest upper-bound key over all its items reaches the threshold (a superset).
__device__ __forceinline__ unsigned candidate_slots(unsigned mhi, unsigned cnt, const unsigned (&thr)[4]) {
    unsigned f = 0u;
#pragma unroll
    for (int q = 0; q < 4; q++) f |= (unsigned)((((cnt >> (8 * q)) & 0xffu) != 0u) & (mhi >= thr[q])) << q;
    return f;
}

template <typename T> __device__ __forceinline__ T sel4(int c, const T (&v)[4]) {
    T r = v[0];
    if (c == 1) r = v[1];
    if (c == 2) r = v[2];
    if (c == 3) r = v[3];
    return r;
}

// Exact best of every slot over all items of the tile -> sm.best (whole CTA).
template <typename P, typename Fetch>
__device__ __noinline__ void resolve_tile_exhaustive(RoundSmem<P> &sm, int nslot, int nItems, Fetch fetch,
                                                     int &exact_c) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    ICand<P> b[4] = {no_icand<P>(), no_icand<P>(), no_icand<P>(), no_icand<P>()};
    for (int i = threadIdx.x; i < nItems; i += NT) {
        const int j = i / NT;
        const int c = (int)((sm.clsPack[j >> 3][threadIdx.x] >> (4 * (j & 7))) & 15u);
        if (c == CLS_NONE) continue;
        float px, py;
        int idx;
        fetch(i, px, py, idx);
        imerge(b[c], icand_of(sm, c, mk_cand(px, py, idx)), c, sm, exact_c);
    }
    for (int q = 0; q < nslot; q++) {
        for (int d = 16; d >= 1; d >>= 1) imerge(b[q], shfl_icand(b[q], lane ^ d), q, sm, exact_c);
        if (lane == 0) sm.wbest[w][q] = b[q];
    }
    __syncthreads();
    if (threadIdx.x < nslot) {
        ICand<P> r = no_icand<P>();
        for (int k = 0; k < NWARP; k++) imerge(r, sm.wbest[k][threadIdx.x], threadIdx.x, sm, exact_c);
        sm.best[threadIdx.x] = r;
    }
}

// Threads q < 4 after the barrier that follows pass1_commit: the warp offsets
// of slot q and the tile's reservation on the child's cursor.  The returned
// base is used only after the candidate pass, so the atomic's round trip
// overlaps it; the caller stores it to sm.base[q] before the next barrier.
template <typename P> __device__ __forceinline__ int tile_reserve_issue(RoundSmem<P> &sm, int nslot,
                                                                        int *const (&cursor)[4]) {
    const int q = threadIdx.x;
    int run = 0;
    if (q < nslot) {
        for (int w = 0; w < NWARP; w++) {
            sm.warpOff[w][q] = run;
            run += (int)sm.warpCnt[w][q];
        }
    }
    sm.tot[q] = run;
    return run ? atomicAdd(cursor[q], run) : 0;
}

// Exact best candidate per slot -> sm.best[q], written by thread q (q < nslot),
// which may use it without a further barrier.  The candidate lists are complete
// (offered before a barrier the caller has passed), so there is no barrier
// here: threads q < nslot resolve while the others write their survivors.
// Usually a slot has one candidate; overflowing lists (massive exact ties) fall
// back to a full exact reduction over the tile (the whole CTA).
template <typename P, typename Fetch>
__device__ __forceinline__ void resolve_candidates_ready(RoundSmem<P> &sm, int nslot, int nItems, Fetch &&fetch,
                                                         int &exact_c) {
    if (!sm.candOver) {
        if (threadIdx.x < nslot) {
            const int q = threadIdx.x, n = sm.nq[q];
            ICand<P> b = n ? sm.candq[q][0] : no_icand<P>();
            for (int j = 1; j < n; j++) imerge(b, sm.candq[q][j], q, sm, exact_c);
            sm.best[q] = b;
        }
    } else {
        resolve_tile_exhaustive(sm, nslot, nItems, fetch, exact_c);
    }
}

// The per-tile lists, thresholds and overflow flag: reset after the barrier
// that starts a tile (every read of the previous tile's values precedes it).
template <typename P> __device__ __forceinline__ void tile_reset(RoundSmem<P> &sm) {
    if (threadIdx.x < 4) {
        sm.maxLo[threadIdx.x] = 0u;
        sm.nq[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) sm.candOver = 0;
}

template <typename P> __device__ __forceinline__ void tile_extremes_reset(RoundSmem<P> &sm) {
    if (threadIdx.x == 0) {
        sm.tk[0] = sm.tk[2] = 0xffffffffu;
        sm.tk[1] = sm.tk[3] = 0u;
    }
}

// --------------------------------------------------------------------------
// extremes (Sec. 4.2)
// --------------------------------------------------------------------------
// Coordinate extremes of the thread's items of a tile; a full tile needs no
// per-item bound test.
template <bool FULL>
__device__ __forceinline__ void ext_pass_a(const float2 *xs, int dx, int nItems, float &mnx, float &mxx, float &mny,
                                           float &mxy, bool &nan) {
#pragma unroll 4
    for (int j = 0; j < IPT; j++) {
        const int i = j * NT + threadIdx.x;
        if (FULL || i < nItems) {
            const float2 v = xs[i + dx];
            mnx = fminf(mnx, v.x);
            mxx = fmaxf(mxx, v.x);
            mny = fminf(mny, v.y);
            mxy = fmaxf(mxy, v.y);
            nan |= (v.x != v.x) | (v.y != v.y);
        }
    }
}

template <typename P>
__device__ __noinline__ bool phase_extremes(const Params &p, unsigned long long &gI,
                                            unsigned long long &gC) {
    RoundSmem<P> &sm = round_smem<P>();
    const long long T = __ldcg(&p.ctl->bigTiles), G = gridDim.x;
    const long long cb = (long long)blockIdx.x * T / G, ce = ((long long)blockIdx.x + 1) * T / G;
    const long long cnt = ce - cb;
    TileSeq q;
    q.first = cb;
    q.step = 1;
    q.cnt = cnt;
    q.kind = 0;
    q.S = q.cur = q.src = 0;
    q.ts = __ldcg(&p.ctl->setTile);
    q.L = 0;
    tile_extremes_reset(sm);
    pipe_start<P>(p, q, gI);
    Ext acc = ext_empty();
    int accInst = -1, segTiles = 0;
    long long segFirst = 0;
    for (long long k = 0; k < cnt; k++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain<P>(p, gI, gC);
            return false;
        }
        const TileRec &R = desc_of(sm, k);
        const int inst = R.inst;
        if (inst != accInst) {
            if (accInst >= 0) ext_flush<P>(p, acc, accInst, segFirst, segTiles);
            acc = ext_empty();
            accInst = inst;
            segFirst = R.t;
            segTiles = 0;
        }
        const int nItems = R.nItems, dx = R.g[0].dx;
        const int base = (int)(R.lt * q.ts);
        const float2 *xs = sm.stage[s].xy;
        // pass A: the tile's coordinate extremes (fminf/fmaxf skip NaN, flagged apart)
        float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
        bool nan = false;
        if (nItems == TILE)
            ext_pass_a<true>(xs, dx, nItems, mnx, mxx, mny, mxy, nan);
        else
            ext_pass_a<false>(xs, dx, nItems, mnx, mxx, mny, mxy, nan);
        if (nan) acc.nonfinite = 1;
        {
            const unsigned k0 = __reduce_min_sync(0xffffffffu, fkey(mnx));
            const unsigned k1 = __reduce_max_sync(0xffffffffu, fkey(mxx));
            const unsigned k2 = __reduce_min_sync(0xffffffffu, fkey(mny));
            const unsigned k3 = __reduce_max_sync(0xffffffffu, fkey(mxy));
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&sm.tk[0], k0);
                atomicMax(&sm.tk[1], k1);
                atomicMin(&sm.tk[2], k2);
                atomicMax(&sm.tk[3], k3);
            }
        }
        __syncthreads();
        const float t0 = fkey_inv(sm.tk[0]), t1 = fkey_inv(sm.tk[1]), t2 = fkey_inv(sm.tk[2]),
                    t3 = fkey_inv(sm.tk[3]);
        if (!(fabsf(t0) <= FLT_MAX && fabsf(t1) <= FLT_MAX && fabsf(t2) <= FLT_MAX && fabsf(t3) <= FLT_MAX))
            acc.nonfinite = 1;
        // pass B: only points on a tile extreme can be a set extreme.  Hits are
        // taken in increasing index order, so strict comparisons keep the lowest
        // index among equal coordinates.
        unsigned hm = 0u;
#pragma unroll UNROLL_ITEMS
        for (int j = 0; j < IPT; j++) {
            const int i = j * NT + threadIdx.x;
            const float2 v = xs[i + dx];  // inside the stage for every j
            const bool hit = (v.x == t0) | (v.x == t1) | (v.y == t2) | (v.y == t3);
            hm |= (unsigned)(hit & (i < nItems)) << j;
        }
        while (hm) {
            const int j = __ffs(hm) - 1;
            hm &= hm - 1u;
            const int i = j * NT + threadIdx.x;
            const float2 v = xs[i + dx];
            const int id = base + i;
            if (acc.a.idx < 0 || v.x < acc.a.x || (v.x == acc.a.x && v.y < acc.a.y)) acc.a = mk_cand(v.x, v.y, id);
            if (acc.b.idx < 0 || v.x > acc.b.x || (v.x == acc.b.x && v.y > acc.b.y)) acc.b = mk_cand(v.x, v.y, id);
            if (acc.bot.idx < 0 || v.y < acc.bot.y || (v.y == acc.bot.y && v.x < acc.bot.x))
                acc.bot = mk_cand(v.x, v.y, id);
            if (acc.top.idx < 0 || v.y > acc.top.y || (v.y == acc.top.y && v.x > acc.top.x))
                acc.top = mk_cand(v.x, v.y, id);
        }
        segTiles++;
        __syncthreads();
        tile_extremes_reset(sm);
        pipe_refill<P>(p, q, k, s, gI);
    }
    if (accInst >= 0) ext_flush<P>(p, acc, accInst, segFirst, segTiles);
    return true;
}

// --------------------------------------------------------------------------
// round 0: the initial split
// --------------------------------------------------------------------------
template <typename P>
__device__ __noinline__ bool phase_round0(const Params &p, unsigned long long &gI,
                                          unsigned long long &gC, int &exact_o, int &exact_c, long long &survivors) {
    RoundSmem<P> &sm = round_smem<P>();
    const long long T = __ldcg(&p.ctl->bigTiles), G = gridDim.x;
    const long long first = chunk_start(blockIdx.x, T, G);
    const long long cnt = chunk_start(blockIdx.x + 1, T, G) - first;
    TileSeq q;
    q.first = first;
    q.step = 1;
    q.cnt = cnt;
    q.kind = 1;
    q.S = q.cur = q.src = 0;
    q.ts = __ldcg(&p.ctl->setTile);
    q.L = 0;
    tile_reset(sm);
    pipe_start<P>(p, q, gI);
    const unsigned lt = lanemask_lt();
    const int w = threadIdx.x >> 5;
    for (long long kt = 0; kt < cnt; kt++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain<P>(p, gI, gC);
            return false;
        }
        tile_reset(sm);
        const TileRec &R = desc_of(sm, kt);
        const int K = R.K, nItems = R.nItems;
        if (K == 0) {  // degenerate or rejected set: no segments
            __syncthreads();
            pipe_refill<P>(p, q, kt, s, gI);
            continue;
        }
        if (sm.run.node >= 0 && sm.run.node != R.inst) flush_run<P>(p, 1, T, exact_c);  // the previous set's run
        if (sm.run.node < 0) run_start(sm.run, R.inst, K, R.t, 0, 0, R.tile0, R.tile0 + R.tiles - 1, 0);
        if (threadIdx.x < K) {
            const Cand u = R.poly[threadIdx.x], v = R.poly[(threadIdx.x + 1) % K];
            sm.edge[threadIdx.x] = make_edge<P>(u.x, u.y, v.x, v.y);
            sm.vend[threadIdx.x][0] = v.x;
            sm.vend[threadIdx.x][1] = v.y;
        }
        __syncthreads();
        // pass 1: each point against its lower- and upper-chain candidate edge
        const int iB = R.iB, dx = R.g[0].dx;
        const bool hasBot = iB == 2, hasTop = K - iB == 2;
        const float botx = R.poly[1].x, topx = R.poly[(iB + 1) & 3].x;
        const float2 *xs = sm.stage[s].xy;
        const int jn = item_groups_end(nItems);
        unsigned cp0 = 0u, cp1 = 0u, pc = 0u, um = 0u;
        unsigned mlo[4] = {0u, 0u, 0u, 0u}, mhi = 0u;
#pragma unroll UNROLL_ITEMS
        for (int j = 0; j < IPT; j++) {
            if (j % UNROLL_ITEMS == 0 && j >= jn) break;
            const int i = j * NT + threadIdx.x;
            const bool in = i < nItems;
            const float2 v = xs[i + dx];  // inside the stage for every j; masked below
            int e0, e1;
            split_edges(v.x, hasBot, botx, hasTop, topx, iB, e0, e1);
            P lo, hi;
            bool unsure;
            int c = classify_fast(sm, e0, e1, v.x, v.y, lo, hi, unsure);
            c = in ? c : CLS_NONE;
            um |= (unsigned)(unsure & in) << j;
            note_item(j, c, max(pkey(lo), 1u), max(pkey_up(hi), 1u), cp0, cp1, pc, mlo, mhi);
        }
        while (um) {  // decisions the filter could not certify
            const int j = __ffs(um) - 1;
            um &= um - 1u;
            const float2 v = xs[j * NT + threadIdx.x + dx];
            int e0, e1;
            split_edges(v.x, hasBot, botx, hasTop, topx, iB, e0, e1);
            P lo, hi;
            const int c = classify_exact<P>(e0, e1, v.x, v.y, lo, hi, exact_o);
            renote_item(j, c, max(pkey(lo), 1u), max(pkey_up(hi), 1u), cp0, cp1, pc, mlo, mhi);
        }
        mark_unused_items(jn, cp0, cp1);
        pass1_commit(sm, cp0, cp1, pc, mlo);
        Inst *W = &p.inst[R.inst];
        int *const cursors[4] = {&W->chCount[0], &W->chCount[1], &W->chCount[2], &W->chCount[3]};
        const int idBase = (int)(R.lt * q.ts);
        // reservation in flight while the farthest-point candidates are offered
        __syncthreads();
        unsigned thr[4];
#pragma unroll
        for (int qq = 0; qq < 4; qq++) thr[qq] = sm.maxLo[qq];
        const int resv = threadIdx.x < 4 ? tile_reserve_issue(sm, K, cursors) : 0;
        if (const unsigned fl = candidate_slots(mhi, pc, thr)) {
            for (unsigned m = items_in_slots(fl, cp0, cp1); m; m &= m - 1u) {
                const int j = __ffs(m) - 1;
                const int c = item_cls(j, cp0, cp1);
                const int i = j * NT + threadIdx.x;
                const float2 v = xs[i + dx];
                offer_candidate(sm, c, sel4(c, thr), v.x, v.y, idBase + i);
            }
        }
        if (threadIdx.x < 4) sm.base[threadIdx.x] = resv;
        __syncthreads();
        // pass 2: write the survivors (threads q < K then resolve slot q's candidates)
        const long long off = R.setOff, n = R.setN;
        int wr[4];
#pragma unroll
        for (int qq = 0; qq < 4; qq++) wr[qq] = sm.base[qq] + sm.warpOff[w][qq];
        float2 *oxy = p.xy[0];
        int *oid = p.id[0];
        bool bad = false;
#pragma unroll UNROLL_ITEMS
        for (int j = 0; j < IPT; j++) {
            if (j % UNROLL_ITEMS == 0 && j >= jn) break;
            const int i = j * NT + threadIdx.x;
            const int c = item_cls(j, cp0, cp1);
            const int rank = slot_rank(c, wr, lt);
            const float2 v = xs[i + dx];
            const long long b = (c < 2 ? 0ll : p.ncap) + off;
            const long long pos = (c & 1) ? b + n - 1 - rank : b + rank;
            const bool live = c != CLS_NONE;
            bad |= live & (rank >= n);  // guard: never write outside the set's range
            if (live & (rank < n)) {
                __stcg(&oxy[pos], v);
                __stcg(&oid[pos], idBase + i);
            }
        }
        if (bad) set_err(p.ctl, E_INTERNAL);
        auto fetch = [&](int i, float &px, float &py, int &idx) {
            const float2 v = xs[i + dx];
            px = v.x;
            py = v.y;
            idx = idBase + i;
        };
        resolve_candidates_ready(sm, K, nItems, fetch, exact_c);
        if (threadIdx.x < K) imerge(sm.run.best[threadIdx.x], sm.best[threadIdx.x], threadIdx.x, sm, exact_c);
        if (threadIdx.x == 0) {
            sm.run.tiles++;
            survivors += (long long)sm.tot[0] + sm.tot[1] + sm.tot[2] + sm.tot[3];
        }
        __syncthreads();  // every read of this tile's stage precedes its refill
        pipe_refill<P>(p, q, kt, s, gI);
    }
    __syncthreads();
    if (sm.run.node >= 0) flush_run<P>(p, 1, T, exact_c);
    return true;
}

// --------------------------------------------------------------------------
// round r >= 1
// --------------------------------------------------------------------------
// Points per tile of a grid round over L live points: the full tile, halved
// (down to TILE_MIN) while every CTA still gets at most one tile, so a short
// round spreads over more CTAs and each one's tile ends sooner.  Segments of a
// round hold more than cut >= TILE points, so a smaller tile still meets at
// most two of them.
__device__ __forceinline__ int round_tile_points(long long L, long long G) {
    int ts = TILE;
    while (ts > TILE_MIN && (L + ts / 2 - 1) / (ts / 2) <= G) ts /= 2;
    return ts;
}

template <typename P>
__device__ __noinline__ bool phase_round(const Params &p, unsigned long long &gI,
                                         unsigned long long &gC, int r, int S, long long L, int cur, int &exact_o,
                                         int &exact_c, long long &survivors) {
    RoundSmem<P> &sm = round_smem<P>();
    const int src = (r - 1) & 1, dst = r & 1;
    const long long G = gridDim.x;
    const int ts = round_tile_points(L, G);
    const long long T = (L + ts - 1) / ts;
    const long long first = chunk_start(blockIdx.x, T, G);
    const long long cnt = chunk_start(blockIdx.x + 1, T, G) - first;
    TileSeq q;
    q.first = first;
    q.step = 1;
    q.cnt = cnt;
    q.kind = 2;
    q.S = S;
    q.cur = cur;
    q.src = src;
    q.ts = ts;
    q.L = L;
    tile_reset(sm);
    pipe_start<P>(p, q, gI);
    const unsigned lt = lanemask_lt();
    const int w = threadIdx.x >> 5;
    for (long long kt = 0; kt < cnt; kt++) {
        const int s = (int)(gC % NS);
        const unsigned par = (unsigned)((gC / NS) & 1ull);
        gC++;
        if (!__syncthreads_and(pipe_wait(p, sm, s, par))) {
            pipe_drain<P>(p, gI, gC);
            return false;
        }
        tile_reset(sm);
        const TileRec &R = desc_of(sm, kt);
        const int valid = R.valid, np = R.np, nItems = R.nItems;
        if (!valid) {
            __syncthreads();
            pipe_refill<P>(p, q, kt, s, gI);
            continue;
        }
        if (sm.run.node >= 0 && sm.run.node != R.node[0]) flush_run<P>(p, 2, T, exact_c);  // the previous segment
        if (sm.run.node < 0) {
            const long long vs = R.vstart[0], cn = R.count[0];
            run_start(sm.run, R.node[0], 2, R.t, 0, 0, vs / ts, (vs + cn - 1) / ts, (vs % ts) != 0 ? 2 : 0);
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
        const int vB = np == 2 ? R.g[1].vofs : TILE;
        const int dx0 = R.g[0].dx, dx1 = R.g[1].dx, di0 = R.g[0].di, di1 = R.g[1].di;
        const float2 *xs = sm.stage[s].xy;
        const int *is = sm.stage[s].id;
        // pass 1: strictly right of h->c (first child) or of c->e (second child).
        // A short tile stops after the groups of items that hold points (jn is
        // the same in the whole CTA).
        const int jn = item_groups_end(nItems);
        unsigned cp0 = 0u, cp1 = 0u, pc = 0u, um = 0u;
        unsigned mlo[4] = {0u, 0u, 0u, 0u}, mhi = 0u;
#pragma unroll UNROLL_ITEMS
        for (int j = 0; j < IPT; j++) {
            if (j % UNROLL_ITEMS == 0 && j >= jn) break;
            const int i = j * NT + threadIdx.x;
            const bool in = i < nItems;
            const bool pb = i >= vB;
            const float2 v = xs[i + (pb ? dx1 : dx0)];  // inside the stage for every j; masked below
            P lo, hi;
            bool unsure;
            const int s0 = pb ? 2 : 0;
            int c = classify_fast(sm, s0, s0 + 1, v.x, v.y, lo, hi, unsure);
            c = in ? c : CLS_NONE;
            um |= (unsigned)(unsure & in) << j;
            note_item(j, c, max(pkey(lo), 1u), max(pkey_up(hi), 1u), cp0, cp1, pc, mlo, mhi);
        }
        while (um) {  // decisions the filter could not certify
            const int j = __ffs(um) - 1;
            um &= um - 1u;
            const int i = j * NT + threadIdx.x;
            const bool pb = i >= vB;
            const float2 v = xs[i + (pb ? dx1 : dx0)];
            P lo, hi;
            const int s0 = pb ? 2 : 0;
            const int c = classify_exact<P>(s0, s0 + 1, v.x, v.y, lo, hi, exact_o);
            renote_item(j, c, max(pkey(lo), 1u), max(pkey_up(hi), 1u), cp0, cp1, pc, mlo, mhi);
        }
        mark_unused_items(jn, cp0, cp1);
        pass1_commit(sm, cp0, cp1, pc, mlo);
        Node *NA = &p.nodes[R.node[0]];
        Node *NB = &p.nodes[R.node[np == 2 ? 1 : 0]];
        int *const cursors[4] = {&NA->chCount[0], &NA->chCount[1], &NB->chCount[0], &NB->chCount[1]};
        // reservation in flight while the farthest-point candidates are offered
        __syncthreads();
        unsigned thr[4];
#pragma unroll
        for (int qq = 0; qq < 4; qq++) thr[qq] = sm.maxLo[qq];
        const int resv = threadIdx.x < 4 ? tile_reserve_issue(sm, 2 * np, cursors) : 0;
        if (const unsigned fl = candidate_slots(mhi, pc, thr)) {
            for (unsigned m = items_in_slots(fl, cp0, cp1); m; m &= m - 1u) {
                const int j = __ffs(m) - 1;
                const int c = item_cls(j, cp0, cp1);
                const int i = j * NT + threadIdx.x;
                const bool pb = (c == 2) | (c == 3);
                const float2 v = xs[i + (pb ? dx1 : dx0)];
                offer_candidate(sm, c, sel4(c, thr), v.x, v.y, is[i + (pb ? di1 : di0)]);
            }
        }
        if (threadIdx.x < 4) sm.base[threadIdx.x] = resv;
        __syncthreads();
        // pass 2: write the survivors (threads q < 2 np then resolve slot q's candidates)
        const long long ps0 = R.pstart[0], ps1 = R.pstart[1];
        const int cn0 = R.count[0], cn1 = R.count[1];
        int wr[4];
#pragma unroll
        for (int qq = 0; qq < 4; qq++) wr[qq] = sm.base[qq] + sm.warpOff[w][qq];
        float2 *oxy = p.xy[dst];
        int *oid = p.id[dst];
        const long long lim = 2 * p.ncap;
        bool bad = false;
#pragma unroll UNROLL_ITEMS
        for (int j = 0; j < IPT; j++) {
            if (j % UNROLL_ITEMS == 0 && j >= jn) break;
            const int i = j * NT + threadIdx.x;
            const int c = item_cls(j, cp0, cp1);
            const int rank = slot_rank(c, wr, lt);
            const bool pb = (c == 2) | (c == 3);  // second part (never for a discarded item)
            const float2 v = xs[i + (pb ? dx1 : dx0)];
            const int idx = is[i + (pb ? di1 : di0)];
            const long long ps = pb ? ps1 : ps0;
            const int cn = pb ? cn1 : cn0;
            const long long pos = (c & 1) ? ps + cn - 1 - rank : ps + rank;
            const bool live = c != CLS_NONE;
            const bool okp = (rank < cn) & (pos < lim);
            bad |= live & !okp;  // guard: a child never leaves its parent's range
            if (live & okp) {
                __stcg(&oxy[pos], v);
                __stcg(&oid[pos], idx);
            }
        }
        if (bad) set_err(p.ctl, E_INTERNAL);
        auto fetch = [&](int i, float &px, float &py, int &idx) {
            const bool pb = i >= vB;
            const float2 v = xs[i + (pb ? dx1 : dx0)];
            px = v.x;
            py = v.y;
            idx = is[i + (pb ? di1 : di0)];
        };
        resolve_candidates_ready(sm, 2 * np, nItems, fetch, exact_c);
        if (threadIdx.x < 2) imerge(sm.run.best[threadIdx.x], sm.best[threadIdx.x], threadIdx.x, sm, exact_c);
        if (threadIdx.x == 0) {
            sm.run.tiles++;
            sm.run.edgeOff = 0;
            survivors += (long long)sm.tot[0] + sm.tot[1] + sm.tot[2] + sm.tot[3];
        }
        if (np == 2) {  // the first segment ends in this tile; the second starts here
            __syncthreads();
            flush_run<P>(p, 2, T, exact_c);
            const long long vs = R.vstart[1], cn = R.count[1];
            run_start(sm.run, R.node[1], 2, R.t, 2, 2, vs / ts, (vs + cn - 1) / ts, 2);
            __syncthreads();
            if (threadIdx.x < 2) sm.run.best[threadIdx.x] = sm.best[2 + threadIdx.x];
            if (threadIdx.x == 0) sm.run.tiles = 1;
        }
        __syncthreads();  // every read of this tile's stage precedes its refill
        pipe_refill<P>(p, q, kt, s, gI);
    }
    __syncthreads();
    if (sm.run.node >= 0) flush_run<P>(p, 2, T, exact_c);
    return true;
}

// --------------------------------------------------------------------------
// level construction (leader of the grid barrier that ends a round)
// --------------------------------------------------------------------------
// Segment records of level r live in ring slot r & 1 (the level a round reads
// and the level it creates); the segment tree (TNode) keeps every level, so the
// depth of the recursion is bounded by the tables' sizes only: a set of n
// points has at most 2n tree nodes, at most n small segments and fewer than n
// levels (a split segment loses at least its farthest point).

__device__ __forceinline__ int node_kind(int count, int cut) {
    return count == 0 ? K_LEAF : (count <= cut ? K_SMALL : K_BIG);
}

// Per-thread tallies of a level's new segments: big ones (and their points)
// for the next round, small ones finished alone, small ones packed (and their
// pack weight).
struct LevelTally {
    long long v[5];  // big, big points, solo small, packed small, pack weight
};
__device__ __forceinline__ void tally_child(LevelTally &t, int kind, int cnt) {
    if (kind == K_BIG) {
        t.v[0]++;
        t.v[1] += cnt;
    } else if (kind == K_SMALL) {
        if (cnt <= PACK_MAX) {
            t.v[3]++;
            t.v[4] += cnt + PACK_W;
        } else {
            t.v[2]++;
        }
    }
}

// Where a level's lists go: running positions of this thread after the scan.
struct LevelCursor {
    long long xb, xp, xs, xk, xw;
    int *bl;
    long long *vs;
};

// Scan the tallies and check the list capacities; false (uniform) on overflow.
// The level's packs start at a fresh pack, so a pack's segments share their level.
template <typename P>
__device__ __forceinline__ bool level_lists_open(const Params &p, LevelTally &t, long long (&tot)[5], int dstBuf,
                                                 long long s0, long long k0, long long pw, LevelCursor &c) {
    RoundSmem<P> &sm = round_smem<P>();
    block_excl_scan5(t.v, tot, scan5_scratch<P>());
    if (tot[0] > p.maxBig || s0 + tot[2] > p.maxSmall || k0 + tot[3] > p.maxSmall) {
        if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
        return false;
    }
    const long long w0 = (pw + PACK_B - 1) / PACK_B * PACK_B;
    c.xb = t.v[0];
    c.xp = t.v[1];
    c.xs = s0 + t.v[2];
    c.xk = k0 + t.v[3];
    c.xw = w0 + t.v[4];
    c.bl = p.bigList[dstBuf];
    c.vs = p.vstart[dstBuf];
    return true;
}

// Enter new segment q of the level in its list (a big one for the next round,
// a small one in the solo or the packed queue).
__device__ __forceinline__ void level_list_put(const Params &p, LevelCursor &c, int q, int kind, int cnt, int hIdx,
                                               int eIdx, int cIdx, long long pstart, int level, int inst, int tree) {
    if (kind == K_BIG) {
        __stcg(&c.bl[c.xb], q);
        __stcg(&c.vs[c.xb], c.xp);
        c.xb++;
        c.xp += cnt;
    } else if (kind == K_SMALL) {
        SmallRec *d;
        if (cnt <= PACK_MAX) {
            __stcg(&p.packOff[c.xk], c.xw);
            c.xw += cnt + PACK_W;
            d = &p.pack[c.xk++];
        } else {
            d = &p.small[c.xs++];
        }
        __stcg(reinterpret_cast<int4 *>(d), make_int4(hIdx, eIdx, cIdx, cnt));
        __stcg(reinterpret_cast<int4 *>(d) + 1, make_int4((int)pstart, level, inst, tree));
    }
}

// Publish the level's list sizes for the next round (thread 0).
__device__ __forceinline__ void level_lists_close(const Params &p, const long long (&tot)[5], int dstBuf,
                                                  long long s0, long long k0, long long pw) {
    if (threadIdx.x == 0) {
        const long long w0 = (pw + PACK_B - 1) / PACK_B * PACK_B;
        __stcg(&p.vstart[dstBuf][tot[0]], tot[1]);
        p.ctl->S = (int)tot[0];
        p.ctl->L = tot[1];
        p.ctl->tiles = (tot[1] + TILE - 1) / TILE;
        p.ctl->cur = dstBuf;
        p.ctl->nSmall = (int)(s0 + tot[2]);
        p.ctl->nPack = (int)(k0 + tot[3]);
        if (tot[3]) p.ctl->packW = w0 + tot[4];
    }
}

// List the new segments of ring entries [first, first + count) (level 0).
template <typename P>
__device__ void build_biglist(const Params &p, int first, int count, int dstBuf) {
    const int per = (count + NT - 1) / NT;
    const int b = min(count, threadIdx.x * per), e = min(count, b + per);
    const long long s0 = __ldcg(&p.ctl->nSmall), k0 = __ldcg(&p.ctl->nPack), pw = __ldcg(&p.ctl->packW);
    LevelTally t = {{0, 0, 0, 0, 0}};
    for (int k = b; k < e; k++) {
        const Node *N = &p.nodes[first + k];
        tally_child(t, __ldcg(&N->kind), __ldcg(&N->count));
    }
    long long tot[5];
    LevelCursor c;
    if (!level_lists_open<P>(p, t, tot, dstBuf, s0, k0, pw, c)) return;
    for (int k = b; k < e; k++) {
        const int q = first + k;
        const Node *N = &p.nodes[q];
        level_list_put(p, c, q, __ldcg(&N->kind), __ldcg(&N->count), __ldcg(&N->h.idx), __ldcg(&N->e.idx),
                       __ldcg(&N->c.idx), __ldcg(&N->pstart), __ldcg(&N->level), __ldcg(&N->inst),
                       __ldcg(&N->tree));
    }
    level_lists_close(p, tot, dstBuf, s0, k0, pw);
    __syncthreads();  // the grid release that follows publishes the lists
}

// A tree node: leaves start with one vertex (their head; a small segment adds
// its inner vertices when it is finished).
__device__ __forceinline__ void put_tnode(const Params &p, int t, int head, int inst) {
    __stcg(reinterpret_cast<int4 *>(&p.tnodes[t]), make_int4(-1, head, 1, inst));
}

template <typename P> __device__ __noinline__ void build_level0(const Params &p) {
    RoundSmem<P> &sm = round_smem<P>();
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
        if (carry + tot > p.slotCap || carry + tot > p.maxTNodes) {
            if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
            return;
        }
        if (j < nBig) {
            Inst *I = &p.inst[i];
            const int q0 = (int)(carry + x);  // ring slot 0 and tree nodes both start at 0
            __stcg(&I->level0, q0);
            const long long off = __ldcg(&I->off), n = __ldcg(&I->n);
            for (int k = 0; k < K; k++) {
                Node *N = &p.nodes[q0 + k];
                const int cnt = __ldcg(&I->chCount[k]);
                const Cand h = ldcg_cand(&I->poly[k]);
                stcg_cand(&N->h, h);
                stcg_cand(&N->e, ldcg_cand(&I->poly[(k + 1) % K]));
                stcg_cand(&N->c, ldcg_cand(&I->chC[k]));
                __stcg(&N->count, cnt);
                __stcg(&N->kind, node_kind(cnt, p.cut));
                __stcg(&N->pstart, (k < 2 ? 0ll : p.ncap) + off + ((k & 1) ? n - cnt : 0ll));
                __stcg(&N->buf, 0);
                __stcg(&N->inst, i);
                __stcg(&N->level, 0);
                __stcg(&N->tree, q0 + k);
                __stcg(&N->chCount[0], 0);
                __stcg(&N->chCount[1], 0);
                __stcg(&N->tdone, 0u);
                put_tnode(p, q0 + k, h.idx, i);
            }
        }
        carry += tot;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctl->nNodes = (int)carry;
        p.ctl->nLevels = 1;
        p.levelBase[0] = 0;
        p.levelBase[1] = (int)carry;
    }
    build_biglist<P>(p, 0, (int)carry, 0);
}

// Level r from the big segments of level r - 1 (ring slot (r - 1) & 1): each
// (h, e) with farthest point c becomes (h, c) and (c, e) in slot r & 1, and
// the new segments go to their lists in the same pass.  Thread t takes a
// contiguous range of parents, so one scan of the per-thread tallies gives
// every list position; the second visit of a parent re-reads its record (an
// L2 hit) instead of the children just written.
template <typename P> __device__ __noinline__ void build_level(const Params &p, int r) {
    const int S = __ldcg(&p.ctl->S);
    const int cur = __ldcg(&p.ctl->cur);
    const int base = __ldcg(&p.ctl->nNodes);
    const long long s0 = __ldcg(&p.ctl->nSmall), k0 = __ldcg(&p.ctl->nPack), pw = __ldcg(&p.ctl->packW);
    if ((long long)base + 2ll * S > p.maxTNodes || 2ll * S > p.slotCap || r + 1 > p.maxLevels) {
        if (threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
        return;
    }
    const int slot = (r & 1) * p.slotCap;
    const int *bl = p.bigList[cur];
    const int per = (S + NT - 1) / NT;
    const int jb = min(S, (int)threadIdx.x * per), je = min(S, jb + per);
    LevelTally t = {{0, 0, 0, 0, 0}};
    for (int j = jb; j < je; j++) {
        const int q = __ldcg(&bl[j]);
        const Node *Q = &p.nodes[q];
        const Cand h = ldcg_cand(&Q->h), e = ldcg_cand(&Q->e), c = ldcg_cand(&Q->c);
        const Cand c0 = ldcg_cand(&Q->chC[0]), c1 = ldcg_cand(&Q->chC[1]);
        const long long ps = __ldcg(&Q->pstart);
        const int cnt = __ldcg(&Q->count), buf = __ldcg(&Q->buf), inst = __ldcg(&Q->inst), tree = __ldcg(&Q->tree);
        const int cc0 = __ldcg(&Q->chCount[0]), cc1 = __ldcg(&Q->chCount[1]);
        __stcg(&p.tnodes[tree].child, base + 2 * j);
#pragma unroll
        for (int w = 0; w < 2; w++) {
            Node *N = &p.nodes[slot + 2 * j + w];
            const int cc = w ? cc1 : cc0;
            const int kind = node_kind(cc, p.cut);
            stcg_cand(&N->h, w ? c : h);
            stcg_cand(&N->e, w ? e : c);
            stcg_cand(&N->c, w ? c1 : c0);
            __stcg(&N->count, cc);
            __stcg(&N->kind, kind);
            __stcg(&N->pstart, w ? ps + cnt - cc : ps);
            __stcg(&N->buf, buf ^ 1);
            __stcg(&N->inst, inst);
            __stcg(&N->level, r);
            __stcg(&N->tree, base + 2 * j + w);
            __stcg(&N->chCount[0], 0);
            __stcg(&N->chCount[1], 0);
            __stcg(&N->tdone, 0u);
            put_tnode(p, base + 2 * j + w, w ? c.idx : h.idx, inst);
            tally_child(t, kind, cc);
        }
    }
    long long tot[5];
    LevelCursor lc;
    if (!level_lists_open<P>(p, t, tot, cur ^ 1, s0, k0, pw, lc)) return;
    for (int j = jb; j < je; j++) {
        const Node *Q = &p.nodes[__ldcg(&bl[j])];
        const int hI = __ldcg(&Q->h.idx), eI = __ldcg(&Q->e.idx), cI = __ldcg(&Q->c.idx);
        const int c0I = __ldcg(&Q->chC[0].idx), c1I = __ldcg(&Q->chC[1].idx);
        const long long ps = __ldcg(&Q->pstart);
        const int cnt = __ldcg(&Q->count), inst = __ldcg(&Q->inst);
        const int cc0 = __ldcg(&Q->chCount[0]), cc1 = __ldcg(&Q->chCount[1]);
        level_list_put(p, lc, slot + 2 * j, node_kind(cc0, p.cut), cc0, hI, cI, c0I, ps, r, inst, base + 2 * j);
        level_list_put(p, lc, slot + 2 * j + 1, node_kind(cc1, p.cut), cc1, cI, eI, c1I, ps + cnt - cc1, r, inst,
                       base + 2 * j + 1);
    }
    level_lists_close(p, tot, cur ^ 1, s0, k0, pw);
    if (threadIdx.x == 0) {
        p.ctl->nNodes = base + 2 * S;
        p.ctl->nLevels = r + 1;
        p.levelBase[r + 1] = base + 2 * S;
        p.ctl->rounds = r;
    }
    __syncthreads();  // the grid release that follows publishes the level
}

// --------------------------------------------------------------------------
// the kernel
// --------------------------------------------------------------------------
template <typename P> __global__ void __launch_bounds__(NT, MINB) rounds_kernel(Params p) {
    RoundSmem<P> &sm = round_smem<P>();
    unsigned phase = 0;
    int exact_o = 0, exact_c = 0;
    long long surv = 0;
    unsigned long long gI = 0, gC = 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) mbar_init(&sm.mbar[s], 1u);
        fence_mbar_init();
        sm.run.node = -1;
    }
    __syncthreads();
    stamp(p.ctl, 0);
    if (blockIdx.x == 0) {
        prep<P>(p);
    }
    if (!grid_sync(p.ctl, phase, p.spinLimit)) goto out;
    stamp(p.ctl, 1);

    phase_extremes<P>(p, gI, gC);
    if (!grid_sync(p.ctl, phase, p.spinLimit)) goto out;
    stamp(p.ctl, 2);

    phase_round0<P>(p, gI, gC, exact_o, exact_c, surv);
    if (threadIdx.x == 0 && surv) {
        atomicAdd((unsigned long long *)&p.ctl->live[0], (unsigned long long)surv);
        atomicAdd((unsigned long long *)&p.ctl->gridWritten, (unsigned long long)surv);
    }
    surv = 0;
    {
        const int role = grid_arrive(p.ctl, phase, p.spinLimit);
        if (role < 0) goto out;
        if (role == 1) {  // the last CTA builds the first level
            build_level0<P>(p);
            if (!grid_release(p.ctl, phase)) goto out;
        }
    }
    stamp(p.ctl, 3);

    for (int r = 1;; r++) {
        const int S = __ldcg(&p.ctl->S);
        if (S == 0) break;
        const long long L = __ldcg(&p.ctl->L);
        const int cur = __ldcg(&p.ctl->cur);
        const int ts = round_tile_points(L, gridDim.x);
        if ((L + ts - 1) / ts > p.maxTiles) {
            if (blockIdx.x == 0 && threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
            break;
        }
        phase_round<P>(p, gI, gC, r, S, L, cur, exact_o, exact_c, surv);
        if (threadIdx.x == 0 && surv) {
            atomicAdd((unsigned long long *)&p.ctl->live[min(r, MAX_GEN - 1)], (unsigned long long)surv);
            atomicAdd((unsigned long long *)&p.ctl->gridWritten, (unsigned long long)surv);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->gridRead += L;
        surv = 0;
        const int role = grid_arrive(p.ctl, phase, p.spinLimit);
        if (role < 0) goto out;
        if (role == 1) {  // the last CTA builds the next level
            build_level<P>(p, r);
            if (!grid_release(p.ctl, phase)) goto out;
        }
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

}  // namespace QH_VARIANT_NS
}  // namespace qh
