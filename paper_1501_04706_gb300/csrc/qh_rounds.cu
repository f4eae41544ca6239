// Grid-wide part of segmented QuickHull: one cooperative, persistent launch.
//
// Phases (separated by bounded grid barriers):
//   prep       CTA 0 classifies the sets: empty, small (<= FIN_MAX points, left
//              to the block finisher) or big (tiled here).
//   extremes   per big set, the four extreme points of Sec. 4.2 (lexicographic
//              min/max of (x, y) and of (y, x), ties to the lower index), as a
//              tile reduction whose last tile merges the set's partials.
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
// Compaction is a single pass with a decoupled look-back over tiles of TILE
// points.  Segments are contiguous ranges of a live buffer; a child never
// leaves its parent's range: the first child grows upward from the parent's
// start, the second downward from its end, so the positions only need the
// parent-local (segmented) counts that the look-back carries, together with
// the farthest point seen so far (the segmented argmax).  Segments with at
// most `cut` points (cut >= TILE) leave the grid-wide rounds for the block
// finisher, so a tile of a round spans at most two segments.
#include "qh_internal.cuh"

namespace qh {

template <typename P> struct RoundSmem {
    // tile descriptors
    Edge<P> edge[4];
    float vend[4][2];  // end point of each slot's chord (for the exact fallback)
    long long pstart[2], vstart[2];
    int count[2], node[2];
    int nparts, inst, kflag;
    long long lt;
    // ranks
    unsigned long long warpTot[IPT * NWARP];
    unsigned long long tileTot;
    // farthest point
    unsigned maxLo[4];
    int ncand;
    Cand best[4];
    Carry carry;
    long long scanTmp[NWARP + 1];
    Ext wext[NWARP];
    Cand cand[TILE];
    unsigned char cslot[TILE];
};

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
// look-back helpers (thread 0 only)
// --------------------------------------------------------------------------
__device__ __forceinline__ void publish(const Params &p, long long t, unsigned epoch, unsigned state,
                                        const Carry &c, int nslot) {
    Carry *dst = state == 2u ? &p.tinc[t] : &p.tagg[t];
    for (int s = 0; s < nslot; s++) {
        __stcg(&dst->cnt[s], c.cnt[s]);
        stcg_cand(&dst->best[s], c.best[s]);
    }
    __threadfence();
    st_release(&p.tstatus[t], (epoch << 2) | state);
}

template <typename P>
__device__ __forceinline__ void carry_merge(Carry &acc, const Carry &x, int nslot, const RoundSmem<P> &sm,
                                            int &exact_c) {
    for (int s = 0; s < nslot; s++) {
        acc.cnt[s] += x.cnt[s];
        const Edge<P> &e = sm.edge[s];
        const Cand &a = x.best[s];
        const Cand &b = acc.best[s];
        if (a.idx < 0) continue;
        if (b.idx < 0) {
            acc.best[s] = a;
            continue;
        }
        DistIv<P> da = dist_interval(orient_approx(e, a.x, a.y));
        DistIv<P> db = dist_interval(orient_approx(e, b.x, b.y));
        if (farther(e, sm.vend[s][0], sm.vend[s][1], a.x, a.y, a.idx, da, b.x, b.y, b.idx, db, exact_c))
            acc.best[s] = a;
    }
}

// Exclusive carry of tile t for its first parent: sum of the predecessors'
// payloads back to (and including) the first inclusive one.
template <typename P>
__device__ bool lookback(const Params &p, long long t, unsigned epoch, int nslot, const RoundSmem<P> &sm,
                         Carry &acc, int &exact_c) {
    for (int s = 0; s < 4; s++) {
        acc.cnt[s] = 0u;
        acc.best[s] = no_cand();
    }
    for (long long u = t - 1; u >= 0; u--) {
        unsigned st, it = 0;
        for (;;) {
            st = ld_acquire(&p.tstatus[u]);
            if ((st >> 2) == epoch && (st & 3u) != 0u) break;
            if (ld_volatile(&p.ctl->err) != 0u) return false;
            if (++it > SPIN_LIMIT) {
                set_err(p.ctl, E_TIMEOUT);
                return false;
            }
            __nanosleep(32);
        }
        const Carry *src = (st & 3u) == 2u ? &p.tinc[u] : &p.tagg[u];
        Carry x;
        for (int s = 0; s < nslot; s++) {
            x.cnt[s] = __ldcg(&src->cnt[s]);
            x.best[s] = ldcg_cand(&src->best[s]);
        }
        carry_merge(acc, x, nslot, sm, exact_c);
        if ((st & 3u) == 2u) return true;
    }
    set_err(p.ctl, E_INTERNAL);  // a chain must end at an inclusive tile
    return false;
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

// Farthest point of each slot within the tile, exactly: the largest lower
// bound per slot, then every item whose upper bound reaches it is a candidate,
// and thread s picks the best candidate of slot s with the exact order.
template <typename P>
__device__ __forceinline__ void tile_farthest(const int (&slot)[IPT], const float (&x)[IPT], const float (&y)[IPT],
                                              const int (&idx)[IPT], const P (&lo)[IPT], const P (&hi)[IPT],
                                              RoundSmem<P> &sm, int &exact_c) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 4) sm.maxLo[threadIdx.x] = 0u;
    if (threadIdx.x == 0) sm.ncand = 0;
    __syncthreads();
    unsigned mk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < IPT; k++) {
#pragma unroll
        for (int s = 0; s < 4; s++)
            if (slot[k] == s) mk[s] = max(mk[s], pkey(lo[k]));
    }
#pragma unroll
    for (int s = 0; s < 4; s++) {
        unsigned v = __reduce_max_sync(0xffffffffu, mk[s]);
        if (lane == 0 && v != 0u) atomicMax(&sm.maxLo[s], v);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        if (slot[k] >= 0) {
            P thr = (P)fkey_inv(sm.maxLo[slot[k]]);
            if (hi[k] >= thr) {
                int j = atomicAdd(&sm.ncand, 1);
                sm.cand[j] = mk_cand(x[k], y[k], idx[k]);
                sm.cslot[j] = (unsigned char)slot[k];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int s = threadIdx.x;
        const Edge<P> &e = sm.edge[s];
        Cand b = no_cand();
        DistIv<P> db;
        db.lo = db.hi = P(0);
        const int nc = sm.ncand;
        for (int j = 0; j < nc; j++) {
            if (sm.cslot[j] != s) continue;
            const Cand a = sm.cand[j];
            DistIv<P> da = dist_interval(orient_approx(e, a.x, a.y));
            if (farther(e, sm.vend[s][0], sm.vend[s][1], a.x, a.y, a.idx, da, b.x, b.y, b.idx, db, exact_c)) {
                b = a;
                db = da;
            }
        }
        sm.best[s] = b;
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
// prep: classify sets (CTA 0)
// --------------------------------------------------------------------------
template <typename P> __device__ void prep(const Params &p, RoundSmem<P> &sm) {
    long long *scr = sm.scanTmp;
    long long carryBig = 0, carrySmall = 0, carryTiles = 0;
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
// extremes (Sec. 4.2)
// --------------------------------------------------------------------------
template <typename P> __device__ void locate_tile(const Params &p, RoundSmem<P> &sm, long long t) {
    if (threadIdx.x == 0) {
        const int nBig = __ldcg(&p.ctl->nBig);
        long long j = upper_bound_ll(p.bigTilePrefix, nBig + 1, t) - 1;
        sm.inst = __ldcg(&p.bigInst[j]);
        sm.lt = t - __ldcg(&p.bigTilePrefix[j]);
    }
    __syncthreads();
}

template <typename P> __device__ void extremes_tile(const Params &p, RoundSmem<P> &sm, long long t) {
    locate_tile(p, sm, t);
    const int i = sm.inst;
    const long long lt = sm.lt;
    const Inst *I = &p.inst[i];
    const long long off = __ldcg(&I->off), n = __ldcg(&I->n);
    const int tiles = __ldcg(&I->tiles);
    const long long tile0 = __ldcg(&I->tile0);
    Ext e = ext_empty();
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const long long v = lt * TILE + (long long)k * NT + threadIdx.x;
        if (v < n) {
            const float2 q = __ldg(&p.pts[off + v]);
            if (!isfinite(q.x) || !isfinite(q.y)) {
                e.nonfinite = 1;
            } else {
                const int id = (int)v;
                if (lex_less(q.x, q.y, id, e.a.x, e.a.y, e.a.idx)) e.a = mk_cand(q.x, q.y, id);
                if (lex_greater(q.x, q.y, id, e.b.x, e.b.y, e.b.idx)) e.b = mk_cand(q.x, q.y, id);
                if (lex_less(q.y, q.x, id, e.bot.y, e.bot.x, e.bot.idx)) e.bot = mk_cand(q.x, q.y, id);
                if (lex_greater(q.y, q.x, id, e.top.y, e.top.x, e.top.idx)) e.top = mk_cand(q.x, q.y, id);
            }
        }
    }
    e = warp_ext_reduce(e);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm.wext[w] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext r = sm.wext[0];
        for (int k = 1; k < NWARP; k++) ext_merge(r, sm.wext[k]);
        st_ext(&p.text[t], r);
        __threadfence();
        unsigned prev = atomicAdd(&p.inst[i].done, 1u);
        sm.kflag = (prev == (unsigned)tiles - 1u);
        __threadfence();
    }
    __syncthreads();
    if (!sm.kflag) return;
    // last tile of set i: merge all partials
    Ext r = ext_empty();
    for (int k = threadIdx.x; k < tiles; k += NT) ext_merge(r, ld_ext(&p.text[tile0 + k]));
    r = warp_ext_reduce(r);
    __syncthreads();
    if (lane == 0) sm.wext[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext a = sm.wext[0];
        for (int k = 1; k < NWARP; k++) ext_merge(a, sm.wext[k]);
        Inst &W = p.inst[i];
        int K = 0;
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
            poly[K++] = a.b;
            if (quad && !same_xy(a.top, a.a) && !same_xy(a.top, a.b)) poly[K++] = a.top;
        }
        W.kind = kind;
        W.K = K;
        for (int k = 0; k < 4; k++) W.poly[k] = (k < K || (kind == I_DEGEN && k == 0)) ? poly[k] : no_cand();
        __threadfence();
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// round 0: the initial split
// --------------------------------------------------------------------------
template <typename P>
__device__ void round0_tile(const Params &p, RoundSmem<P> &sm, long long t, int &exact_o, int &exact_c,
                            long long &survivors) {
    locate_tile(p, sm, t);
    const int i = sm.inst;
    const long long lt = sm.lt;
    const Inst *I = &p.inst[i];
    const int K = __ldcg(&I->K);
    if (K == 0) return;  // degenerate or rejected set: no segments
    const long long off = __ldcg(&I->off), n = __ldcg(&I->n);
    const int tiles = __ldcg(&I->tiles);
    if (threadIdx.x < 4) {
        const int s = threadIdx.x;
        if (s < K) {
            const Cand u = ldcg_cand(&I->poly[s]);
            const Cand v = ldcg_cand(&I->poly[(s + 1) % K]);
            sm.edge[s] = make_edge<P>(u.x, u.y, v.x, v.y);
            sm.vend[s][0] = v.x;
            sm.vend[s][1] = v.y;
        }
    }
    __syncthreads();

    float x[IPT], y[IPT];
    int idx[IPT], slot[IPT], rank[IPT];
    P lo[IPT], hi[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const long long v = lt * TILE + (long long)k * NT + threadIdx.x;
        slot[k] = -1;
        lo[k] = hi[k] = P(0);
        x[k] = y[k] = 0.f;
        idx[k] = (int)v;
        if (v < n) {
            const float2 q = __ldg(&p.pts[off + v]);
            x[k] = q.x;
            y[k] = q.y;
            for (int s = 0; s < K; s++) {
                if (right_of(sm.edge[s], sm.vend[s][0], sm.vend[s][1], q.x, q.y, lo[k], hi[k], exact_o)) {
                    slot[k] = s;
                    break;
                }
            }
        }
    }
    unsigned tot[4];
    tile_ranks(slot, rank, tot, sm);
    tile_farthest(slot, x, y, idx, lo, hi, sm, exact_c);

    const unsigned epoch = 1u;
    if (threadIdx.x == 0) {
        Carry local;
        for (int s = 0; s < 4; s++) {
            local.cnt[s] = tot[s];
            local.best[s] = sm.best[s];
        }
        Carry c;
        bool ok = true;
        if (lt == 0) {
            publish(p, t, epoch, 2u, local, K);
            for (int s = 0; s < 4; s++) {
                c.cnt[s] = 0u;
                c.best[s] = no_cand();
            }
        } else {
            publish(p, t, epoch, 1u, local, K);
            ok = lookback(p, t, epoch, K, sm, c, exact_c);
            Carry inc = c;
            carry_merge(inc, local, K, sm, exact_c);
            publish(p, t, epoch, 2u, inc, K);
        }
        sm.carry = c;
        sm.kflag = ok;
        if (ok && lt == tiles - 1) {
            Carry f = c;
            carry_merge(f, local, K, sm, exact_c);
            Inst *W = &p.inst[i];
            for (int s = 0; s < K; s++) {
                __stcg(&W->chCount[s], (int)f.cnt[s]);
                stcg_cand(&W->chC[s], f.best[s]);
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (!sm.kflag) return;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const int s = slot[k];
        if (s < 0) continue;
        const long long base = (s < 2 ? 0ll : p.ncap) + off;
        const long long r = (long long)sm.carry.cnt[s] + rank[k];
        const long long pos = (s & 1) ? base + n - 1 - r : base + r;
        if (pos < base || pos >= base + n) {  // guard: never write outside the set's range
            set_err(p.ctl, E_INTERNAL);
            continue;
        }
        __stcg(&p.xy[0][pos], make_float2(x[k], y[k]));
        __stcg(&p.id[0][pos], idx[k]);
    }
    if (threadIdx.x == 0) survivors += (long long)tot[0] + tot[1] + tot[2] + tot[3];
}

// --------------------------------------------------------------------------
// round r >= 1
// --------------------------------------------------------------------------
template <typename P>
__device__ void round_tile(const Params &p, RoundSmem<P> &sm, long long t, int r, int S, long long L, int cur,
                           int &exact_o, int &exact_c, long long &survivors) {
    const int src = (r - 1) & 1, dst = r & 1;
    const long long v0 = t * TILE;
    const long long v1 = min(v0 + (long long)TILE, L);
    const long long *vs = p.vstart[cur];
    const int *bl = p.bigList[cur];
    if (threadIdx.x == 0) {
        const long long sA = upper_bound_ll(vs, (long long)S + 1, v0) - 1;
        int np = 1;
        sm.node[0] = __ldcg(&bl[sA]);
        sm.vstart[0] = __ldcg(&vs[sA]);
        if (sA + 1 < S && __ldcg(&vs[sA + 1]) < v1) {
            np = 2;
            sm.node[1] = __ldcg(&bl[sA + 1]);
            sm.vstart[1] = __ldcg(&vs[sA + 1]);
        }
        sm.nparts = np;
    }
    __syncthreads();
    if (threadIdx.x < 2 * sm.nparts) {
        const int part = threadIdx.x >> 1, which = threadIdx.x & 1;
        const Node *N = &p.nodes[sm.node[part]];
        const Cand h = ldcg_cand(&N->h), e = ldcg_cand(&N->e), c = ldcg_cand(&N->c);
        const Cand u = which ? c : h;
        const Cand v = which ? e : c;
        sm.edge[2 * part + which] = make_edge<P>(u.x, u.y, v.x, v.y);
        sm.vend[2 * part + which][0] = v.x;
        sm.vend[2 * part + which][1] = v.y;
        if (!which) {
            sm.pstart[part] = __ldcg(&N->pstart);
            sm.count[part] = __ldcg(&N->count);
        }
    }
    __syncthreads();
    const int np = sm.nparts;

    float x[IPT], y[IPT];
    int idx[IPT], slot[IPT], rank[IPT];
    P lo[IPT], hi[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const long long v = v0 + (long long)k * NT + threadIdx.x;
        slot[k] = -1;
        lo[k] = hi[k] = P(0);
        x[k] = y[k] = 0.f;
        idx[k] = -1;
        if (v < v1) {
            const int part = (np == 2 && v >= sm.vstart[1]) ? 1 : 0;
            const long long phys = sm.pstart[part] + (v - sm.vstart[part]);
            if (phys < 0 || phys >= 2 * p.ncap) {  // guard: never read outside the live buffer
                set_err(p.ctl, E_INTERNAL);
                continue;
            }
            const float2 q = __ldcg(&p.xy[src][phys]);
            x[k] = q.x;
            y[k] = q.y;
            idx[k] = __ldcg(&p.id[src][phys]);
            const int s0 = 2 * part;
            if (right_of(sm.edge[s0], sm.vend[s0][0], sm.vend[s0][1], q.x, q.y, lo[k], hi[k], exact_o))
                slot[k] = s0;
            else if (right_of(sm.edge[s0 + 1], sm.vend[s0 + 1][0], sm.vend[s0 + 1][1], q.x, q.y, lo[k], hi[k],
                              exact_o))
                slot[k] = s0 + 1;
        }
    }
    unsigned tot[4];
    tile_ranks(slot, rank, tot, sm);
    tile_farthest(slot, x, y, idx, lo, hi, sm, exact_c);

    const unsigned epoch = (unsigned)r + 1u;
    if (threadIdx.x == 0) {
        Carry la, lb;
        for (int s = 0; s < 2; s++) {
            la.cnt[s] = tot[s];
            la.best[s] = sm.best[s];
            lb.cnt[s] = tot[2 + s];
            lb.best[s] = sm.best[2 + s];
        }
        for (int s = 2; s < 4; s++) {
            la.cnt[s] = lb.cnt[s] = 0u;
            la.best[s] = lb.best[s] = no_cand();
        }
        const bool contA = sm.vstart[0] < v0;
        Carry c;
        for (int s = 0; s < 4; s++) {
            c.cnt[s] = 0u;
            c.best[s] = no_cand();
        }
        bool ok = true;
        if (np == 2)
            publish(p, t, epoch, 2u, lb, 2);
        else if (!contA)
            publish(p, t, epoch, 2u, la, 2);
        else
            publish(p, t, epoch, 1u, la, 2);
        if (contA) {
            ok = lookback(p, t, epoch, 2, sm, c, exact_c);
            if (np == 1) {
                Carry inc = c;
                carry_merge(inc, la, 2, sm, exact_c);
                publish(p, t, epoch, 2u, inc, 2);
            }
        }
        sm.carry = c;
        sm.kflag = ok;
        if (ok) {
            if (sm.vstart[0] + sm.count[0] <= v1) {  // part A ends in this tile
                Carry f = c;
                carry_merge(f, la, 2, sm, exact_c);
                Node *N = &p.nodes[sm.node[0]];
                for (int s = 0; s < 2; s++) {
                    __stcg(&N->chCount[s], (int)f.cnt[s]);
                    stcg_cand(&N->chC[s], f.best[s]);
                }
            }
            if (np == 2 && sm.vstart[1] + sm.count[1] <= v1) {  // part B starts and ends here
                Node *N = &p.nodes[sm.node[1]];
                for (int s = 0; s < 2; s++) {
                    __stcg(&N->chCount[s], (int)lb.cnt[s]);
                    stcg_cand(&N->chC[s], lb.best[s]);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (!sm.kflag) return;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const int s = slot[k];
        if (s < 0) continue;
        const int part = s >> 1;
        const long long rr = (long long)(part == 0 ? sm.carry.cnt[s] : 0u) + rank[k];
        const long long pos = (s & 1) ? sm.pstart[part] + sm.count[part] - 1 - rr : sm.pstart[part] + rr;
        if (pos < sm.pstart[part] || pos >= sm.pstart[part] + sm.count[part] || pos >= 2 * p.ncap) {
            set_err(p.ctl, E_INTERNAL);  // guard: a child never leaves its parent's range
            continue;
        }
        __stcg(&p.xy[dst][pos], make_float2(x[k], y[k]));
        __stcg(&p.id[dst][pos], idx[k]);
    }
    if (threadIdx.x == 0) survivors += (long long)tot[0] + tot[1] + tot[2] + tot[3];
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

template <typename P> __device__ void build_level0(const Params &p, RoundSmem<P> &sm) {
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

template <typename P> __device__ void build_level(const Params &p, RoundSmem<P> &sm, int r) {
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
template <typename P> __global__ void __launch_bounds__(NT, 2) rounds_kernel(Params p) {
    __shared__ RoundSmem<P> sm;
    unsigned phase = 0, donePhase = 0;
    int exact_o = 0, exact_c = 0;
    long long surv = 0;

    if (blockIdx.x == 0) prep(p, sm);
    if (!grid_sync(p.ctl, phase)) goto out;

    {
        const long long T = __ldcg(&p.ctl->bigTiles);
        for (long long t = blockIdx.x; t < T; t += gridDim.x) extremes_tile(p, sm, t);
    }
    if (!grid_sync(p.ctl, phase)) goto out;

    {
        const long long T = __ldcg(&p.ctl->bigTiles);
        for (long long t = blockIdx.x; t < T; t += gridDim.x) round0_tile(p, sm, t, exact_o, exact_c, surv);
        if (threadIdx.x == 0 && surv) atomicAdd((unsigned long long *)&p.ctl->live[0], (unsigned long long)surv);
        surv = 0;
        if (last_cta(p.ctl, donePhase, &sm.kflag)) build_level0(p, sm);
    }
    if (!grid_sync(p.ctl, phase)) goto out;

    for (int r = 1;; r++) {
        const int S = __ldcg(&p.ctl->S);
        if (S == 0) break;
        const long long L = __ldcg(&p.ctl->L);
        const long long T = __ldcg(&p.ctl->tiles);
        const int cur = __ldcg(&p.ctl->cur);
        if (T > p.maxTiles) {
            if (blockIdx.x == 0 && threadIdx.x == 0) set_err(p.ctl, E_CAPACITY);
            break;
        }
        for (long long t = blockIdx.x; t < T; t += gridDim.x)
            round_tile(p, sm, t, r, S, L, cur, exact_o, exact_c, surv);
        if (threadIdx.x == 0 && surv)
            atomicAdd((unsigned long long *)&p.ctl->live[min(r, MAX_GEN - 1)], (unsigned long long)surv);
        surv = 0;
        if (last_cta(p.ctl, donePhase, &sm.kflag)) build_level(p, sm, r);
        if (!grid_sync(p.ctl, phase)) goto out;
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

cudaError_t launch_rounds(const Params &p, int prec, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    if (prec)
        return cudaLaunchCooperativeKernel((void *)rounds_kernel<double>, dim3(grid), dim3(NT), args, 0, s);
    return cudaLaunchCooperativeKernel((void *)rounds_kernel<float>, dim3(grid), dim3(NT), args, 0, s);
}

int rounds_max_ctas_per_sm(int prec) {
    int b = 0;
    if (prec)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rounds_kernel<double>, NT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rounds_kernel<float>, NT, 0);
    return b;
}

}  // namespace qh
