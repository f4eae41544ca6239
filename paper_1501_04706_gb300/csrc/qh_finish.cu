// Block-level parts of segmented QuickHull.
//
// finish_kernel  one thread block per small problem: a segment of at most
//                `cut` points left by the grid-wide rounds, a pack of up to
//                PACK_SEGS segments of at most PACK_MAX points each (all from
//                one level, so they share their generations), or a whole set of
//                at most FIN_MAX points.  The block runs the remaining
//                generations of Sec. 4.4 with all state in shared memory: per
//                point the id of its segment; per live segment its place in the
//                CCW list of segment heads (a pack lists each segment's chord
//                h -> e, the end marked as a boundary); per generation the
//                farthest point of each new segment and the classification
//                against the two new edges.
// emit_kernel    one block per set: walks the binary tree of segments built by
//                the grid-wide rounds (each big segment (h, e) split at its
//                farthest point c into (h, c), (c, e)), computes the output
//                offset of every leaf in CCW order, and writes the heads.
// copy_kernel    copies the inner vertices found by the finisher to their
//                output offsets.
#include "qh_internal.cuh"

namespace qh {

constexpr int FM = FIN_MAX;
constexpr unsigned short NONE16 = 0xffffu;

struct OrdE {
    unsigned short head, live, c, bnd;  // head point, live segment id (or NONE16), its farthest point;
                                        // bnd: the end of a packed segment's chord
};
constexpr int ORDCAP = FM + 2 * PACK_SEGS + 8;  // heads: one per point, plus every chord's two ends

static_assert(FM % FIN_NT == 0, "the live list is split into FM / FIN_NT entries per thread");
constexpr int FIN_PER = FM / FIN_NT;

struct FinSmem {
    float2 pxy[FM + 2 * PACK_SEGS];  // the points, then the chord ends
    unsigned short seg[FM];  // per point: live segment / child code, NONE16 = discarded
    unsigned short lst[FM];  // the points still live (any order); nLive of them
    OrdE ordA[ORDCAP], ordB[ORDCAP];
    unsigned short memStart[PACK_SEGS + 1];  // pack: first point of every segment
    const int *gidx;         // solo segment: original index of every point
    int gmode;               // point -> original index: 0 identity (set), 1 gidx, 2 pack
    int mem0, nMem, packBuf; // pack: first segment in the pack queue, segments, live buffer
    unsigned short lpos[FM];  // live segment -> position in the ord list
    unsigned cnt2[FM];        // per live segment: packed child counts (low: first child, high: second)
    unsigned maxLo[2 * FM];   // per child: largest lower distance bound (orderable key)
    unsigned short best[2 * FM];
    unsigned short newId[2 * FM];
    int scan[FIN_NT / 32 + 1];
    int ticket, cLocal, nOrd, S, K, degenerate, nonfinite, nLive;
    long long liveCount;
    unsigned short poly[4];
    Ext wext[FIN_NT / 32];
};

// Original index (local to its set) of problem point k.
__device__ __forceinline__ int fin_gidx(const Params &p, const FinSmem &s, int k) {
    if (s.gmode == 0) return k;
    if (s.gmode == 1) return __ldg(&s.gidx[k]);
    int lo = 0, hi = s.nMem;  // the packed segment holding k: memStart[lo] <= k < memStart[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s.memStart[mid] <= k) lo = mid; else hi = mid;
    }
    const SmallRec *R = &p.pack[s.mem0 + lo];
    return __ldg(&p.id[s.packBuf][__ldg(&R->pstart) + (k - s.memStart[lo])]);
}

__device__ __forceinline__ Cand shfl_c(const Cand &c, int src) {
    Cand o;
    o.x = __shfl_sync(0xffffffffu, c.x, src);
    o.y = __shfl_sync(0xffffffffu, c.y, src);
    o.idx = __shfl_sync(0xffffffffu, c.idx, src);
    o.pad = 0;
    return o;
}

__device__ __forceinline__ void ext_merge_f(Ext &a, const Ext &b) {
    if (lex_less(b.a.x, b.a.y, b.a.idx, a.a.x, a.a.y, a.a.idx)) a.a = b.a;
    if (lex_greater(b.b.x, b.b.y, b.b.idx, a.b.x, a.b.y, a.b.idx)) a.b = b.b;
    if (lex_less(b.bot.y, b.bot.x, b.bot.idx, a.bot.y, a.bot.x, a.bot.idx)) a.bot = b.bot;
    if (lex_greater(b.top.y, b.top.x, b.top.idx, a.top.y, a.top.x, a.top.idx)) a.top = b.top;
    a.nonfinite |= b.nonfinite;
}

// Chord (u, v) of child c: initial edges of the polygon, or the two edges
// (h, C), (C, e) of live segment c >> 1.
__device__ __forceinline__ void child_chord(const FinSmem &s, const OrdE *ord, int nOrd, bool initial, int c, int &u,
                                            int &v) {
    if (initial) {
        u = s.poly[c];
        v = s.poly[(c + 1) % s.K];
    } else {
        const int pos = s.lpos[c >> 1];
        const OrdE &o = ord[pos];
        if (c & 1) {
            u = o.c;
            v = ord[(pos + 1) % nOrd].head;
        } else {
            u = o.head;
            v = o.c;
        }
    }
}

template <typename P>
__device__ __forceinline__ bool fin_right_of(const FinSmem &s, int u, int v, float px, float py, P &lo, P &hi,
                                             int &exact_o) {
    const float2 a = s.pxy[u], b = s.pxy[v];
    const Edge<P> e = make_edge<P>(a.x, a.y, b.x, b.y);
    Approx<P> o = orient_approx(e, px, py);
    if (orient_sign(e, b.x, b.y, px, py, o, exact_o) < 0) {
        DistIv<P> d = dist_interval(o);
        lo = d.lo;
        hi = d.hi;
        return true;
    }
    return false;
}

// One generation.  Classification (pass 1), exact farthest point per child
// (pass 2), rebuild of the CCW head list and of the live segments, relabelling.
// Returns (the same in the whole block) whether the generation failed or, when
// pollErr is set, another block has reported an error.
template <typename P>
__device__ bool fin_generation(const Params &p, FinSmem &s, int m, bool initial, OrdE *&ord, OrdE *&ordN,
                               int gen, bool pollErr, int &exact_o, int &exact_c) {
    const int S = s.S, nOrd = s.nOrd;
    const int nch = initial ? s.K : 2 * S;
    for (int c = threadIdx.x; c < nch; c += FIN_NT) {
        s.maxLo[c] = 0u;
        s.best[c] = NONE16;
    }
    for (int j = threadIdx.x; j < (initial ? s.K : S); j += FIN_NT) s.cnt2[j] = 0u;
    __syncthreads();
    // pass 1: classify.  The per-child counters are updated once per group of
    // lanes that share a child (same-address shared atomics would serialise).
    const int nL = s.nLive;
    for (int i0 = 0; i0 < nL; i0 += FIN_NT) {
        const int i = i0 + threadIdx.x;
        int child = -1;
        unsigned key = 0u;
        if (i < nL) {
            const int k = s.lst[i];
            const unsigned short j = s.seg[k];
            if (j != NONE16) {
                const float2 q = s.pxy[k];
                P lo = P(0), hi = P(0);
                if (initial) {
                    for (int c = 0; c < s.K; c++) {
                        int u, v;
                        child_chord(s, ord, nOrd, true, c, u, v);
                        if (fin_right_of(s, u, v, q.x, q.y, lo, hi, exact_o)) {
                            child = c;
                            break;
                        }
                    }
                } else {
                    int u, v;
                    child_chord(s, ord, nOrd, false, 2 * j, u, v);
                    if (fin_right_of(s, u, v, q.x, q.y, lo, hi, exact_o)) {
                        child = 2 * j;
                    } else {
                        child_chord(s, ord, nOrd, false, 2 * j + 1, u, v);
                        if (fin_right_of(s, u, v, q.x, q.y, lo, hi, exact_o)) child = 2 * j + 1;
                    }
                }
                s.seg[k] = child < 0 ? NONE16 : (unsigned short)child;
                key = max(pkey(lo), 1u);
            }
        }
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        const unsigned grp = __match_any_sync(full, child);
        const bool leader = child >= 0 && lane == __ffs(grp) - 1;
        unsigned leaders = __ballot_sync(full, leader);
        if (__popc(leaders) <= 4) {
            while (leaders) {
                const int l = __ffs(leaders) - 1;
                const int c = __shfl_sync(full, child, l);
                const unsigned mx = __reduce_max_sync(full, child == c ? key : 0u);
                if (lane == l) {
                    const unsigned cnt = __popc(grp);
                    if (initial)
                        atomicAdd(&s.cnt2[c], cnt);
                    else
                        atomicAdd(&s.cnt2[c >> 1], (c & 1) ? cnt << 16 : cnt);
                    atomicMax(&s.maxLo[c], mx);
                }
                leaders &= leaders - 1;
            }
        } else if (child >= 0) {
            if (initial)
                atomicAdd(&s.cnt2[child], 1u);
            else
                atomicAdd(&s.cnt2[child >> 1], (child & 1) ? 0x10000u : 1u);
            atomicMax(&s.maxLo[child], key);
        }
    }
    __syncthreads();
    // pass 2: exact farthest point among the candidates of each child
    for (int i = threadIdx.x; i < nL; i += FIN_NT) {
        const int k = s.lst[i];
        const unsigned short c = s.seg[k];
        if (c == NONE16) continue;
        int u, v;
        child_chord(s, ord, nOrd, initial, c, u, v);
        const float2 a = s.pxy[u], b = s.pxy[v];
        const Edge<P> e = make_edge<P>(a.x, a.y, b.x, b.y);
        const float2 q = s.pxy[k];
        DistIv<P> dq = dist_interval(orient_approx(e, q.x, q.y));
        const P thr = (P)fkey_inv(s.maxLo[c]);
        if (!(dq.hi >= thr)) continue;
        unsigned short cur = s.best[c];
        for (int it = 0; it < 1 << 20; it++) {
            bool mine;
            if (cur == NONE16) {
                mine = true;
            } else {
                const float2 w = s.pxy[cur];
                if (q.x == w.x && q.y == w.y) {
                    // equal points: the original indices decide (a global load for
                    // a segment's points, so only here)
                    mine = fin_gidx(p, s, k) < fin_gidx(p, s, cur);
                } else {  // the local indices only stand for "a point" here
                    DistIv<P> dw = dist_interval(orient_approx(e, w.x, w.y));
                    mine = farther(e, b.x, b.y, q.x, q.y, k, dq, w.x, w.y, (int)cur, dw, exact_c);
                }
            }
            if (!mine) break;
            const unsigned short prev = atomicCAS(&s.best[c], cur, (unsigned short)k);
            if (prev == cur) break;
            cur = prev;
        }
    }
    __syncthreads();
    // children that hold points become the new live segments (one scan of the
    // packed per-thread counts: live children in the high half, their points in
    // the low half; both totals stay below 2^16)
    {
        const int per = (nch + FIN_NT - 1) / FIN_NT;
        const int b = min(nch, (int)threadIdx.x * per), e = min(nch, b + per);
        int packed = 0;
        for (int c = b; c < e; c++) {
            const unsigned cnt = initial ? s.cnt2[c] : ((s.cnt2[c >> 1] >> (16 * (c & 1))) & 0xffffu);
            packed += (cnt > 0u ? 1 << 16 : 0) + (int)cnt;
        }
        int tot;
        int x = block_excl_scan_open<int, FIN_NT>(packed, s.scan, tot) >> 16;  // a barrier follows
        for (int c = b; c < e; c++) {
            const unsigned cnt = initial ? s.cnt2[c] : ((s.cnt2[c >> 1] >> (16 * (c & 1))) & 0xffffu);
            s.newId[c] = cnt > 0u ? (unsigned short)(x++) : NONE16;
        }
        if (threadIdx.x == 0) {
            s.S = tot >> 16;
            s.liveCount = tot & 0xffff;
        }
    }
    __syncthreads();
    // The new CCW list of heads and the relabelled, compacted list of live
    // points, with one scan of the packed per-thread sizes (list entries in the
    // high half, live points in the low half).  Each thread reads its ranges
    // (at most FIN_PER points) before the scan's barriers and writes after them.
    {
        int w = 0, bo = 0, eo = 0;
        if (!initial) {
            const int per = (nOrd + FIN_NT - 1) / FIN_NT;
            bo = min(nOrd, (int)threadIdx.x * per);
            eo = min(nOrd, bo + per);
            for (int q = bo; q < eo; q++) w += ord[q].live != NONE16 ? 2 : 1;
        }
        const int b = min(nL, (int)threadIdx.x * FIN_PER), e = min(nL, b + FIN_PER);
        unsigned short keep[FIN_PER];
        unsigned km = 0u;
#pragma unroll
        for (int j = 0; j < FIN_PER; j++) {
            keep[j] = 0;
            if (b + j < e) {
                const unsigned short k = s.lst[b + j];
                const unsigned short c = s.seg[k];
                const unsigned short nc = c != NONE16 ? s.newId[c] : NONE16;
                s.seg[k] = nc;
                keep[j] = k;
                km |= (unsigned)(nc != NONE16) << j;
            }
        }
        int tot;
        const int x = block_excl_scan_open<int, FIN_NT>((w << 16) + __popc(km), s.scan, tot);
        if (!initial && (tot >> 16) > ORDCAP - 8) {  // guard: at most one head per point plus the chord ends
            if (threadIdx.x == 0) {
                set_err(p.ctl, E_INTERNAL);
                s.S = 0;
                s.nOrd = 0;
            }
            return __syncthreads_or(1);
        }
        int xl = x & 0xffff;
#pragma unroll
        for (int j = 0; j < FIN_PER; j++)
            if ((km >> j) & 1u) s.lst[xl++] = keep[j];
        if (initial) {
            for (int c = threadIdx.x; c < s.K; c += FIN_NT) {
                OrdE o;
                o.head = s.poly[c];
                o.live = s.newId[c];
                o.c = o.live != NONE16 ? s.best[c] : NONE16;
                o.bnd = 0;
                ordN[c] = o;
                if (o.live != NONE16) s.lpos[o.live] = (unsigned short)c;
            }
        } else {
            int np = x >> 16;
            for (int q = bo; q < eo; q++) {
                const OrdE o = ord[q];
                if (o.live == NONE16) {
                    ordN[np++] = o;
                    continue;
                }
                const int j = o.live;
                for (int wch = 0; wch < 2; wch++) {
                    OrdE n;
                    n.head = wch ? o.c : o.head;
                    n.live = s.newId[2 * j + wch];
                    n.c = n.live != NONE16 ? s.best[2 * j + wch] : NONE16;
                    n.bnd = 0;
                    ordN[np] = n;
                    if (n.live != NONE16) s.lpos[n.live] = (unsigned short)np;
                    np++;
                }
            }
        }
        if (threadIdx.x == 0) {
            s.nOrd = initial ? s.K : (tot >> 16);
            s.nLive = tot & 0xffff;
        }
    }
    if (threadIdx.x == 0)
        atomicAdd((unsigned long long *)&p.ctl->live[min(gen, MAX_GEN - 1)], (unsigned long long)s.liveCount);
    OrdE *t = ord;
    ord = ordN;
    ordN = t;
    return __syncthreads_or(threadIdx.x == 0 && pollErr && ld_volatile(&p.ctl->err) != 0u);
}

template <typename P> __device__ void fin_solve(const Params &p, FinSmem &s, bool isNode, int id, int &exact_o,
                                                int &exact_c) {
    int m;
    const float2 *src;
    const int *gidx = nullptr;
    long long outOff = 0;
    int gen = 0;
    Cand H = no_cand(), E = no_cand(), C = no_cand();
    long long pstart = 0;
    int tree = -1;
    if (isNode) {
        const SmallRec *R = &p.small[id];
        m = R->count;
        if (threadIdx.x == 0) atomicAdd((unsigned long long *)&p.ctl->smallPoints, (unsigned long long)m);
        const int level = R->level;
        const long long setOff = p.inst[R->inst].off;
        pstart = R->pstart;
        src = p.xy[level & 1] + pstart;  // level r was written by round r into buffer r & 1
        gidx = p.id[level & 1] + pstart;
        gen = level + 1;
        tree = R->tree;
        const float2 hp = __ldg(&p.pts[setOff + R->hIdx]), ep = __ldg(&p.pts[setOff + R->eIdx]);
        H = mk_cand(hp.x, hp.y, R->hIdx);
        E = mk_cand(ep.x, ep.y, R->eIdx);
        C.idx = R->cIdx;
    } else {
        const Inst *I = &p.inst[id];
        m = (int)I->n;
        outOff = I->off;
        src = p.pts + I->off;
    }
    if (m < 1 || m > FM) {  // guard: shared-memory tables hold FIN_MAX points
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        return;
    }
    if (threadIdx.x == 0) {
        s.cLocal = -1;
        s.nonfinite = 0;
        s.degenerate = 0;
        s.gmode = isNode ? 1 : 0;
        s.gidx = gidx;
    }
    __syncthreads();
    Ext ex;
    ex.a = ex.b = ex.bot = ex.top = no_cand();
    ex.nonfinite = 0;
    if (threadIdx.x == 0) s.nLive = m;
    for (int k = threadIdx.x; k < m; k += FIN_NT) {
        const float2 q = __ldg(&src[k]);
        s.pxy[k] = q;
        s.lst[k] = (unsigned short)k;
        if (isNode) {
            s.seg[k] = 0;
            if (__ldg(&gidx[k]) == C.idx) s.cLocal = k;
        } else {
            if (!isfinite(q.x) || !isfinite(q.y)) {
                ex.nonfinite = 1;
            } else {
                if (lex_less(q.x, q.y, k, ex.a.x, ex.a.y, ex.a.idx)) ex.a = mk_cand(q.x, q.y, k);
                if (lex_greater(q.x, q.y, k, ex.b.x, ex.b.y, ex.b.idx)) ex.b = mk_cand(q.x, q.y, k);
                if (lex_less(q.y, q.x, k, ex.bot.y, ex.bot.x, ex.bot.idx)) ex.bot = mk_cand(q.x, q.y, k);
                if (lex_greater(q.y, q.x, k, ex.top.y, ex.top.x, ex.top.idx)) ex.top = mk_cand(q.x, q.y, k);
            }
            s.seg[k] = 0;
        }
    }
    OrdE *ord = s.ordA, *ordN = s.ordB;
    if (isNode) {
        if (threadIdx.x == 0) {
            s.pxy[m] = make_float2(H.x, H.y);
            s.pxy[m + 1] = make_float2(E.x, E.y);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s.cLocal < 0) set_err(p.ctl, E_INTERNAL);
            OrdE a, b;
            a.head = (unsigned short)m;
            a.live = 0;
            a.c = (unsigned short)max(s.cLocal, 0);
            a.bnd = 0;
            b.head = (unsigned short)(m + 1);
            b.live = NONE16;
            b.c = NONE16;
            b.bnd = 0;
            ord[0] = a;
            ord[1] = b;
            s.lpos[0] = 0;
            s.nOrd = 2;
            s.S = 1;
        }
        __syncthreads();
        if (s.cLocal < 0) return;
    } else {
        // extreme points of the set (Sec. 4.2) and the initial polygon
        for (int d = 16; d >= 1; d >>= 1) {
            Ext o;
            const int l = (threadIdx.x & 31) ^ d;
            o.a = shfl_c(ex.a, l);
            o.b = shfl_c(ex.b, l);
            o.bot = shfl_c(ex.bot, l);
            o.top = shfl_c(ex.top, l);
            o.nonfinite = __shfl_sync(0xffffffffu, ex.nonfinite, l);
            ext_merge_f(ex, o);
        }
        if ((threadIdx.x & 31) == 0) s.wext[threadIdx.x >> 5] = ex;
        __syncthreads();
        if (threadIdx.x == 0) {
            Ext a = s.wext[0];
            for (int w = 1; w < FIN_NT / 32; w++) ext_merge_f(a, s.wext[w]);
            int K = 0;
            if (a.nonfinite) {
                s.nonfinite = 1;
            } else if (a.a.x == a.b.x && a.a.y == a.b.y) {
                s.degenerate = 1;
                s.poly[0] = (unsigned short)a.a.idx;
            } else {
                const bool quad = (p.mode == 0);
                s.poly[K++] = (unsigned short)a.a.idx;
                if (quad && !(a.bot.x == a.a.x && a.bot.y == a.a.y) && !(a.bot.x == a.b.x && a.bot.y == a.b.y))
                    s.poly[K++] = (unsigned short)a.bot.idx;
                s.poly[K++] = (unsigned short)a.b.idx;
                if (quad && !(a.top.x == a.a.x && a.top.y == a.a.y) && !(a.top.x == a.b.x && a.top.y == a.b.y))
                    s.poly[K++] = (unsigned short)a.top.idx;
            }
            s.K = K;
            s.S = 0;
            s.nOrd = 0;
        }
        __syncthreads();
        if (s.nonfinite) {
            if (threadIdx.x == 0) p.outCounts[id] = -2;
            return;
        }
        if (s.degenerate) {
            if (threadIdx.x == 0) {
                p.outIdx[outOff] = s.poly[0];
                p.outCounts[id] = 1;
            }
            return;
        }
        fin_generation<P>(p, s, m, true, ord, ordN, 0, false, exact_o, exact_c);
        gen = 1;
    }
    const int genLimit = gen + m + 4;  // every generation removes at least one point per live segment
    bool stop = false;
    while (s.S > 0) {
        if (stop || gen > genLimit) {  // the same in the whole block
            if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
            return;
        }
        // another block's error is polled every fourth generation (a global round trip)
        stop = fin_generation<P>(p, s, m, false, ord, ordN, gen, (gen & 3) == 0, exact_o, exact_c);
        gen++;
    }
    const int nOrd = s.nOrd;
    if (nOrd > m + (isNode ? 2 : 0)) {  // guard: the output never exceeds the problem's points
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        __syncthreads();
        return;
    }
    if (isNode) {
        // heads strictly between h (entry 0) and e (last entry)
        for (int q = 1 + threadIdx.x; q < nOrd - 1; q += FIN_NT) p.vscratch[pstart + q - 1] = __ldg(&gidx[ord[q].head]);
        if (threadIdx.x == 0) {
            p.small[id].cIdx = nOrd - 2;     // inner vertices, for the copy pass
            p.tnodes[tree].val = nOrd - 1;   // the leaf's vertices: its head and the inner ones
        }
    } else {
        for (int q = threadIdx.x; q < nOrd; q += FIN_NT) p.outIdx[outOff + q] = ord[q].head;
        if (threadIdx.x == 0) p.outCounts[id] = nOrd;
    }
    __syncthreads();
}

// Pack k: the packed segments whose weight offsets lie in [k PACK_B,
// (k + 1) PACK_B), all of one level, solved as one problem.  Every segment
// enters the CCW head list as its chord h -> e (e marked as a boundary);
// the generations then treat the live segments of all of them together, and
// each segment's inner vertices are the heads between its h and its e.
template <typename P> __device__ void fin_solve_pack(const Params &p, FinSmem &s, long long k, int &exact_o,
                                                     int &exact_c) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const long long n = p.ctl->nPack, lo = k * PACK_B, hi = lo + PACK_B;
        long long a = 0, b = n;  // first offset >= lo
        while (a < b) {
            const long long mid = (a + b) >> 1;
            if (__ldcg(&p.packOff[mid]) < lo) a = mid + 1; else b = mid;
        }
        long long c = a, d = n;  // first offset >= hi
        while (c < d) {
            const long long mid = (c + d) >> 1;
            if (__ldcg(&p.packOff[mid]) < hi) c = mid + 1; else d = mid;
        }
        s.mem0 = (int)a;
        s.nMem = (int)(c - a);
        s.gmode = 2;
        s.gidx = nullptr;
    }
    __syncthreads();
    const int a = s.mem0, nm = s.nMem;
    if (nm <= 0) return;
    if (nm > PACK_SEGS) {  // guard: the weights bound a pack to PACK_SEGS segments
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        return;
    }
    const int cnt = threadIdx.x < nm ? __ldg(&p.pack[a + threadIdx.x].count) : 0;
    int m;
    const int st = block_excl_scan<int, FIN_NT>(cnt, s.scan, m);
    const int level = __ldg(&p.pack[a].level), buf = level & 1;  // level r lives in buffer r & 1
    if (threadIdx.x < nm) s.memStart[threadIdx.x] = (unsigned short)st;
    if (threadIdx.x == 0) {
        s.memStart[nm] = (unsigned short)m;
        s.packBuf = buf;
        s.nLive = m;
        s.nOrd = 2 * nm;
        s.S = nm;
        atomicAdd((unsigned long long *)&p.ctl->smallPoints, (unsigned long long)m);
    }
    for (int i = threadIdx.x; i < nm; i += FIN_NT) s.newId[i] = NONE16;  // farthest point of segment i
    if (m < 1 || m > FM) {
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        return;
    }
    __syncthreads();
    // the points, segment by segment (one warp per segment), and the chord ends
    for (int i = wp; i < nm; i += FIN_NT / 32) {
        const SmallRec *R = &p.pack[a + i];
        const int c0 = __ldg(&R->count), ps = __ldg(&R->pstart), cIdx = __ldg(&R->cIdx), b0 = s.memStart[i];
        for (int j = lane; j < c0; j += 32) {
            s.pxy[b0 + j] = __ldg(&p.xy[buf][ps + j]);
            s.seg[b0 + j] = (unsigned short)i;
            s.lst[b0 + j] = (unsigned short)(b0 + j);
            if (__ldg(&p.id[buf][ps + j]) == cIdx) s.newId[i] = (unsigned short)(b0 + j);
        }
        if (lane == 0) {
            const long long setOff = p.inst[__ldg(&R->inst)].off;
            s.pxy[m + 2 * i] = __ldg(&p.pts[setOff + __ldg(&R->hIdx)]);
            s.pxy[m + 2 * i + 1] = __ldg(&p.pts[setOff + __ldg(&R->eIdx)]);
        }
    }
    __syncthreads();
    OrdE *ord = s.ordA, *ordN = s.ordB;
    bool ok = true;
    for (int i = threadIdx.x; i < nm; i += FIN_NT) {
        const unsigned short c = s.newId[i];
        ok &= c != NONE16;
        OrdE h, e;
        h.head = (unsigned short)(m + 2 * i);
        h.live = (unsigned short)i;
        h.c = c == NONE16 ? 0 : c;
        h.bnd = 0;
        e.head = (unsigned short)(m + 2 * i + 1);
        e.live = NONE16;
        e.c = NONE16;
        e.bnd = 1;
        ord[2 * i] = h;
        ord[2 * i + 1] = e;
        s.lpos[i] = (unsigned short)(2 * i);
    }
    if (!__syncthreads_and(ok)) {  // a segment's farthest point is one of its own points
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        return;
    }
    int gen = level + 1;
    const int genLimit = gen + m + 4;
    bool stop = false;
    while (s.S > 0) {
        if (stop || gen > genLimit) {  // the same in the whole block
            if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
            return;
        }
        // another block's error is polled every fourth generation (a global round trip)
        stop = fin_generation<P>(p, s, m, false, ord, ordN, gen, (gen & 3) == 0, exact_o, exact_c);
        gen++;
    }
    const int nOrd = s.nOrd;
    if (nOrd > m + 2 * nm) {  // guard: the output never exceeds the points and the chord ends
        if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
        __syncthreads();
        return;
    }
    // positions of every segment's h (entry after a boundary) and e (its boundary)
    unsigned short *posH = s.lpos;
    unsigned *posE = s.cnt2;
    const int per = (nOrd + FIN_NT - 1) / FIN_NT;
    const int qb = min(nOrd, (int)threadIdx.x * per), qe = min(nOrd, qb + per);
    int nb = 0;
    for (int q = qb; q < qe; q++) nb += ord[q].bnd;
    int tot;
    const int mb = block_excl_scan<int, FIN_NT>(nb, s.scan, tot);
    int mm = mb;
    for (int q = qb; q < qe; q++) {
        if (ord[q].bnd) {
            posE[mm++] = q;
        } else if (q == 0 || ord[q - 1].bnd) {
            posH[mm] = (unsigned short)q;
        }
    }
    __syncthreads();
    mm = mb;
    for (int q = qb; q < qe; q++) {
        if (ord[q].bnd) {
            mm++;
        } else if (!(q == 0 || ord[q - 1].bnd) && mm < nm) {
            const int ps = __ldg(&p.pack[a + mm].pstart);
            p.vscratch[ps + q - posH[mm] - 1] = fin_gidx(p, s, ord[q].head);
        }
    }
    for (int i = threadIdx.x; i < nm; i += FIN_NT) {
        const int inner = (int)posE[i] - (int)posH[i] - 1;
        p.pack[a + i].cIdx = inner;                       // inner vertices, for the copy pass
        p.tnodes[__ldg(&p.pack[a + i].tree)].val = inner + 1;  // the leaf's vertices
    }
    __syncthreads();
}

template <typename P> __global__ void __launch_bounds__(FIN_NT, 1) finish_kernel(Params p) {
    extern __shared__ __align__(16) unsigned char fin_smem_raw[];
    FinSmem &s = *reinterpret_cast<FinSmem *>(fin_smem_raw);
    if (p.ctl->err != 0u) return;
    const int nSI = p.ctl->nSmallInst, nSN = p.ctl->nSmall;
    const long long nPk = (p.ctl->packW + PACK_B - 1) / PACK_B;  // packs (some of them may be empty)
    int exact_o = 0, exact_c = 0;
    for (;;) {
        if (threadIdx.x == 0) s.ticket = (int)atomicAdd(&p.ctl->finTicket, 1u);
        __syncthreads();
        const long long w = s.ticket;
        __syncthreads();
        if (w >= nSI + nSN + nPk) break;
        if (w < nSI)
            fin_solve<P>(p, s, false, p.smallInst[w], exact_o, exact_c);
        else if (w < nSI + nSN)
            fin_solve<P>(p, s, true, (int)(w - nSI), exact_o, exact_c);
        else
            fin_solve_pack<P>(p, s, w - nSI - nSN, exact_o, exact_c);
    }
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

// --------------------------------------------------------------------------
// emit: output offsets of the segment tree of every big set
// --------------------------------------------------------------------------
__device__ __forceinline__ int status_of(unsigned err) {
    if (err & E_ARG) return 1;
    if (err & E_TIMEOUT) return 6;
    if (err & E_CAPACITY) return 5;
    return 7;
}

constexpr int EMIT_NT = 256;
constexpr int EMIT_CAP = 2048;  // tree nodes of a single set that the output pass stages in shared memory

// Nodes of set i in level r of the segment tree: [lo, hi).
__device__ __forceinline__ void set_level_range(const Params &p, const Inst *I, int i, int K, int r, int &lo,
                                                int &hi) {
    if (r == 0) {
        lo = I->level0;
        hi = lo + K;
        return;
    }
    const int a = __ldcg(&p.levelBase[r]), b = __ldcg(&p.levelBase[r + 1]);
    if (p.numSets == 1) {  // one set: the level is its node range
        lo = a;
        hi = b;
        return;
    }
    int l = a, h = b;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (__ldcg(&p.tnodes[mid].inst) < i) l = mid + 1; else h = mid;
    }
    int l2 = l, h2 = b;
    while (l2 < h2) {
        const int mid = (l2 + h2) >> 1;
        if (__ldcg(&p.tnodes[mid].inst) <= i) l2 = mid + 1; else h2 = mid;
    }
    lo = l;
    hi = l2;
}

// One block per set.  Bottom-up over the levels of the segment tree, every
// split segment's vertex count is the sum of its children's; top-down, the
// children of a segment at output offset o start at o and o + (vertices of
// the first child), and every leaf writes its head at its offset (the copy
// pass adds the inner vertices of small segments after it).  The levels live
// in global memory, so the tree may be of any depth.
__global__ void __launch_bounds__(EMIT_NT) emit_kernel(Params p) {
    __shared__ int child_s[EMIT_CAP], val_s[EMIT_CAP], head_s[EMIT_CAP];
    const int i = blockIdx.x;
    if (i >= p.numSets) return;
    const unsigned err = p.ctl->err;
    if (err != 0u) {
        if (threadIdx.x == 0) p.outCounts[i] = -status_of(err);
        return;
    }
    const Inst *I = &p.inst[i];
    const int kind = I->kind;
    if (kind == I_EMPTY || kind == I_SMALL) return;
    if (kind == I_NONFINITE) {
        if (threadIdx.x == 0) p.outCounts[i] = -2;
        return;
    }
    const long long off = I->off, n = I->n;
    if (kind == I_DEGEN) {
        if (threadIdx.x == 0) {
            p.outIdx[off] = I->poly[0].idx;
            p.outCounts[i] = 1;
        }
        return;
    }
    const int nL = p.ctl->nLevels;
    const int K = I->K;
    const int nN = __ldcg(&p.levelBase[nL]);
    if (p.numSets == 1 && I->level0 == 0 && nN <= EMIT_CAP) {
        // One set with a small tree (its nodes are 0 .. nN - 1): the same two
        // passes on a shared-memory copy of the tree.
        for (int q = threadIdx.x; q < nN; q += EMIT_NT) {
            const int4 t = __ldcg(reinterpret_cast<const int4 *>(&p.tnodes[q]));
            child_s[q] = t.x;
            head_s[q] = t.y;
            val_s[q] = t.z;
        }
        __syncthreads();
        for (int r = nL - 1; r >= 0; r--) {
            int lo, hi;
            set_level_range(p, I, i, K, r, lo, hi);
            for (int q = lo + threadIdx.x; q < hi; q += EMIT_NT) {
                const int c = child_s[q];
                if (c < 0) continue;
                if (c + 1 < nN) {
                    val_s[q] = val_s[c] + val_s[c + 1];
                } else {
                    set_err(p.ctl, E_INTERNAL);
                    val_s[q] = 0;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            int o = 0;
            for (int k = 0; k < K; k++) {
                const int v = val_s[k];
                val_s[k] = o;
                o += v;
            }
            p.outCounts[i] = o;
        }
        __syncthreads();
        for (int r = 0; r < nL; r++) {
            int lo, hi;
            set_level_range(p, I, i, K, r, lo, hi);
            for (int q = lo + threadIdx.x; q < hi; q += EMIT_NT) {
                const int c = child_s[q], o = val_s[q];
                if (c >= 0) {
                    if (c + 1 >= nN) continue;
                    const int a = val_s[c];
                    val_s[c] = o;
                    val_s[c + 1] = o + a;
                } else if (o >= 0 && o < n) {
                    p.outIdx[off + o] = head_s[q];
                    p.tnodes[q].val = o;  // where the copy pass puts a small segment's inner vertices
                } else {
                    set_err(p.ctl, E_INTERNAL);
                }
            }
            __syncthreads();
        }
        return;
    }
    for (int r = nL - 1; r >= 0; r--) {
        int lo, hi;
        set_level_range(p, I, i, K, r, lo, hi);
        for (int q = lo + threadIdx.x; q < hi; q += EMIT_NT) {
            TNode *N = &p.tnodes[q];
            const int c = N->child;
            if (c < 0) continue;
            if (c + 1 < nN) {
                N->val = __ldcg(&p.tnodes[c].val) + __ldcg(&p.tnodes[c + 1].val);
            } else {
                set_err(p.ctl, E_INTERNAL);
                N->val = 0;
            }
        }
        __threadfence_block();
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int o = 0;
        for (int k = 0; k < K; k++) {
            TNode *N = &p.tnodes[I->level0 + k];
            const int v = __ldcg(&N->val);
            N->val = o;
            o += v;
        }
        p.outCounts[i] = o;
    }
    __threadfence_block();
    __syncthreads();
    for (int r = 0; r < nL; r++) {
        int lo, hi;
        set_level_range(p, I, i, K, r, lo, hi);
        for (int q = lo + threadIdx.x; q < hi; q += EMIT_NT) {
            const TNode *N = &p.tnodes[q];
            const int c = N->child, o = __ldcg(&N->val);
            if (c >= 0) {
                if (c + 1 >= nN) continue;
                const int a = __ldcg(&p.tnodes[c].val);
                p.tnodes[c].val = o;
                p.tnodes[c + 1].val = o + a;
            } else if (o >= 0 && o < n) {
                p.outIdx[off + o] = N->head;
            } else {
                set_err(p.ctl, E_INTERNAL);
            }
        }
        __threadfence_block();
        __syncthreads();
    }
}

// The inner vertices of every small segment after its head.
__global__ void copy_kernel(Params p) {
    if (p.ctl->err != 0u) return;
    const int nSN = p.ctl->nSmall, nPk = p.ctl->nPack;
    for (int w = blockIdx.x; w < nSN + nPk; w += gridDim.x) {
        const SmallRec *R = w < nSN ? &p.small[w] : &p.pack[w - nSN];
        const int inner = R->cIdx, count = R->count;
        const Inst *I = &p.inst[R->inst];
        const int o = p.tnodes[R->tree].val;
        if (o < 0 || o + 1 + (long long)inner > I->n || inner > count || inner < 0) {
            if (threadIdx.x == 0) set_err(p.ctl, E_INTERNAL);
            continue;
        }
        int *dst = p.outIdx + I->off + o + 1;
        const int *src = p.vscratch + R->pstart;
        for (int k = threadIdx.x; k < inner; k += blockDim.x) dst[k] = src[k];
    }
}

// --------------------------------------------------------------------------
// predicate check kernels
// --------------------------------------------------------------------------
template <typename P> __global__ void check_orient_kernel(const float *tri, long long n, int *sign, int *cert) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float *t = tri + 6 * k;
    const Edge<P> e = make_edge<P>(t[0], t[1], t[2], t[3]);
    const Approx<P> o = orient_approx(e, t[4], t[5]);
    int used = 0;
    sign[k] = orient_sign(e, t[2], t[3], t[4], t[5], o, used);
    cert[k] = used == 0;
}

__global__ void check_dist_kernel(const float *q, long long n, int *sign) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float *t = q + 8 * k;
    const Edge<float> e = make_edge<float>(t[0], t[1], t[2], t[3]);
    const DistIv<float> a = dist_interval(orient_approx(e, t[4], t[5]));
    const DistIv<float> b = dist_interval(orient_approx(e, t[6], t[7]));
    int s;
    if (a.lo > b.hi)
        s = 1;
    else if (b.lo > a.hi)
        s = -1;
    else
        s = dist_cmp_exact(t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7]);
    sign[k] = s;
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
int finish_smem_bytes() { return (int)sizeof(FinSmem); }

cudaError_t launch_finish(const Params &p, int prec, int grid, cudaStream_t s) {
    const int bytes = finish_smem_bytes();
    cudaError_t e;
    if (prec) {
        e = cudaFuncSetAttribute(finish_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        finish_kernel<double><<<grid, FIN_NT, bytes, s>>>(p);
    } else {
        e = cudaFuncSetAttribute(finish_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        finish_kernel<float><<<grid, FIN_NT, bytes, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_emit(const Params &p, cudaStream_t s) {
    if (p.numSets > 0) emit_kernel<<<p.numSets, EMIT_NT, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_copy(const Params &p, int grid, cudaStream_t s) {
    copy_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Autotuner check: counts the entries in which a trial's output differs from
// the reference setting's (vertex counts, and every index inside a hull).  Set
// s of a batch owns out[offsets[s] ..][: counts[s]]; one set: offsets == null.
__global__ void compare_hulls_kernel(const int *out, const int *cnt, const int *ref, const int *refCnt,
                                     const long long *offsets, int numSets, long long n, unsigned *diff) {
    unsigned d = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < numSets; s += stride)
        d += cnt[s] != refCnt[s];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        int set = 0;
        long long base = 0;
        if (offsets) {  // the set holding position i: the last s with offsets[s] <= i
            int lo = 0, hi = numSets;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (offsets[mid] <= i) lo = mid; else hi = mid;
            }
            set = lo;
            base = offsets[lo];
        }
        const int c = refCnt[set];
        if (i - base < (long long)c && c > 0) d += out[i] != ref[i];
    }
    if (d) atomicAdd(diff, d);
}

cudaError_t launch_compare_hulls(const int *out, const int *cnt, const int *ref, const int *refCnt,
                                 const long long *offsets, int numSets, long long n, unsigned *diff, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(diff, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const long long work = n > numSets ? n : numSets;
    const int nb = (int)(work / 256 + 1 < 4096 ? work / 256 + 1 : 4096);
    compare_hulls_kernel<<<nb, 256, 0, s>>>(out, cnt, ref, refCnt, offsets, numSets, n, diff);
    return cudaGetLastError();
}

cudaError_t launch_check_orient(const float *tri, long long n, int prec, int *sign, int *cert, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = (int)((n + 255) / 256);
    if (prec)
        check_orient_kernel<double><<<nb, 256, 0, s>>>(tri, n, sign, cert);
    else
        check_orient_kernel<float><<<nb, 256, 0, s>>>(tri, n, sign, cert);
    return cudaGetLastError();
}

cudaError_t launch_check_dist(const float *quads, long long n, int *sign, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    check_dist_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(quads, n, sign);
    return cudaGetLastError();
}

}  // namespace qh
