// Shared definitions of the hull kernels: tunables, device-side records, the
// launch parameter block, and synchronisation helpers (bounded grid barrier,
// acquire/release flags, block scans).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qh_predicates.cuh"

namespace qh {

// ---------------------------------------------------------------------------
// Tunables
// ---------------------------------------------------------------------------
// The grid-wide kernel is compiled once per variant (threads per CTA, CTAs per
// SM); QH_NT / QH_MINB select the variant of a translation unit.
#ifndef QH_NT
#define QH_NT 256
#endif
#ifndef QH_MINB
#define QH_MINB 2
#endif
#ifndef QH_IPT
#define QH_IPT 16
#endif
constexpr int NT = QH_NT;          // threads per CTA of the grid-wide kernel
constexpr int MINB = QH_MINB;      // CTAs per SM the grid-wide kernel is built for
constexpr int NWARP = NT / 32;
constexpr int IPT = QH_IPT;        // points per thread per tile (warp-striped rows): 16 or 8
constexpr int TILE = NT * IPT;     // points per tile
constexpr int TILE_MIN = 128 * 8;  // smallest tile of the compiled variants (sizes the plans)
constexpr int FIN_NT = 512;        // threads per CTA of the block finisher
constexpr int FIN_MAX = 4096;      // largest problem the block finisher holds in shared memory
// Small segments of at most PACK_MAX points are finished many at a time: each
// weighs its points plus PACK_W, and the segments of one level whose weight
// offsets fall in the same span of PACK_B form one problem (a pack), so a pack
// holds at most FIN_MAX points and FIN_MAX / PACK_W segments.
constexpr int PACK_MAX = 1024;
constexpr int PACK_W = 16;
constexpr int PACK_B = FIN_MAX - PACK_MAX - PACK_W;
constexpr int PACK_SEGS = FIN_MAX / PACK_W;
constexpr int MAX_GEN = 512;       // generations tracked in the statistics (deeper ones add to the last)
constexpr int MAX_STAMPS = 64;     // grid-phase timestamps kept in the statistics
constexpr unsigned SPIN_LIMIT = 1u << 22;  // polls (with back-off) before a wait gives up

// device-side error bits (ctl->err)
enum : unsigned { E_TIMEOUT = 1u, E_CAPACITY = 2u, E_INTERNAL = 4u, E_ARG = 8u };

// instance kinds
enum : int { I_EMPTY = 0, I_SMALL = 1, I_BIG = 2, I_DEGEN = 3, I_NONFINITE = 4 };
// segment (node) kinds
enum : int { K_LEAF = 0, K_SMALL = 1, K_BIG = 2 };

// A point record: coordinates and index (idx < 0: none).  16-byte aligned:
// records move through global memory as single 16-byte accesses.
struct __align__(16) Cand {
    float x, y;
    int idx, pad;
};

// One point set of the batch.
struct Inst {
    long long off, n;
    long long tile0;   // first tile of this set in the grid-wide tiling (big sets)
    int kind, K;       // kind, initial polygon size (0: no segments)
    int tiles;         // tiles of this set
    int level0;        // first level-0 node
    unsigned done;     // tiles of the extreme-point pass finished (atomic)
    unsigned done0;    // tiles of the initial split finished (atomic)
    Cand poly[4];      // initial polygon, CCW, starting at the lexicographic minimum
    int iB, pad0;      // index of the rightmost vertex B in poly
    int chCount[4];    // points of each initial segment: output cursors during the split (atomic)
    Cand chC[4];       // farthest point of each initial segment
};

// A segment of the grid-wide rounds while it is active: its chord h->e, its
// points [pstart, pstart + count) of live buffer `buf`, and its farthest point
// c.  Records live in a ring of two levels (the level a round reads and the
// level it creates); the segment tree itself is kept in TNode.
struct Node {
    Cand h, e, c;
    int count, kind;
    long long pstart;
    int buf, inst, level, tree;   // tree: the segment's TNode
    int chCount[2];               // points of the two children: output cursors during the round (atomic)
    Cand chC[2];                  // farthest points of the two children
    unsigned tdone;               // tiles of the round that finished with this segment (atomic)
    int pad2[3];
};

// A node of the segment tree of the grid-wide rounds (16 bytes).  Nodes are
// stored level by level, every level grouped by set in set order.  child: the
// first of the two children of a split segment, -1 for a leaf (a segment that
// ended empty or went to the block finisher).  val: vertices of the subtree,
// then (output pass) the subtree's output offset within its set.
// Every node's head is a distinct hull vertex of its set and a split segment
// has two children, so a set of n points has at most 2n nodes.
struct TNode {
    int child, head, val, inst;
};

// A segment handed to the block finisher.  Coordinates of h and e are read
// from the input through their indices (local to the set).  cIdx is replaced
// by the number of inner vertices once the segment is finished.
struct SmallRec {
    int hIdx, eIdx, cIdx, count;
    int pstart, level, inst, tree;
};

// Extreme points of a tile: lexicographic min/max of (x, y) and of (y, x).
struct Ext {
    Cand a, b, bot, top;
    int nonfinite, pad[3];
};

// The words that waiting CTAs poll (err, bar, gen) sit on their own 128-byte
// lines, so the polls do not queue in front of the ordinary reads of the block.
struct alignas(128) Ctl {
    unsigned err;
    unsigned padErr[31];
    unsigned bar;        // grid barrier arrivals (monotonic within a launch)
    unsigned padBar[31];
    unsigned gen;        // barriers released by their leader (monotonic within a launch)
    unsigned padGen[31];
    int nBig, nSmallInst;
    int setTile;         // points per tile of the extreme-point pass and the initial split
    long long bigTiles;  // tiles over all big sets
    int S;               // big segments of the current round
    int cur;             // bigList buffer of the current round
    long long L;         // points of the current round
    long long tiles;     // tiles of the current round
    int nLevels, nNodes; // levels and TNodes of the segment tree
    int nSmall;          // small-segment queue length (segments finished one per block)
    int nPack;           // packed small-segment queue length
    long long packW;     // weight offset past the last packed segment
    unsigned finTicket;
    int rounds;          // grid-wide rounds run after the initial split
    long long bigPoints;     // points of the sets tiled by the grid-wide kernel
    long long gridRead;      // live points read by grid-wide rounds r >= 1
    long long gridWritten;   // live points written by the initial split and the grid-wide rounds
    long long smallPoints;   // points handled by the block finisher
    int gens;            // generations run (max over sets)
    long long live[MAX_GEN];
    unsigned long long exactOrient, exactCmp;
    unsigned long long tphase[MAX_STAMPS];  // %globaltimer at the kernel start and after each grid barrier
};

struct Params {
    const float2 *pts;
    const long long *offsets;  // nullptr: one set of nSingle points
    long long nSingle;
    int numSets;
    int mode;                  // 0 = quadrilateral, 1 = chord
    long long ncap;            // plan capacity in points
    int *outIdx;
    int *outCounts;
    float2 *xy[2];             // live points, 2 * ncap each
    int *id[2];
    int *vscratch;             // inner vertices of small segments, 2 * ncap
    Cand *tbest;               // per tile and slot: the tile's exact farthest point (4 per tile)
    Ext *text;                 // extreme-point partials per tile
    long long maxTiles;
    Inst *inst;
    int *bigInst, *smallInst;
    long long *bigTilePrefix;  // exclusive prefix of tiles over big sets (nBig + 1)
    Node *nodes;               // ring of two levels of active segments, slotCap each
    int slotCap;
    TNode *tnodes;             // segment tree
    int maxTNodes;
    int *levelBase;            // first TNode of every level (maxLevels + 1 entries)
    int maxLevels;
    SmallRec *small;           // small-segment queue (one block each)
    SmallRec *pack;            // small segments finished in packs, in weight-offset order
    long long *packOff;        // their weight offsets (non-decreasing)
    int maxSmall;
    unsigned spinLimit;        // polls of a grid-barrier wait before it gives up
    int *bigList[2];
    long long *vstart[2];      // exclusive prefix of big-segment sizes (S + 1)
    int maxBig;
    Ctl *ctl;
    int cut;                   // small-segment cutover
};

// ---------------------------------------------------------------------------
// Memory-ordering helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(volatile const unsigned *)p; }
// Counter arrivals.  Release: the caller's writes, and those of its CTA ordered
// before it by a CTA barrier, become visible no later than the increment.
// Acquire (acq_rel): the caller also sees everything released by the earlier
// increments of the same counter.
__device__ __forceinline__ unsigned atom_add_release(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ Cand ldcg_cand(const Cand *p) {
    int4 v = __ldcg(reinterpret_cast<const int4 *>(p));
    Cand c;
    c.x = __int_as_float(v.x);
    c.y = __int_as_float(v.y);
    c.idx = v.z;
    c.pad = v.w;
    return c;
}
__device__ __forceinline__ void stcg_cand(Cand *p, const Cand &c) {
    __stcg(reinterpret_cast<int4 *>(p), make_int4(__float_as_int(c.x), __float_as_int(c.y), c.idx, c.pad));
}

__device__ __forceinline__ Cand no_cand() {
    Cand c;
    c.x = 0.f;
    c.y = 0.f;
    c.idx = -1;
    c.pad = 0;
    return c;
}
__device__ __forceinline__ Cand mk_cand(float x, float y, int idx) {
    Cand c;
    c.x = x;
    c.y = y;
    c.idx = idx;
    c.pad = 0;
    return c;
}

__device__ __forceinline__ void set_err(Ctl *ctl, unsigned bits) { atomicOr(&ctl->err, bits); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Phase timestamp, written by CTA 0 after a grid barrier.
__device__ __forceinline__ void stamp(Ctl *ctl, int k) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && k < MAX_STAMPS) ctl->tphase[k] = global_ns();
}

// Grid-wide barrier for a cooperative launch.  Every CTA increments `bar`
// once per barrier; phase counts barriers passed by this CTA.  The wait is
// bounded: on timeout (or when another CTA reported an error) the error bit is
// set and false is returned so the kernel can leave.
__device__ __forceinline__ bool grid_sync(Ctl *ctl, unsigned &phase, unsigned limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        phase++;
        const unsigned target = phase * gridDim.x;
        atom_add_release(&ctl->bar, 1u);
        unsigned it = 0, ns = 32;
        int ok = 1;
        while (ld_acquire(&ctl->bar) < target) {
            if ((it & 7u) == 0u && ld_volatile(&ctl->err) != 0u) {
                ok = 0;
                break;
            }
            if (++it > limit) {
                set_err(ctl, E_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(ns);  // back-off: 32 ns doubling to 256 ns
            ns = ns < 256u ? 2u * ns : ns;
        }
        if (ld_volatile(&ctl->err) != 0u) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide barrier with a serial step: the last CTA to arrive (the leader)
// returns 1 in all its threads, runs the step and calls grid_release; the
// other CTAs wait for that release and return 0.  -1: an error was reported
// or the wait timed out (the error bit is set).  One atomic round trip
// instead of a separate "last CTA" count followed by a barrier.
__device__ __forceinline__ int grid_arrive(Ctl *ctl, unsigned &phase, unsigned limit) {
    __shared__ int s_role;
    __syncthreads();
    if (threadIdx.x == 0) {
        phase++;
        const unsigned d = atom_add_acq_rel(&ctl->bar, 1u);  // the leader acquires every arrival's writes
        int role = 0;
        if (d == phase * gridDim.x - 1u) {
            role = 1;
        } else {
            unsigned it = 0, ns = 32;
            while (ld_acquire(&ctl->gen) < phase) {
                if ((it & 7u) == 0u && ld_volatile(&ctl->err) != 0u) {
                    role = -1;
                    break;
                }
                if (++it > limit) {
                    set_err(ctl, E_TIMEOUT);
                    role = -1;
                    break;
                }
                __nanosleep(ns);
                ns = ns < 256u ? 2u * ns : ns;
            }
        }
        if (ld_volatile(&ctl->err) != 0u) role = -1;
        s_role = role;
    }
    __syncthreads();
    return s_role;
}
// The leader's release (after its serial step); false when an error was reported.
__device__ __forceinline__ bool grid_release(Ctl *ctl, unsigned phase) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        st_release(&ctl->gen, phase);
        s_ok = ld_volatile(&ctl->err) == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Block-wide scans (exclusive), NTHREADS threads, scratch of NTHREADS/32 + 1 entries.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <typename T, int NTHREADS>
__device__ __forceinline__ T block_excl_scan(T v, T *scratch, T &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = NTHREADS / 32;
    T inc = warp_incl_scan(v);
    if (lane == 31) scratch[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < NW ? scratch[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < NW) scratch[lane] = si - s;
        if (lane == NW - 1) scratch[NW] = si;
    }
    __syncthreads();
    T r = scratch[w] + inc - v;
    total = scratch[NW];
    __syncthreads();
    return r;
}

// The same without the closing barrier, for callers that pass a CTA barrier
// before the scratch is written again.
template <typename T, int NTHREADS>
__device__ __forceinline__ T block_excl_scan_open(T v, T *scratch, T &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = NTHREADS / 32;
    T inc = warp_incl_scan(v);
    if (lane == 31) scratch[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < NW ? scratch[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < NW) scratch[lane] = si - s;
        if (lane == NW - 1) scratch[NW] = si;
    }
    __syncthreads();
    total = scratch[NW];
    return scratch[w] + inc - v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Orderable 32-bit key of a float: unsigned comparison matches float order.
__device__ __forceinline__ unsigned fkey(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ unsigned pkey(float f) { return fkey(f); }
__device__ __forceinline__ unsigned pkey(double d) { return fkey(__double2float_rd(d)); }
// Key of an upper bound (rounded up to float).
__device__ __forceinline__ unsigned pkey_up(float f) { return fkey(f); }
__device__ __forceinline__ unsigned pkey_up(double d) { return fkey(__double2float_ru(d)); }

// Host launchers (defined in the .cu files).
// Grid-wide kernel variants (threads per CTA x points per thread), each
// compiled in its own namespace.
#define QH_DECLARE_VARIANT(ns)                                                      \
    namespace ns {                                                                  \
    cudaError_t launch_rounds(const Params &p, int prec, int grid, cudaStream_t s); \
    int rounds_max_ctas_per_sm(int prec);                                           \
    }
QH_DECLARE_VARIANT(v256)
QH_DECLARE_VARIANT(v256i8)
QH_DECLARE_VARIANT(v128)
QH_DECLARE_VARIANT(v128i8)
#undef QH_DECLARE_VARIANT
struct RoundsVariant {
    int threads, ipt, tile;
    cudaError_t (*launch)(const Params &, int, int, cudaStream_t);
    int (*max_ctas_per_sm)(int);
};
constexpr int NUM_ROUNDS_VARIANTS = 4;
inline const RoundsVariant &rounds_variant(int v) {
    static const RoundsVariant table[NUM_ROUNDS_VARIANTS] = {
        {256, 16, 256 * 16, &v256::launch_rounds, &v256::rounds_max_ctas_per_sm},
        {256, 8, 256 * 8, &v256i8::launch_rounds, &v256i8::rounds_max_ctas_per_sm},
        {128, 16, 128 * 16, &v128::launch_rounds, &v128::rounds_max_ctas_per_sm},
        {128, 8, 128 * 8, &v128i8::launch_rounds, &v128i8::rounds_max_ctas_per_sm}};
    return table[v];
}
cudaError_t launch_finish(const Params &p, int prec, int grid, cudaStream_t s);
int finish_smem_bytes();
cudaError_t launch_emit(const Params &p, cudaStream_t s);
cudaError_t launch_copy(const Params &p, int grid, cudaStream_t s);
cudaError_t launch_compare_hulls(const int *out, const int *cnt, const int *ref, const int *refCnt,
                                 const long long *offsets, int numSets, long long n, unsigned *diff, cudaStream_t s);
cudaError_t launch_check_orient(const float *tri, long long n, int prec, int *sign, int *cert, cudaStream_t s);
cudaError_t launch_check_dist(const float *quads, long long n, int *sign, cudaStream_t s);

}  // namespace qh
