// C ABI of the hull library: plans (device scratch), the launch sequence and
// statistics.  See include/qh.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/qh.h"
#include "qh_internal.cuh"
#include "qh_sorted.cuh"

using namespace qh;

struct qh_plan_s {
    int device = 0;
    long long ncap = 0;
    int maxSets = 0;
    unsigned flags = 0;
    int cut = FIN_MAX;   // small-segment cutover (>= the tile of the variant)
    int variant = 0;     // grid-wide kernel variant (rounds_variant)
    int timing = 0;
    int ctasPerSm = 0;
    int numSMs = 0;
    // device scratch
    float2 *xy[2] = {nullptr, nullptr};
    int *id[2] = {nullptr, nullptr};
    int *vscratch = nullptr;
    Cand *tbest = nullptr;
    Ext *text = nullptr;
    long long maxTiles = 0;
    Inst *inst = nullptr;
    int *bigInst = nullptr, *smallInst = nullptr;
    long long *bigTilePrefix = nullptr;
    Node *nodes = nullptr;  // ring of two levels
    int slotCap = 0;
    TNode *tnodes = nullptr;
    int maxTNodes = 0;
    int *levelBase = nullptr;
    int maxLevels = 0;
    SmallRec *small = nullptr;
    SmallRec *pack = nullptr;
    long long *packOff = nullptr;
    int maxSmall = 0;
    int *bigList[2] = {nullptr, nullptr};
    long long *vstart[2] = {nullptr, nullptr};
    int maxBig = 0;
    Ctl *ctl = nullptr;
    // debug limits (0: defaults)
    unsigned dbgSpin = 0;
    int dbgTNodes = 0;
    // host side
    Ctl *hctl = nullptr;  // pinned
    cudaStream_t last = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool evRecorded = false;
    int lastSets = 0;
    // end-to-end staging
    float *stIn = nullptr;
    int *stOut = nullptr;
    int *stCnt = nullptr;     // 8 counters (see qh_hull2d_host)
    long long stCap = 0;
    // overlapped host path: side copy stream, its events, and the merge of the two halves' hulls
    cudaStream_t cpStream = nullptr;
    cudaEvent_t cpEv[2] = {nullptr, nullptr};
    float2 *mPts = nullptr;     // vertices of the first half's hull
    int *mOut = nullptr;        // hull of those vertices and the second half (local indices)
    int *fOut = nullptr;        // final indices
    long long *mOff = nullptr;  // that set's range in the staging buffer
    // scratch of the x-sorted form, allocated by its first call
    sx::SortedWs *sorted = nullptr;
};

namespace {

qh_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return QH_OK;
    if (e == cudaErrorMemoryAllocation) return QH_ERR_OOM;
    return QH_ERR_CUDA;
}

template <typename T> cudaError_t dalloc(T **p, long long count) {
    if (count < 1) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)count);
}

void plan_free(qh_plan p) {
    if (!p) return;
    cudaFree(p->xy[0]);
    cudaFree(p->xy[1]);
    cudaFree(p->id[0]);
    cudaFree(p->id[1]);
    cudaFree(p->vscratch);
    cudaFree(p->tbest);
    cudaFree(p->text);
    cudaFree(p->inst);
    cudaFree(p->bigInst);
    cudaFree(p->smallInst);
    cudaFree(p->bigTilePrefix);
    cudaFree(p->nodes);
    cudaFree(p->tnodes);
    cudaFree(p->levelBase);
    cudaFree(p->small);
    cudaFree(p->pack);
    cudaFree(p->packOff);
    cudaFree(p->bigList[0]);
    cudaFree(p->bigList[1]);
    cudaFree(p->vstart[0]);
    cudaFree(p->vstart[1]);
    cudaFree(p->ctl);
    cudaFree(p->stIn);
    cudaFree(p->stOut);
    cudaFree(p->stCnt);
    cudaFree(p->mPts);
    cudaFree(p->mOut);
    cudaFree(p->fOut);
    cudaFree(p->mOff);
    for (auto &e : p->cpEv)
        if (e) cudaEventDestroy(e);
    if (p->cpStream) cudaStreamDestroy(p->cpStream);
    if (p->sorted) {
        sx::sorted_free(*p->sorted);
        delete p->sorted;
    }
    if (p->hctl) cudaFreeHost(p->hctl);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    delete p;
}

qh_status plan_alloc(qh_plan p) {
    const long long N = p->ncap;
    cudaError_t e = cudaSuccess;
#define QH_ALLOC(ptr, cnt)                   \
    do {                                     \
        e = dalloc(&(ptr), (cnt));           \
        if (e != cudaSuccess) return cuda_status(e); \
    } while (0)
    QH_ALLOC(p->xy[0], 2 * N);
    QH_ALLOC(p->xy[1], 2 * N);
    QH_ALLOC(p->id[0], 2 * N);
    QH_ALLOC(p->id[1], 2 * N);
    QH_ALLOC(p->vscratch, 2 * N);
    p->maxTiles = N / TILE_MIN + p->maxSets + 16;
    QH_ALLOC(p->tbest, 4 * p->maxTiles);
    QH_ALLOC(p->text, p->maxTiles);
    QH_ALLOC(p->inst, p->maxSets);
    QH_ALLOC(p->bigInst, p->maxSets + 1);
    QH_ALLOC(p->smallInst, p->maxSets + 1);
    QH_ALLOC(p->bigTilePrefix, p->maxSets + 2);
    // Every big segment holds more than a tile of points (the smallest tile of
    // the variants), so a level has at most N / TILE_MIN of them.
    p->maxBig = (int)(N / TILE_MIN + 16);
    long long bigSets = N / (FIN_MAX + 1) + 1;
    if (bigSets > p->maxSets) bigSets = p->maxSets;
    // Ring slot: the K <= 4 initial segments of every big set, or the two
    // children of every big segment of a level.
    const long long slot = (4 * bigSets > 2ll * p->maxBig ? 4 * bigSets : 2ll * p->maxBig) + 16;
    p->slotCap = (int)slot;
    QH_ALLOC(p->nodes, 2 * slot);
    // Segment tree: every node's head is a distinct hull vertex of its set, so
    // a set of n points has at most n leaves and n - 1 split segments; a split
    // segment loses at least its farthest point, so there are fewer than N
    // levels; every small segment holds a point.  No input of at most N points
    // exceeds these tables.
    p->maxTNodes = (int)(2 * N + 64);
    p->maxLevels = (int)(N + 2);
    p->maxSmall = (int)(N + 64);
    QH_ALLOC(p->tnodes, p->maxTNodes);
    QH_ALLOC(p->levelBase, p->maxLevels + 2);
    QH_ALLOC(p->small, p->maxSmall);
    QH_ALLOC(p->pack, p->maxSmall);
    QH_ALLOC(p->packOff, p->maxSmall);
    QH_ALLOC(p->bigList[0], p->maxBig + 1);
    QH_ALLOC(p->bigList[1], p->maxBig + 1);
    QH_ALLOC(p->vstart[0], p->maxBig + 2);
    QH_ALLOC(p->vstart[1], p->maxBig + 2);
    QH_ALLOC(p->ctl, 1);
#undef QH_ALLOC
    e = cudaMallocHost((void **)&p->hctl, sizeof(Ctl));
    if (e != cudaSuccess) return cuda_status(e);
    memset(p->hctl, 0, sizeof(Ctl));
    for (auto &ev : p->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return QH_OK;
}

Params make_params(qh_plan pl, const float *points, const long long *offsets, long long nSingle, int numSets,
                   int *outIdx, int *outCounts) {
    Params p;
    memset(&p, 0, sizeof(p));
    p.pts = reinterpret_cast<const float2 *>(points);
    p.offsets = offsets;
    p.nSingle = nSingle;
    p.numSets = numSets;
    p.mode = (pl->flags & QH_MODE_CHORD) ? 1 : 0;
    p.ncap = pl->ncap;
    p.outIdx = outIdx;
    p.outCounts = outCounts;
    for (int b = 0; b < 2; b++) {
        p.xy[b] = pl->xy[b];
        p.id[b] = pl->id[b];
        p.bigList[b] = pl->bigList[b];
        p.vstart[b] = pl->vstart[b];
    }
    p.vscratch = pl->vscratch;
    p.tbest = pl->tbest;
    p.text = pl->text;
    p.maxTiles = pl->maxTiles;
    p.inst = pl->inst;
    p.bigInst = pl->bigInst;
    p.smallInst = pl->smallInst;
    p.bigTilePrefix = pl->bigTilePrefix;
    p.nodes = pl->nodes;
    p.slotCap = pl->slotCap;
    p.tnodes = pl->tnodes;
    p.maxTNodes = pl->dbgTNodes > 0 && pl->dbgTNodes < pl->maxTNodes ? pl->dbgTNodes : pl->maxTNodes;
    p.levelBase = pl->levelBase;
    p.maxLevels = pl->maxLevels;
    p.small = pl->small;
    p.pack = pl->pack;
    p.packOff = pl->packOff;
    p.maxSmall = pl->maxSmall;
    p.spinLimit = pl->dbgSpin > 0 ? pl->dbgSpin : SPIN_LIMIT;
    p.maxBig = pl->maxBig;
    p.ctl = pl->ctl;
    p.cut = pl->cut;
    return p;
}

qh_status run(qh_plan pl, const float *points, const long long *offsets, long long nSingle, int numSets,
              int *outIdx, int *outCounts, cudaStream_t s) {
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != pl->device) return QH_ERR_INVALID_ARG;
    const int prec = (pl->flags & QH_PREC_F64) ? 1 : 0;
    Params p = make_params(pl, points, offsets, nSingle, numSets, outIdx, outCounts);
    cudaError_t e = cudaMemsetAsync(pl->ctl, 0, sizeof(Ctl), s);
    if (e != cudaSuccess) return cuda_status(e);
    const bool tm = pl->timing != 0;
    if (tm) cudaEventRecord(pl->ev[0], s);
    const RoundsVariant &V = rounds_variant(pl->variant);
    int per = V.max_ctas_per_sm(prec);
    if (pl->ctasPerSm > 0 && pl->ctasPerSm < per) per = pl->ctasPerSm;
    // automatic: a single set of at most 2^19 points runs one CTA per SM -- its
    // phases are short, and fewer CTAs shorten every grid barrier and merge
    // (square-100K 161 -> 154 us in FP32, 215 -> 197 us in FP64; at 2M points
    // the full occupancy is faster again, and at 1M about even)
    if (pl->ctasPerSm == 0 && !offsets && nSingle <= (1ll << 19)) per = 1;
    if (per < 1) return QH_ERR_CUDA;
    e = V.launch(p, prec, pl->numSMs * per, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (tm) cudaEventRecord(pl->ev[1], s);
    e = launch_finish(p, prec, pl->numSMs, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (tm) cudaEventRecord(pl->ev[2], s);
    e = launch_emit(p, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (tm) cudaEventRecord(pl->ev[3], s);
    e = launch_copy(p, pl->numSMs * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (tm) cudaEventRecord(pl->ev[4], s);
    pl->evRecorded = tm;
    pl->last = s;
    pl->lastSets = numSets;
    return QH_OK;
}

// The overlapped host path hulls the first half of a large set while the
// second half is still being copied, then hulls the first half's vertices
// together with the second half: every vertex of the whole hull is a vertex of
// the first half's hull or a point of the second half.  The first half's
// vertices are placed right before the second half, so their indices (all
// below the second half's) come first and coordinate duplicates still resolve
// to the lowest input index.
__global__ void merge_gather_kernel(const float2 *pts, long long n1, long long n, const int *hull1, const int *c1p,
                                    float2 *mPts, long long *mOff, int *mSt) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c1 = *c1p;
    if (c1 < 0) {
        if (gt == 0) {
            mOff[0] = 0;
            mOff[1] = 0;
            *mSt = c1;
        }
        return;
    }
    for (long long k = gt; k < c1; k += (long long)gridDim.x * blockDim.x) mPts[k] = pts[hull1[k]];
    if (gt == 0) {
        mOff[0] = n1 - c1;
        mOff[1] = n;
        *mSt = 0;
    }
}

// The gathered vertices into the places right before the second half (a
// separate launch: the gather reads the first half where this one writes).
__global__ void merge_place_kernel(float2 *pts, long long n1, const int *c1p, const float2 *mPts) {
    const int c1 = *c1p;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < c1; k += (long long)gridDim.x * blockDim.x)
        pts[n1 - c1 + k] = mPts[k];
}

__global__ void merge_map_kernel(long long n1, const int *hull1, const int *c1p, const int *mOut, const int *mCnt,
                                 const int *mSt, int *out, int *count) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int st = *mSt, h = *mCnt, c1 = *c1p;
    if (st < 0 || h < 0) {
        if (gt == 0) *count = st < 0 ? st : h;
        return;
    }
    const int *res = mOut + (n1 - c1);  // the merged set's output starts at its offset
    for (long long k = gt; k < h; k += (long long)gridDim.x * blockDim.x) {
        const int j = res[k];
        out[k] = j < c1 ? hull1[j] : (int)(n1 + (j - c1));
    }
    if (gt == 0) *count = h;
}

struct DefaultPlans {
    std::mutex mu;
    qh_plan plan[64] = {};
};
DefaultPlans &defaults() {
    static DefaultPlans d;
    return d;
}

}  // namespace

extern "C" {

int32_t qh_version(void) { return 10000; }

const char *qh_status_string(qh_status s) {
    switch (s) {
    case QH_OK: return "ok";
    case QH_ERR_INVALID_ARG: return "invalid argument";
    case QH_ERR_NONFINITE: return "non-finite input coordinate";
    case QH_ERR_CUDA: return "CUDA runtime error";
    case QH_ERR_OOM: return "out of device memory";
    case QH_ERR_CAPACITY: return "capacity exceeded";
    case QH_ERR_TIMEOUT: return "device-side wait timed out";
    case QH_ERR_INTERNAL: return "internal error";
    case QH_ERR_UNSUPPORTED: return "unsupported in this context";
    }
    return "unknown status";
}

qh_status qh_plan_create(int64_t max_points, int32_t max_sets, uint32_t flags, qh_plan *out) {
    if (!out || max_points < 1 || max_sets < 1 || (flags & ~3u)) return QH_ERR_INVALID_ARG;
    if (max_points > QH_MAX_PLAN_POINTS) return QH_ERR_CAPACITY;  // int32 indices, nested ranges 2x, tree 2x
    *out = nullptr;
    qh_plan p = new (std::nothrow) qh_plan_s();
    if (!p) return QH_ERR_OOM;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->numSMs, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_status(e);
    }
    p->ncap = max_points;
    p->maxSets = max_sets;
    p->flags = flags;
    p->cut = FIN_MAX;
    qh_status st = plan_alloc(p);
    if (st != QH_OK) {
        plan_free(p);
        return st;
    }
    *out = p;
    return QH_OK;
}

qh_status qh_plan_destroy(qh_plan plan) {
    if (!plan) return QH_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    return QH_OK;
}

qh_status qh_plan_set_flags(qh_plan plan, uint32_t flags) {
    if (!plan || (flags & ~3u)) return QH_ERR_INVALID_ARG;
    plan->flags = flags;
    return QH_OK;
}

qh_status qh_plan_set_tuning(qh_plan plan, int32_t cutover, int32_t timing, int32_t grid_ctas_per_sm) {
    if (!plan || grid_ctas_per_sm < 0) return QH_ERR_INVALID_ARG;
    if (cutover < rounds_variant(plan->variant).tile || cutover > FIN_MAX) return QH_ERR_INVALID_ARG;
    plan->cut = cutover;
    plan->timing = timing ? 1 : 0;
    plan->ctasPerSm = grid_ctas_per_sm;
    return QH_OK;
}

namespace {
qh_status select_variant(qh_plan plan, int threads, int ipt) {
    for (int v = 0; v < NUM_ROUNDS_VARIANTS; v++)
        if (rounds_variant(v).threads == threads && rounds_variant(v).ipt == ipt) {
            plan->variant = v;
            if (plan->cut < rounds_variant(v).tile) plan->cut = rounds_variant(v).tile;
            plan->ctasPerSm = 0;
            return QH_OK;
        }
    return QH_ERR_INVALID_ARG;
}
}  // namespace

qh_status qh_plan_set_block(qh_plan plan, int32_t threads_per_block) {
    if (!plan) return QH_ERR_INVALID_ARG;
    return select_variant(plan, threads_per_block, rounds_variant(plan->variant).ipt);
}

qh_status qh_plan_set_items_per_thread(qh_plan plan, int32_t items_per_thread) {
    if (!plan) return QH_ERR_INVALID_ARG;
    return select_variant(plan, rounds_variant(plan->variant).threads, items_per_thread);
}

qh_status qh_plan_set_debug(qh_plan plan, uint32_t spin_limit, int32_t max_tree_nodes) {
    if (!plan || max_tree_nodes < 0) return QH_ERR_INVALID_ARG;
    plan->dbgSpin = spin_limit;
    plan->dbgTNodes = max_tree_nodes;
    return QH_OK;
}

qh_status qh_plan_get_tuning(qh_plan plan, int32_t *threads_per_block, int32_t *items_per_thread, int32_t *cutover,
                             int32_t *grid_ctas_per_sm) {
    if (!plan) return QH_ERR_INVALID_ARG;
    const RoundsVariant &V = rounds_variant(plan->variant);
    if (threads_per_block) *threads_per_block = V.threads;
    if (items_per_thread) *items_per_thread = V.ipt;
    if (cutover) *cutover = plan->cut;
    if (grid_ctas_per_sm) {
        const int mx = V.max_ctas_per_sm((plan->flags & QH_PREC_F64) ? 1 : 0);
        *grid_ctas_per_sm = (plan->ctasPerSm > 0 && plan->ctasPerSm < mx) ? plan->ctasPerSm : mx;
    }
    return QH_OK;
}

// Time every candidate setting (grid-kernel variant, grid CTAs per SM, small-segment cutover) on the
// caller's input and keep the fastest in the plan.  The outputs are written by every trial; after the
// call they hold the result of the last one, which is the same hull (every setting is exact).
qh_status qh_plan_autotune(qh_plan plan, const float *points, const int64_t *offsets, int32_t num_sets, int64_t n,
                           int32_t *out_idx, int32_t *out_counts, int32_t reps, qh_stream_t stream) {
    if (!plan || reps < 1 || reps > 64) return QH_ERR_INVALID_ARG;
    if (offsets && num_sets <= 0) return num_sets == 0 ? QH_OK : QH_ERR_INVALID_ARG;
    if (!out_counts || (!offsets && n < 0)) return QH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    auto call = [&]() -> qh_status {
        return offsets ? qh_hull2d_batched(plan, points, offsets, num_sets, out_idx, out_counts, stream)
                       : qh_hull2d_p(plan, points, n, out_idx, out_counts, stream);
    };
    const int sets = offsets ? num_sets : 1;
    long long total = n;
    if (offsets) {
        int64_t last = 0;
        cudaError_t e = cudaMemcpyAsync(&last, offsets + num_sets, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        total = last;
    }
    // The reference: the plan's setting before tuning.  Every candidate's output
    // must equal it (the hull is unique); a candidate that differs is never chosen.
    int *ref = nullptr, *refCnt = nullptr;
    unsigned *diff = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto release = [&]() {
        cudaFree(ref);
        cudaFree(refCnt);
        cudaFree(diff);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    };
    cudaError_t e = cudaMalloc((void **)&ref, sizeof(int) * (size_t)(total > 0 ? total : 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&refCnt, sizeof(int) * (size_t)sets);
    if (e == cudaSuccess) e = cudaMalloc((void **)&diff, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        release();
        return cuda_status(e);
    }
    const int saveTiming = plan->timing;
    plan->timing = 0;
    qh_status st = call();
    if (st == QH_OK && total > 0)
        e = cudaMemcpyAsync(ref, out_idx, sizeof(int) * (size_t)total, cudaMemcpyDeviceToDevice, s);
    if (st == QH_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(refCnt, out_counts, sizeof(int) * (size_t)sets, cudaMemcpyDeviceToDevice, s);
    if (st == QH_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st == QH_OK && e != cudaSuccess) st = cuda_status(e);
    float best = -1.f;
    int bestV = plan->variant, bestCut = plan->cut, bestCtas = plan->ctasPerSm;
    int rejected = 0;
    const int prec = (plan->flags & QH_PREC_F64) ? 1 : 0;
    for (int v = 0; v < NUM_ROUNDS_VARIANTS && st == QH_OK; v++) {
        const RoundsVariant &V = rounds_variant(v);
        const int mx = V.max_ctas_per_sm(prec);
        for (int ctas = mx; ctas >= 1 && ctas >= mx / 2 && st == QH_OK; ctas--) {
            for (int cut = V.tile; cut <= FIN_MAX && st == QH_OK; cut += 1024) {
                plan->variant = v;
                plan->ctasPerSm = ctas;
                plan->cut = cut;
                st = call();  // warm-up (first use of the variant, caches), then the check
                unsigned d = 0u;
                if (st == QH_OK) {
                    e = launch_compare_hulls(out_idx, out_counts, ref, refCnt,
                                             reinterpret_cast<const long long *>(offsets), sets, total, diff, s);
                    if (e == cudaSuccess) e = cudaMemcpyAsync(&d, diff, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) st = cuda_status(e);
                }
                if (st != QH_OK) break;
                if (d != 0u) {
                    rejected++;
                    continue;
                }
                float tot = 0.f;
                for (int r = 0; r < reps && st == QH_OK; r++) {
                    cudaEventRecord(a, s);
                    st = call();
                    cudaEventRecord(b, s);
                    if (cudaEventSynchronize(b) != cudaSuccess) st = QH_ERR_CUDA;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, b);
                    tot += ms;
                }
                if (st == QH_OK && (best < 0.f || tot < best)) {
                    best = tot;
                    bestV = v;
                    bestCut = cut;
                    bestCtas = ctas;
                }
            }
        }
    }
    plan->variant = bestV;
    plan->cut = bestCut;
    plan->ctasPerSm = bestCtas;
    plan->timing = saveTiming;
    release();
    if (st != QH_OK) return st;
    return rejected ? QH_ERR_INTERNAL : QH_OK;
}

qh_status qh_hull2d_p(qh_plan plan, const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                      qh_stream_t stream) {
    if (!plan || n < 0 || !out_count || (n > 0 && (!points || !out_idx))) return QH_ERR_INVALID_ARG;
    if (((uintptr_t)points & 7u) != 0) return QH_ERR_INVALID_ARG;
    if (n > plan->ncap) return QH_ERR_CAPACITY;
    return run(plan, points, nullptr, n, 1, out_idx, out_count, (cudaStream_t)stream);
}

qh_status qh_hull2d(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count, qh_stream_t stream) {
    if (n < 0 || !out_count || (n > 0 && (!points || !out_idx))) return QH_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return QH_ERR_INVALID_ARG;
    DefaultPlans &d = defaults();
    std::lock_guard<std::mutex> lock(d.mu);
    qh_plan &pl = d.plan[dev];
    if (!pl || pl->ncap < n) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing((cudaStream_t)stream, &cs);
        if (cs != cudaStreamCaptureStatusNone) return QH_ERR_UNSUPPORTED;
        long long cap = n < (1 << 20) ? (1 << 20) : n;
        if (pl) {
            if (cap < 2 * pl->ncap) cap = 2 * pl->ncap;
            if (cap > (1ll << 30)) cap = n;
            qh_plan_destroy(pl);
            pl = nullptr;
        }
        qh_status st = qh_plan_create(cap, 1, QH_MODE_QUAD | QH_PREC_F32, &pl);
        if (st != QH_OK) {
            pl = nullptr;
            return st;
        }
    }
    return qh_hull2d_p(pl, points, n, out_idx, out_count, stream);
}

qh_status qh_hull2d_batched(qh_plan plan, const float *points, const int64_t *offsets, int32_t num_sets,
                            int32_t *out_idx, int32_t *out_counts, qh_stream_t stream) {
    if (!plan || num_sets < 0 || (num_sets > 0 && (!offsets || !out_counts || !points || !out_idx)))
        return QH_ERR_INVALID_ARG;
    if (((uintptr_t)points & 7u) != 0) return QH_ERR_INVALID_ARG;
    if (num_sets > plan->maxSets) return QH_ERR_CAPACITY;
    if (num_sets == 0) return QH_OK;
    return run(plan, points, reinterpret_cast<const long long *>(offsets), 0, num_sets, out_idx, out_counts,
               (cudaStream_t)stream);
}

qh_status qh_hull2d_sorted(qh_plan plan, const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                           qh_stream_t stream) {
    if (!plan || n < 0 || !out_count || (n > 0 && (!points || !out_idx))) return QH_ERR_INVALID_ARG;
    if (((uintptr_t)points & 7u) != 0) return QH_ERR_INVALID_ARG;
    if (n > plan->ncap) return QH_ERR_CAPACITY;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->device) return QH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_status(e);
    if (cs != cudaStreamCaptureStatusNone) return QH_ERR_UNSUPPORTED;  // the host reads the end flag
    if (!plan->sorted) {
        sx::SortedWs *w = new (std::nothrow) sx::SortedWs();
        if (!w) return QH_ERR_OOM;
        e = sx::sorted_alloc(*w, plan->ncap);
        if (e != cudaSuccess) {
            sx::sorted_free(*w);
            delete w;
            return cuda_status(e);
        }
        plan->sorted = w;
    }
    plan->last = s;
    plan->lastSets = 1;
    plan->evRecorded = false;
    if (n == 0) {
        e = cudaMemsetAsync(plan->ctl, 0, sizeof(Ctl), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(out_count, 0, sizeof(int32_t), s);
        return cuda_status(e);
    }
    const bool tm = plan->timing != 0;
    const int st = sx::sorted_run(*plan->sorted, reinterpret_cast<const float2 *>(points), (int)n,
                                  (plan->flags & QH_MODE_CHORD) ? 1 : 0, (plan->flags & QH_PREC_F64) ? 1 : 0, out_idx,
                                  out_count, plan->ctl, plan->numSMs, s, tm ? plan->ev : nullptr);
    plan->evRecorded = tm && st == QH_OK;
    return (qh_status)st;
}

namespace {
// Sets of at least this many points take the overlapped host path: the copy of
// the second half runs on a side stream while the first half is hulled.  The
// path pays a second hull call (~0.15 ms of fixed cost) to hide half of the
// copy (~0.038 ms per million points at the host link's ~210 GB/s); on a GB300
// it is slower below ~11M points (4.2M: 0.544 vs 0.469 ms, 10M: 0.832 vs 0.775
// ms) and faster above (12M: 0.85 vs 0.88 ms, 20M: 1.17 vs 1.37 ms).
#ifndef QH_HOST_SPLIT_MIN
#define QH_HOST_SPLIT_MIN 11000000ll
#endif
constexpr long long HOST_SPLIT_MIN = QH_HOST_SPLIT_MIN;

qh_status host_staging(qh_plan plan, long long n, bool split, cudaStream_t s) {
    if (plan->stCap >= n && plan->stIn && (!split || plan->mPts)) return QH_OK;
    cudaStreamSynchronize(s);
    cudaFree(plan->stIn);
    cudaFree(plan->stOut);
    cudaFree(plan->stCnt);
    cudaFree(plan->mPts);
    cudaFree(plan->mOut);
    cudaFree(plan->fOut);
    cudaFree(plan->mOff);
    plan->stIn = nullptr;
    plan->stOut = nullptr;
    plan->stCnt = nullptr;
    plan->mPts = nullptr;
    plan->mOut = nullptr;
    plan->fOut = nullptr;
    plan->mOff = nullptr;
    plan->stCap = 0;
    const long long cap = n < 1024 ? 1024 : n;
    cudaError_t e = cudaMalloc((void **)&plan->stIn, sizeof(float) * 2 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc((void **)&plan->stOut, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc((void **)&plan->stCnt, sizeof(int) * 8);
    if (e == cudaSuccess && split) e = cudaMalloc((void **)&plan->mPts, sizeof(float2) * (size_t)cap);
    if (e == cudaSuccess && split) e = cudaMalloc((void **)&plan->mOut, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess && split) e = cudaMalloc((void **)&plan->fOut, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess && split) e = cudaMalloc((void **)&plan->mOff, sizeof(long long) * 2);
    if (e == cudaSuccess && split && !plan->cpStream) e = cudaStreamCreateWithFlags(&plan->cpStream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess && split; k++)
        if (!plan->cpEv[k]) e = cudaEventCreateWithFlags(&plan->cpEv[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    plan->stCap = cap;
    return QH_OK;
}

// Enqueue the overlapped host path; the result goes to plan->fOut and plan->stCnt[4].
qh_status host_split_hull(qh_plan plan, const float *host_points, long long n, cudaStream_t s) {
    const long long n1 = n / 2, n2 = n - n1;
    int *cnt = plan->stCnt;  // [0]: the first half's hull; [2]: the merged set's; [3]: merge status; [4]: final
    float2 *pts = reinterpret_cast<float2 *>(plan->stIn);
    cudaError_t e = cudaEventRecord(plan->cpEv[0], s);  // the buffers' earlier users on s are done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->cpStream, plan->cpEv[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pts, host_points, sizeof(float2) * (size_t)n1, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pts + n1, host_points + 2 * n1, sizeof(float2) * (size_t)n2, cudaMemcpyHostToDevice,
                            plan->cpStream);
    if (e == cudaSuccess) e = cudaEventRecord(plan->cpEv[1], plan->cpStream);
    if (e != cudaSuccess) return cuda_status(e);
    qh_status st = qh_hull2d_p(plan, plan->stIn, n1, plan->stOut, cnt, (qh_stream_t)s);
    if (st != QH_OK) return st;
    const int g = plan->numSMs * 4;
    merge_gather_kernel<<<g, 256, 0, s>>>(pts, n1, n, plan->stOut, cnt, plan->mPts, plan->mOff, cnt + 3);
    merge_place_kernel<<<g, 256, 0, s>>>(pts, n1, cnt, plan->mPts);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->cpEv[1], 0);
    if (e != cudaSuccess) return cuda_status(e);
    st = qh_hull2d_batched(plan, plan->stIn, reinterpret_cast<const int64_t *>(plan->mOff), 1, plan->mOut, cnt + 2,
                           (qh_stream_t)s);
    if (st != QH_OK) return st;
    merge_map_kernel<<<g, 256, 0, s>>>(n1, plan->stOut, cnt, plan->mOut, cnt + 2, cnt + 3, plan->fOut, cnt + 4);
    return cuda_status(cudaGetLastError());
}
}  // namespace

qh_status qh_hull2d_host(qh_plan plan, const float *host_points, int64_t n, int32_t *host_out_idx,
                         int32_t *host_out_count, qh_stream_t stream) {
    if (!plan || n < 0 || !host_out_count || (n > 0 && (!host_points || !host_out_idx))) return QH_ERR_INVALID_ARG;
    if (n > plan->ncap) return QH_ERR_CAPACITY;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->device) return QH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool split = n >= HOST_SPLIT_MIN;
    qh_status st = host_staging(plan, n, split, s);
    if (st != QH_OK) return st;
    const int *resIdx = plan->stOut, *resCnt = plan->stCnt;
    cudaError_t e = cudaSuccess;
    if (split) {
        st = host_split_hull(plan, host_points, n, s);
        resIdx = plan->fOut;
        resCnt = plan->stCnt + 4;
    } else {
        e = cudaMemcpyAsync(plan->stIn, host_points, sizeof(float) * 2 * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
        st = qh_hull2d_p(plan, plan->stIn, n, plan->stOut, plan->stCnt, stream);
    }
    if (st != QH_OK) return st;
    // The count and the first indices come back together (one synchronisation for
    // every hull of up to EAGER vertices); a larger hull reads the rest after.
    constexpr long long EAGER = 65536;
    const long long first = n < EAGER ? n : EAGER;
    e = cudaMemcpyAsync(host_out_count, resCnt, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && first > 0)
        e = cudaMemcpyAsync(host_out_idx, resIdx, sizeof(int) * (size_t)first, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    const int h = *host_out_count;
    if (h > first) {
        e = cudaMemcpyAsync(host_out_idx + first, resIdx + first, sizeof(int) * (size_t)(h - first),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
    } else if (h < 0) {
        return (qh_status)(-h);
    }
    return QH_OK;
}

qh_status qh_plan_get_stats(qh_plan plan, qh_stats *out) {
    if (!plan || !out) return QH_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(plan->last);
    if (e == cudaSuccess) e = cudaMemcpy(plan->hctl, plan->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    const Ctl &c = *plan->hctl;
    memset(out, 0, sizeof(*out));
    unsigned err = c.err;
    out->device_status = err == 0u ? 0 : (err & E_ARG) ? QH_ERR_INVALID_ARG : (err & E_TIMEOUT) ? QH_ERR_TIMEOUT
                                     : (err & E_CAPACITY) ? QH_ERR_CAPACITY : QH_ERR_INTERNAL;
    out->global_rounds = c.rounds;
    out->small_problems = c.nSmall + c.nPack + c.nSmallInst;
    out->nodes = c.nNodes;
    out->big_sets = c.nBig;
    int last = -1;
    for (int g = 0; g < QH_MAX_GEN && g < MAX_GEN; g++) {
        out->live[g] = c.live[g];
        if (c.live[g] > 0) last = g;
    }
    out->generations = last < 0 ? 1 : last + 2;
    out->levels = c.nLevels;
    out->exact_orient = (int64_t)c.exactOrient;
    out->grid_points = c.bigPoints;
    out->grid_read = c.gridRead;
    out->grid_written = c.gridWritten;
    out->small_points = c.smallPoints;
    out->exact_compare = (int64_t)c.exactCmp;
    for (int k = 0; k < 16; k++) {
        const int hi = k + 1;
        if (hi >= MAX_STAMPS || c.tphase[hi] == 0ull || c.tphase[k] == 0ull) break;
        out->grid_phase_us[k] = (float)((double)(c.tphase[hi] - c.tphase[k]) * 1e-3);
    }
    if (plan->evRecorded) {
        for (int k = 0; k < 4; k++) cudaEventElapsedTime(&out->phase_ms[k], plan->ev[k], plan->ev[k + 1]);
        cudaEventElapsedTime(&out->phase_ms[4], plan->ev[0], plan->ev[4]);
    }
    return QH_OK;
}

// ------------------------------------------------------------------------
// predicate check hooks
// ------------------------------------------------------------------------
qh_status qh_check_orient_host(const float *tri, int64_t n, int32_t prec, int32_t *sign, int32_t *certified) {
    if (n < 0 || (n > 0 && (!tri || !sign || !certified))) return QH_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n; k++) {
        const float *t = tri + 6 * k;
        int used = 0;
        if (prec) {
            const Edge<double> e = make_edge<double>(t[0], t[1], t[2], t[3]);
            sign[k] = orient_sign(e, t[2], t[3], t[4], t[5], orient_approx(e, t[4], t[5]), used);
        } else {
            const Edge<float> e = make_edge<float>(t[0], t[1], t[2], t[3]);
            sign[k] = orient_sign(e, t[2], t[3], t[4], t[5], orient_approx(e, t[4], t[5]), used);
        }
        certified[k] = used == 0;
    }
    return QH_OK;
}

qh_status qh_check_orient_device(const float *tri, int64_t n, int32_t prec, int32_t *sign, int32_t *certified,
                                 qh_stream_t stream) {
    if (n < 0 || (n > 0 && (!tri || !sign || !certified))) return QH_ERR_INVALID_ARG;
    return cuda_status(launch_check_orient(tri, n, prec, sign, certified, (cudaStream_t)stream));
}

qh_status qh_check_dist_host(const float *quads, int64_t n, int32_t *sign) {
    if (n < 0 || (n > 0 && (!quads || !sign))) return QH_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n; k++) {
        const float *t = quads + 8 * k;
        const Edge<float> e = make_edge<float>(t[0], t[1], t[2], t[3]);
        const DistIv<float> a = dist_interval(orient_approx(e, t[4], t[5]));
        const DistIv<float> b = dist_interval(orient_approx(e, t[6], t[7]));
        if (a.lo > b.hi)
            sign[k] = 1;
        else if (b.lo > a.hi)
            sign[k] = -1;
        else
            sign[k] = dist_cmp_exact(t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7]);
    }
    return QH_OK;
}

qh_status qh_check_dist_device(const float *quads, int64_t n, int32_t *sign, qh_stream_t stream) {
    if (n < 0 || (n > 0 && (!quads || !sign))) return QH_ERR_INVALID_ARG;
    return cuda_status(launch_check_dist(quads, n, sign, (cudaStream_t)stream));
}

}  // extern "C"
