// qh_hull2d_noalloc: the single-set hull for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at the moment they need a hull: a
// real-time loop for which cudaMalloc's implicit device synchronisation and
// unbounded latency are not acceptable, or a plug-in hosted by an application
// that owns the whole device-memory budget and forbids allocations by its
// components.  This entry point takes its scratch from one file-scope
// __device__ array of fixed size instead of a plan, so it allocates nothing
// (the array is part of the library's device image: every GPU that loads the
// library holds it, about 31 MB, until the process exits).
//
// The work itself is the library's regular kernel sequence (grid-wide rounds in
// the 256-thread variant,
// block finisher, emit, copy) with the quadrilateral initial split and FP32
// filtered predicates, so its results are those of qh_hull2d.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/qh.h"
#include "qh_internal.cuh"

namespace qh {
namespace {

constexpr long long NA_N = QH_NOALLOC_MAX_POINTS;
constexpr long long NA_SETS = 1;
constexpr long long NA_TILES = NA_N / TILE_MIN + NA_SETS + 16;
constexpr long long NA_BIG = NA_N / TILE_MIN + 16;
// Ring slot of active segments, and the segment tree, small-segment queue and
// level table sized for any input of NA_N points (as in a plan).
constexpr long long NA_SLOT = (4 * NA_SETS > 2 * NA_BIG ? 4 * NA_SETS : 2 * NA_BIG) + 16;
constexpr long long NA_TNODES = 2 * NA_N + 64;
constexpr long long NA_LEVELS = NA_N + 2;
constexpr long long NA_SMALL = NA_N + 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte sizes of the carved buffers, in carving order.
constexpr size_t NA_SIZES[] = {
    sizeof(float2) * 2 * NA_N,       // xy[0]
    sizeof(float2) * 2 * NA_N,       // xy[1]
    sizeof(int) * 2 * NA_N,          // id[0]
    sizeof(int) * 2 * NA_N,          // id[1]
    sizeof(int) * 2 * NA_N,          // vscratch
    sizeof(Cand) * 4 * NA_TILES,     // tbest
    sizeof(Ext) * NA_TILES,          // text
    sizeof(Inst) * NA_SETS,          // inst
    sizeof(int) * (NA_SETS + 1),     // bigInst
    sizeof(int) * (NA_SETS + 1),     // smallInst
    sizeof(long long) * (NA_SETS + 2),  // bigTilePrefix
    sizeof(Node) * 2 * NA_SLOT,      // nodes (ring of two levels)
    sizeof(int) * (NA_BIG + 1),      // bigList[0]
    sizeof(int) * (NA_BIG + 1),      // bigList[1]
    sizeof(long long) * (NA_BIG + 2),   // vstart[0]
    sizeof(long long) * (NA_BIG + 2),   // vstart[1]
    sizeof(TNode) * NA_TNODES,       // tnodes
    sizeof(int) * (NA_LEVELS + 2),   // levelBase
    sizeof(SmallRec) * NA_SMALL,     // small
    sizeof(SmallRec) * NA_SMALL,     // pack
    sizeof(long long) * NA_SMALL,    // packOff
    sizeof(Ctl),                     // ctl
};
constexpr int NA_NBUF = sizeof(NA_SIZES) / sizeof(NA_SIZES[0]);

constexpr size_t na_total() {
    size_t t = 0;
    for (int k = 0; k < NA_NBUF; k++) t += align256(NA_SIZES[k]);
    return t;
}
constexpr size_t NA_BYTES = na_total();

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol: never pass it to a kernel; use the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char qh_noalloc_scratch[NA_BYTES];

struct DeviceScratch {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of qh_noalloc_scratch on this device
    int numSMs = 0;
    int ctasPerSm = 0;
};

std::mutex na_mu;
DeviceScratch na_dev[64];

// Resolve the scratch address and launch constants of the current device (once).
qh_status na_setup(int dev, DeviceScratch &d) {
    if (d.ready) return QH_OK;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, qh_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return QH_ERR_CUDA;
    e = cudaDeviceGetAttribute(&d.numSMs, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return QH_ERR_CUDA;
    d.ctasPerSm = rounds_variant(0).max_ctas_per_sm(0);
    if (d.ctasPerSm < 1) return QH_ERR_CUDA;
    d.base = static_cast<unsigned char *>(ptr);
    d.ready = true;
    return QH_OK;
}

Params na_params(const DeviceScratch &d, const float *points, long long n, int *out_idx, int *out_count) {
    unsigned char *b[NA_NBUF];
    size_t off = 0;
    for (int k = 0; k < NA_NBUF; k++) {
        b[k] = d.base + off;
        off += align256(NA_SIZES[k]);
    }
    Params p;
    memset(&p, 0, sizeof(p));
    p.pts = reinterpret_cast<const float2 *>(points);
    p.offsets = nullptr;
    p.nSingle = n;
    p.numSets = 1;
    p.mode = 0;  // quadrilateral initial split
    p.ncap = NA_N;
    p.outIdx = out_idx;
    p.outCounts = out_count;
    p.xy[0] = reinterpret_cast<float2 *>(b[0]);
    p.xy[1] = reinterpret_cast<float2 *>(b[1]);
    p.id[0] = reinterpret_cast<int *>(b[2]);
    p.id[1] = reinterpret_cast<int *>(b[3]);
    p.vscratch = reinterpret_cast<int *>(b[4]);
    p.tbest = reinterpret_cast<Cand *>(b[5]);
    p.text = reinterpret_cast<Ext *>(b[6]);
    p.maxTiles = NA_TILES;
    p.inst = reinterpret_cast<Inst *>(b[7]);
    p.bigInst = reinterpret_cast<int *>(b[8]);
    p.smallInst = reinterpret_cast<int *>(b[9]);
    p.bigTilePrefix = reinterpret_cast<long long *>(b[10]);
    p.nodes = reinterpret_cast<Node *>(b[11]);
    p.slotCap = (int)NA_SLOT;
    p.bigList[0] = reinterpret_cast<int *>(b[12]);
    p.bigList[1] = reinterpret_cast<int *>(b[13]);
    p.vstart[0] = reinterpret_cast<long long *>(b[14]);
    p.vstart[1] = reinterpret_cast<long long *>(b[15]);
    p.maxBig = (int)NA_BIG;
    p.tnodes = reinterpret_cast<TNode *>(b[16]);
    p.maxTNodes = (int)NA_TNODES;
    p.levelBase = reinterpret_cast<int *>(b[17]);
    p.maxLevels = (int)NA_LEVELS;
    p.small = reinterpret_cast<SmallRec *>(b[18]);
    p.pack = reinterpret_cast<SmallRec *>(b[19]);
    p.packOff = reinterpret_cast<long long *>(b[20]);
    p.maxSmall = (int)NA_SMALL;
    p.ctl = reinterpret_cast<Ctl *>(b[21]);
    p.spinLimit = SPIN_LIMIT;
    p.cut = FIN_MAX;
    return p;
}

}  // namespace
}  // namespace qh

extern "C" qh_status qh_hull2d_noalloc(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                                        qh_stream_t stream) {
    using namespace qh;
    if (n < 0 || !out_count || (n > 0 && (!points || !out_idx))) return QH_ERR_INVALID_ARG;
    if (((uintptr_t)points & 7u) != 0) return QH_ERR_INVALID_ARG;
    if (n > QH_NOALLOC_MAX_POINTS) return QH_ERR_CAPACITY;  // the scratch holds this many points at most
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QH_ERR_CUDA;
    DeviceScratch d;
    {
        std::lock_guard<std::mutex> lock(na_mu);
        qh_status st = na_setup(dev, na_dev[dev]);
        if (st != QH_OK) return st;
        d = na_dev[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    Params p = na_params(d, points, n, out_idx, out_count);
    // the scratch keeps the previous call's contents: reset the control block
    // (counters, barrier, statistics, error bits); every other buffer is
    // initialised by the kernels before it is read
    cudaError_t e = cudaMemsetAsync(p.ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) e = rounds_variant(0).launch(p, 0, d.numSMs * d.ctasPerSm, s);
    if (e == cudaSuccess) e = launch_finish(p, 0, d.numSMs, s);
    if (e == cudaSuccess) e = launch_emit(p, s);
    if (e == cudaSuccess) e = launch_copy(p, d.numSMs * 4, s);
    return e == cudaSuccess ? QH_OK : QH_ERR_CUDA;
}
