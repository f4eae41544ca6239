// The x-sorted form of the rounds (Sec. 3, Sec. 4.2-4.4): device state and
// scratch of qh_hull2d_sorted, and its host-side driver.
#pragma once

#include <cuda_runtime.h>

#include "qh_internal.cuh"

namespace qh {
namespace sx {

constexpr int SNT = 256;               // threads per CTA of every kernel of this form
constexpr int SIPT = 16;               // items per thread
constexpr int STILE = SNT * SIPT;      // items per tile (4096)
constexpr int SNW = SNT / 32;
constexpr int BINS = 512;              // radix bins: 2 chains x 256 digit values
constexpr int MAX_PARTIALS = 1024;     // CTAs of the extreme-point pass
constexpr int ROUND_BATCH = 8;         // rounds enqueued between two host checks of the end flag
constexpr unsigned IDX_MASK = 0x1FFFFFFFu;  // item payload: input index (< 2^29),
constexpr unsigned HEAD_BIT = 0x80000000u;  // initial-polygon vertex flag and its rank << 29

// Extreme points of a range of the input (lexicographic min/max of (x, y) and of (y, x)).
struct Ext4 {
    Cand a, b, bot, top;
    int nonfinite, pad[3];
};

// Device state of one call.
struct SxState {
    Cand poly[4];        // initial polygon, CCW from the lexicographic minimum A
    int K, iB;           // its size (1: all points coincide, 0: non-finite input) and the rank of B
    int nonfinite, done; // done: no segment holds a point
    unsigned c0, c1;     // items of the lower chain (front) and of the upper chain (back) after the split
    int m, mNew;         // polygon length (a copy of A follows at index m) this round / next round
    int S, SNew;         // heads (= segments) this round / next round
    int cur, gen;        // buffer of this round; generation the round produces
    long long liveNew;   // points the round keeps in segments
    long long liveLast;  // points held in segments before the round
    unsigned ticket;     // CTAs finished (the last one of a kernel runs its closing step)
    int pad;
};

// Buffers of the rounds, selected by SxState::cur.
struct SxBufs {
    float *X[2], *Y[2];  // polygon coordinates (capacity + a tile + the copy of A)
    int *I[2];           // input indices
    int *hp[2];          // head positions, ascending, then m
    int *best[2];        // per segment: position of its farthest point (-1: none yet)
    int2 *tcnt;          // per tile of a round: (kept items, kept heads), then their exclusive offsets
};

struct SortedWs {
    long long cap = 0;
    unsigned *key[2] = {nullptr, nullptr};
    unsigned *val[2] = {nullptr, nullptr};
    SxBufs b = {};
    int *hist = nullptr;     // radix counts, bin-major: BINS x tiles
    int *rowTot = nullptr;   // per bin: total
    int *binBase = nullptr;  // per bin: exclusive offset
    Ext4 *part = nullptr;    // extreme-point partials
    SxState *st = nullptr;
    int *hDone = nullptr;    // pinned copy of SxState::done
};

cudaError_t sorted_alloc(SortedWs &w, long long cap);
void sorted_free(SortedWs &w);
// Status (qh_status value) of enqueueing and running one hull; ev: 5 events or nullptr.
int sorted_run(SortedWs &w, const float2 *pts, int n, int mode, int prec, int *outIdx, int *outCount, Ctl *ctl,
               int numSMs, cudaStream_t s, cudaEvent_t *ev);

}  // namespace sx
}  // namespace qh
