/*
 * qh.h -- C ABI of the GB300 segmented-QuickHull library (libqh.so).
 *
 * Method: Zhang, Mei, Xu, Zhao, "A Novel Implementation of QuickHull Algorithm
 * on the GPU".  The library computes the convex hull of planar FP32 point sets
 * (Sec. 1: the smallest convex polygon containing every point) with the
 * segmented, generation-synchronous QuickHull of Sec. 3-4: extreme points and an
 * initial split (Sec. 4.2-4.3), then rounds of farthest point per segment
 * (Sec. 4.4.1), segment update (Sec. 4.4.2, 4.4.4) and discard of interior
 * points (Sec. 4.4.3) until no segment holds points.
 *
 * Output convention (every entry point): indices of the strictly convex hull
 * vertices, counter-clockwise, starting at the lexicographically smallest
 * (x, then y) point.  Points on a hull edge are not vertices.  Points with
 * identical coordinates (compared by value, -0 == +0) are represented by their
 * lowest index.  Every geometric decision is exact: FP32 (or FP64) arithmetic
 * with a certified error bound, and an exact fallback where the bound cannot
 * decide.
 *
 * Memory: every pointer argument named "device" must be device memory of the
 * current CUDA device; "host" pointers are host memory.  Points are interleaved
 * x, y float pairs (8-byte aligned).  The caller owns inputs and outputs; a
 * plan owns all scratch memory.  Calls are stream-ordered and asynchronous
 * unless stated otherwise: the results are valid once the stream has reached
 * the call.  Host-detected errors return immediately; errors detected on the
 * device are written into the output counts as the negated status code.
 * A plan must not be used by two streams at the same time.
 */
#ifndef QH_H
#define QH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Compatible with cudaStream_t. */
typedef struct CUstream_st *qh_stream_t;

typedef enum {
    QH_OK = 0,
    QH_ERR_INVALID_ARG = 1, /* bad pointer, size or flag */
    QH_ERR_NONFINITE = 2,   /* an input coordinate is NaN or infinite */
    QH_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    QH_ERR_OOM = 4,         /* device memory allocation failed */
    QH_ERR_CAPACITY = 5,    /* input larger than the plan, or a device table overflowed */
    QH_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (status word set) */
    QH_ERR_INTERNAL = 7,    /* inconsistent device state */
    QH_ERR_UNSUPPORTED = 8  /* not possible in this context (e.g. growing a plan during capture) */
} qh_status;

/* Plan flags. */
#define QH_MODE_QUAD 0x0u   /* initial quadrilateral of the 4 extreme points (paper's Mode 1, Sec. 4.2) */
#define QH_MODE_CHORD 0x1u  /* initial chord leftmost->rightmost only (paper's Mode 2, Sec. 4.3) */
#define QH_PREC_F32 0x0u    /* FP32 predicates with certified bound + exact fallback */
#define QH_PREC_F64 0x2u    /* plain FP64 predicates with bound + the same exact fallback */

#define QH_MAX_GEN 512

/* Largest plan (points): int32 indices, two nested copies of the points, up to 2n tree nodes. */
#define QH_MAX_PLAN_POINTS (1ll << 29)

typedef struct qh_plan_s *qh_plan;

typedef struct {
    int32_t device_status;      /* 0, or the qh_status of the first device-side failure */
    int32_t global_rounds;      /* grid-wide rounds after the initial split */
    int32_t generations;        /* generations run (initial split = generation 0) */
    int32_t small_problems;     /* segments and sets finished by one thread block each */
    int32_t nodes;              /* segments created by grid-wide rounds */
    int32_t big_sets;           /* point sets that took the grid-wide path */
    int32_t levels;             /* levels of the segment tree (initial segments = level 0) */
    int32_t pad0;
    int64_t live[QH_MAX_GEN];   /* points held by segments after each generation (all sets);
                                   generations past the last entry add to it */
    int64_t exact_orient;       /* orientation tests decided by the exact fallback */
    int64_t exact_compare;      /* farthest-point comparisons decided by the exact fallback */
    float phase_ms[5];          /* with timing on: grid rounds, finisher, emit, copy, total */
    float grid_phase_us[16];    /* inside the grid-wide kernel: set prep, extreme points, initial
                                   split, then grid-wide rounds 1.. (device clock) */
    int64_t grid_points;        /* points of the sets tiled by the grid-wide kernel (read twice:
                                   extreme points and initial split) */
    int64_t grid_read;          /* live points read by grid-wide rounds after the initial split */
    int64_t grid_written;       /* live points written by the initial split and grid-wide rounds */
    int64_t small_points;       /* points handled by the block finisher (small segments and sets) */
} qh_stats;

/*
 * qh_plan_create -- allocate a plan for up to max_points points in up to
 * max_sets sets.  flags: QH_MODE_* | QH_PREC_*.  The plan holds roughly
 * 165 bytes of device scratch per point: two nested copies of the live points,
 * and a segment tree, small-segment queues and level table sized for any input
 * (a set of n points has at most 2n tree nodes, n small segments and n levels),
 * so no input within max_points exceeds it, however deep the recursion.
 * Errors: QH_ERR_INVALID_ARG (sizes < 1), QH_ERR_CAPACITY (max_points above
 * QH_MAX_PLAN_POINTS), QH_ERR_OOM, QH_ERR_CUDA.
 */
qh_status qh_plan_create(int64_t max_points, int32_t max_sets, uint32_t flags, qh_plan *out);

/* Release a plan (synchronizes the device first).  NULL is accepted. */
qh_status qh_plan_destroy(qh_plan plan);

/* Change mode/precision flags of an existing plan (no reallocation). */
qh_status qh_plan_set_flags(qh_plan plan, uint32_t flags);

/*
 * Tuning knobs.  cutover: segments with at most this many points are finished
 * by one thread block in shared memory; from the grid-wide tile of the plan's
 * kernel variant (32 x points per thread, so a tile never spans more than two
 * segments) to 4096.  timing: 1 records CUDA events between the kernels so
 * qh_plan_get_stats can report per-phase times.  grid_ctas_per_sm: 0 =
 * automatic (one CTA per SM for a single set of at most 2^19 points, else the
 * occupancy maximum).
 */
qh_status qh_plan_set_tuning(qh_plan plan, int32_t cutover, int32_t timing, int32_t grid_ctas_per_sm);

/*
 * Kernel variant of the grid-wide rounds: threads per block (256 or 128) and points per thread per tile (16
 * or 8; a tile is threads x points per thread points).  Each call keeps the other knob, raises
 * the cutover to the new tile if needed and resets grid_ctas_per_sm to the occupancy maximum.  Other values:
 * QH_ERR_INVALID_ARG.  (Not in the paper: its kernels are Thrust calls with library-chosen launch shapes.)
 */
qh_status qh_plan_set_block(qh_plan plan, int32_t threads_per_block);
qh_status qh_plan_set_items_per_thread(qh_plan plan, int32_t items_per_thread);

/*
 * Debug limits for tests of the device-side error paths (not in the paper).  spin_limit: polls (each
 * followed by a ~100 ns sleep) before a grid-barrier wait gives up with QH_ERR_TIMEOUT; 0 restores the
 * default (2^22).  max_tree_nodes: lowers the segment-tree capacity so that a deep enough input reports
 * QH_ERR_CAPACITY; 0 restores the full table.  Both errors reach the output counts as -status, the
 * kernels leave at their next barrier, and the plan works normally again once the limits are reset.
 */
qh_status qh_plan_set_debug(qh_plan plan, uint32_t spin_limit, int32_t max_tree_nodes);

/* The plan's current tuning: block size, points per thread, small-segment cutover, grid CTAs per SM (when
 * automatic: the occupancy maximum, which single sets of at most 2^19 points do not use). */
qh_status qh_plan_get_tuning(qh_plan plan, int32_t *threads_per_block, int32_t *items_per_thread,
                             int32_t *cutover, int32_t *grid_ctas_per_sm);

/*
 * Autotuner (not in the paper): hulls the caller's input with the plan's current setting (the reference),
 * then once per candidate setting -- every kernel variant (block size x points per thread), grid CTAs per
 * SM from the occupancy maximum down to half of it, and every cutover from the variant's tile to 4096 in
 * steps of 1024 -- and checks on the device that each candidate's output equals the reference's (vertex
 * counts and every index; the hull is unique).  A candidate that agrees is timed over `reps` runs with
 * CUDA events on `stream`; the fastest agreeing candidate is kept in the plan.  offsets == NULL: one set
 * of n points (as qh_hull2d_p); otherwise a CSR batch (as qh_hull2d_batched, n ignored).  Allocates a copy
 * of the reference output for the duration of the call and synchronizes the stream; out_idx / out_counts
 * end up holding the result of the last trial.  Errors: QH_ERR_INVALID_ARG (reps outside [1, 64]),
 * QH_ERR_INTERNAL (some candidate's output differed from the reference; the best agreeing setting is
 * kept), a failing trial's status (the best setting so far is kept).
 */
qh_status qh_plan_autotune(qh_plan plan, const float *points, const int64_t *offsets, int32_t num_sets,
                           int64_t n, int32_t *out_idx, int32_t *out_counts, int32_t reps, qh_stream_t stream);

/*
 * qh_hull2d_p -- hull of one point set (Sec. 1).
 *   points:    device, float[2*n] interleaved x,y; read only.
 *   n:         number of points, 0 <= n <= the plan's max_points.
 *   out_idx:   device int32[n] (any capacity >= n); receives the hull vertex
 *              indices (CCW from the lexicographic minimum).
 *   out_count: device int32[1]; receives the vertex count, or -status on a
 *              device-detected error (QH_ERR_NONFINITE, QH_ERR_TIMEOUT, ...).
 *   stream:    CUDA stream (NULL = legacy default stream).
 * Returns QH_OK once the work is enqueued.
 */
qh_status qh_hull2d_p(qh_plan plan, const float *points, int64_t n, int32_t *out_idx,
                      int32_t *out_count, qh_stream_t stream);

/*
 * qh_hull2d -- as qh_hull2d_p with a per-device default plan (QUAD, FP32) that
 * grows on demand.  Growing synchronizes the device and is refused
 * (QH_ERR_UNSUPPORTED) while the stream is being captured.
 */
qh_status qh_hull2d(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                    qh_stream_t stream);

/*
 * qh_hull2d_batched -- hulls of num_sets independent point sets in one call.
 *   points:     device, float[2*N] interleaved x,y of all sets.
 *   offsets:    device int64[num_sets+1], non-decreasing, offsets[0] >= 0,
 *               offsets[num_sets] <= the plan's max_points; set s is
 *               points[offsets[s] .. offsets[s+1]).
 *   out_idx:    device int32[offsets[num_sets]]; set s's hull (indices local
 *               to the set) is written at out_idx + offsets[s].
 *   out_counts: device int32[num_sets]; vertex count of each set, or -status.
 * The result equals num_sets separate qh_hull2d_p calls.  No host
 * synchronization; the call can be captured in a CUDA graph.
 */
qh_status qh_hull2d_batched(qh_plan plan, const float *points, const int64_t *offsets, int32_t num_sets,
                            int32_t *out_idx, int32_t *out_counts, qh_stream_t stream);

/*
 * qh_hull2d_sorted -- the hull of one set by the paper's own arrangement of the
 * rounds (Sec. 3, Sec. 4.2-4.4): after the first split the points are sorted by
 * x (the lower subset ascending, the upper one descending), so that all of them
 * read as one polygon from the lexicographic minimum; every round marks the
 * farthest point of each segment as a head in place and a stable compaction
 * removes the points that are not strictly right of their new chord.  The
 * result equals qh_hull2d_p's (same vertices, same order, same per-generation
 * live counts in the statistics) for the plan's mode and precision flags.
 *   points, n, out_idx, out_count, stream: as for qh_hull2d_p.
 * Scratch: the first call allocates about 60 bytes per point of the plan's
 * capacity in the plan (kept until qh_plan_destroy).  The host reads an end
 * flag after every 8 rounds, so the call synchronizes the stream and returns
 * once the hull is written; it cannot be captured in a CUDA graph
 * (QH_ERR_UNSUPPORTED while the stream is capturing).  With timing on, the
 * statistics' phase_ms hold: first split (with the extreme points), sort,
 * rounds (including the host's checks), output, total.
 * Errors: as qh_hull2d_p; QH_ERR_INTERNAL when the device state is inconsistent.
 */
qh_status qh_hull2d_sorted(qh_plan plan, const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                           qh_stream_t stream);

/*
 * qh_hull2d_host -- end-to-end form of qh_hull2d_p with HOST buffers: copies
 * host_points (float[2*n]) to the device, computes, copies the hull to
 * host_out_idx (int32[n]) and the count to *host_out_count, and synchronizes
 * the stream before returning.  Entries of host_out_idx past the count are
 * unspecified (the first min(n, 65536) entries are read back together with the
 * count).  Pinned host memory gives the fastest copies.
 * Sets of at least 11,000,000 points overlap the copy with the computation: the
 * second half is copied on a side stream of the plan while the first half is
 * hulled, then the first half's hull vertices are hulled together with the
 * second half (the same output).  The plan's statistics then describe that
 * second hull.  Scratch: staging for the copies (about 12 bytes
 * per point) and, for the overlapped form, about 16 more, kept in the plan.
 * Errors: as qh_hull2d_p, QH_ERR_INVALID_ARG when the current device is not the
 * plan's.
 */
qh_status qh_hull2d_host(qh_plan plan, const float *host_points, int64_t n, int32_t *host_out_idx,
                         int32_t *host_out_count, qh_stream_t stream);

/*
 * qh_hull2d_noalloc -- the hull of one set (same output as qh_hull2d: quadrilateral
 * initial split, FP32 filtered predicates with exact fallback) for callers that
 * must not allocate device memory when they need a hull: real-time loops that
 * cannot afford cudaMalloc's implicit device synchronisation, or plug-ins whose
 * host application owns the device-memory budget.  The paper has no counterpart:
 * this is an interface addition.
 *   points, n, out_idx, out_count, stream: as for qh_hull2d_p.
 *   n must not exceed QH_NOALLOC_MAX_POINTS; larger sets return QH_ERR_CAPACITY
 *   without touching the device.
 * Scratch: one fixed array in the library's device image (about 43 MB on every
 * GPU that loads the library, held until the process exits); no cudaMalloc,
 * cudaFree or other allocating call is made.  The first call on a device looks up
 * the array's address for that device (it must come before any stream capture)
 * and keeps it for the life of the process: a cudaDeviceReset after that first
 * call invalidates the kept address and is not supported.
 * All calls share the array: calls that overlap on the GPU (other streams, other
 * host threads) race and corrupt each other's results; serialise them.
 */
#define QH_NOALLOC_MAX_POINTS 262144
qh_status qh_hull2d_noalloc(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                            qh_stream_t stream);

/* Statistics of the plan's last call; synchronizes the plan's last stream. */
qh_status qh_plan_get_stats(qh_plan plan, qh_stats *out);

/* Static description of a status code. */
const char *qh_status_string(qh_status s);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t qh_version(void);

/*
 * Predicate check hooks (used by the test suite; the hull itself never calls
 * them).  qh_check_orient_host evaluates, on the CPU, the same filtered
 * orientation code the kernels run: sign[k] is the decided sign of
 * orient(a_k, b_k, c_k) for the triples tri[6k .. 6k+6) = ax ay bx by cx cy,
 * and certified[k] is 1 when the filter (prec: 0 = FP32, 1 = FP64) decided it
 * without the exact fallback.  qh_check_orient_device runs the same on the
 * GPU with device arrays.  qh_check_dist_* return sign(dist(P) - dist(Q)) for
 * quads[8k .. 8k+8) = ux uy vx vy px py qx qy, where dist(X) is the distance
 * of X to the right of the chord u->v.
 */
qh_status qh_check_orient_host(const float *tri, int64_t n, int32_t prec, int32_t *sign, int32_t *certified);
qh_status qh_check_orient_device(const float *tri, int64_t n, int32_t prec, int32_t *sign, int32_t *certified,
                                 qh_stream_t stream);
qh_status qh_check_dist_host(const float *quads, int64_t n, int32_t *sign);
qh_status qh_check_dist_device(const float *quads, int64_t n, int32_t *sign, qh_stream_t stream);


#ifdef __cplusplus
}
#endif

#endif /* QH_H */
