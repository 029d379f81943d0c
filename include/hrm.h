/*
 * hrm.h -- C ABI of libhrm: exact running median / order-statistic filters
 * ("hierarchical recursive running median") on NVIDIA GB300 (sm_103a).
 *
 * Problem statement (Section II): for every pixel, the output is the median
 * (more generally the k-th order statistic) of the pixel values inside the
 * n x n (or n x n x n) window centred on it.  Windows use n = 2*radius+1;
 * coordinates outside the image are clamped to the nearest edge (replicate
 * border), and clamped pixels count with multiplicity, so every window holds
 * N = n^2 (2D) or n^3 (3D) values.  The median is the element of 0-based rank
 * (N-1)/2 of the sorted window -- the "n^2/2 position" of Section II; the
 * hierarchical method returns exactly this element (Section III, proof of
 * get_order_statistic), so every entry point below is bit-exact.
 *
 * General conventions
 *  - Pointers named src/dst are DEVICE pointers (cudaMalloc / torch CUDA
 *    memory) unless the name says host.  The caller owns all buffers and
 *    keeps them alive until the work on `stream` has finished.
 *  - Pitches are in BYTES between consecutive rows (pitch >= width * elem
 *    size) and, for volumes, between consecutive slices (slice_pitch >=
 *    height * pitch).  Padding bytes of dst are never written; padding bytes
 *    of src are never read.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Filter calls are asynchronous: they enqueue kernels and return.
 *  - src and dst must not overlap (HRM_EINVAL).
 *  - Return values are hrm_status codes; on error, hrm_last_error() returns a
 *    thread-local message.  No C++ exception crosses this boundary.
 *  - The library keeps a per-device workspace (small: level tables, counters)
 *    that it allocates on first use and reuses; calls on the same device and
 *    stream serialise through it, and concurrent calls on different streams of
 *    one device take separate workspace slices.
 */
#ifndef HRM_H
#define HRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HRM_VERSION 110 /* 1.1.0 */

typedef enum { HRM_U8 = 1, HRM_U16 = 2 } hrm_dtype;

/* Border handling.  Replicate (clamped coordinates) is the only mode; any
 * other value is rejected with HRM_EINVAL. */
enum { HRM_BORDER_REPLICATE = 0 };

/* Flags (bitmask).  Unknown bits are rejected with HRM_EINVAL.
 *  HRM_ADAPTIVE: build data-driven level boundaries before filtering
 *    (Section III-C, adaptive interval-occurrences tree: split the value range
 *    so that frequently used intervals get shorter paths, from a 1:1 mix of
 *    the source's global histogram and a median-estimate histogram).  It
 *    changes speed only, never the output. */
enum { HRM_ADAPTIVE = 1u << 0 };

typedef enum {
    HRM_OK = 0,
    HRM_EAGAIN = 1,        /* hrm_poll / hrm_submit: not done yet / queue full   */
    HRM_EINVAL = -1,       /* bad argument                                     */
    HRM_ENOMEM = -2,       /* device workspace / arena / host allocation failed */
    HRM_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed      */
    HRM_ETIMEDOUT = -4,    /* hrm_poll timed out                               */
    HRM_ECANCELED = -5,    /* request cancelled (server destroyed)             */
    HRM_ENOTSUP = -6,      /* valid but unsupported combination                */
    HRM_EDEVICE = -7       /* a kernel reported an internal error flag         */
} hrm_status;

/* Largest supported radii.  2D: column counts are stored in 8 bits
 * (n <= 255) and window counts in 16 bits (n^2 <= 65025).  3D: window counts
 * n^3 must fit 16 bits (n <= 39). */
#define HRM_MAX_RADIUS_2D 127
#define HRM_MAX_RADIUS_3D 19

/* hrm_filter2d -- exact 2D median filter (Section II problem statement;
 * Section III algorithm: per-column histograms organised as a hierarchy of
 * levels, updated recursively as the window slides, and a level-by-level walk
 * to the rank-(N+1)/2 value).
 *   dtype      HRM_U8 or HRM_U16 (pixels are uint8_t / uint16_t)
 *   src, dst   device pointers to width x height images, row pitch in bytes
 *   radius     0..HRM_MAX_RADIUS_2D (0 copies src to dst)
 *   border     HRM_BORDER_REPLICATE
 *   flags      0 or HRM_ADAPTIVE
 *   stream     cudaStream_t or NULL
 * Radius <= 5 uses register selection networks (3x3, 5x5 and pruned k x k
 * networks); larger radii use the hierarchical histogram kernels.  Empty
 * images (width or height 0) are a no-op returning HRM_OK. */
int hrm_filter2d(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                 int width, int height, int radius, int border, unsigned flags, void* stream);

/* hrm_filter3d -- exact 3D median with a cubic n x n x n window (Section III,
 * extension of the recursion to N dimensions).  src/dst are width x height x
 * depth volumes: element (x, y, z) at base + z*slice_pitch + y*pitch +
 * x*elemsize.  radius 0..HRM_MAX_RADIUS_3D. */
int hrm_filter3d(int dtype, const void* src, size_t src_pitch, size_t src_slice_pitch,
                 void* dst, size_t dst_pitch, size_t dst_slice_pitch,
                 int width, int height, int depth, int radius, int border, unsigned flags,
                 void* stream);

/* hrm_rank_filter2d / hrm_rank_filter3d -- any order statistic (Section III:
 * get_order_statistic finds the element of rank K = k*n^2 for a requested
 * percentile k).  rank is the 0-based position in the sorted window,
 * 0 <= rank < N; rank 0 is the minimum filter, N-1 the maximum filter,
 * (N-1)/2 the median.  Other arguments as for hrm_filter2d/3d. */
int hrm_rank_filter2d(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                      int width, int height, int radius, long rank, int border, unsigned flags,
                      void* stream);
int hrm_rank_filter3d(int dtype, const void* src, size_t src_pitch, size_t src_slice_pitch,
                      void* dst, size_t dst_pitch, size_t dst_slice_pitch,
                      int width, int height, int depth, int radius, long rank, int border,
                      unsigned flags, void* stream);

/* hrm_filter2d_lowprec -- reduced-precision 2D median (Section III-D,
 * variable precision: the level walk stops before the leaves and returns the
 * lower bound of the last interval visited).  With drop_bits = s the output
 * is the exact median with its s lowest bits cleared (the uniform tree is
 * anchored at 0, so every interval at that depth is 2^s wide and aligned);
 * 0 <= s <= 12.  s = 0 equals hrm_filter2d.  Not bit-exact by design. */
int hrm_filter2d_lowprec(int dtype, const void* src, size_t src_pitch, void* dst,
                         size_t dst_pitch, int width, int height, int radius, int drop_bits,
                         void* stream);

/* ---- frame streams: the previous frame's medians as the median estimate ----
 *
 * Section III-C names the previous frame's median as one source of the
 * median estimate that shapes the adaptive tree.  A topology object carries
 * that estimate from one frame to the next: hrm_filter2d_video filters a
 * frame with the top level derived from the previous frame's output (the
 * first frame, or a frame of another dtype, uses the image's own adaptive
 * pre-pass), then histograms its own output for the next frame.  Outputs are
 * always the exact median (identical to hrm_filter2d); only the speed
 * depends on how well consecutive frames agree.
 *
 * The topology holds device state (about 17 KB, allocated by create on the
 * current device) that each call reads and rewrites asynchronously on its
 * stream: calls that share a topology must be ordered (one stream, or events),
 * and the topology must outlive them.  create: HRM_ENOMEM if the allocation
 * fails.  video: HRM_EINVAL for a null topology or one created on another
 * device, plus hrm_filter2d's argument errors.  Frames also run inside
 * batches (hrm_job.topo) and through the serving loop (hrm_request.topo). */
typedef struct hrm_topology hrm_topology;
int hrm_topology_create(hrm_topology** out);
int hrm_topology_destroy(hrm_topology* topo);
int hrm_filter2d_video(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                       int width, int height, int radius, hrm_topology* topo, void* stream);

/* The top level a topology currently holds (what the next frame will use).
 * dtype = 0 until a frame has been filtered with it.  mode 1: the 16 top
 * intervals are [edge[i], edge[i+1]), edge[16] = vmax + 1; mode 0: the
 * uniform tree over [0, vmax] (edge[] all 0).  Waits for `stream` (the one
 * the topology's last frame ran on) before reading the device state.
 * HRM_EINVAL for a null argument. */
typedef struct {
    int dtype;
    unsigned mode, vmin, vmax;
    unsigned edge[17];
} hrm_topology_info;
int hrm_topology_get(hrm_topology* topo, void* stream, hrm_topology_info* out);

/* ---- batched form: many images of uneven size and radius, one launch ----
 *
 * hrm_filter_batch runs every job in ONE persistent kernel launch (plus the
 * level pre-passes) over a device tile work queue: each resident warp
 * repeatedly takes the next (job, tile) work item until the queue is empty.
 * Jobs may mix dtype, dims, size and radius.  Outputs are bit-identical to
 * the corresponding single-image calls.  A job with a topology is one frame
 * of that stream: its top level comes from the topology (or from its own
 * adaptive pre-pass when the topology holds none of its dtype) and its output
 * becomes the topology's next estimate after the launch; a topology may
 * appear in at most one job per call (HRM_EINVAL otherwise), and a graph
 * (hrm_batch_graph_create) takes topology jobs only once each topology holds
 * a top level of its job's dtype. */
typedef struct {
    int dtype;              /* HRM_U8 / HRM_U16                               */
    int dims;               /* 2 or 3                                          */
    const void* src;        /* device pointer                                  */
    size_t src_pitch;       /* bytes                                           */
    size_t src_slice_pitch; /* bytes (3D only)                                 */
    void* dst;              /* device pointer                                  */
    size_t dst_pitch;
    size_t dst_slice_pitch;
    int width, height, depth; /* depth = 1 for 2D                              */
    int radius;
    long rank;              /* -1 = median, else 0-based order statistic       */
    unsigned flags;         /* 0 or HRM_ADAPTIVE                               */
    hrm_topology* topo;     /* NULL, or a frame stream: 2D median, flags 0;   */
                            /* the job runs as hrm_filter2d_video would       */
} hrm_job;

int hrm_filter_batch(const hrm_job* jobs, int njobs, void* stream);

/* hrm_filter_batch_noalloc -- the same batched filter, for callers that must
 * not allocate device memory.  (The paper has no counterpart: this is a
 * deployment entry point.)  Some callers cannot call cudaMalloc: frame loops
 * with a hard latency budget (an allocation may synchronise the whole
 * device and stall every stream), and programs whose device memory is handed
 * out by their own pooling allocator, where a library allocating behind the
 * pool's back breaks its accounting or fails once the pool has reserved the
 * memory.
 *
 * This call allocates nothing: its scratch (job table, tile offsets, level
 * descriptors, queue counter, error word, pre-pass histograms) is one
 * file-scope device array of 64 KiB that every GPU loading the library holds
 * until the process exits.  It takes at most 64 jobs per call and rejects
 * more with HRM_EINVAL.  The first call on each device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current.  All calls
 * share the one array and it keeps the last call's contents (the call clears
 * what must start at zero), so calls whose work overlaps on the GPU -- on
 * different streams, or from different threads without ordering -- race:
 * serialise them.  The job tables are copied from host memory on the
 * caller's thread (cudaMemcpyAsync from pageable memory returns once the
 * source has been read).  A kernel error raised by this path stays set in the
 * array until hrm_device_status (any stream of the device; it allocates
 * nothing) reads and clears it.  Outputs are bit-identical to
 * hrm_filter_batch.  Other arguments as for hrm_filter_batch. */
int hrm_filter_batch_noalloc(const hrm_job* jobs, int njobs, void* stream);

/* hrm_batch_graph_* -- capture the batched launch for a FIXED job list into a
 * CUDA graph once and replay it (no host-side planning or per-job launches on
 * replay).  The job list (pointers included) is frozen at create time. */
typedef struct hrm_batch_graph hrm_batch_graph;
int hrm_batch_graph_create(const hrm_job* jobs, int njobs, void* stream, hrm_batch_graph** out);
int hrm_batch_graph_launch(hrm_batch_graph* g, void* stream);
/* Wait for `stream`, then report (and clear) the error word the graph's
 * kernels write: HRM_OK or HRM_EDEVICE (replays accumulate until read). */
int hrm_batch_graph_status(hrm_batch_graph* g, void* stream);
int hrm_batch_graph_destroy(hrm_batch_graph* g);

/* ---- planning / autotuning ---------------------------------------------
 *
 * The hierarchical kernels are parameterised by tile width (output columns
 * per 4-warp tile: 128 or 256, i.e. one or two outputs per thread), strip
 * length (rows or slices walked per tile), the shared memory per tile for
 * cached tree nodes, and the tree's top level.  Every level below the top is
 * 16-ary (one 16-byte counter record per node and column); the top level is
 * either 16 equal intervals over the image's value range (the uniform
 * interval-occurrence tree, Section III) or the adaptive split: intervals of
 * one power-of-16 width over the central range of a block-median estimate,
 * which also fixes how many levels lie below (Section III-C).  A plan's
 * `tree` field overrides the call's HRM_ADAPTIVE flag; the output is the same
 * either way, only the speed differs.  hrm_autotune times candidate plans
 * for one problem class on `stream` -- first the default plan and the
 * default with the other top level, then tile widths, slot budgets and strip
 * lengths under the faster top level -- and caches the fastest (the default
 * unless another plan is at least 3 % faster); later calls of
 * the same class (dtype, dims, size, radius, flags) use it.  The timing runs
 * on `sample` (device pointer, the caller's pitches) when it is not NULL --
 * speed depends on the data, so a representative image is best -- and on a
 * synthetic image otherwise.  hrm_autotune allocates and frees its own output
 * (and synthetic input) buffers and blocks until the timing finishes.  The
 * cache is per process; hrm_plan_save / hrm_plan_load persist it as text
 * (one line per class; a line without the trailing tree field loads with
 * tree 0).
 * Environment, read once per process: HRM_PLAN_CACHE=<file> loads a saved
 * plan file before the first call (a missing or malformed file is ignored);
 * HRM_FORCE_PATH=hist or =sortnet forces the histogram kernel or the
 * selection networks (where one exists for the problem) in every call
 * without an explicit plan.  Outputs never depend on the plan.
 *
 * Node-cache feedback (2D single-image calls of a class with no set, tuned
 * or forced plan): the first call counts how many tree nodes its tiles had to
 * build and copies the count back asynchronously; the second call of the
 * class waits for that 4-byte copy and, if the tile rows built more than 0.75
 * nodes on average, tries as many cached nodes as fit in up to 200 KB per
 * tile (one or two tiles per SM) instead of the default four tiles per SM;
 * that trial call is counted too, the third call waits for its count, and the
 * class keeps the large cache only if it cut the node builds at least
 * 3-fold.  From the third call on, every call of the class runs the same
 * settled plan.  hrm_get_plan reports the plan a single call of the class
 * would use now, feedback included. */
typedef struct {
    int tile_width;     /* output columns per tile: 128 or 256 (0 = default) */
    int strip_height;   /* output rows (2D) or slices (3D) per tile (0 = default) */
    int slot_kbytes;    /* shared memory per tile, KB (0 = default)            */
    int path;           /* 0 = auto, 1 = selection network, 2 = histogram     */
    int tree;           /* top level: 0 = as the call's flags say,
                           1 = uniform, 2 = adaptive (histogram path only)   */
} hrm_plan;

int hrm_autotune(int dtype, int dims, int width, int height, int depth, int radius,
                 unsigned flags, const void* sample, size_t sample_pitch,
                 size_t sample_slice_pitch, void* stream, hrm_plan* best);
int hrm_get_plan(int dtype, int dims, int width, int height, int depth, int radius,
                 unsigned flags, hrm_plan* plan);
int hrm_set_plan(int dtype, int dims, int width, int height, int depth, int radius,
                 unsigned flags, const hrm_plan* plan);
int hrm_plan_save(const char* path);
int hrm_plan_load(const char* path);

/* ---- serving loop: continuous batching -----------------------------------
 *
 * A server owns a device arena carved from caller-provided device memory
 * (arena_dev_ptr, arena_bytes; e.g. a torch uint8 CUDA tensor).  Requests are
 * admitted while their resident bytes (input + output copies in the arena)
 * fit the arena and fewer than max_inflight are admitted; each admitted
 * request's tiles join the next persistent-kernel wave, so requests that
 * arrive while others run are added as memory and slots free up.  A
 * background host thread drives copies and waves on the server's own
 * streams.  Frame streams (Section III-C, previous frame as the median
 * estimate): requests that name the same topology are filtered in submission
 * order, each with the top level left by the one before it; two frames of one
 * stream never share a wave (the later one waits for the next), and a wave
 * on the other compute stream waits for the wave that last used the
 * topology.  The topology must outlive its requests, and while the server
 * holds requests for it no other call may use it (the server's streams are
 * not ordered with the caller's). */
typedef struct hrm_server hrm_server;

typedef struct {
    int dtype;                /* HRM_U8 / HRM_U16                              */
    int width, height;        /* 2D requests                                   */
    int radius;               /* 0..HRM_MAX_RADIUS_2D                          */
    unsigned flags;           /* 0 or HRM_ADAPTIVE                             */
    const void* src;          /* host or device pointer (see src_on_host)      */
    size_t src_pitch;
    void* dst;                /* host or device pointer (see dst_on_host)      */
    size_t dst_pitch;
    int src_on_host;          /* 1: src is host memory (pinned is fastest)     */
    int dst_on_host;          /* 1: dst is host memory                         */
    hrm_topology* topo;       /* NULL, or the frame stream this frame belongs  */
                              /* to (flags must then be 0)                     */
} hrm_request;

typedef struct {
    uint64_t submitted, admitted, completed, rejected, waves;
    uint64_t bytes_resident, bytes_high_water, arena_bytes;
    int inflight, queued;
} hrm_server_stats;

/* Create a server on the current CUDA device.  max_inflight bounds admitted,
 * unfinished requests; the submit queue holds up to max_queue requests
 * (0 = 4096). */
int hrm_server_create(void* arena_dev_ptr, size_t arena_bytes, int max_inflight, int max_queue,
                      hrm_server** out);
/* Queue a request; returns immediately with a ticket.  HRM_EAGAIN if the
 * submit queue is full, HRM_EINVAL if the request can never fit the arena.
 * The caller keeps src/dst valid until hrm_poll returns HRM_OK. */
int hrm_submit(hrm_server* s, const hrm_request* req, uint64_t* ticket);
/* Wait up to timeout_us (0 = just check, < 0 = forever) for a ticket:
 * HRM_OK = done (dst holds the result), HRM_EAGAIN = still pending when
 * timeout_us == 0, HRM_ETIMEDOUT = still pending after a positive timeout,
 * HRM_ECANCELED, or the request's error status.  A ticket that returned
 * HRM_OK is retired and unknown afterwards (HRM_EINVAL). */
int hrm_poll(hrm_server* s, uint64_t ticket, int timeout_us);
/* Per-ticket latency in microseconds (submit -> completion event).  Known
 * once hrm_poll returned HRM_OK for the ticket; the server remembers the
 * latencies of the most recent 1,000,000 retired tickets.  Negative for a ticket
 * that is unknown, still pending, or older than that. */
double hrm_ticket_latency_us(hrm_server* s, uint64_t ticket);
int hrm_server_stats_get(hrm_server* s, hrm_server_stats* out);
/* Stop the loop; pending requests end as HRM_ECANCELED. */
int hrm_server_destroy(hrm_server* s);

/* Wait for `stream`, then report (and clear) any error flag raised by the
 * kernels of this stream's workspace (single-image calls and
 * hrm_filter_batch) or by hrm_filter_batch_noalloc on the current device:
 * HRM_OK or HRM_EDEVICE.  Kernels never trap; internal limits that cannot be
 * met set this flag instead.  Allocates nothing.  Graphs report through
 * hrm_batch_graph_status. */
int hrm_device_status(void* stream);

/* Thread-local description of the last error on this thread. */
const char* hrm_last_error(void);
int hrm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HRM_H */
