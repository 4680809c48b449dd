/*
 * ws.h -- C ABI of libws, a GB300-native (sm_103a) watershed and waterfall
 * partitioning library.
 *
 * The method is the one of "Parallel Watershed Partitioning: GPU-Based
 * Hierarchical Image Segmentation" (Yeghiazaryan, Gabrielyan, Voiculescu,
 * arXiv 2410.08946):
 *   - watershed (Sec. 3, Alg. 1): step I states and steepest-descent arrows
 *     (Eq. 1), step II fair resolution of non-minimal plateaux (Sec. 3.3,
 *     Alg. 3), step III path reduction to the minima (Sec. 3.1, Fig. 4),
 *     step IV Union-Find merge of minimal plateaux (Sec. 3.1);
 *   - waterfall (Sec. 4, Alg. 4, Alg. 5): lowest pass of each basin, then the
 *     basins joined across their lowest passes, NL levels in all.
 *
 * Conventions for every entry point
 *   Images are dense, row-major, x fastest: a 2D pixel (x, y) is p = y*W + x,
 *   a 3D voxel (x, y, z) is p = (z*H + y)*W + x (the row-major order of
 *   Sec. 3.1).  N = W*H*D must be below 2^31.  Neighbourhoods contain in-image
 *   pixels only (no padding, no wrap-around).
 *
 *   Labels are canonical: the K regions of a level are numbered 0..K-1 in the
 *   order of each region's smallest pixel index.  (The paper's labels are the
 *   index of a representative pixel, Sec. 3.1; any two equivalent labellings
 *   map to the same canonical one.)
 *
 *   Buffers named *_d are device pointers owned by the caller; the library
 *   never frees or keeps them after the call's work completes.  *_h are host
 *   pointers (pinned memory gives the fastest copies).  Workspace (label and
 *   parent arrays, edge tables) is owned by the context and stays resident
 *   between calls; it grows on demand within the context's byte budget.
 *
 *   Device-side calls only enqueue work on `stream` (NULL = the legacy
 *   default stream) and return without waiting for it.  Argument errors are
 *   returned at once and enqueue nothing.  Errors found by the device (an
 *   iteration cap reached, a full edge table) are recorded in the context's
 *   device status word and returned by ws_context_check().  No call aborts,
 *   throws or traps; every device loop is bounded.
 *
 *   A context may be used from one host thread at a time.  Calls on one
 *   context must not overlap on the device (they share its workspace): use
 *   one stream per context, or one context per stream.
 */
#ifndef WS_H
#define WS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* same type as cudaStream_t / CUstream */
typedef struct CUstream_st *ws_stream_t;

typedef enum {
    WS_OK = 0,
    WS_ERR_INVALID = 1,      /* bad argument: pointer, shape, dtype, connectivity, NL */
    WS_ERR_UNSUPPORTED = 2,  /* valid request that this build does not implement */
    WS_ERR_OOM = 3,          /* workspace budget or device memory exhausted, or edge table full */
    WS_ERR_CUDA = 4,         /* a CUDA runtime call failed (see ws_last_error) */
    WS_ERR_NONCONVERGED = 5, /* a device loop hit its iteration cap */
    WS_ERR_TIMEOUT = 6,      /* a device-wide barrier waited longer than its time limit */
    WS_ERR_NOT_READY = 7,    /* ws_poll: the request has not finished yet */
    WS_ERR_CANCELLED = 8     /* ws_poll: the request was cancelled */
} ws_status;

typedef enum { WS_U8 = 0, WS_U16 = 1 } ws_dtype;

/* dims[0] = W (fastest), dims[1] = H, dims[2] = D (ignored when ndim == 2) */
typedef struct {
    int32_t ndim;
    int32_t pad_;
    int64_t dims[3];
} ws_shape;

typedef struct ws_context ws_context;

/* Tuning knobs (all optional; zero = library default). */
typedef struct {
    int32_t plateau_round_cap;   /* max global rounds of the step II distance relaxation */
    int32_t jump_round_cap;      /* max global rounds of step III pointer jumping */
    int32_t jumps_per_round;     /* pointer hops per pixel per round (the paper's RR, Sec. 3.1) */
    int32_t barrier_timeout_ms;  /* device-wide barrier wait limit */
    int64_t edge_capacity;       /* slots of the region-adjacency table and edge lists (0: pixels x forward
                                    neighbours, rounded up to a power of two, at most 2^28) */
    int32_t levels_ctas_per_sm;  /* CTAs per SM of the cooperative waterfall-level kernel (1..32) */
    int32_t barrier_withhold;    /* failure-detection tests only: 1 arms a one-shot hold, 0 = off.  In
                                    the next cooperative kernel the context launches, block 0 does not
                                    arrive at its first device-wide barrier, so the other blocks' waits
                                    run out after barrier_timeout_ms; the call then reports
                                    WS_ERR_TIMEOUT through ws_context_check.  Nothing faults or hangs,
                                    and the hold is disarmed once it has been handed to a launch. */
    int32_t tile_shape;          /* 2D uint8 images: tile shape and threads per tile of the tiled kernels:
                                    0 = 64 x 32 pixels / 256 threads (default), 1 = 32 x 32 / 256,
                                    2 = 128 x 16 / 256, 3 = 64 x 32 / 512.  Other images use their
                                    fixed shape (2D uint16: 64 x 32 / 256; 3D: 32 x 16 x 16 / 512).
                                    No shape changes a result. */
    int32_t pad_;                /* reserved, 0 */
} ws_tuning;

/* ------------------------------------------------------------------------ */
/* context                                                                   */
/* ------------------------------------------------------------------------ */

/* Creates a context on CUDA device `device`.  workspace_budget_bytes bounds
 * the device memory the context may hold (0 = no bound).  Nothing is
 * allocated until the first call that needs workspace. */
ws_status ws_context_create(ws_context **out, int device, size_t workspace_budget_bytes);

/* Frees the context and its workspace.  The caller must make sure no work of
 * this context is still running (synchronise its streams first). */
void ws_context_destroy(ws_context *ctx);

/* Waits for `stream`, then reads and clears the device status word: WS_OK if
 * every call enqueued on this context since the last check completed, else
 * the first error recorded (WS_ERR_NONCONVERGED, WS_ERR_TIMEOUT, WS_ERR_OOM). */
ws_status ws_context_check(ws_context *ctx, ws_stream_t stream);

/* Human-readable message for the last error of this context ("" if none).
 * The pointer stays valid until the next call on the context. */
const char *ws_last_error(const ws_context *ctx);

/* Replaces the tuning knobs (zero fields keep their defaults). */
ws_status ws_context_set_tuning(ws_context *ctx, const ws_tuning *t);

/* Device bytes currently held by the context's workspace. */
size_t ws_context_workspace_bytes(const ws_context *ctx);

/* ------------------------------------------------------------------------ */
/* tracing                                                                   */
/* ------------------------------------------------------------------------ */

/* Turns per-phase CUDA-event timing on (enable != 0) or off.  When on, every
 * phase a call enqueues is bracketed by two events on the call's stream. */
ws_status ws_context_set_profiling(ws_context *ctx, int enable);

/* Number of timed phases, and the name of phase i ("step1", "plateau", ...). */
int ws_phase_count(void);
const char *ws_phase_name(int phase);

/* Waits for the events recorded since the last call, then writes the summed
 * device time (ms) and the number of timed instances of each phase into
 * total_ms[0..n) and calls[0..n) (either may be NULL) and resets the sums. */
ws_status ws_context_phase_times(ws_context *ctx, double *total_ms, long long *calls, int n);

/* Number of CUDA kernels this context has enqueued since it was created. */
unsigned long long ws_context_launches(const ws_context *ctx);

/* Counts the device kept for the last watershed call of this context (for a
 * batch: over all its images), after waiting for `stream`.  out[0..n) gets,
 * in this order (as many as n asks for, at most WS_NUM_COUNTERS):
 *   0  global rounds of the step II distance relaxation (Alg. 3's fixpoint)
 *   1  global rounds of step III pointer jumping on plateau tiles
 *   2  level-0 edge records of the waterfall (pairs of adjacent basins; a 2D
 *      call lists a pair once per tile that sees it)
 *   3  K0, the basins of level 0
 *   4  3D 6-connectivity: in-tile path ends chased across tiles
 *   5  tiles that hold plateau pixels
 *   6  2D: plateau pixels (states 2 and 3 of Eq. 1)
 * Returns WS_ERR_INVALID for a NULL context or out. */
#define WS_NUM_COUNTERS 7
ws_status ws_context_counters(ws_context *ctx, ws_stream_t stream, int64_t *out, int n);

/* ------------------------------------------------------------------------ */
/* hot path                                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Pipeline steps 1-2 of Sec. 1 (minimal smoothing, gradient magnitude; Fig. 2
 * marks both optional).  The paper names no operator; this library uses a
 * 5x5 binomial blur [1 4 6 4 1]^2 with (sum + 128) >> 8, a 3x3 integer
 * Sobel, the exact floor square root of gx^2 + gy^2 clipped to 255, then
 * >> quant_shift (0..7).  Borders replicate the edge pixel.
 *   img_d   uint8 [H*W] (2D only; shape->ndim must be 2)
 *   grad_d  uint8 [H*W] output; must not overlap img_d
 */
ws_status ws_gradient(ws_context *ctx, const uint8_t *img_d, const ws_shape *shape, int quant_shift,
                      uint8_t *grad_d, ws_stream_t stream);

/*
 * The same two steps for a volume (the paper names no operator; these are the
 * 3D counterparts of ws_gradient's): 5x5x5 binomial blur [1 4 6 4 1]^3 with
 * (sum + 2048) >> 12, 3x3x3 Sobel (central difference along one axis, [1 2 1]
 * along the other two), exact floor square root of gx^2 + gy^2 + gz^2, then
 * >> shift (0..31) and clipped to 65535.  Borders replicate the edge voxel.
 *   vol_d   uint8 or uint16 (dtype) [D*H*W], shape->ndim must be 3
 *   grad_d  uint16 [D*H*W] output; must not overlap vol_d
 */
ws_status ws_gradient3d(ws_context *ctx, const void *vol_d, ws_dtype dtype, const ws_shape *shape, int shift,
                        uint16_t *grad_d, ws_stream_t stream);

/*
 * Watershed, steps I-IV of Alg. 1 with the step II result of Sec. 3.3 / Alg. 3
 * (each non-minimal plateau pixel drains towards the nearest lower border of
 * its plateau; ties between equally near neighbours go to the larger pixel
 * index, as Eq. 1 does for steepest descent).
 *   grad_d        gradient samples, dtype WS_U8 or WS_U16, [N]
 *   connectivity  4 or 8 (ndim 2), 6 or 26 (ndim 3): the face neighbours, or
 *                 every voxel of the 3x3x3 cube around (Sec. 3.1: unit distance
 *                 in the chosen metric)
 *   labels_d      int32 [N] output, canonical basin ids 0..K-1
 *   count_d       int32 [1] output, K (may be NULL)
 */
ws_status ws_watershed(ws_context *ctx, const void *grad_d, ws_dtype dtype, const ws_shape *shape,
                       int connectivity, int32_t *labels_d, int32_t *count_d, ws_stream_t stream);

/*
 * Waterfall levels 1..NL-1 above given level-0 basins (Sec. 4, Alg. 4 with the
 * lowest passes of Alg. 5 step V).  pass(A, B) is the smallest
 * max(G(p), G(q)) over adjacent pixels p in A, q in B; newmin(A) is A's
 * lowest pass.  Level k+1 joins A and B whenever pass(A, B) equals newmin(A)
 * or newmin(B) (chains of such joins merge), so every level is a union of
 * regions of the level below.
 *   labels0_d  int32 [N] canonical level-0 labels (as ws_watershed writes them)
 *   NL         number of levels counting level 0 (Sec. 4), NL >= 1
 *   levels_d   int32 [(NL-1)*N] output, level k at offset (k-1)*N
 *   counts_d   int32 [NL] output, region count of levels 0..NL-1 (may be NULL)
 */
ws_status ws_waterfall(ws_context *ctx, const int32_t *labels0_d, const void *grad_d, ws_dtype dtype,
                       const ws_shape *shape, int connectivity, int NL, int32_t *levels_d,
                       int32_t *counts_d, ws_stream_t stream);

/*
 * The paper's own waterfall (Alg. 4 with the image reconstruction of Alg. 5):
 * level 0 is the watershed of G; for every further level, step V takes each
 * region's lowest pass newmin(A) (the smallest max(I(p), I(q)) over its
 * border pairs; M = 255 / 65535 when A has no neighbour), step VI raises every
 * pixel below newmin(L(p)) to it, and the watershed of the raised image is the
 * next level.  Unlike ws_segment's graph form, a level need not be a union of
 * regions of the level below (a pixel can change basin).  The caller's
 * gradient is not modified (the raised image lives in the workspace).
 *   levels_d  int32 [NL*N] output, level 0 first, canonical ids per level
 *   counts_d  int32 [NL] output (may be NULL);  1 <= NL <= 64
 */
ws_status ws_waterfall_reconstruct(ws_context *ctx, const void *grad_d, ws_dtype dtype, const ws_shape *shape,
                                   int connectivity, int NL, int32_t *levels_d, int32_t *counts_d,
                                   ws_stream_t stream);

/*
 * Region graph of one labelling, for graph-network pre-processing (Sec. 6: the
 * regions of a waterfall level replace superpixels as the nodes of the graph).
 * Node A is region id A (0..K-1, K = largest id + 1; ids no pixel carries are
 * isolated nodes of size 0).  Regions A != B share an edge when a pixel of A
 * has a pixel of B in its neighbourhood N(p) (Sec. 3.1, the connectivity
 * below); the edge weight is pass(A, B) of Alg. 5 step V, the smallest
 * max(G(p), G(q)) over those pixel pairs.  The graph is built into the context
 * and read out with ws_region_graph_read.  This call synchronises `stream`
 * (the sizes of the result are returned to the host).
 *   labels_d      int32 [N] ids >= 0 and below N (a level plane of ws_segment,
 *                 or any labelling); otherwise WS_ERR_INVALID
 *   grad_d        gradient [N] of `dtype`, the heights of the pass values
 *   values_d      value image for the node features: `channels` planes of N
 *                 samples, channel-major, WS_U8 or WS_U16 (NULL if channels = 0)
 *   regions       host int64 output: K (may be NULL)
 *   entries       host int64 output: CSR entries, twice the edge count (may be NULL)
 * Errors: WS_ERR_OOM when the region table is full (raise
 * ws_tuning.edge_capacity) or the workspace budget is exhausted.
 */
ws_status ws_region_graph(ws_context *ctx, const int32_t *labels_d, const void *grad_d, ws_dtype dtype,
                          const ws_shape *shape, int connectivity, const void *values_d, ws_dtype values_dtype,
                          int channels, int64_t *regions, int64_t *entries, ws_stream_t stream);

/*
 * Copies the last graph built by ws_region_graph in this context into caller
 * device buffers (each may be NULL to skip it); enqueued on `stream`:
 *   row_ptr_d  int64  [K+1]      CSR row starts (symmetric adjacency)
 *   col_d      int32  [entries]  neighbours of each row, increasing ids
 *   pass_d     uint32 [entries]  pass(A, B) of each entry
 *   size_d     int64  [K]        pixels per region
 *   sum_d      uint64 [K*channels]  value sums, region-major
 *   mean_d     double [K*channels]  sum / size (0 for an empty id)
 * WS_ERR_INVALID if no graph has been built.
 */
ws_status ws_region_graph_read(ws_context *ctx, int64_t *row_ptr_d, int32_t *col_d, uint32_t *pass_d,
                               int64_t *size_d, uint64_t *sum_d, double *mean_d, ws_stream_t stream);

/*
 * The whole hierarchy of Alg. 4: ws_watershed followed by ws_waterfall.
 *   levels_d  int32 [NL*N] output, level 0 first
 *   counts_d  int32 [NL] output (may be NULL)
 */
ws_status ws_segment(ws_context *ctx, const void *grad_d, ws_dtype dtype, const ws_shape *shape,
                     int connectivity, int NL, int32_t *levels_d, int32_t *counts_d,
                     ws_stream_t stream);

/*
 * ws_segment on HOST buffers: copies grad_h to the device, runs the
 * hierarchy, copies levels and counts back, and waits for completion before
 * returning (this call does synchronise `stream`).  Returns the device status
 * as ws_context_check would.
 *   grad_h    host gradient [N];  levels_h  host int32 [NL*N];  counts_h  host int32 [NL]
 */
ws_status ws_segment_host(ws_context *ctx, const void *grad_h, ws_dtype dtype, const ws_shape *shape,
                          int connectivity, int NL, int32_t *levels_h, int32_t *counts_h,
                          ws_stream_t stream);

/* ------------------------------------------------------------------------ */
/* batches                                                                   */
/* ------------------------------------------------------------------------ */

/* One image of a batch. */
typedef struct {
    const void *grad_d;   /* gradient samples [N], the batch's dtype */
    ws_shape shape;       /* its own size; every image of a batch has the same ndim */
    int32_t *levels_d;    /* int32 [NL*N] output, level 0 first (as ws_segment) */
    int32_t *counts_d;    /* int32 [NL] output (may be NULL) */
} ws_item;

/*
 * ws_segment for n images of uneven sizes at once (the hierarchy of Alg. 4
 * for each image).  The images are processed together: their pixels and tiles
 * are concatenated in the context's workspace and each phase is one launch
 * over all of them, so small images do not leave the GPU idle.  Every image's
 * result is exactly what ws_segment returns for it alone.
 *   items         n descriptors (host memory, read during the call)
 *   dtype, connectivity, NL   shared by all images; NL <= 64
 * The images' pixels must total below 2^31.
 */
ws_status ws_segment_batch(ws_context *ctx, int n, const ws_item *items, ws_dtype dtype, int connectivity, int NL,
                           ws_stream_t stream);

typedef struct ws_graph ws_graph;

/*
 * Records ws_segment_batch for this exact batch (same buffers) into a CUDA
 * graph: one eager run sizes the workspace and uploads the image descriptors
 * into memory owned by the graph, then the pipeline is captured.  Replaying it
 * with ws_graph_launch costs one graph launch per batch.  The graph uses the
 * context's workspace: calls on the context that grow the workspace
 * invalidate it (ws_graph_launch then returns WS_ERR_INVALID), and calls
 * whose work overlaps a replay on the device race with it.
 */
ws_status ws_graph_create(ws_context *ctx, int n, const ws_item *items, ws_dtype dtype, int connectivity, int NL,
                          ws_stream_t stream, ws_graph **out);
ws_status ws_graph_launch(ws_graph *g, ws_stream_t stream);
void ws_graph_destroy(ws_graph *g);

/* ------------------------------------------------------------------------ */
/* serving: a request loop with continuous batching                          */
/* ------------------------------------------------------------------------ */

typedef struct ws_server ws_server;

/* One partitioning request (the hierarchy of Alg. 4 for one image). */
typedef struct {
    const void *grad;     /* gradient samples [N]: host memory if on_host, else device memory */
    int32_t on_host;      /* 1: grad and the outputs are host memory (copied by the server) */
    int32_t connectivity; /* 4 / 8 (2D) or 6 / 26 (3D) */
    ws_dtype dtype;
    int32_t NL;           /* levels, counting level 0 */
    ws_shape shape;
    int32_t *levels;      /* int32 [NL*N] output (host or device, as grad) */
    int32_t *counts;      /* int32 [NL] output (may be NULL) */
} ws_request;

/*
 * Starts a server on `device`: a scheduler thread and n_lanes lanes, each with
 * its own context, stream and resident staging buffers.  Requests wait in a
 * queue; whenever a lane is free the scheduler takes the queued requests that
 * share the oldest one's dtype, connectivity, dimensionality and NL (up to
 * max_batch of them, within the lane's share of the memory budget) and runs
 * them as one batch (ws_segment_batch), so requests that arrive while others
 * are running are admitted as soon as a lane frees up and their work overlaps
 * on the device.  budget_bytes is split evenly between the lanes: a lane
 * admits requests while the sum of their estimated device footprints
 * (workspace, and staging of host buffers) fits its share, and its context's
 * workspace is capped at that share; 0 = no bound.  Host buffers should be
 * pinned (page-locked) so that their copies overlap other lanes' work.
 */
ws_status ws_server_create(ws_server **out, int device, size_t budget_bytes, int n_lanes, int max_batch);

/* Queues a request (its descriptor is copied; its buffers must stay valid
 * until ws_poll reports it finished).  Returns WS_ERR_OOM if the request
 * alone cannot fit a lane's share of the budget. */
ws_status ws_submit(ws_server *srv, const ws_request *req, uint64_t *ticket);

/* Waits up to timeout_us microseconds (0: do not wait, < 0: no limit) for a
 * request: WS_OK when its outputs are complete (host outputs included),
 * WS_ERR_NOT_READY if not yet, WS_ERR_CANCELLED, or the error that failed its
 * batch.  Once a final status has been returned the ticket is forgotten
 * (polling it again returns WS_ERR_INVALID). */
ws_status ws_poll(ws_server *srv, uint64_t ticket, int64_t timeout_us);

/* Cancels a request that is still queued (WS_OK); one already running
 * finishes normally (WS_ERR_NOT_READY is returned). */
ws_status ws_cancel(ws_server *srv, uint64_t ticket);

/* Stops the scheduler: queued requests are cancelled, running batches finish,
 * then every resource is released. */
void ws_server_destroy(ws_server *srv);

/* ------------------------------------------------------------------------ */
/* step-level entry points (for parity checks of individual steps)           */
/* ------------------------------------------------------------------------ */

/*
 * Step I alone (Alg. 1 step I, Eq. 1).
 *   states_d  uint8 [N] output: 0 lower neighbour, 1 strict minimum (or no
 *             neighbour), 2 plateau pixel whose chosen equal neighbour has a
 *             larger index, 3 one whose equal neighbours all have smaller ones
 *   arrows_d  int32 [N] output: q for states 0 and 2, p itself for 1 and 3
 */
ws_status ws_step1(ws_context *ctx, const void *grad_d, ws_dtype dtype, const ws_shape *shape,
                   int connectivity, uint8_t *states_d, int32_t *arrows_d, ws_stream_t stream);

/*
 * Step II distances (the fixpoint of Alg. 3, where -S is the distance):
 *   dist_d  int32 [N] output: 0 for state-0 pixels, the equal-valued path
 *           length to the nearest state-0 pixel of the plateau for plateau
 *           pixels that have one, -1 otherwise (state 1, minimal plateaux)
 */
ws_status ws_plateau_distance(ws_context *ctx, const void *grad_d, ws_dtype dtype,
                              const ws_shape *shape, int connectivity, int32_t *dist_d,
                              ws_stream_t stream);

/* ------------------------------------------------------------------------ */
/* watershed without device-memory allocation                                */
/* ------------------------------------------------------------------------ */

/* Largest image, in pixels, that ws_watershed_static accepts. */
#define WS_STATIC_MAX_PIXELS 524288

/* Size of the device array that holds all scratch of ws_watershed_static
 * (about 15.5 MB; the library checks this figure against its layout). */
#define WS_STATIC_SCRATCH_BYTES 15504384

/*
 * The result of ws_watershed (the same labels and the same count) for callers
 * that cannot allocate device memory: hosts that reserve all of the GPU's
 * memory for their own allocator, and latency-critical loops that cannot
 * afford the device-wide synchronisation of cudaMalloc and cudaFree.  The
 * paper has no counterpart: this is a deployment variant of the watershed.
 *
 * It needs no ws_context and allocates nothing.  All of its scratch lives in
 * one fixed device array inside the library (WS_STATIC_SCRATCH_BYTES), which
 * every GPU that loads the library holds until the process exits.
 *   - Images of at most WS_STATIC_MAX_PIXELS pixels; a larger image returns
 *     WS_ERR_INVALID and enqueues nothing (use ws_watershed instead).
 *   - grad_d, dtype, shape, connectivity, labels_d as in ws_watershed.
 *     count_d is required: it receives K, or -1 if the device detected an
 *     error during the call (an iteration or time limit reached).
 *   - Runs on the current device.  The first call on each device looks up the
 *     array's device address (cudaGetSymbolAddress) and keeps it; make that
 *     first call before any stream capture.
 *   - Every call uses the same array: calls whose work overlaps on the GPU
 *     (on different streams, or from different host threads) race and
 *     corrupt each other's results.  Issue them one after another on one
 *     stream, or synchronise between them.  Host threads may call it at the
 *     same time without harm to the library's host state (each call works on
 *     its own copy of it), but the results of GPU work that overlaps are
 *     undefined.
 *   - Each call starts by clearing the error state a failed earlier call may
 *     have left, so one call's device error never leaks into the next.
 */
ws_status ws_watershed_static(const void *grad_d, ws_dtype dtype, const ws_shape *shape, int connectivity,
                              int32_t *labels_d, int32_t *count_d, ws_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* WS_H */
