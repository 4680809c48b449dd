// ws_internal.h -- host-side internals of libws shared by its translation
// units: the context (workspace, tuning, device status word) and the
// per-(dtype, connectivity) launcher table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ws.h"
#include "ws_device.cuh"

namespace ws {

// Tile shapes of the step II relaxation (one CTA relaxes one tile in shared
// memory with a one-pixel frozen halo).
struct TileGeo {
    int TX, TY, TZ;
    int ntx, nty, ntz;
    int ntiles;
};

// Workspace held by a context; every array is sized for the largest image
// seen so far and stays resident between calls.
struct Workspace {
    size_t N = 0;           // pixels the per-pixel arrays can hold
    int32_t *par = nullptr; // in-tile path ends, then roots (3D 6-connectivity:
                            // the arrows of plateau tiles only)              [N]
    int32_t *aux = nullptr; // smallest index per root, then canonical id    [N]
    int32_t *dist = nullptr;// step II distances (plateau tiles only)        [N]
    size_t ntiles = 0;
    uint8_t *plat = nullptr;  // tile holds plateau pixels                   [ntiles]
    uint8_t *act = nullptr;   // active-tile flags, two rounds               [2*ntiles]
    int32_t *tlist = nullptr; // list of plateau tiles                       [ntiles]
    size_t rmax = 0;
    int32_t *roots = nullptr; // list of basin roots                         [rmax]
    int32_t *rootm = nullptr; // smallest pixel index of each listed root    [rmax]
    int32_t *counters = nullptr;  // plateau tiles, roots, path ends, ...    [4]
    // 3D path ends: per pixel the slot of its in-tile path end, per tile the
    // span of its slots in `ends` ((end pixel, next pixel of its path), then
    // (root, root))
    size_t ncode = 0, ntends = 0;
    uint16_t *code = nullptr;     // [ncode]
    int2 *ends = nullptr;         // [ncode]
    int2 *tends = nullptr;        // (first slot, slot count) per tile  [ntends]
    // 2D path: the plateau pixels of every tile (tile-local indices), per tile
    // the span of its entries in plist
    size_t nplist = 0, npspan = 0;
    uint16_t *plist = nullptr;    // [nplist]
    int2 *pspan = nullptr;        // (first entry, entry count) per tile [npspan]
    size_t nwords = 0, ngroups = 0, nchunks = 0;
    uint32_t *bitmap = nullptr;   // one bit per pixel index (kept zero)     [nwords]
    int32_t *gcnt = nullptr;      // popcount per 32-word group, then prefix [ngroups]
    int32_t *csum = nullptr;      // scan chunk sums                         [nchunks + 1]
    size_t nbatch = 0;
    void *descs = nullptr;        // image descriptors of a batch            [nbatch]
    int32_t *rbase = nullptr;     // global id of each image's first basin   [nbatch + 1]
    // region adjacency hash table
    size_t edge_cap = 0;            // power of two
    unsigned long long *keys = nullptr;  // (a << 32 | b), empty = ~0
    uint32_t *vals = nullptr;       // pass value (min height), empty = ~0
    int32_t *slots = nullptr;       // used slots, in insertion order [edge_cap]
    int32_t *ecount = nullptr;      // number of used slots             [1]
    void *ea = nullptr, *eb = nullptr;  // region-graph edge lists (a, b, pass), 12 B each [edge_cap]
    int32_t *ecnt = nullptr;        // edges of each level             [kMaxLevels]
    // region graph arrays (level-0 region count K0 <= kmax)
    size_t kmax = 0;
    int levels_cap = 0;             // NL-1 the gmap array can hold
    int32_t *gmap = nullptr;        // level-0 id -> level-k id, [levels_cap][kmax]
    uint32_t *newmin = nullptr;     // [kmax]
    int32_t *uf = nullptr;          // [kmax]
    int32_t *rank = nullptr;        // [kmax]
    int32_t *bsum = nullptr;        // per-block sums for device-wide scans [4096]
    int32_t *kcount = nullptr;      // K0 of the last watershed [1]
    int32_t *lcount = nullptr;      // region count per level of the last batch [kMaxLevels]
    // region-graph export (ws_region_graph): the last graph built
    struct RGraph {
        long long K = 0, nnz = 0;   // regions, directed entries (twice the edges)
        int C = 0;                  // value channels
        int valid = 0;              // a graph is held
        int sorted = 0;             // which key/val buffer holds the sorted entries
        int shift = 0;              // bits of a column in a key
        size_t kcap = 0, scap = 0, ecap = 0, hcap = 0;
        unsigned long long *size = nullptr;   // pixels per region          [kcap]
        unsigned long long *sum = nullptr;    // value sums, region-major   [scap]
        int32_t *row = nullptr;               // CSR row starts             [kcap + 1]
        unsigned long long *key[2] = {};      // (row << shift | col)       [ecap]
        uint32_t *val[2] = {};                // pass values                [ecap]
        int32_t *hist = nullptr;              // radix digit counts, then offsets [hcap]
        int32_t *hsum = nullptr;              // scan chunk sums            [hcap / 2048 + 2]
        int32_t *misc = nullptr;              // largest id, negative-id flag, edges, K [4]
    } rg;
    // reconstructed image of the paper-literal waterfall
    size_t rec_n = 0;
    void *rec = nullptr;
    // host-copy staging for ws_segment_host
    size_t host_n = 0, grad_n = 0;
    uint8_t *grad_stage = nullptr;  // device copy of a host gradient
    int32_t *levels_stage = nullptr;
    int32_t *counts_stage = nullptr;
};

// Phases timed by the optional event profiler (ws_context_set_profiling).
enum Phase {
    PH_STEP1 = 0,     // Eq. 1 states and arrows
    PH_PLATEAU,       // step II distances
    PH_RESOLVE,       // step II pointer choice + step IV Union
    PH_JUMP,          // step III pointer jumping + smallest index per basin
    PH_COMPACT,       // canonical ids
    PH_RAG,           // region adjacency (pass values)
    PH_LEVELS,        // lowest-pass merging on the region graph
    PH_LEVEL_WRITE,   // per-pixel level planes
    PH_CLEANUP,       // edge table reset
    PH_GRADIENT,      // blur + Sobel
    PH_COPY,          // host <-> device copies of ws_segment_host
    PH_CHASE,         // roots of the 3D tiles' path ends
    PH_EXPORT,        // region-graph export
    PH_RECON,         // image reconstruction (Alg. 5 steps V-VI)
    NPHASE
};

struct Prof {
    int on = 0;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double total_ms[NPHASE] = {};
    long long calls[NPHASE] = {};
};

}  // namespace ws

struct ws_context {
    int device = 0;
    size_t budget = 0;       // 0 = unbounded
    size_t held = 0;         // bytes held by the workspace
    std::string err;
    ws_tuning tun{};
    ws::DevStatus *status = nullptr;
    ws::Workspace w;
    int num_sms = 0;
    unsigned long long launches = 0;  // kernels enqueued by this context
    unsigned long long generation = 0; // bumped whenever workspace is reallocated
    int hold_armed = 0;                // ws_tuning.barrier_withhold, not yet handed to a launch
    ws::Prof prof;
};

namespace ws {

// Brackets one phase with timing events when profiling is on.
struct PhaseScope {
    ws_context *c;
    int ph;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(ws_context *c_, int ph_, cudaStream_t s_);
    ~PhaseScope();
};

// Largest NL of a batched call (per-level totals are kept in a fixed array).
constexpr int kMaxLevels = 64;

// Bytes reserved per image descriptor of a batch (>= sizeof(ImgDesc)).
constexpr size_t kDescBytes = 128;

// Effective tuning values.
int tune_plateau_cap(const ws_context *c);
int tune_jump_cap(const ws_context *c);
int tune_rr(const ws_context *c);
int tune_levels_ctas(const ws_context *c);
// The barrier time limit of the next cooperative launch (it also hands over
// an armed ws_tuning.barrier_withhold, once).
unsigned long long tune_timeout_ns(ws_context *c);

// Workspace management (ws_api.cu).
ws_status ensure_pixels(ws_context *c, size_t N, size_t ntiles);
ws_status ensure_edges(ws_context *c, size_t cap, cudaStream_t s);
ws_status ensure_regions(ws_context *c, size_t kmax, int levels);
ws_status ensure_batch(ws_context *c, size_t n);
ws_status ensure_ends(ws_context *c, size_t N, size_t ntiles);
ws_status ensure_plist(ws_context *c, size_t N, size_t ntiles);

ws_status ensure_rgraph(ws_context *c, size_t K, size_t sums, size_t entries);
ws_status ensure_rec(ws_context *c, size_t bytes);
// Region-table slots of a call over npix pixels (c: the context's tuning, or nullptr).
size_t edge_slots(size_t npix, int conn, const ws_context *c);
// Upper bound of the workspace bytes a call (a batch of nimg images, npix
// pixels and ntiles tiles in all) needs; additive: a per-request bound whose
// sum over a batch bounds the batch.
size_t workspace_bound(size_t npix, size_t ntiles, size_t nimg, int conn, int NL, bool additive);
// Frees every workspace array of the context (after a device synchronisation).
void release_workspace(ws_context *c);
ws_status set_error_msg(ws_context *c, ws_status st, const char *msg);
ws_status set_cuda_error(ws_context *c, cudaError_t e, const char *what);

// Launchers instantiated per (sample type, connectivity).
struct Launchers {
    ws_status (*watershed)(ws_context *, const void *grad, const Geo &, int32_t *labels,
                           int32_t *count, cudaStream_t);
    ws_status (*step1)(ws_context *, const void *grad, const Geo &, uint8_t *states, int32_t *arrows,
                       cudaStream_t);
    ws_status (*plateau_distance)(ws_context *, const void *grad, const Geo &, int32_t *dist,
                                  cudaStream_t);
    ws_status (*waterfall)(ws_context *, const int32_t *labels0, const void *grad, const Geo &, int NL,
                           int32_t *levels, int32_t *counts, size_t kmax, cudaStream_t);
    ws_status (*segment)(ws_context *, const void *grad, const Geo &, int NL, int32_t *levels, int32_t *counts,
                         cudaStream_t);
    ws_status (*segment_batch)(ws_context *, int n, const Geo *geos, const ws_item *items, int NL,
                               const void *descs_dev, cudaStream_t);
    size_t desc_bytes;                // sizeof one image descriptor
    void (*descs)(int n, const Geo *geos, const ws_item *items, void *out);  // host descriptors, desc_bytes each
    ws_status (*reconstruct)(ws_context *, const void *grad, const Geo &, int NL, int32_t *levels, int32_t *counts,
                             cudaStream_t);
};

// dtype: 0 = u8, 1 = u16; conn: 4, 8, 6, 26.  Returns nullptr when unsupported.
const Launchers *launchers(int dtype, int conn);
// The same for a context: 2D uint8 images take the tile shape of its tuning.
const Launchers *launchers_for(const ws_context *c, int dtype, int conn);

// Instantiation entry points (one per translation unit).
const Launchers *launchers_u8(int conn);
const Launchers *launchers_u16(int conn);
// 2D uint8 on tile shape 1..3 (ws_tuning.tile_shape); nullptr otherwise.
const Launchers *launchers_u8_shape(int conn, int shape);

// K0 = max(labels) + 1 into c->w.kcount (ws_gradient.cu).
ws_status launch_count_labels(ws_context *c, const int32_t *labels, int N, cudaStream_t s);

// Region-graph export (ws_rgraph.cu): builds the graph of `labels` into c->w.rg
// and returns K and the directed entry count (synchronises the stream).
ws_status region_graph_build(ws_context *c, const int32_t *labels, const void *grad, int dtype, const Geo &g,
                             int conn, const void *values, int vdtype, int C, long long *K, long long *nnz,
                             cudaStream_t s);
ws_status region_graph_read(ws_context *c, int64_t *row_ptr, int32_t *col, uint32_t *pass, int64_t *size,
                            uint64_t *sum, double *mean, cudaStream_t s);

// Gradient (ws_gradient.cu).
ws_status launch_gradient(ws_context *c, const uint8_t *img, int W, int H, int shift, uint8_t *grad,
                          cudaStream_t s);
ws_status launch_gradient3d(ws_context *c, const void *vol, int bps, int W, int H, int D, int shift,
                            uint16_t *grad, cudaStream_t s);

}  // namespace ws
