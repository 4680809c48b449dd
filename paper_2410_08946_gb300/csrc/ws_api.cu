// ws_api.cu -- the C ABI of libws (declared in include/ws.h): contexts,
// workspace management under a byte budget, argument validation, dispatch to
// the per-(dtype, connectivity) pipelines, the device status word.
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "ws_internal.h"

using namespace ws;

namespace ws {

int tune_plateau_cap(const ws_context *c) { return c->tun.plateau_round_cap > 0 ? c->tun.plateau_round_cap : (1 << 24); }
int tune_jump_cap(const ws_context *c) { return c->tun.jump_round_cap > 0 ? c->tun.jump_round_cap : 4096; }
int tune_rr(const ws_context *c) { return c->tun.jumps_per_round > 0 ? c->tun.jumps_per_round : 6; }
int tune_levels_ctas(const ws_context *c) { return c->tun.levels_ctas_per_sm > 0 ? c->tun.levels_ctas_per_sm : 4; }
unsigned long long tune_timeout_ns(ws_context *c)
{
    long long ms = c->tun.barrier_timeout_ms > 0 ? c->tun.barrier_timeout_ms : 4000;
    unsigned long long ns = (unsigned long long)ms * 1000000ull;
    if (c->hold_armed) {   // the one-shot hold of ws_tuning.barrier_withhold goes to this launch
        c->hold_armed = 0;
        ns |= kHold;
    }
    return ns;
}

ws_status set_cuda_error(ws_context *c, cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    c->err = buf;
    return e == cudaErrorMemoryAllocation ? WS_ERR_OOM : WS_ERR_CUDA;
}

static ws_status set_error(ws_context *c, ws_status st, const char *msg)
{
    c->err = msg;
    return st;
}

ws_status set_error_msg(ws_context *c, ws_status st, const char *msg) { return set_error(c, st, msg); }

template <typename P> static ws_status dalloc(ws_context *c, P **p, size_t bytes)
{
    if (c->budget && c->held + bytes > c->budget) {
        char buf[160];
        snprintf(buf, sizeof buf, "workspace budget exceeded: need %zu more bytes, %zu of %zu held", bytes,
                 c->held, c->budget);
        c->err = buf;
        return WS_ERR_OOM;
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_cuda_error(c, e, "cudaMalloc");
    }
    c->held += bytes;
    c->generation++;
    *p = (P *)q;
    return WS_OK;
}

template <typename P> static void dfree(ws_context *c, P **p, size_t bytes)
{
    if (*p) {
        cudaFree((void *)*p);
        c->held -= bytes;
        *p = nullptr;
    }
}

// Capacity to allocate when a workspace array of `unit` bytes per element must
// grow from `have` to at least `need` elements: 1.5x the old capacity (so that
// a stream of growing requests reallocates rarely; cudaFree synchronises the
// device), or exactly `need` when asked to or when the larger capacity would
// not fit the context's budget.
static size_t grown(const ws_context *c, size_t need, size_t have, bool exact, size_t unit)
{
    if (exact || have == 0) return need;
    const size_t g = have + have / 2;
    if (g <= need) return need;
    if (c->budget && c->held - have * unit + g * unit > c->budget) return need;
    return g;
}

static ws_status alloc_pixels(ws_context *c, size_t N)
{
    Workspace &w = c->w;
    ws_status st;
    // sizes first, so that free_pixels releases exactly what a partial failure allocated
    w.N = N;
    w.rmax = N / 2 + 2;
    w.nwords = (N + 31) / 32;
    w.ngroups = (w.nwords + 31) / 32;
    w.nchunks = (w.ngroups + 2047) / 2048;
    if ((st = dalloc(c, &w.par, N * 4)) || (st = dalloc(c, &w.aux, N * 4)) || (st = dalloc(c, &w.dist, N * 4)) ||
        (st = dalloc(c, &w.roots, w.rmax * 4)) || (st = dalloc(c, &w.rootm, w.rmax * 4)) ||
        (st = dalloc(c, &w.bitmap, w.nwords * 4)) || (st = dalloc(c, &w.gcnt, (w.ngroups + 1) * 4)) ||
        (st = dalloc(c, &w.csum, (w.nchunks + 1) * 4)))
        return st;
    cudaError_t e = cudaMemset(w.bitmap, 0, w.nwords * 4);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    return WS_OK;
}

static void free_pixels(ws_context *c)
{
    Workspace &w = c->w;
    dfree(c, &w.par, w.N * 4);
    dfree(c, &w.aux, w.N * 4);
    dfree(c, &w.dist, w.N * 4);
    dfree(c, &w.roots, w.rmax * 4);
    dfree(c, &w.rootm, w.rmax * 4);
    dfree(c, &w.bitmap, w.nwords * 4);
    dfree(c, &w.gcnt, (w.ngroups + 1) * 4);
    dfree(c, &w.csum, (w.nchunks + 1) * 4);
    w.N = w.rmax = w.nwords = w.ngroups = w.nchunks = 0;
}

ws_status ensure_pixels(ws_context *c, size_t N, size_t ntiles)
{
    Workspace &w = c->w;
    ws_status st = WS_OK;
    if (N > w.N) {
        const size_t have = w.N;
        free_pixels(c);
        if ((st = alloc_pixels(c, grown(c, N, have, false, 17))) != WS_OK) {
            free_pixels(c);
            if ((st = alloc_pixels(c, N)) != WS_OK) return st;
        }
    }
    if (ntiles > w.ntiles) {
        const size_t have = w.ntiles;
        for (int exact = 0; exact < 2; exact++) {
            dfree(c, &w.plat, w.ntiles);
            dfree(c, &w.act, w.ntiles * 2);
            dfree(c, &w.tlist, w.ntiles * 4);
            w.ntiles = 0;
            const size_t n = grown(c, ntiles, have, exact, 7);
            if ((st = dalloc(c, &w.plat, n)) || (st = dalloc(c, &w.act, n * 2)) || (st = dalloc(c, &w.tlist, n * 4))) {
                w.ntiles = n;  // so that the frees above release what was allocated
                continue;
            }
            w.ntiles = n;
            return WS_OK;
        }
        dfree(c, &w.plat, w.ntiles);
        dfree(c, &w.act, w.ntiles * 2);
        dfree(c, &w.tlist, w.ntiles * 4);
        w.ntiles = 0;
        return st;
    }
    return WS_OK;
}

// Grows the region table to cap slots.  The old arrays are released by
// cudaFree (which waits for the work that may still use them); the new ones
// are initialised on `s`, ahead of the calls that use them.
ws_status ensure_edges(ws_context *c, size_t cap, cudaStream_t s)
{
    Workspace &w = c->w;
    if (cap <= w.edge_cap) return WS_OK;
    dfree(c, &w.keys, w.edge_cap * 8);
    dfree(c, &w.vals, w.edge_cap * 4);
    dfree(c, &w.slots, w.edge_cap * 4);
    dfree(c, (uint8_t **)&w.ea, w.edge_cap * 12);
    dfree(c, (uint8_t **)&w.eb, w.edge_cap * 12);
    w.edge_cap = 0;
    ws_status st;
    if ((st = dalloc(c, &w.keys, cap * 8)) || (st = dalloc(c, &w.vals, cap * 4)) ||
        (st = dalloc(c, &w.slots, cap * 4)) || (st = dalloc(c, (uint8_t **)&w.ea, cap * 12)) ||
        (st = dalloc(c, (uint8_t **)&w.eb, cap * 12)))
        return st;
    cudaError_t e = cudaMemsetAsync(w.keys, 0xff, cap * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.vals, 0xff, cap * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ecount, 0, 4, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    w.edge_cap = cap;
    return WS_OK;
}

ws_status ensure_regions(ws_context *c, size_t kmax, int levels)
{
    Workspace &w = c->w;
    if (kmax <= w.kmax && levels <= w.levels_cap) return WS_OK;
    size_t nk = kmax > w.kmax ? kmax : w.kmax;
    int nl = levels > w.levels_cap ? levels : w.levels_cap;
    dfree(c, &w.gmap, w.kmax * 4 * (size_t)w.levels_cap);
    dfree(c, &w.newmin, w.kmax * 4);
    dfree(c, &w.uf, w.kmax * 4);
    dfree(c, &w.rank, w.kmax * 4);
    w.kmax = 0;
    w.levels_cap = 0;
    ws_status st;
    if ((st = dalloc(c, &w.gmap, nk * 4 * (size_t)nl)) || (st = dalloc(c, &w.newmin, nk * 4)) ||
        (st = dalloc(c, &w.uf, nk * 4)) || (st = dalloc(c, &w.rank, nk * 4)))
        return st;
    w.kmax = nk;
    w.levels_cap = nl;
    return WS_OK;
}

static cudaEvent_t prof_event(ws_context *c)
{
    if (!c->prof.pool.empty()) {
        cudaEvent_t e = c->prof.pool.back();
        c->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

PhaseScope::PhaseScope(ws_context *c_, int ph_, cudaStream_t s_) : c(c_), ph(ph_), s(s_)
{
    if (!c->prof.on) return;
    a = prof_event(c);
    if (a) cudaEventRecord(a, s);
}

PhaseScope::~PhaseScope()
{
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    if (!b) {
        c->prof.pool.push_back(a);
        return;
    }
    cudaEventRecord(b, s);
    c->prof.pending.push_back({ph, a, b});
}

static const char *const PHASE_NAMES[NPHASE] = {"step1",       "plateau", "resolve_union", "jump",
                                                "compact",     "rag",     "levels",        "level_write",
                                                "cleanup",     "gradient", "copy",          "chase",
                                                "export",      "reconstruct"};

ws_status ensure_ends(ws_context *c, size_t N, size_t ntiles)
{
    Workspace &w = c->w;
    ws_status st;
    if (N > w.ncode) {
        const size_t have = w.ncode;
        dfree(c, &w.code, w.ncode * 2);
        dfree(c, &w.ends, w.ncode * 8);
        w.ncode = grown(c, N, have, false, 10);
        if ((st = dalloc(c, &w.code, w.ncode * 2)) || (st = dalloc(c, &w.ends, w.ncode * 8))) {
            dfree(c, &w.code, w.ncode * 2);
            dfree(c, &w.ends, w.ncode * 8);
            w.ncode = 0;
            return st;
        }
    }
    if (ntiles > w.ntends) {
        const size_t have = w.ntends;
        dfree(c, &w.tends, w.ntends * 8);
        w.ntends = grown(c, ntiles, have, false, 8);
        if ((st = dalloc(c, &w.tends, w.ntends * 8))) {
            w.ntends = 0;
            return st;
        }
    }
    return WS_OK;
}

ws_status ensure_plist(ws_context *c, size_t N, size_t ntiles)
{
    Workspace &w = c->w;
    ws_status st;
    if (N > w.nplist) {
        const size_t have = w.nplist;
        dfree(c, &w.plist, w.nplist * 2);
        w.nplist = grown(c, N, have, false, 2);
        if ((st = dalloc(c, &w.plist, w.nplist * 2))) {
            w.nplist = 0;
            return st;
        }
    }
    if (ntiles > w.npspan) {
        const size_t have = w.npspan;
        dfree(c, &w.pspan, w.npspan * 8);
        w.npspan = grown(c, ntiles, have, false, 8);
        if ((st = dalloc(c, &w.pspan, w.npspan * 8))) {
            w.npspan = 0;
            return st;
        }
    }
    return WS_OK;
}

// Region-graph export arrays: K regions (node sizes and CSR row starts), `sums`
// value sums, `entries` directed edge entries (two key/value buffers for the
// radix sort, digit counts of 4096-entry tiles).
ws_status ensure_rgraph(ws_context *c, size_t K, size_t sums, size_t entries)
{
    Workspace::RGraph &r = c->w.rg;
    ws_status st;
    if (!r.misc && (st = dalloc(c, &r.misc, 16))) return st;
    if (K > r.kcap) {
        const size_t have = r.kcap;
        dfree(c, &r.size, r.kcap * 8);
        dfree(c, &r.row, (r.kcap + 1) * 4);
        r.kcap = grown(c, K, have, false, 12);
        if ((st = dalloc(c, &r.size, r.kcap * 8)) || (st = dalloc(c, &r.row, (r.kcap + 1) * 4))) {
            dfree(c, &r.size, r.kcap * 8);
            r.kcap = 0;
            return st;
        }
    }
    if (sums > r.scap) {
        const size_t have = r.scap;
        dfree(c, &r.sum, r.scap * 8);
        r.scap = grown(c, sums, have, false, 8);
        if ((st = dalloc(c, &r.sum, r.scap * 8))) {
            r.scap = 0;
            return st;
        }
    }
    if (entries > r.ecap) {
        const size_t have = r.ecap;
        for (int i = 0; i < 2; i++) {
            dfree(c, &r.key[i], r.ecap * 8);
            dfree(c, &r.val[i], r.ecap * 4);
        }
        dfree(c, &r.hist, r.hcap * 4);
        dfree(c, &r.hsum, (r.hcap / 2048 + 2) * 4);
        r.ecap = grown(c, entries, have, false, 24);
        r.hcap = 256 * ((r.ecap + 4095) / 4096);
        for (int i = 0; i < 2; i++)
            if ((st = dalloc(c, &r.key[i], r.ecap * 8)) || (st = dalloc(c, &r.val[i], r.ecap * 4))) break;
        if (st == WS_OK && !(st = dalloc(c, &r.hist, r.hcap * 4))) st = dalloc(c, &r.hsum, (r.hcap / 2048 + 2) * 4);
        if (st) {
            for (int i = 0; i < 2; i++) {
                dfree(c, &r.key[i], r.ecap * 8);
                dfree(c, &r.val[i], r.ecap * 4);
            }
            dfree(c, &r.hist, r.hcap * 4);
            dfree(c, &r.hsum, (r.hcap / 2048 + 2) * 4);
            r.ecap = r.hcap = 0;
            return st;
        }
    }
    return WS_OK;
}

ws_status ensure_rec(ws_context *c, size_t bytes)
{
    Workspace &w = c->w;
    if (bytes <= w.rec_n) return WS_OK;
    const size_t have = w.rec_n;
    dfree(c, (uint8_t **)&w.rec, w.rec_n);
    w.rec_n = grown(c, bytes, have, false, 1);
    ws_status st = dalloc(c, (uint8_t **)&w.rec, w.rec_n);
    if (st) w.rec_n = 0;
    return st;
}

// Edge-table slots of a call over npix pixels (the sizing in run_core).
size_t edge_slots(size_t npix, int conn, const ws_context *c)
{
    // every pixel puts at most one pair per forward neighbour (halfn of them),
    // so npix * halfn slots never overflow below the 2^28 cap (a checkerboard
    // of strict minima comes close: a pair for almost every forward neighbour)
    const int halfn = conn == 26 ? 13 : conn / 2;
    size_t want = npix * (size_t)halfn;
    if (c && c->tun.edge_capacity > 0) want = (size_t)c->tun.edge_capacity;
    size_t cap = 1 << 16;
    while (cap < want && cap < ((size_t)1 << 28)) cap <<= 1;
    return cap;
}

size_t workspace_bound(size_t npix, size_t ntiles, size_t nimg, int conn, int NL, bool additive)
{
    size_t b = npix * 17 + ntiles * 7 + 4096;                      // per-pixel and per-tile arrays
    if (conn == 6) b += npix * 10 + ntiles * 8;                    // 3D slot codes, path ends, slot spans
    if (conn == 4 || conn == 8) b += npix * 2 + ntiles * 8;        // 2D plateau pixel lists
    if (nimg > 1) b += nimg * (kDescBytes + 4);                    // batch descriptors
    if (NL > 1) {
        const size_t kmax = npix / 2 + nimg + 2;
        b += kmax * (4 * (size_t)(NL - 1) + 12);                   // region graph arrays
        // region table and edge lists; additive: a bound that holds for any
        // batch summing such requests (twice the wanted slots covers the
        // power-of-two rounding of the sum)
        const int halfn = conn == 26 ? 13 : conn / 2;
        b += (additive ? 2 * npix * (size_t)halfn + ((size_t)1 << 16) : edge_slots(npix, conn, nullptr)) * 40;
    }
    return b;
}

void release_workspace(ws_context *c)
{
    Workspace &w = c->w;
    cudaDeviceSynchronize();
    free_pixels(c);
    dfree(c, &w.plat, w.ntiles);
    dfree(c, &w.act, w.ntiles * 2);
    dfree(c, &w.tlist, w.ntiles * 4);
    w.ntiles = 0;
    dfree(c, &w.code, w.ncode * 2);
    dfree(c, &w.ends, w.ncode * 8);
    w.ncode = 0;
    dfree(c, &w.tends, w.ntends * 8);
    w.ntends = 0;
    dfree(c, &w.plist, w.nplist * 2);
    w.nplist = 0;
    dfree(c, &w.pspan, w.npspan * 8);
    w.npspan = 0;
    dfree(c, &w.keys, w.edge_cap * 8);
    dfree(c, &w.vals, w.edge_cap * 4);
    dfree(c, &w.slots, w.edge_cap * 4);
    dfree(c, (uint8_t **)&w.ea, w.edge_cap * 12);
    dfree(c, (uint8_t **)&w.eb, w.edge_cap * 12);
    w.edge_cap = 0;
    dfree(c, &w.gmap, w.kmax * 4 * (size_t)w.levels_cap);
    dfree(c, &w.newmin, w.kmax * 4);
    dfree(c, &w.uf, w.kmax * 4);
    dfree(c, &w.rank, w.kmax * 4);
    w.kmax = 0;
    w.levels_cap = 0;
    dfree(c, &w.descs, w.nbatch * kDescBytes);
    dfree(c, &w.rbase, (w.nbatch + 1) * 4);
    w.nbatch = 0;
}

ws_status ensure_batch(ws_context *c, size_t n)
{
    Workspace &w = c->w;
    if (n <= w.nbatch) return WS_OK;
    dfree(c, &w.descs, w.nbatch * kDescBytes);
    dfree(c, &w.rbase, (w.nbatch + 1) * 4);
    w.nbatch = 0;
    ws_status st;
    if ((st = dalloc(c, (uint8_t **)&w.descs, n * kDescBytes)) || (st = dalloc(c, &w.rbase, (n + 1) * 4))) return st;
    w.nbatch = n;
    return WS_OK;
}

const Launchers *launchers(int dtype, int conn)
{
    if (dtype == WS_U8) return launchers_u8(conn);
    if (dtype == WS_U16) return launchers_u16(conn);
    return nullptr;
}

const Launchers *launchers_for(const ws_context *c, int dtype, int conn)
{
    if (dtype == WS_U8 && (conn == 4 || conn == 8) && c->tun.tile_shape > 0)
        return launchers_u8_shape(conn, c->tun.tile_shape);
    return launchers(dtype, conn);
}

}  // namespace ws

// ---------------------------------------------------------------------------
// argument validation
// ---------------------------------------------------------------------------

static ws_status make_geo(ws_context *c, const ws_shape *shape, Geo *g)
{
    if (!shape) return set_error(c, WS_ERR_INVALID, "shape is NULL");
    if (shape->ndim != 2 && shape->ndim != 3) return set_error(c, WS_ERR_INVALID, "ndim must be 2 or 3");
    int64_t W = shape->dims[0], H = shape->dims[1], D = shape->ndim == 3 ? shape->dims[2] : 1;
    if (W < 1 || H < 1 || D < 1) return set_error(c, WS_ERR_INVALID, "every dimension must be >= 1");
    if (W > 0x7fffffff || H > 0x7fffffff || D > 0x7fffffff || W * H > 0x7fffffffLL ||
        W * H * D > 0x7fffffffLL)
        return set_error(c, WS_ERR_INVALID, "image too large: N must be below 2^31");
    g->W = (int)W;
    g->H = (int)H;
    g->D = (int)D;
    g->HW = (int)(W * H);
    g->N = (int)(W * H * D);
    return WS_OK;
}

static ws_status check_conn(ws_context *c, const ws_shape *shape, int conn)
{
    if (shape->ndim == 2 && (conn == 4 || conn == 8)) return WS_OK;
    if (shape->ndim == 3 && (conn == 6 || conn == 26)) return WS_OK;
    return set_error(c, WS_ERR_INVALID, "connectivity must be 4 or 8 (2D) or 6 or 26 (3D)");
}

static ws_status prep(ws_context *c, const void *grad, int dtype, const ws_shape *shape, int conn, Geo *g,
                      const Launchers **L)
{
    if (!c) return WS_ERR_INVALID;
    c->err.clear();
    ws_status st = make_geo(c, shape, g);
    if (st) return st;
    if ((st = check_conn(c, shape, conn))) return st;
    if (dtype != WS_U8 && dtype != WS_U16) return set_error(c, WS_ERR_INVALID, "dtype must be WS_U8 or WS_U16");
    if (!grad) return set_error(c, WS_ERR_INVALID, "gradient pointer is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != c->device) {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return set_cuda_error(c, e, "cudaSetDevice");
    }
    *L = launchers_for(c, dtype, conn);
    if (!*L) return set_error(c, WS_ERR_UNSUPPORTED, "no pipeline for this dtype / connectivity");
    return WS_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

ws_status ws_context_create(ws_context **out, int device, size_t budget)
{
    if (!out) return WS_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 ? WS_ERR_INVALID : WS_ERR_CUDA;
    }
    ws_context *c = new (std::nothrow) ws_context();
    if (!c) return WS_ERR_OOM;
    c->device = device;
    c->budget = budget;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        return WS_ERR_CUDA;
    }
    ws_status st = dalloc(c, &c->status, sizeof(DevStatus));
    if (st == WS_OK) st = dalloc(c, &c->w.ecount, 4);
    if (st == WS_OK) st = dalloc(c, &c->w.bsum, 4096 * 4);
    if (st == WS_OK) st = dalloc(c, &c->w.kcount, 4);
    if (st == WS_OK) st = dalloc(c, &c->w.counters, 16);
    if (st == WS_OK) st = dalloc(c, &c->w.lcount, kMaxLevels * 4);
    if (st == WS_OK) st = dalloc(c, &c->w.ecnt, kMaxLevels * 4);
    if (st == WS_OK) {
        e = cudaMemset(c->status, 0, sizeof(DevStatus));
        if (e == cudaSuccess) e = cudaMemset(c->w.ecount, 0, 4);
        if (e == cudaSuccess) e = cudaMemset(c->w.kcount, 0, 4);
        if (e != cudaSuccess) st = WS_ERR_CUDA;
    }
    if (st != WS_OK) {
        ws_context_destroy(c);
        return st;
    }
    *out = c;
    return WS_OK;
}

void ws_context_destroy(ws_context *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    Workspace &w = c->w;
    cudaFree(c->status);
    void *ptrs[] = {w.par,   w.aux,    w.dist,   w.plat,   w.act,    w.tlist,  w.roots,  w.rootm,
                    w.counters, w.bitmap, w.gcnt, w.csum,   w.keys,   w.vals,   w.slots,  w.ecount,
                    w.gmap,  w.newmin, w.uf,     w.rank,   w.bsum,   w.kcount, w.grad_stage, w.levels_stage,
                    w.counts_stage, w.descs, w.rbase, w.lcount, w.ea, w.eb, w.ecnt, w.code, w.ends, w.tends,
                    w.plist, w.pspan};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    const Workspace::RGraph &r = w.rg;
    void *rptrs[] = {r.size, r.sum, r.row, r.key[0], r.key[1], r.val[0], r.val[1], r.hist, r.hsum, r.misc, w.rec};
    for (void *p : rptrs)
        if (p) cudaFree(p);
    for (auto &r : c->prof.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    delete c;
}

ws_status ws_context_check(ws_context *c, ws_stream_t stream)
{
    if (!c) return WS_ERR_INVALID;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(c, e, "stream synchronize");
    DevStatus h;
    e = cudaMemcpy(&h, c->status, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(c, e, "status read");
    if (h.code == 0) return WS_OK;
    cudaMemset(c->status, 0, sizeof(DevStatus));
    char buf[200];
    const char *what = "device error";
    switch (h.where) {
    case 2: what = "step II plateau relaxation reached its round cap"; break;
    case 3: what = "Union retry cap reached"; break;
    case 4: what = "Union retry cap reached"; break;
    case 5: what = "step III pointer jumping reached its round cap"; break;
    case 6: what = "region adjacency table full (raise ws_tuning.edge_capacity)"; break;
    case 7: what = "step II found a plateau pixel with no neighbour one step closer"; break;
    case 8: what = "level-0 labels out of range (expected canonical ids 0..K-1)"; break;
    case 9: what = "root chase exceeded its hop cap"; break;
    case 100: what = "device-wide barrier timed out"; break;
    }
    snprintf(buf, sizeof buf, "%s (code %d, site %d)", what, h.code, h.where);
    c->err = buf;
    return (ws_status)h.code;
}

const char *ws_last_error(const ws_context *c) { return c ? c->err.c_str() : "no context"; }

ws_status ws_context_set_profiling(ws_context *c, int enable)
{
    if (!c) return WS_ERR_INVALID;
    c->prof.on = enable != 0;
    return WS_OK;
}

int ws_phase_count(void) { return NPHASE; }

const char *ws_phase_name(int phase) { return (phase >= 0 && phase < NPHASE) ? PHASE_NAMES[phase] : ""; }

ws_status ws_context_phase_times(ws_context *c, double *total_ms, long long *calls, int n)
{
    if (!c || n < 0) return WS_ERR_INVALID;
    cudaSetDevice(c->device);
    Prof &P = c->prof;
    for (auto &r : P.pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        P.total_ms[r.phase] += ms;
        P.calls[r.phase] += 1;
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    P.pending.clear();
    for (int i = 0; i < n && i < NPHASE; i++) {
        if (total_ms) total_ms[i] = P.total_ms[i];
        if (calls) calls[i] = P.calls[i];
    }
    for (int i = 0; i < NPHASE; i++) {
        P.total_ms[i] = 0;
        P.calls[i] = 0;
    }
    return WS_OK;
}

unsigned long long ws_context_launches(const ws_context *c) { return c ? c->launches : 0; }

ws_status ws_context_counters(ws_context *c, ws_stream_t stream, int64_t *out, int n)
{
    if (!c || !out) return WS_ERR_INVALID;
    DevStatus st{};
    int32_t cnt[4] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&st, c->status, sizeof st, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && c->w.counters) e = cudaMemcpy(cnt, c->w.counters, sizeof cnt, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(c, e, "counters");
    const int64_t v[WS_NUM_COUNTERS] = {st.rounds_plateau, st.rounds_jump, st.edges, cnt[1], cnt[2], cnt[0], cnt[3]};
    for (int i = 0; i < n && i < WS_NUM_COUNTERS; i++) out[i] = v[i];
    return WS_OK;
}

ws_status ws_context_set_tuning(ws_context *c, const ws_tuning *t)
{
    if (!c || !t) return WS_ERR_INVALID;
    if (t->plateau_round_cap < 0 || t->jump_round_cap < 0 || t->jumps_per_round < 0 || t->barrier_timeout_ms < 0 ||
        t->edge_capacity < 0 || t->levels_ctas_per_sm < 0)
        return set_error(c, WS_ERR_INVALID, "tuning values must be >= 0");
    if (t->levels_ctas_per_sm > 32) return set_error(c, WS_ERR_INVALID, "levels_ctas_per_sm must be <= 32");
    if (t->barrier_withhold != 0 && t->barrier_withhold != 1)
        return set_error(c, WS_ERR_INVALID, "barrier_withhold must be 0 or 1");
    if (t->tile_shape < 0 || t->tile_shape > 3) return set_error(c, WS_ERR_INVALID, "tile_shape must be in 0..3");
    c->tun = *t;
    c->hold_armed = t->barrier_withhold;
    c->tun.barrier_withhold = 0;
    return WS_OK;
}

size_t ws_context_workspace_bytes(const ws_context *c) { return c ? c->held : 0; }

ws_status ws_gradient(ws_context *c, const uint8_t *img_d, const ws_shape *shape, int quant_shift, uint8_t *grad_d,
                      ws_stream_t stream)
{
    if (!c) return WS_ERR_INVALID;
    c->err.clear();
    Geo g;
    ws_status st = make_geo(c, shape, &g);
    if (st) return st;
    if (shape->ndim != 2) return set_error(c, WS_ERR_UNSUPPORTED, "ws_gradient takes 2D images");
    if (!img_d || !grad_d) return set_error(c, WS_ERR_INVALID, "NULL buffer");
    if (quant_shift < 0 || quant_shift > 7) return set_error(c, WS_ERR_INVALID, "quant_shift must be 0..7");
    if ((const void *)img_d == (const void *)grad_d) return set_error(c, WS_ERR_INVALID, "img and grad overlap");
    cudaSetDevice(c->device);
    return launch_gradient(c, img_d, g.W, g.H, quant_shift, grad_d, (cudaStream_t)stream);
}

ws_status ws_gradient3d(ws_context *c, const void *vol_d, ws_dtype dtype, const ws_shape *shape, int shift,
                        uint16_t *grad_d, ws_stream_t stream)
{
    if (!c) return WS_ERR_INVALID;
    c->err.clear();
    Geo g;
    ws_status st = make_geo(c, shape, &g);
    if (st) return st;
    if (shape->ndim != 3) return set_error(c, WS_ERR_UNSUPPORTED, "ws_gradient3d takes volumes (ndim 3)");
    if (!vol_d || !grad_d) return set_error(c, WS_ERR_INVALID, "NULL buffer");
    if (dtype != WS_U8 && dtype != WS_U16) return set_error(c, WS_ERR_INVALID, "dtype must be WS_U8 or WS_U16");
    if (shift < 0 || shift > 31) return set_error(c, WS_ERR_INVALID, "shift must be 0..31");
    if (g.D > 65535 * 8) return set_error(c, WS_ERR_UNSUPPORTED, "depth above 524280");
    const size_t bps = dtype == WS_U8 ? 1 : 2;
    const char *a = (const char *)vol_d, *b = (const char *)grad_d;
    if (a < b + (size_t)g.N * 2 && b < a + (size_t)g.N * bps)
        return set_error(c, WS_ERR_INVALID, "volume and gradient overlap");
    cudaSetDevice(c->device);
    return launch_gradient3d(c, vol_d, (int)bps, g.W, g.H, g.D, shift, grad_d, (cudaStream_t)stream);
}

ws_status ws_step1(ws_context *c, const void *grad_d, ws_dtype dtype, const ws_shape *shape, int conn,
                   uint8_t *states_d, int32_t *arrows_d, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!states_d || !arrows_d) return set_error(c, WS_ERR_INVALID, "NULL output");
    return L->step1(c, grad_d, g, states_d, arrows_d, (cudaStream_t)stream);
}

ws_status ws_plateau_distance(ws_context *c, const void *grad_d, ws_dtype dtype, const ws_shape *shape, int conn,
                              int32_t *dist_d, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!dist_d) return set_error(c, WS_ERR_INVALID, "NULL output");
    return L->plateau_distance(c, grad_d, g, dist_d, (cudaStream_t)stream);
}

ws_status ws_watershed(ws_context *c, const void *grad_d, ws_dtype dtype, const ws_shape *shape, int conn,
                       int32_t *labels_d, int32_t *count_d, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!labels_d) return set_error(c, WS_ERR_INVALID, "NULL labels");
    return L->watershed(c, grad_d, g, labels_d, count_d, (cudaStream_t)stream);
}

ws_status ws_waterfall(ws_context *c, const int32_t *labels0_d, const void *grad_d, ws_dtype dtype,
                       const ws_shape *shape, int conn, int NL, int32_t *levels_d, int32_t *counts_d,
                       ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!labels0_d) return set_error(c, WS_ERR_INVALID, "NULL labels0");
    if (NL < 1) return set_error(c, WS_ERR_INVALID, "NL must be >= 1");
    if (NL > 1 && !levels_d) return set_error(c, WS_ERR_INVALID, "NULL levels");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = launch_count_labels(c, labels0_d, g.N, s))) return st;
    return L->waterfall(c, labels0_d, grad_d, g, NL, levels_d, counts_d, (size_t)g.N, s);
}

ws_status ws_waterfall_reconstruct(ws_context *c, const void *grad_d, ws_dtype dtype, const ws_shape *shape,
                                   int conn, int NL, int32_t *levels_d, int32_t *counts_d, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!levels_d) return set_error(c, WS_ERR_INVALID, "NULL levels");
    if (NL < 1 || NL > kMaxLevels) return set_error(c, WS_ERR_INVALID, "NL must be in 1..64");
    return L->reconstruct(c, grad_d, g, NL, levels_d, counts_d, (cudaStream_t)stream);
}

ws_status ws_region_graph(ws_context *c, const int32_t *labels_d, const void *grad_d, ws_dtype dtype,
                          const ws_shape *shape, int conn, const void *values_d, ws_dtype values_dtype, int channels,
                          int64_t *regions, int64_t *entries, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!labels_d) return set_error(c, WS_ERR_INVALID, "NULL labels");
    if (channels < 0 || channels > 65536) return set_error(c, WS_ERR_INVALID, "channels must be in 0..65536");
    if (channels > 0 && !values_d) return set_error(c, WS_ERR_INVALID, "NULL values with channels > 0");
    if (channels > 0 && values_dtype != WS_U8 && values_dtype != WS_U16)
        return set_error(c, WS_ERR_INVALID, "values dtype must be WS_U8 or WS_U16");
    long long K = 0, n = 0;
    st = region_graph_build(c, labels_d, grad_d, dtype, g, conn, values_d, values_dtype, channels, &K, &n,
                            (cudaStream_t)stream);
    if (st) return st;
    if (regions) *regions = K;
    if (entries) *entries = n;
    return WS_OK;
}

ws_status ws_region_graph_read(ws_context *c, int64_t *row_ptr_d, int32_t *col_d, uint32_t *pass_d,
                               int64_t *size_d, uint64_t *sum_d, double *mean_d, ws_stream_t stream)
{
    if (!c) return WS_ERR_INVALID;
    c->err.clear();
    cudaSetDevice(c->device);
    return region_graph_read(c, row_ptr_d, col_d, pass_d, size_d, sum_d, mean_d, (cudaStream_t)stream);
}

ws_status ws_segment(ws_context *c, const void *grad_d, ws_dtype dtype, const ws_shape *shape, int conn, int NL,
                     int32_t *levels_d, int32_t *counts_d, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_d, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!levels_d) return set_error(c, WS_ERR_INVALID, "NULL levels");
    if (NL < 1) return set_error(c, WS_ERR_INVALID, "NL must be >= 1");
    return L->segment(c, grad_d, g, NL, levels_d, counts_d, (cudaStream_t)stream);
}

ws_status ws_segment_host(ws_context *c, const void *grad_h, ws_dtype dtype, const ws_shape *shape, int conn,
                          int NL, int32_t *levels_h, int32_t *counts_h, ws_stream_t stream)
{
    Geo g;
    const Launchers *L = nullptr;
    ws_status st = prep(c, grad_h, dtype, shape, conn, &g, &L);
    if (st) return st;
    if (!levels_h || NL < 1) return set_error(c, WS_ERR_INVALID, "NULL levels or NL < 1");
    Workspace &w = c->w;
    // staging buffers, grown on demand (host_n = bytes of the levels buffer,
    // grad_n = bytes of the gradient buffer)
    size_t b = dtype == WS_U8 ? 1 : 2;
    size_t levels_bytes = (size_t)NL * g.N * 4, grad_bytes = (size_t)g.N * b;
    if (levels_bytes > w.host_n) {
        dfree(c, &w.levels_stage, w.host_n);
        w.host_n = 0;
        if ((st = dalloc(c, &w.levels_stage, levels_bytes))) return st;
        w.host_n = levels_bytes;
    }
    if (grad_bytes > w.grad_n) {
        dfree(c, &w.grad_stage, w.grad_n);
        w.grad_n = 0;
        if ((st = dalloc(c, &w.grad_stage, grad_bytes))) return st;
        w.grad_n = grad_bytes;
    }
    if (!w.counts_stage && (st = dalloc(c, &w.counts_stage, 64 * 4))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    {
        PhaseScope ps(c, PH_COPY, s);
        e = cudaMemcpyAsync(w.grad_stage, grad_h, (size_t)g.N * b, cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "H2D copy");
    int32_t *cnt = NL <= 64 ? w.counts_stage : nullptr;
    if ((st = L->segment(c, w.grad_stage, g, NL, w.levels_stage, cnt, s))) return st;
    {
        PhaseScope ps(c, PH_COPY, s);
        e = cudaMemcpyAsync(levels_h, w.levels_stage, levels_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && counts_h && cnt)
            e = cudaMemcpyAsync(counts_h, cnt, (size_t)NL * 4, cudaMemcpyDeviceToHost, s);
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "D2H copy");
    return ws_context_check(c, stream);
}

static ws_status prep_batch(ws_context *c, int n, const ws_item *items, ws_dtype dtype, int conn, int NL,
                            std::vector<Geo> &geos, const Launchers **L)
{
    if (!c) return WS_ERR_INVALID;
    c->err.clear();
    if (n < 1 || !items) return set_error(c, WS_ERR_INVALID, "empty batch");
    if (NL < 1 || NL > kMaxLevels) return set_error(c, WS_ERR_INVALID, "NL must be in 1..64 for a batch");
    geos.resize((size_t)n);
    for (int i = 0; i < n; i++) {
        ws_status st = make_geo(c, &items[i].shape, &geos[i]);
        if (st) return st;
        if (items[i].shape.ndim != items[0].shape.ndim) return set_error(c, WS_ERR_INVALID, "mixed ndim in a batch");
        if (!items[i].grad_d || !items[i].levels_d) return set_error(c, WS_ERR_INVALID, "NULL buffer in a batch item");
    }
    ws_status st = check_conn(c, &items[0].shape, conn);
    if (st) return st;
    if (dtype != WS_U8 && dtype != WS_U16) return set_error(c, WS_ERR_INVALID, "dtype must be WS_U8 or WS_U16");
    cudaSetDevice(c->device);
    *L = launchers_for(c, dtype, conn);
    if (!*L) return set_error(c, WS_ERR_UNSUPPORTED, "no pipeline for this dtype / connectivity");
    return WS_OK;
}

ws_status ws_segment_batch(ws_context *c, int n, const ws_item *items, ws_dtype dtype, int conn, int NL,
                           ws_stream_t stream)
{
    std::vector<Geo> geos;
    const Launchers *L = nullptr;
    ws_status st = prep_batch(c, n, items, dtype, conn, NL, geos, &L);
    if (st) return st;
    return L->segment_batch(c, n, geos.data(), items, NL, nullptr, (cudaStream_t)stream);
}

struct ws_graph {
    ws_context *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *descs = nullptr;        // the batch's image descriptors (owned)
    unsigned long long generation = 0;
};

void ws_graph_destroy(ws_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->descs) cudaFree(g->descs);
    delete g;
}

ws_status ws_graph_create(ws_context *c, int n, const ws_item *items, ws_dtype dtype, int conn, int NL,
                          ws_stream_t stream, ws_graph **out)
{
    if (!out) return WS_ERR_INVALID;
    *out = nullptr;
    std::vector<Geo> geos;
    const Launchers *L = nullptr;
    ws_status st = prep_batch(c, n, items, dtype, conn, NL, geos, &L);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // eager run: sizes the workspace and checks the batch
    if ((st = L->segment_batch(c, n, geos.data(), items, NL, nullptr, s))) return st;
    if ((st = ws_context_check(c, stream))) return st;
    ws_graph *g = new (std::nothrow) ws_graph();
    if (!g) return WS_ERR_OOM;
    g->ctx = c;
    std::vector<unsigned char> host(L->desc_bytes * (size_t)n);
    L->descs(n, geos.data(), items, host.data());
    cudaError_t e = cudaMalloc(&g->descs, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->descs, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ws_graph_destroy(g);
        return set_cuda_error(c, e, "graph descriptors");
    }
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cap) cudaStreamDestroy(cap);
        ws_graph_destroy(g);
        return set_cuda_error(c, e, "begin capture");
    }
    const int prof = c->prof.on;
    c->prof.on = 0;
    const unsigned long long gen = c->generation;
    st = L->segment_batch(c, n, geos.data(), items, NL, g->descs, cap);
    c->prof.on = prof;
    e = cudaStreamEndCapture(cap, &g->graph);
    cudaStreamDestroy(cap);
    if (st == WS_OK && e == cudaSuccess && c->generation != gen)
        st = set_error(c, WS_ERR_INVALID, "workspace changed during capture");
    if (st != WS_OK || e != cudaSuccess) {
        ws_graph_destroy(g);
        return st != WS_OK ? st : set_cuda_error(c, e, "capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        ws_graph_destroy(g);
        return set_cuda_error(c, e, "graph instantiate");
    }
    g->generation = gen;
    *out = g;
    return WS_OK;
}

ws_status ws_graph_launch(ws_graph *g, ws_stream_t stream)
{
    if (!g || !g->exec) return WS_ERR_INVALID;
    if (g->ctx->generation != g->generation)
        return set_error(g->ctx, WS_ERR_INVALID, "the context's workspace changed since the graph was recorded");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? WS_OK : set_cuda_error(g->ctx, e, "graph launch");
}

}  // extern "C"
