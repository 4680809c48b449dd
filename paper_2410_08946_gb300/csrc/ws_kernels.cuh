// ws_kernels.cuh -- the kernels and device helpers of libws that are not
// tiled: the union-find, the scans, the region table and the
// graph-form waterfall, and Alg. 5's image reconstruction; templated on the
// gradient sample type T (uint8_t / uint16_t) and the connectivity CONN (4, 8
// in 2D; 6, 26 in 3D) where they touch pixels.  The tiled watershed pipeline
// (steps I-IV, canonical ids, adjacency, level planes) is in ws_tiles.cuh.
//
//   uf_find/uf_union global union-find (path halving; atomicCAS links the
//                    larger root under the smaller)
//   k_scan_chunks / k_scan / k_scan_add
//                    device-wide exclusive scan in chunks of 2048
//   edge_insert_slot / edge_insert / append_slots
//                    the region table: open addressing on (a << 32 | b) with
//                    the min pass per pair, new slots listed (one counter
//                    atomic per warp where the caller is warp-uniform)
//   k_rag            Alg. 5 step V on pixel pairs of a caller's labelling:
//                    pass(A,B) = min over adjacent pixels of max(G(p), G(q)),
//                    warp-deduplicated into the region table
//   EdgeSink, sink_put1 / sink_put_warp
//                    where the segmentation path's adjacency kernels put
//                    their pairs of basins: an appended list (2D) or the
//                    region table (3D)
//   k_edges_compact  region table -> dense edge list in canonical level-0 ids
//                    (and the table emptied)
//   k_edges_ids      the segmentation path's edge list -> canonical level-0
//                    ids, in place
//   k_levels         NL-1 rounds of lowest-pass merging on the region graph
//                    (newmin, Union over kept edges, canonical ids, the next
//                    level's id per region, contracted edges); cooperative
//   k_level_write    levels[k][p] = map_k[L0[p]] for all k in one pass
//   k_fill_newmin, k_newmin, k_raise
//                    ws_waterfall_reconstruct: Alg. 5 steps V and VI between
//                    two watersheds of the paper-literal hierarchy (Alg. 4)
#pragma once

#include <cooperative_groups.h>

#include "ws_device.cuh"
#include "ws_internal.h"

namespace ws {

constexpr int INF_D = 0x3fffffff;   // "no distance" (INF_D + 1 does not overflow)
constexpr int NTHR = 256;           // threads per CTA of the per-pixel kernels
constexpr unsigned long long EMPTY_KEY = ~0ull;

template <int CONN> struct PTile {
    static constexpr int ND = Dim<CONN>::nd;
    static constexpr int TX = ND == 2 ? 32 : 16;
    static constexpr int TY = ND == 2 ? 32 : 8;
    static constexpr int TZ = ND == 2 ? 1 : 8;
    static constexpr int HX = TX + 2, HY = TY + 2, HZ = ND == 2 ? 1 : TZ + 2;
    static constexpr int HS = HX * HY * HZ;
    static constexpr int NPIX = TX * TY * TZ;
    static constexpr int PER_THR = NPIX / NTHR;
};

template <int CONN> inline TileGeo make_tilegeo(const Geo &g)
{
    using PT = PTile<CONN>;
    TileGeo t;
    t.TX = PT::TX;
    t.TY = PT::TY;
    t.TZ = PT::TZ;
    t.ntx = (g.W + PT::TX - 1) / PT::TX;
    t.nty = (g.H + PT::TY - 1) / PT::TY;
    t.ntz = (g.D + PT::TZ - 1) / PT::TZ;
    t.ntiles = t.ntx * t.nty * t.ntz;
    return t;
}

static __device__ __forceinline__ void coords(const Geo &g, int p, int &x, int &y, int &z)
{
    z = p / g.HW;
    int r = p - z * g.HW;
    y = r / g.W;
    x = r - y * g.W;
}

template <int CONN>
static __device__ __forceinline__ bool nb_at(const Geo &g, int x, int y, int z, int i, int &q)
{
    int xx = x + Nb<CONN>::dx(i), yy = y + Nb<CONN>::dy(i), zz = z + Nb<CONN>::dz(i);
    if (xx < 0 || xx >= g.W || yy < 0 || yy >= g.H || zz < 0 || zz >= g.D) return false;
    q = (zz * g.H + yy) * g.W + xx;
    return true;
}

// ---------------------------------------------------------------------------
// Union-Find (step IV of Alg. 1 and the region graph merge)
// ---------------------------------------------------------------------------

static __device__ __forceinline__ int uf_find(int32_t *par, int a)
{
    volatile int32_t *vp = par;
    for (;;) {
        int b = vp[a];
        if (b == a) return a;
        int c = vp[b];
        if (c == b) return b;
        vp[a] = c;  // path halving: c is an ancestor of a
        a = c;
    }
}

static __device__ __forceinline__ void uf_union(int32_t *par, int a, int b, DevStatus *s)
{
    for (int it = 0; it < (1 << 20); it++) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) return;
        if (a < b) {
            int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(par + a, a, b) == a) return;
    }
    record_error(s, DEV_NONCONVERGED, 4);
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------

// Exclusive scan of blk[0..n) in place, total to blk[n] (one CTA of 1024).
static __global__ void __launch_bounds__(1024) k_scan(int32_t *blk, int n, int32_t *total_out)
{
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < n ? blk[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int excl = carry + (wid ? wsum[wid - 1] : 0) + x - v;
        if (i < n) blk[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        blk[n] = carry;
        if (total_out) *total_out = carry;
    }
}

// Device-wide exclusive scan, step 1: each CTA scans SCAN_CHUNK elements of
// a in place and writes the chunk total to sums[blockIdx.x].
constexpr int SCAN_CHUNK = 2048;
static __global__ void __launch_bounds__(NTHR) k_scan_chunks(int32_t *a, int n, int32_t *sums)
{
    __shared__ int wsum[NTHR / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int base = blockIdx.x * SCAN_CHUNK;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int j = 0; j < SCAN_CHUNK; j += NTHR) {
        const int i = base + j + threadIdx.x;
        const int v = i < n ? a[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        int off = carry;
        for (int w = 0; w < wid; w++) off += wsum[w];
        if (i < n) a[i] = off + x - v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < NTHR / 32; w++) s += wsum[w];
            carry += s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = carry;
}

// step 3: add the scanned chunk offsets
static __global__ void __launch_bounds__(NTHR) k_scan_add(int32_t *a, int n, const int32_t *__restrict__ sums)
{
    const int off = sums[blockIdx.x];
    for (int j = threadIdx.x; j < SCAN_CHUNK; j += NTHR) {
        const int i = blockIdx.x * SCAN_CHUNK + j;
        if (i < n) a[i] += off;
    }
}

static __global__ void k_copy_int(const int32_t *src, int32_t *dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
}

// ---------------------------------------------------------------------------
// waterfall: region adjacency (Alg. 5 step V on pixel pairs)
// ---------------------------------------------------------------------------

// One edge of the region graph: regions a < b and their pass value.
struct Edge {
    int a, b;
    unsigned h;
};

// Where the segmentation path's adjacency kernels put their pairs of basins
// (a < b, root pixels) with the lowest pass each one saw:
//   - a list (HASHED = false): records appended at e[*n], a pair found by several
//     tiles once per tile.  The waterfall needs no more (its merge rule reads a
//     pair's minimum over all its records), and appends cost far less than
//     the table's atomics; 2D images, whose small basins rarely meet across
//     tiles, take it.  A record past cap is dropped and reported as a full
//     table.
//   - the region table (HASHED = true): one record per pair; 3D volumes,
//     whose large basins meet across many tiles, take it.
// The choice is fixed per kernel instantiation (a template parameter of the
// put functions), so a kernel carries the code of one of them only.
struct EdgeSink {
    Edge *e;
    int32_t *n;
    int cap;
    unsigned long long *keys;
    uint32_t *vals;
    int32_t *slots;
    int32_t *ecount;
    unsigned long long gmask;
};

static __device__ __forceinline__ unsigned long long mix64(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Inserts (key, h) into the region table (open addressing, min of h per key).
// Returns the slot when this call created the key -- the caller then lists
// it in `slots` -- and -1 otherwise (or when the table is full: error 6).
static __device__ __forceinline__ int edge_insert_slot(unsigned long long key, unsigned h, unsigned long long *keys,
                                                      uint32_t *vals, unsigned long long mask, DevStatus *status)
{
    unsigned long long s = mix64(key) & mask;
    for (int probe = 0; probe < 4096; probe++) {
        unsigned long long k = *(volatile unsigned long long *)(keys + s);
        if (k == key) {
            atomicMin(vals + s, h);
            return -1;
        }
        if (k == EMPTY_KEY) {
            unsigned long long old = atomicCAS(keys + s, EMPTY_KEY, key);
            if (old == EMPTY_KEY) {
                atomicMin(vals + s, h);
                return (int)s;
            }
            if (old == key) {
                atomicMin(vals + s, h);
                return -1;
            }
        }
        s = (s + 1) & mask;
    }
    record_error(status, DEV_EDGE_TABLE_FULL, 6);
    return -1;
}

// One lane's insert, listing a new key at once.
static __device__ __forceinline__ void edge_insert(unsigned long long key, unsigned h, unsigned long long *keys,
                                                   uint32_t *vals, int32_t *slots, int32_t *ecount,
                                                   unsigned long long mask, DevStatus *status)
{
    const int s = edge_insert_slot(key, h, keys, vals, mask, status);
    if (s >= 0) slots[atomicAdd(ecount, 1)] = s;
}

// Called by all 32 lanes of a warp: lists the lanes' new slots (s >= 0) with
// one atomic on the slot counter for the whole warp.
static __device__ __forceinline__ void append_slots(int s, int32_t *slots, int32_t *ecount)
{
    const unsigned m = __ballot_sync(0xffffffffu, s >= 0);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(ecount, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (s >= 0) slots[base + __popc(m & ((1u << lane) - 1u))] = s;
}

static __device__ __forceinline__ void list_put(const EdgeSink &S, int i, unsigned a, unsigned b, unsigned h,
                                                DevStatus *status)
{
    if (i >= S.cap) {
        record_error(status, DEV_EDGE_TABLE_FULL, 14);
        return;
    }
    int *q = reinterpret_cast<int *>(S.e + i);
    q[0] = (int)a;
    q[1] = (int)b;
    q[2] = (int)h;
}

// One pair from any thread.
template <bool HASHED>
static __device__ __forceinline__ void sink_put1(const EdgeSink &S, unsigned a, unsigned b, unsigned h,
                                                 DevStatus *status)
{
    if (HASHED)
        edge_insert(((unsigned long long)a << 32) | b, h, S.keys, S.vals, S.slots, S.ecount, S.gmask, status);
    else
        list_put(S, atomicAdd(S.n, 1), a, b, h, status);
}

// The pairs of the lanes with have == true; every lane of the warp calls it
// (one counter atomic per warp).
template <bool HASHED>
static __device__ __forceinline__ void sink_put_warp(const EdgeSink &S, bool have, unsigned a, unsigned b,
                                                     unsigned h, DevStatus *status)
{
    if (HASHED) {
        const int sl = have ? edge_insert_slot(((unsigned long long)a << 32) | b, h, S.keys, S.vals, S.gmask, status)
                            : -1;
        append_slots(sl, S.slots, S.ecount);
        return;
    }
    const unsigned m = __ballot_sync(0xffffffffu, have);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(S.n, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (have) list_put(S, base + __popc(m & ((1u << lane) - 1u)), a, b, h, status);
}

template <typename T, int CONN>
static __global__ void __launch_bounds__(NTHR) k_rag(const T *__restrict__ g, Geo geo, const int32_t *__restrict__ L,
                                              unsigned long long *keys, uint32_t *vals, int32_t *slots,
                                              int32_t *ecount, unsigned long long mask, DevStatus *status)
{
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * NTHR;
    const int nIter = (geo.N + stride - 1) / stride;
    for (int it = 0; it < nIter; it++) {
        int p = it * stride + blockIdx.x * NTHR + threadIdx.x;
        bool in = p < geo.N;
        int x = 0, y = 0, z = 0, A = 0;
        unsigned gp = 0;
        if (in) {
            coords(geo, p, x, y, z);
            A = L[p];
            gp = g[p];
        }
#pragma unroll
        for (int i = Half<CONN>::first; i < Nb<CONN>::n; i++) {
            int q;
            bool has = false;
            unsigned long long key = 0;
            unsigned h = 0;
            if (in && nb_at<CONN>(geo, x, y, z, i, q)) {
                int B = L[q];
                if (B != A && A >= 0 && B >= 0) {
                    has = true;
                    int a = imin(A, B), b = imax(A, B);
                    key = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
                    unsigned gq = g[q];
                    h = gp > gq ? gp : gq;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, has);
            if (!m) continue;   // warp-uniform
            int sl = -1;
            if (has) {
                const unsigned grp = __match_any_sync(m, key);
                const unsigned hmin = __reduce_min_sync(grp, h);
                if (lane == __ffs(grp) - 1) sl = edge_insert_slot(key, hmin, keys, vals, mask, status);
            }
            append_slots(sl, slots, ecount);
        }
    }
}

// ---------------------------------------------------------------------------
// paper-literal waterfall: image reconstruction (Alg. 5 steps V, VI)
// ---------------------------------------------------------------------------

// newmin[0..K) = ~0 (K read on the device: the watershed's region count).
static __global__ void __launch_bounds__(NTHR) k_fill_newmin(uint32_t *newmin, const int32_t *kptr)
{
    const int K = *kptr;
    for (int a = blockIdx.x * NTHR + threadIdx.x; a < K; a += gridDim.x * NTHR) newmin[a] = 0xffffffffu;
}

// Step V: newmin(L(p)) = min over neighbours q in another region of
// max(I(p), I(q)).  Each unordered pixel pair is visited once (forward
// neighbours) and lowers both regions; a lane reads the current value first
// and issues the atomic only when it lowers it.
template <typename T, int CONN>
static __global__ void __launch_bounds__(NTHR) k_newmin(const T *__restrict__ I, Geo geo, const int32_t *__restrict__ L,
                                                        uint32_t *newmin)
{
    for (int p = blockIdx.x * NTHR + threadIdx.x; p < geo.N; p += gridDim.x * NTHR) {
        int x, y, z;
        coords(geo, p, x, y, z);
        const int A = L[p];
        const unsigned ip = I[p];
#pragma unroll
        for (int i = Half<CONN>::first; i < Nb<CONN>::n; i++) {
            int q;
            if (!nb_at<CONN>(geo, x, y, z, i, q)) continue;
            const int B = L[q];
            if (B == A) continue;
            const unsigned iq = I[q];
            const unsigned h = ip > iq ? ip : iq;
            if (h < __ldcg(newmin + A)) atomicMin(newmin + A, h);
            if (h < __ldcg(newmin + B)) atomicMin(newmin + B, h);
        }
    }
}

// Step VI: out(p) = newmin(L(p)) where I(p) is below it, else I(p); a region
// with no neighbour has newmin = M, the sample type's maximum.  in == out is
// allowed (element-wise).
template <typename T>
static __global__ void __launch_bounds__(NTHR) k_raise(const T *in, T *out, const int32_t *__restrict__ L,
                                                       const uint32_t *__restrict__ newmin, int N)
{
    constexpr unsigned M = sizeof(T) == 1 ? 0xffu : 0xffffu;
    for (int p = blockIdx.x * NTHR + threadIdx.x; p < N; p += gridDim.x * NTHR) {
        unsigned nm = __ldg(newmin + L[p]);
        nm = nm < M ? nm : M;
        const unsigned v = in[p];
        out[p] = (T)(v < nm ? nm : v);
    }
}

// ---------------------------------------------------------------------------
// waterfall: lowest-pass merging on the region graph (cooperative)
// ---------------------------------------------------------------------------

static __device__ __forceinline__ int block_sum(int v, int *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    return s;
}

// Edge lists are rewritten between levels by other CTAs: read them from L2.
__device__ __forceinline__ Edge ld_edge(const Edge *p)
{
    const int *q = reinterpret_cast<const int *>(p);
    Edge e;
    e.a = __ldcg(q);
    e.b = __ldcg(q + 1);
    e.h = (unsigned)__ldcg(q + 2);
    return e;
}

// Region table -> dense edge list in canonical level-0 ids (idmap maps the
// table's keys, root pixels, to ids; nullptr: keys are ids already).  Every
// used slot is returned to empty on the way, and the slot count is reset.
static __global__ void __launch_bounds__(NTHR) k_edges_compact(unsigned long long *keys, uint32_t *vals,
                                                               const int32_t *__restrict__ slots, int32_t *ecount,
                                                               const int32_t *__restrict__ idmap,
                                                               const int32_t *__restrict__ k0_ptr, Edge *edges,
                                                               int32_t *lcnt, DevStatus *status)
{
    const int E = *ecount;
    const int K0 = *k0_ptr;
    for (int e = blockIdx.x * NTHR + threadIdx.x; e < E; e += gridDim.x * NTHR) {
        const int s = slots[e];
        const unsigned long long key = keys[s];
        int a = (int)(key >> 32), b = (int)(key & 0xffffffffu);
        if (idmap) {
            a = idmap[a];
            b = idmap[b];
        }
        Edge ed;
        if ((unsigned)a < (unsigned)K0 && (unsigned)b < (unsigned)K0) {
            ed.a = a < b ? a : b;
            ed.b = a < b ? b : a;
            ed.h = vals[s];
        } else {  // only after an earlier device error: a self-loop is ignored
            ed.a = ed.b = 0;
            ed.h = 0;
        }
        edges[e] = ed;
        keys[s] = EMPTY_KEY;
        vals[s] = 0xffffffffu;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) status->edges = E;
    (void)lcnt;
}

// The segmentation path's edge list (lcnt[0] records, at most cap kept) ->
// the level-0 edge list in canonical ids, in place; lcnt[0] clamped to cap
// and lcnt[1..nl-1] cleared for k_levels.
static __global__ void __launch_bounds__(NTHR) k_edges_ids(Edge *edges, int32_t *lcnt, int nl, int cap,
                                                           const int32_t *__restrict__ idmap, int npix,
                                                           const int32_t *__restrict__ k0_ptr, DevStatus *status)
{
    const int E = min(*(volatile int32_t *)lcnt, cap);
    const int K0 = *k0_ptr;
    for (int e = blockIdx.x * NTHR + threadIdx.x; e < E; e += gridDim.x * NTHR) {
        int *q = reinterpret_cast<int *>(edges + e);
        const int ra = q[0], rb = q[1];
        const int a = (unsigned)ra < (unsigned)npix ? idmap[ra] : -1;
        const int b = (unsigned)rb < (unsigned)npix ? idmap[rb] : -1;
        if ((unsigned)a < (unsigned)K0 && (unsigned)b < (unsigned)K0) {
            q[0] = a < b ? a : b;
            q[1] = a < b ? b : a;
        } else {  // only after an earlier device error: a self-loop is ignored
            q[0] = q[1] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        for (int k = 1 + threadIdx.x; k < nl; k += 32) lcnt[k] = 0;
        if (threadIdx.x == 0) status->edges = E;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && E < *(volatile int32_t *)lcnt) lcnt[0] = E;   // records dropped
}

static __global__ void k_edges_reset(int32_t *ecount, int32_t *lcnt, int nl)
{
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            lcnt[0] = *ecount;  // edges of level 0
            *ecount = 0;
        }
        for (int k = 1 + threadIdx.x; k < nl; k += 32) lcnt[k] = 0;
    }
}

// NL-1 levels of lowest-pass merging on the region graph (cooperative).
// Level k works on an edge list in level-k ids (ecnt[k] edges, in ebuf[k&1]):
// newmin(A) = min pass of A's edges; Union across every edge that is the
// lowest pass of one endpoint; level-(k+1) ids = ranks of the Union roots
// (the smallest level-k id of each new region, so ids stay ordered by each
// region's smallest pixel); the edges that stay between two different new
// regions are relabelled into ebuf[(k+1)&1].  Multi-edges are kept: a
// region's lowest pass over several parallel edges is their minimum either way.
static __global__ void __launch_bounds__(NTHR) k_levels(Edge *e0, Edge *e1, int32_t *ecnt,
                                                        const int32_t *k0_ptr, int NL, int32_t *gmap, size_t kstride,
                                                        uint32_t *newmin, int32_t *uf, int32_t *rank, int32_t *bsum,
                                                        int32_t *counts, DevStatus *status,
                                                        unsigned long long timeout_ns)
{
    __shared__ int red[NTHR / 32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gsz = gridDim.x * NTHR;
    const int K0 = *k0_ptr;
    if (K0 < 1 || (size_t)K0 > kstride) {
        if (blockIdx.x == 0 && tid == 0) record_error(status, DEV_BAD_LABELS, 8);
        return;  // uniform: every CTA leaves before the first barrier
    }
    if (blockIdx.x == 0 && tid == 0 && counts) counts[0] = K0;
    int Kk = K0;
    for (int k = 0; k + 1 < NL; k++) {
        const int32_t *gm = k == 0 ? nullptr : gmap + (size_t)(k - 1) * kstride;
        int32_t *gout = gmap + (size_t)k * kstride;
        const Edge *cur = (k & 1) ? e1 : e0;
        Edge *nxt = (k & 1) ? e0 : e1;
        const int E = *(volatile int32_t *)(ecnt + k);
        // A: reset
        for (int a = blockIdx.x * NTHR + tid; a < Kk; a += gsz) {
            newmin[a] = 0xffffffffu;
            uf[a] = a;
        }
        if (!grid_barrier(status, timeout_ns)) return;
        // B: newmin(A) = lowest pass of A (newmin only falls: an edge whose
        // pass is not below the value it reads issues no atomic)
        for (int e = blockIdx.x * NTHR + tid; e < E; e += gsz) {
            const Edge ed = ld_edge(cur + e);
            if (ed.a != ed.b) {
                if (ed.h < __ldcg(newmin + ed.a)) atomicMin(newmin + ed.a, ed.h);
                if (ed.h < __ldcg(newmin + ed.b)) atomicMin(newmin + ed.b, ed.h);
            }
        }
        if (!grid_barrier(status, timeout_ns)) return;
        // C: Union across every edge that is the lowest pass of one endpoint
        for (int e = blockIdx.x * NTHR + tid; e < E; e += gsz) {
            const Edge ed = ld_edge(cur + e);
            if (ed.a != ed.b && (ed.h == __ldcg(newmin + ed.a) || ed.h == __ldcg(newmin + ed.b)))
                uf_union(uf, ed.a, ed.b, status);
        }
        if (!grid_barrier(status, timeout_ns)) return;
        // D: count roots per contiguous chunk (order-preserving scan)
        const int chunk = (Kk + gridDim.x - 1) / gridDim.x;
        const int c0 = blockIdx.x * chunk, c1 = min(Kk, c0 + chunk);
        int cnt = 0;
        for (int a = c0 + tid; a < c1; a += NTHR) cnt += uf_find(uf, a) == a;
        int tot = block_sum(cnt, red);
        if (tid == 0) bsum[blockIdx.x] = tot;
        if (!grid_barrier(status, timeout_ns)) return;
        // E: ranks of the roots
        int off = 0, all = 0;
        for (int b = tid; b < (int)gridDim.x; b += NTHR) {
            const int v = *(volatile int *)(bsum + b);
            all += v;
            if (b < (int)blockIdx.x) off += v;
        }
        off = block_sum(off, red);
        all = block_sum(all, red);
        if (tid == 0) carry = off;
        __syncthreads();
        for (int a0 = c0; a0 < c1; a0 += NTHR) {
            const int a = a0 + tid;
            int isr = 0;
            if (a < c1) isr = uf_find(uf, a) == a;
            const unsigned bl = __ballot_sync(0xffffffffu, isr);
            __syncthreads();
            if (lane == 0) red[wid] = __popc(bl);
            __syncthreads();
            int o = carry;
            for (int w = 0; w < wid; w++) o += red[w];
            if (isr) rank[a] = o + __popc(bl & ((1u << lane) - 1u));
            __syncthreads();
            if (tid == 0) {
                int s = 0;
                for (int w = 0; w < NTHR / 32; w++) s += red[w];
                carry += s;
            }
            __syncthreads();
        }
        if (blockIdx.x == 0 && tid == 0 && counts) counts[k + 1] = all;
        if (!grid_barrier(status, timeout_ns)) return;
        // F: every level-k region's level-(k+1) id, once (newmin is dead after
        // C and holds it); then compose the level-0 -> level-(k+1) map and
        // contract the edge list with one lookup per id
        int32_t *lab = reinterpret_cast<int32_t *>(newmin);
        for (int a = blockIdx.x * NTHR + tid; a < Kk; a += gsz) lab[a] = __ldcg(rank + uf_find(uf, a));
        if (!grid_barrier(status, timeout_ns)) return;
        for (int c = blockIdx.x * NTHR + tid; c < K0; c += gsz) {
            const int A = gm ? __ldcg(gm + c) : c;
            gout[c] = __ldcg(lab + A);
        }
        if (k + 2 < NL) {
            // the edges between different level-(k+1) regions, relabelled; each
            // block compacts one contiguous range of the list (counted first, so
            // that it takes its span of the next list with one atomic), in order
            auto next_edge = [&](int e, Edge &ne) -> bool {
                const Edge ed = ld_edge(cur + e);
                if (ed.a == ed.b) return false;
                const int A = __ldcg(lab + ed.a), B = __ldcg(lab + ed.b);
                if (A == B) return false;
                ne.a = A < B ? A : B;
                ne.b = A < B ? B : A;
                ne.h = ed.h;
                return true;
            };
            const int per = (E + (int)gridDim.x - 1) / (int)gridDim.x;
            const int r0 = min(E, (int)blockIdx.x * per), r1 = min(E, r0 + per);
            int cnt = 0;
            for (int e = r0 + tid; e < r1; e += NTHR) {
                Edge ne;
                cnt += next_edge(e, ne) ? 1 : 0;
            }
            const int tot = block_sum(cnt, red);
            if (tid == 0) carry = tot ? atomicAdd(ecnt + k + 1, tot) : 0;
            __syncthreads();
            int pos = carry;
            for (int e0 = r0; e0 < r1; e0 += NTHR) {   // trip count uniform in the block
                const int e = e0 + tid;
                Edge ne{0, 0, 0};
                const bool keep = e < r1 && next_edge(e, ne);
                const unsigned bl = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) red[wid] = __popc(bl);
                __syncthreads();
                int o = pos, all_w = 0;
                for (int w = 0; w < NTHR / 32; w++) {
                    if (w < wid) o += red[w];
                    all_w += red[w];
                }
                if (keep) nxt[o + __popc(bl & ((1u << lane) - 1u))] = ne;
                pos += all_w;
                __syncthreads();
            }
        }
        Kk = all;
        if (!grid_barrier(status, timeout_ns)) return;
    }
}

static __global__ void __launch_bounds__(NTHR) k_level_write(int N, const int32_t *__restrict__ L0,
                                                      const int32_t *__restrict__ gmap, size_t kstride,
                                                      int nlev, int32_t *__restrict__ out)
{
    for (int p = blockIdx.x * NTHR + threadIdx.x; p < N; p += gridDim.x * NTHR) {
        int c = L0[p];
        bool ok = c >= 0 && (size_t)c < kstride;
        for (int k = 0; k < nlev; k++) __stcs(out + (size_t)k * N + p, ok ? gmap[(size_t)k * kstride + c] : -1);
    }
}

}  // namespace ws
