// ws_launch.cuh -- host launchers of the watershed and waterfall pipelines,
// templated on the sample type and connectivity.  Included by the
// per-sample-type translation units (ws_inst_u8.cu, ws_inst_u16.cu).
#pragma once

#include <stddef.h>
#include <string.h>

#include <vector>

#include "ws_tiles.cuh"

namespace ws {

// Grid size of a cooperative launch: every CTA must be co-resident.
template <typename K> static int coop_grid(ws_context *c, K kernel, int threads, size_t smem, int want)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const int maxg = per_sm * c->num_sms;
    if (want < 1) want = 1;
    return want < maxg ? want : maxg;
}

static inline int pixel_grid(ws_context *c, long long work)
{
    long long g = (work + NTHR - 1) / NTHR;
    long long cap = (long long)c->num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// Clears the barrier counter and the round-change counters of the status word.
static inline cudaError_t reset_barrier(ws_context *c, cudaStream_t s)
{
    return cudaMemsetAsync(&c->status->bar_count, 0,
                           offsetof(DevStatus, rounds_plateau) - offsetof(DevStatus, bar_count), s);
}

template <typename K, typename... Args>
static cudaError_t launch_coop(K kernel, int grid, int threads, size_t smem, cudaStream_t s, Args... args)
{
    void *argv[] = {(void *)&args...};
    return cudaLaunchCooperativeKernel((const void *)kernel, dim3(grid), dim3(threads), argv, smem, s);
}

template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// ---------------------------------------------------------------------------
// the tiled watershed core (one image, or a batch of images)
// ---------------------------------------------------------------------------

static_assert(sizeof(ImgDesc) <= kDescBytes, "image descriptor larger than its workspace slot");

template <int CONN> static ImgDesc make_desc(const Geo &g, int base, int tile0, const void *grad, int32_t *out,
                                             int32_t *counts)
{
    const TileGeo tg = tiles_for<CONN>(g);
    ImgDesc d{};
    d.W = g.W;
    d.H = g.H;
    d.D = g.D;
    d.HW = g.HW;
    d.N = g.N;
    d.base = base;
    d.tile0 = tile0;
    d.ntx = tg.ntx;
    d.nty = tg.nty;
    d.ntz = tg.ntz;
    d.grad = grad;
    d.out = out;
    d.counts = counts;
    return d;
}

template <int CONN> static Batch single_batch(const Geo &g, const void *grad, int32_t *out, int32_t *counts)
{
    Batch b{};
    b.one = make_desc<CONN>(g, 0, 0, grad, out, counts);
    b.d = nullptr;
    b.n = 1;
    b.ntiles = b.one.ntx * b.one.nty * b.one.ntz;
    b.npix = g.N;
    return b;
}

// Steps I and II: leaves in-tile path ends in w.par (3D 6-connectivity: the
// slot codes and path ends, and the arrows of plateau tiles), step II
// distances of the plateau tiles in w.dist, the plateau tiles in w.tlist.
// full: the arrow of every pixel in w.par (3D 6-connectivity; the other
// paths always write every pixel), the states and arrows of Eq. 1 into ex
// when ex.s is set, and no step II when step1_only.
template <typename T, int CONN> static ws_status run_front(ws_context *c, const Batch &b, cudaStream_t s,
                                                           bool full = false, StepExport ex = StepExport{},
                                                           bool step1_only = false)
{
    using C = TC<CONN>;
    Workspace &w = c->w;
    ws_status st = ensure_pixels(c, b.npix, b.ntiles);
    if (st != WS_OK) return st;
    if (CONN == 6 && (st = ensure_ends(c, b.npix, b.ntiles)) != WS_OK) return st;
    if (kPlateauList<CONN> && (st = ensure_plist(c, b.npix, b.ntiles)) != WS_OK) return st;
    cudaError_t e = cudaMemsetAsync(w.act, 0, 2 * (size_t)b.ntiles, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.counters, 0, 16, s);
    if (e == cudaSuccess) e = reset_barrier(c, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_STEP1, s);
        using B = InitBox<T, CONN>;
        CUtensorMap tm;
        const bool tma = !b.d && make_tmap_3d(&tm, b.one.grad, sizeof(T), b.one.W, b.one.H, b.one.D, B::RW, C::HY,
                                              C::HZ);
        if (!tma) memset(&tm, 0, sizeof tm);
        if constexpr (CONN == 6) {
            // k_init6 is the 3D specialisation (it also numbers the path ends)
            using B6 = Init6Box<T>;
            auto kern = tma ? (full ? k_init6<T, true, true> : k_init6<T, true, false>)
                            : (full ? k_init6<T, false, true> : k_init6<T, false, false>);
            const size_t smem = tma ? B6::SMEM_TMA : B6::SMEM_PLAIN;
            if ((e = allow_smem(kern, smem)) != cudaSuccess) return set_cuda_error(c, e, "smem attribute");
            // three CTAs per SM need all of the SM's unified memory as shared memory
            if ((e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
                return set_cuda_error(c, e, "smem carveout");
            // TMA: persistent CTAs (the next tile's box loads during this one); plain loads: one CTA per tile
            const int grid = tma ? coop_grid(c, kern, C::NT, smem, b.ntiles) : b.ntiles;
            kern<<<grid, C::NT, smem, s>>>(tm, b, w.par, w.aux, w.dist, w.plat, w.act, w.tlist, w.roots, w.code,
                                           w.ends, w.tends, w.counters, c->status, ex);
        } else {
            const bool exp = ex.s != nullptr;
            auto kern = tma ? (exp ? k_init<T, CONN, true, true> : k_init<T, CONN, true, false>)
                            : (exp ? k_init<T, CONN, false, true> : k_init<T, CONN, false, false>);
            const size_t smem = tma ? B::SMEM_TMA : B::SMEM_PLAIN;
            if ((e = allow_smem(kern, smem)) != cudaSuccess) return set_cuda_error(c, e, "smem attribute");
            const int grid = tma ? coop_grid(c, kern, C::NT, smem, b.ntiles) : b.ntiles;
            kern<<<grid, C::NT, smem, s>>>(tm, b, w.par, w.aux, w.dist, w.plat, w.act, w.tlist, w.roots, w.counters,
                                           c->status, ex, w.plist, w.pspan);
        }
        c->launches += 1;
    }
    if (step1_only) {
        e = cudaGetLastError();
        return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "step1 launch");
    }
    {
        PhaseScope ps(c, PH_PLATEAU, s);
        // box of G and distances (2D: and the staged plateau pixels with their starting distances)
        const size_t smem = (size_t)C::HS * 8 + (kPlateauList<CONN> ? (size_t)C::NPIX * 6 : 0);
        if ((e = allow_smem(k_plateau2<T, CONN>, smem)) != cudaSuccess) return set_cuda_error(c, e, "smem attribute");
        const int grid = coop_grid(c, k_plateau2<T, CONN>, C::NT, smem, b.ntiles);
        e = launch_coop(k_plateau2<T, CONN>, grid, C::NT, smem, s, b, w.dist, (const uint8_t *)w.plat, w.act,
                        (const int32_t *)w.tlist, (const int32_t *)w.counters, c->status, tune_plateau_cap(c),
                        tune_timeout_ns(c), (const uint16_t *)w.plist, (const int2 *)w.pspan);
        c->launches += 1;
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "plateau launch");
    return WS_OK;
}

// Whole watershed of a batch: roots in w.par, global canonical id of every
// root in w.aux (ids ordered image by image), total K0 in
// w.counters[CNT_ROOTS]; with do_rag, the region table holds every adjacent
// pair of basins (keyed by root pixel) with its pass value.
template <typename T, int CONN> static ws_status run_core(ws_context *c, const Batch &b, bool do_rag, cudaStream_t s)
{
    using C = TC<CONN>;
    ws_status st = run_front<T, CONN>(c, b, s);
    if (st != WS_OK) return st;
    Workspace &w = c->w;
    cudaError_t e = cudaSuccess;
    {
        PhaseScope ps(c, PH_RESOLVE, s);
        const int grid = b.ntiles < c->num_sms * 8 ? b.ntiles : c->num_sms * 8;
        k_resolve2<T, CONN><<<grid, C::NT, 0, s>>>(b, w.par, w.dist, w.plat, w.tlist, w.counters, c->status,
                                                   (const uint16_t *)w.plist, (const int2 *)w.pspan);
        k_union2<T, CONN><<<grid, NTHR, 0, s>>>(b, w.par, w.dist, w.plat, w.tlist, w.counters, c->status);
        c->launches += 2;
    }
    if ((e = reset_barrier(c, s)) != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_JUMP, s);
        // one CTA per tile at most (only plateau tiles have work)
        const int grid = coop_grid(c, k_jump2<CONN>, NTHR, 0, b.ntiles < c->num_sms * 8 ? b.ntiles : c->num_sms * 8);
        e = launch_coop(k_jump2<CONN>, grid, NTHR, 0, s, b, w.par, (const int32_t *)w.dist, (const int32_t *)w.tlist,
                        w.counters, w.roots, tune_rr(c), c->status, tune_jump_cap(c), tune_timeout_ns(c),
                        (const uint8_t *)w.plat, w.ends, (const int2 *)w.tends, (const uint16_t *)w.plist,
                        (const int2 *)w.pspan);
        c->launches += 1;
        if (e != cudaSuccess) return set_cuda_error(c, e, "jump launch");
    }
    if (do_rag) {
        // at most one pair record per pixel and forward neighbour (the 2D list),
        // and as many table slots (a load factor <= 1/2 for the region table's
        // distinct pairs in practice); capped at 2^28 slots
        if ((st = ensure_edges(c, edge_slots((size_t)b.npix, CONN, c), s)) != WS_OK) return st;
        if ((e = cudaMemsetAsync(w.ecnt, 0, 4, s)) != cudaSuccess) return set_cuda_error(c, e, "memset");
    }
    // the adjacency kernels put their pairs of basins here: 2D images append
    // them to a list (k_edges_ids turns it into the level-0 edge list), 3D
    // volumes insert them into the region table (k_edges_compact)
    EdgeSink elist{};
    elist.e = (Edge *)w.ea;
    elist.n = w.ecnt;
    elist.cap = (int)w.edge_cap;
    elist.keys = w.keys;
    elist.vals = w.vals;
    elist.slots = w.slots;
    elist.ecount = w.ecount;
    elist.gmask = w.edge_cap ? w.edge_cap - 1 : 0;
    if constexpr (CONN == 6) {  // 3D: roots of the tiles' path ends
        PhaseScope pc(c, PH_CHASE, s);
        k_chase<<<c->num_sms * 8, NTHR, 0, s>>>(b, w.ends, w.tends, w.code, w.counters, c->status);
        c->launches += 1;
    }
    {
        PhaseScope ps(c, PH_RAG, s);
        using B = LabelBox<T, CONN>;
        CUtensorMap tmp, tmg;
        const bool tma = !b.d && make_tmap_3d(&tmp, w.par, 4, b.one.W, b.one.H, b.one.D, B::RWP, C::BY, C::BZ) &&
                         make_tmap_3d(&tmg, b.one.grad, sizeof(T), b.one.W, b.one.H, b.one.D, B::RWG, C::BY, C::BZ);
        if constexpr (CONN == 6) {
            // 3D: the per-pixel pass over slot codes (roots known from k_chase)
            using B6 = Rag6Box<T>;
            CUtensorMap tmc;
            const bool tma6 = !b.d &&
                              make_tmap_3d(&tmc, w.code, 2, b.one.W, b.one.H, b.one.D, B6::CW, B6::BY, B6::BZ) &&
                              make_tmap_3d(&tmg, b.one.grad, sizeof(T), b.one.W, b.one.H, b.one.D, B6::GW, B6::BY,
                                           B6::BZ);
            if (!tma6) {
                memset(&tmc, 0, sizeof tmc);
                memset(&tmg, 0, sizeof tmg);
            }
            auto kern = tma6 ? k_rag6<T, true> : k_rag6<T, false>;
            if ((e = allow_smem(kern, B6::SMEM)) != cudaSuccess) return set_cuda_error(c, e, "smem attribute");
            // three CTAs per SM need all of the SM's unified memory as shared memory
            if ((e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
                return set_cuda_error(c, e, "smem carveout");
            kern<<<b.ntiles, C::NT, B6::SMEM, s>>>(tmc, tmg, b, w.code, w.ends, w.tends, w.aux, do_rag ? 1 : 0, elist,
                                                   c->status);
        } else if (tma) {
            if ((e = allow_smem(k_label<T, CONN, true>, B::SMEM)) != cudaSuccess)
                return set_cuda_error(c, e, "smem attribute");
            k_label<T, CONN, true><<<b.ntiles, C::NT, B::SMEM, s>>>(tmp, tmg, b, w.par, w.aux, do_rag ? 1 : 0, elist,
                                                                    c->status);
        } else {
            memset(&tmp, 0, sizeof tmp);
            memset(&tmg, 0, sizeof tmg);
            if ((e = allow_smem(k_label<T, CONN, false>, B::SMEM)) != cudaSuccess)
                return set_cuda_error(c, e, "smem attribute");
            k_label<T, CONN, false><<<b.ntiles, C::NT, B::SMEM, s>>>(tmp, tmg, b, w.par, w.aux, do_rag ? 1 : 0, elist,
                                                                     c->status);
        }
        c->launches += 1;
    }
    {
        PhaseScope ps(c, PH_COMPACT, s);
        const int ng = (int)((b.npix + 1023) / 1024), nw = (int)((b.npix + 31) / 32);
        const int nch = (ng + SCAN_CHUNK - 1) / SCAN_CHUNK;
        const int rg = c->num_sms * 4;
        k_rank_mark<<<rg, NTHR, 0, s>>>(b.npix, w.roots, w.counters, w.aux, w.rootm, w.bitmap, c->status);
        k_rank_groups<<<(ng + NTHR / 32 - 1) / (NTHR / 32), NTHR, 0, s>>>(w.bitmap, nw, w.gcnt, ng);
        k_scan_chunks<<<nch, NTHR, 0, s>>>(w.gcnt, ng, w.csum);
        if (nch > 1) {   // one chunk is already scanned
            k_scan<<<1, 1024, 0, s>>>(w.csum, nch, nullptr);
            k_scan_add<<<nch, NTHR, 0, s>>>(w.gcnt, ng, w.csum);
            c->launches += 2;
        }
        k_rank_assign<<<rg, NTHR, 0, s>>>(w.roots, w.counters, w.rootm, w.bitmap, w.gcnt, w.aux);
        c->launches += 4;
        if (b.d) {
            k_rank_bases<<<(b.n + NTHR) / NTHR, NTHR, 0, s>>>(b, w.bitmap, w.gcnt, w.counters, w.rbase);
            c->launches += 1;
        }
        k_rank_clear<<<rg, NTHR, 0, s>>>(w.counters, w.rootm, w.bitmap);
        c->launches += 1;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "watershed launch");
}

// Descriptors of a batch, as run_segment_batch builds them (for callers that
// upload them once, e.g. before capturing a graph).
template <int CONN> static void batch_descs(int n, const Geo *geos, const ws_item *items, std::vector<ImgDesc> &out)
{
    out.resize((size_t)n);
    long long npix = 0, ntiles = 0;
    for (int i = 0; i < n; i++) {
        out[i] = make_desc<CONN>(geos[i], (int)npix, (int)ntiles, items[i].grad_d, items[i].levels_d,
                                 items[i].counts_d);
        npix += geos[i].N;
        ntiles += (long long)out[i].ntx * out[i].nty * out[i].ntz;
    }
}

// One pass writing level 0 (canonical ids) and levels 1..NL-1 of one image.
static inline ws_status run_write(ws_context *c, const Geo &geo, int NL, int32_t *out, bool d3, cudaStream_t s)
{
    Workspace &w = c->w;
    PhaseScope ps(c, PH_LEVEL_WRITE, s);
    if (d3) {   // 3D: from the voxels' end slots, tile by tile
        Batch b{};
        b.one.W = geo.W;
        b.one.H = geo.H;
        b.one.D = geo.D;
        b.one.HW = geo.HW;
        b.one.N = geo.N;
        b.one.out = out;
        const TileGeo tg = tiles_for<6>(geo);
        b.one.ntx = tg.ntx;
        b.one.nty = tg.nty;
        b.one.ntz = tg.ntz;
        b.ntiles = tg.ntiles;
        b.npix = geo.N;
        k_write6<<<b.ntiles, TT<6>::NT, 0, s>>>(b, w.code, w.ends, w.tends, w.aux, w.gmap, w.kmax, NL, nullptr,
                                                w.counters + CNT_ROOTS);
        c->launches += 1;
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "write launch");
    }
    const bool vec = (geo.N % 4 == 0) && (((uintptr_t)out & 15) == 0);
    const int grid = pixel_grid(c, vec ? geo.N / 4 : geo.N);
    if (vec)
        k_write_vec<<<grid, NTHR, 0, s>>>(geo.N, w.par, w.aux, w.gmap, w.kmax, NL, w.counters + CNT_ROOTS, out);
    else
        k_write_scalar<<<grid, NTHR, 0, s>>>(geo.N, w.par, w.aux, w.gmap, w.kmax, NL, w.counters + CNT_ROOTS,
                                              out);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "write launch");
}

// Region-graph merging for levels 1..NL-1: the cooperative k_levels
// contracts the level-0 edge list level by level.  The level-0 list comes
// from the edge list a 2D segmentation appended (list_npix > 0: its records,
// keyed by root pixels below list_npix, mapped to canonical ids through idmap
// in place) or from the filled region table (list_npix == 0: the table
// becomes the list, idmap maps its keys to ids or is nullptr when the keys are
// ids, and the table is emptied for the next call).
static inline ws_status run_levels(ws_context *c, int NL, const int32_t *idmap, const int32_t *k0_ptr,
                                   int32_t *counts, cudaStream_t s, int list_npix = 0)
{
    Workspace &w = c->w;
    cudaError_t e = reset_barrier(c, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_CLEANUP, s);
        if (list_npix > 0) {
            k_edges_ids<<<c->num_sms * 8, NTHR, 0, s>>>((Edge *)w.ea, w.ecnt, NL, (int)w.edge_cap, idmap, list_npix,
                                                        k0_ptr, c->status);
            c->launches += 1;
        } else {
            k_edges_compact<<<c->num_sms * 8, NTHR, 0, s>>>(w.keys, w.vals, w.slots, w.ecount, idmap, k0_ptr,
                                                            (Edge *)w.ea, w.ecnt, c->status);
            k_edges_reset<<<1, 32, 0, s>>>(w.ecount, w.ecnt, NL);
            c->launches += 2;
        }
    }
    PhaseScope ps(c, PH_LEVELS, s);
    int grid = coop_grid(c, k_levels, NTHR, 0, c->num_sms * tune_levels_ctas(c));
    if (grid > 4096) grid = 4096;
    e = launch_coop(k_levels, grid, NTHR, 0, s, (Edge *)w.ea, (Edge *)w.eb, w.ecnt, k0_ptr, NL, w.gmap, w.kmax,
                    w.newmin, w.uf, w.rank, w.bsum, counts, c->status, tune_timeout_ns(c));
    c->launches += 1;
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "levels launch");
}

template <typename T, int CONN> static ws_status run_watershed(ws_context *c, const void *grad, const Geo &geo,
                                                               int32_t *labels, int32_t *count, cudaStream_t s)
{
    const Batch b = single_batch<CONN>(geo, grad, labels, nullptr);
    ws_status st = run_core<T, CONN>(c, b, false, s);
    if (st != WS_OK) return st;
    if ((st = run_write(c, geo, 1, labels, CONN == 6, s)) != WS_OK) return st;
    if (count) {
        k_copy_int<<<1, 32, 0, s>>>(c->w.counters + CNT_ROOTS, count);
        c->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "watershed launch");
}

template <typename T, int CONN> static ws_status run_segment(ws_context *c, const void *grad, const Geo &geo, int NL,
                                                             int32_t *levels, int32_t *counts, cudaStream_t s)
{
    Workspace &w = c->w;
    ws_status st;
    // distinct minimal plateaux are never adjacent, so K0 <= ceil(N / 2)
    if (NL > 1 && (st = ensure_regions(c, (size_t)geo.N / 2 + 2, NL - 1)) != WS_OK) return st;
    const Batch b = single_batch<CONN>(geo, grad, levels, counts);
    if ((st = run_core<T, CONN>(c, b, NL > 1, s)) != WS_OK) return st;
    if (NL > 1) {
        if ((st = run_levels(c, NL, w.aux, w.counters + CNT_ROOTS, counts, s, TC<CONN>::D3 ? 0 : geo.N)) != WS_OK)
            return st;
    } else if (counts) {
        k_copy_int<<<1, 32, 0, s>>>(w.counters + CNT_ROOTS, counts);
        c->launches += 1;
    }
    return run_write(c, geo, NL, levels, CONN == 6, s);
}

// A batch of images (same dtype and connectivity) in one launch per phase:
// the images' pixels and tiles are concatenated in the workspace.
// descs_dev: device copy of the descriptors made by the caller (graph
// capture), or nullptr to upload them into the workspace here.
template <typename T, int CONN> static ws_status run_segment_batch(ws_context *c, int n, const Geo *geos,
                                                                   const ws_item *items, int NL, const void *descs_dev,
                                                                   cudaStream_t s)
{
    Workspace &w = c->w;
    std::vector<ImgDesc> descs((size_t)n);
    long long npix = 0, ntiles = 0, kmax = 0;
    for (int i = 0; i < n; i++) {
        descs[i] = make_desc<CONN>(geos[i], (int)npix, (int)ntiles, items[i].grad_d, items[i].levels_d,
                                   items[i].counts_d);
        npix += geos[i].N;
        ntiles += (long long)descs[i].ntx * descs[i].nty * descs[i].ntz;
        kmax += geos[i].N / 2 + 1;
    }
    if (npix >= 0x7fffffffLL || ntiles >= 0x7fffffffLL)
        return set_error_msg(c, WS_ERR_INVALID, "batch too large: the images' pixels must total below 2^31");
    ws_status st;
    if ((st = ensure_batch(c, (size_t)n)) != WS_OK) return st;
    if (NL > 1 && (st = ensure_regions(c, (size_t)kmax + 2, NL - 1)) != WS_OK) return st;
    cudaError_t e = cudaSuccess;
    if (!descs_dev) {
        e = cudaMemcpyAsync(w.descs, descs.data(), sizeof(ImgDesc) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return set_cuda_error(c, e, "descriptor upload");
    }
    Batch b{};
    b.d = (const ImgDesc *)(descs_dev ? descs_dev : w.descs);
    b.n = n;
    b.ntiles = (int)ntiles;
    b.npix = (int)npix;
    if ((st = run_core<T, CONN>(c, b, NL > 1, s)) != WS_OK) return st;
    // w.lcount[k] = region count of level k over the whole batch
    if (NL > 1 && (st = run_levels(c, NL, w.aux, w.counters + CNT_ROOTS, w.lcount, s, TC<CONN>::D3 ? 0 : b.npix)) !=
                      WS_OK)
        return st;
    {
        PhaseScope ps(c, PH_LEVEL_WRITE, s);
        if (CONN == 6)   // 3D: from the voxels' end slots, tile by tile
            k_write6<<<b.ntiles, TT<6>::NT, 0, s>>>(b, w.code, w.ends, w.tends, w.aux, w.gmap, w.kmax, NL, w.rbase,
                                                    w.counters + CNT_ROOTS);
        else
            k_write_batch<<<pixel_grid(c, b.npix), NTHR, 0, s>>>(b, w.par, w.aux, w.gmap, w.kmax, NL, w.rbase,
                                                                 w.counters + CNT_ROOTS);
        k_counts_batch<<<(n + NTHR - 1) / NTHR, NTHR, 0, s>>>(b, w.gmap, w.kmax, NL, w.rbase, w.lcount);
        c->launches += 2;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "batch launch");
}

template <typename T, int CONN> static ws_status run_plateau_distance(ws_context *c, const void *grad,
                                                                      const Geo &geo, int32_t *dist,
                                                                      cudaStream_t s)
{
    const Batch b = single_batch<CONN>(geo, grad, nullptr, nullptr);
    ws_status st = run_front<T, CONN>(c, b, s, true);   // every pixel's arrow (k_dist_out2 reads them)
    if (st != WS_OK) return st;
    k_dist_out2<<<pixel_grid(c, geo.N), NTHR, 0, s>>>(geo, tiles_for<CONN>(geo), c->w.par, c->w.dist, c->w.plat,
                                                      dist);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "plateau distance");
}

// Step I alone (ws_step1): the states and arrows of Eq. 1 as the tiled step I
// kernels of the segmentation path compute them.
template <typename T, int CONN> static ws_status run_step1(ws_context *c, const void *grad, const Geo &geo,
                                                           uint8_t *states, int32_t *arrows, cudaStream_t s)
{
    const Batch b = single_batch<CONN>(geo, grad, nullptr, nullptr);
    StepExport ex;
    ex.s = states;
    ex.l = arrows;
    return run_front<T, CONN>(c, b, s, true, ex, true);
}

// ---------------------------------------------------------------------------
// waterfall above caller-provided level-0 labels
// ---------------------------------------------------------------------------

template <typename T, int CONN> static ws_status run_waterfall(ws_context *c, const int32_t *labels0,
                                                               const void *grad, const Geo &geo, int NL,
                                                               int32_t *levels, int32_t *counts, size_t kmax,
                                                               cudaStream_t s)
{
    // levels: NL-1 planes.  c->w.kcount holds K0 (from the labels); K0 <= kmax.
    Workspace &w = c->w;
    if (NL <= 1) {
        if (counts) {
            k_copy_int<<<1, 32, 0, s>>>(w.kcount, counts);
            c->launches += 1;
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "waterfall launch");
    }
    ws_status st = ensure_edges(c, edge_slots((size_t)geo.N, CONN, c), s);
    if (st != WS_OK) return st;
    st = ensure_regions(c, kmax, NL - 1);
    if (st != WS_OK) return st;
    const T *g = (const T *)grad;
    {
        PhaseScope ps(c, PH_RAG, s);
        k_rag<T, CONN><<<pixel_grid(c, geo.N), NTHR, 0, s>>>(g, geo, labels0, w.keys, w.vals, w.slots, w.ecount,
                                                             (unsigned long long)(w.edge_cap - 1), c->status);
        c->launches += 1;
    }
    if ((st = run_levels(c, NL, nullptr, w.kcount, counts, s)) != WS_OK) return st;
    {
        PhaseScope ps(c, PH_LEVEL_WRITE, s);
        k_level_write<<<pixel_grid(c, geo.N), NTHR, 0, s>>>(geo.N, labels0, w.gmap, w.kmax, NL - 1, levels);
        c->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "waterfall launch");
}

// ---------------------------------------------------------------------------
// paper-literal waterfall: watershed, then image reconstruction, per level
// ---------------------------------------------------------------------------

// Level n is the watershed of I_n (I_0 = G); I_{n+1} is I_n raised by Alg. 5
// steps V-VI into the workspace image w.rec (the caller's gradient is never
// written).  counts: NL device ints (w.lcount when the caller gives none).
template <typename T, int CONN> static ws_status run_reconstruct(ws_context *c, const void *grad, const Geo &geo,
                                                                 int NL, int32_t *levels, int32_t *counts,
                                                                 cudaStream_t s)
{
    Workspace &w = c->w;
    ws_status st;
    if (NL > 1) {
        if ((st = ensure_rec(c, (size_t)geo.N * sizeof(T))) != WS_OK) return st;
        if ((st = ensure_regions(c, (size_t)geo.N / 2 + 2, 1)) != WS_OK) return st;
    }
    int32_t *cnt = counts ? counts : w.lcount;
    const void *I = grad;
    for (int n = 0; n < NL; n++) {
        int32_t *L = levels + (size_t)n * geo.N;
        if ((st = run_watershed<T, CONN>(c, I, geo, L, cnt + n, s)) != WS_OK) return st;
        if (n == NL - 1) break;
        PhaseScope ps(c, PH_RECON, s);
        k_fill_newmin<<<pixel_grid(c, geo.N / 2 + 2), NTHR, 0, s>>>(w.newmin, cnt + n);
        k_newmin<T, CONN><<<pixel_grid(c, geo.N), NTHR, 0, s>>>((const T *)I, geo, L, w.newmin);
        k_raise<T><<<pixel_grid(c, geo.N), NTHR, 0, s>>>((const T *)I, (T *)w.rec, L, w.newmin, geo.N);
        c->launches += 3;
        I = w.rec;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "reconstruct launch");
}

template <int CONN> static void descs_host(int n, const Geo *geos, const ws_item *items, void *out)
{
    std::vector<ImgDesc> v;
    batch_descs<CONN>(n, geos, items, v);
    memcpy(out, v.data(), sizeof(ImgDesc) * (size_t)n);
}

template <typename T, int CONN> struct Inst {
    static const Launchers *get()
    {
        static const Launchers L = {&run_watershed<T, CONN>, &run_step1<T, CONN>, &run_plateau_distance<T, CONN>,
                                    &run_waterfall<T, CONN % 100>, &run_segment<T, CONN>,
                                    &run_segment_batch<T, CONN>, sizeof(ImgDesc), &descs_host<CONN>,
                                    &run_reconstruct<T, CONN>};
        return &L;
    }
};

}  // namespace ws
