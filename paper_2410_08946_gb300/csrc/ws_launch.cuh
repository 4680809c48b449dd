// ws_launch.cuh -- host launchers of the watershed and waterfall pipelines,
// templated on the sample type and connectivity.  Included by the
// per-sample-type translation units (ws_inst_u8.cu, ws_inst_u16.cu).
#pragma once

#include <stddef.h>

#include "ws_kernels.cuh"

namespace ws {

// Grid size of a cooperative launch: every CTA must be co-resident.
template <typename K> static int coop_grid(ws_context *c, K kernel, int want)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NTHR, 0);
    if (per_sm < 1) per_sm = 1;
    int maxg = per_sm * c->num_sms;
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
static cudaError_t launch_coop(K kernel, int grid, cudaStream_t s, Args... args)
{
    void *argv[] = {(void *)&args...};
    return cudaLaunchCooperativeKernel((const void *)kernel, dim3(grid), dim3(NTHR), argv, 0, s);
}

template <typename T, int CONN> static ws_status run_step1(ws_context *c, const void *grad, const Geo &geo,
                                                           uint8_t *states, int32_t *arrows, cudaStream_t s)
{
    TileGeo tg = make_tilegeo<CONN>(geo);
    PhaseScope ps(c, PH_STEP1, s);
    k_step1<T, CONN><<<pixel_grid(c, geo.N), NTHR, 0, s>>>((const T *)grad, geo, arrows, states, nullptr,
                                                           nullptr, tg);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "step1 launch");
}

// Steps I and II; leaves arrows in w.par, states in w.st, distances in w.aux.
template <typename T, int CONN> static ws_status run_front(ws_context *c, const T *g, const Geo &geo,
                                                           cudaStream_t s)
{
    TileGeo tg = make_tilegeo<CONN>(geo);
    size_t nblk = ((size_t)geo.N + CHUNK - 1) / CHUNK;
    ws_status st = ensure_pixels(c, geo.N, tg.ntiles, nblk);
    if (st != WS_OK) return st;
    Workspace &w = c->w;
    cudaError_t e = cudaMemsetAsync(w.act, 0, 2 * (size_t)tg.ntiles, s);
    if (e == cudaSuccess) e = reset_barrier(c, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_STEP1, s);
        k_step1<T, CONN><<<pixel_grid(c, geo.N), NTHR, 0, s>>>(g, geo, w.par, w.st, w.aux, w.act, tg);
        c->launches += 1;
    }
    {
        PhaseScope ps(c, PH_PLATEAU, s);
        int grid = coop_grid(c, k_plateau<T, CONN>, tg.ntiles);
        e = launch_coop(k_plateau<T, CONN>, grid, s, g, geo, tg, w.aux, w.act, c->status, tune_plateau_cap(c),
                        tune_timeout_ns(c));
        c->launches += 1;
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "plateau launch");
    return WS_OK;
}

template <typename T, int CONN> static ws_status run_plateau_distance(ws_context *c, const void *grad,
                                                                      const Geo &geo, int32_t *dist,
                                                                      cudaStream_t s)
{
    ws_status st = run_front<T, CONN>(c, (const T *)grad, geo, s);
    if (st != WS_OK) return st;
    k_dist_out<<<pixel_grid(c, geo.N), NTHR, 0, s>>>(geo.N, c->w.aux, dist);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "plateau distance");
}

template <typename T, int CONN> static ws_status run_watershed(ws_context *c, const void *grad, const Geo &geo,
                                                               int32_t *labels, int32_t *count, cudaStream_t s)
{
    const T *g = (const T *)grad;
    ws_status st = run_front<T, CONN>(c, g, geo, s);
    if (st != WS_OK) return st;
    Workspace &w = c->w;
    {
        PhaseScope ps(c, PH_RESOLVE, s);
        k_resolve_union<T, CONN><<<pixel_grid(c, geo.N), NTHR, 0, s>>>(g, geo, w.par, w.st, w.aux, c->status);
        c->launches += 1;
    }
    cudaError_t e = reset_barrier(c, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_JUMP, s);
        int grid = coop_grid(c, k_jump, (geo.N + NTHR - 1) / NTHR);
        e = launch_coop(k_jump, grid, s, geo.N, w.par, w.aux, tune_rr(c), c->status, tune_jump_cap(c),
                        tune_timeout_ns(c));
        c->launches += 1;
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "jump launch");
    {
        PhaseScope ps(c, PH_COMPACT, s);
        const int nblk = (geo.N + CHUNK - 1) / CHUNK;
        k_flags<<<nblk, NTHR, 0, s>>>(geo.N, w.par, w.aux, w.st, w.blk);
        k_scan<<<1, 1024, 0, s>>>(w.blk, nblk, w.kcount);
        k_assign<<<nblk, NTHR, 0, s>>>(geo.N, w.par, w.aux, w.st, w.blk);
        k_label<<<pixel_grid(c, geo.N), NTHR, 0, s>>>(geo.N, w.par, w.aux, labels);
        c->launches += 4;
        if (count) {
            k_copy_int<<<1, 32, 0, s>>>(w.kcount, count);
            c->launches += 1;
        }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "watershed launch");
}

template <typename T, int CONN> static ws_status run_waterfall(ws_context *c, const int32_t *labels0,
                                                               const void *grad, const Geo &geo, int NL,
                                                               int32_t *levels, int32_t *counts, size_t kmax,
                                                               cudaStream_t s)
{
    // levels: NL-1 planes.  c->w.kcount holds K0 (set by the watershed, or by
    // the caller of this function from the labels); K0 <= kmax.
    Workspace &w = c->w;
    if (NL <= 1) {
        if (counts) {
            k_copy_int<<<1, 32, 0, s>>>(w.kcount, counts);
            c->launches += 1;
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "waterfall launch");
    }
    const int halfn = Nb<CONN>::n / 2;
    size_t want = (size_t)geo.N * halfn / 2;
    if (c->tun.edge_capacity > 0) want = (size_t)c->tun.edge_capacity;
    size_t cap = 1 << 16;
    while (cap < want && cap < ((size_t)1 << 28)) cap <<= 1;
    ws_status st = ensure_edges(c, cap);
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
    cudaError_t e = reset_barrier(c, s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    {
        PhaseScope ps(c, PH_LEVELS, s);
        int grid = coop_grid(c, k_levels, c->num_sms * 4);
        if (grid > 4096) grid = 4096;
        e = launch_coop(k_levels, grid, s, (const unsigned long long *)w.keys, (const uint32_t *)w.vals,
                        (const int32_t *)w.slots, (const int32_t *)w.ecount, (const int32_t *)w.kcount, NL, w.gmap,
                        w.kmax, w.newmin, w.uf, w.rank, w.bsum, counts, c->status, tune_timeout_ns(c));
        c->launches += 1;
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "levels launch");
    {
        PhaseScope ps(c, PH_LEVEL_WRITE, s);
        k_level_write<<<pixel_grid(c, geo.N), NTHR, 0, s>>>(geo.N, labels0, w.gmap, w.kmax, NL - 1, levels);
        c->launches += 1;
    }
    {
        PhaseScope ps(c, PH_CLEANUP, s);
        k_hash_clear<<<pixel_grid(c, (long long)geo.N / 4 + 1), NTHR, 0, s>>>(w.keys, w.vals, w.slots, w.ecount);
        k_reset_count<<<1, 32, 0, s>>>(w.ecount, c->status);
        c->launches += 2;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "waterfall launch");
}

template <typename T, int CONN> struct Inst {
    static const Launchers *get()
    {
        static const Launchers L = {&run_watershed<T, CONN>, &run_step1<T, CONN>, &run_plateau_distance<T, CONN>,
                                    &run_waterfall<T, CONN>};
        return &L;
    }
};

}  // namespace ws
