// ws_tiles.cuh -- the fused, tiled watershed pipeline of libws.
//
// The image is cut into tiles (2D 64 x 32 pixels, 3D 32 x 16 x 16 voxels);
// one CTA owns one tile.  Pixel work runs in three passes over HBM, with the
// sparse plateau work (Alg. 1 step II, step IV) and the small region-graph
// work in between:
//
//   k_init      Alg. 1 step I (Eq. 1) on the tile + 1-pixel halo staged in
//               shared memory, then step III *inside the tile*: every pixel
//               follows its arrows through shared memory until the path
//               leaves the tile, reaches a minimum, or reaches a plateau
//               pixel.  Writes that end point (par), flags tiles that hold
//               plateau pixels, lists the minima and (2D) lists each tile's
//               plateau pixels.
//   k_plateau2  step II distances on the listed plateau tiles only (in-tile
//               relaxation with a frozen halo, device-wide rounds; the fixed
//               point of Alg. 3); 2D relaxes the tile's listed plateau pixels
//   k_resolve2  step II pointer choice, step IV Union of minimal plateaux
//               inside each tile (2D: and step III along the tile's plateau)
//   k_union2    step IV across tile borders
//   k_jump2     step III for plateau tiles (pointer jumping rounds), lists
//               the minimal-plateau roots
//   k_label     per tile: final root of every pixel (chasing the few
//               tile-to-tile hops left), smallest pixel index per basin, and
//               Alg. 5 step V on pixel pairs (runs of equal neighbour roots
//               merged in registers, then a shared-memory hash, then the
//               edge list (2D) or the global region table (26-connectivity))
// These serve 2D (4-, 8-connectivity) and 3D 26-connectivity.
//
// 3D volumes with 6-connectivity take a variant of this pipeline with one z
// column of the tile per thread:
//   k_init6     as k_init, and numbers the tile's in-tile path ends (slots):
//               per pixel a 16-bit code (the slot of its end), per tile the
//               list of its end pixels, each with the next pixel of its path
//               (the arrow of Eq. 1 out of the tile); par holds the arrows
//               on plateau tiles only
//   k_chase     the root of every listed end, following the next pixels
//               and the slot codes through the next tiles
//   k_rag6      per tile: roots by slot lookup, smallest index per basin,
//               and Alg. 5 step V from per-warp lists of boundary pixels
//   k_rank_*    canonical ids: rank of every basin's smallest pixel index
//               among all of them, by a bitmap over pixel indices
//   k_write6    per tile (3D, 6-connectivity): the canonical and waterfall
//               ids of the tile's slots in a shared table, then every voxel's
//               row of it by its slot code, all NL planes in one pass
//   k_write_vec / k_write_batch
//               per pixel (the other paths): canonical id of its root and its
//               id on every waterfall level, one pass writing all NL planes
#pragma once

#include <type_traits>

#include "ws_kernels.cuh"
#include "ws_tma.cuh"

namespace ws {

// Tile shape and threads per tile.  2D images run on shape 0 (64 x 32
// pixels, 256 threads) unless ws_tuning.tile_shape picks another (uint8
// gradients): 1 = 32 x 32 / 256, 2 = 128 x 16 / 256, 3 = 64 x 32 / 512; the
// template value is CONN + 100 * shape.  TX stays a multiple of 32 (warps
// cover whole runs of one row).
template <int CONN> struct TT;
template <> struct TT<4> {
    static constexpr int TX = 64, TY = 32, TZ = 1, NT = 256;
};
template <> struct TT<8> : TT<4> {};
template <> struct TT<104> {
    static constexpr int TX = 32, TY = 32, TZ = 1, NT = 256;
};
template <> struct TT<108> : TT<104> {};
template <> struct TT<204> {
    static constexpr int TX = 128, TY = 16, TZ = 1, NT = 256;
};
template <> struct TT<208> : TT<204> {};
template <> struct TT<304> {
    static constexpr int TX = 64, TY = 32, TZ = 1, NT = 512;
};
template <> struct TT<308> : TT<304> {};
template <> struct TT<6> {
    static constexpr int TX = 32, TY = 16, TZ = 16, NT = 512;
};
template <> struct TT<26> {
    static constexpr int TX = 32, TY = 16, TZ = 16, NT = 512;
};


template <int CONN> struct TC {
    static constexpr int TX = TT<CONN>::TX, TY = TT<CONN>::TY, TZ = TT<CONN>::TZ, NT = TT<CONN>::NT;
    static constexpr bool D3 = TZ > 1;
    static constexpr int NPIX = TX * TY * TZ;
    static constexpr int PER = NPIX / NT;
    // halo box on both sides (k_init, k_plateau2)
    static constexpr int HX = TX + 2, HY = TY + 2, HZ = D3 ? TZ + 2 : 1;
    static constexpr int HS = HX * HY * HZ;
    // forward box of k_label: +1 on every axis, and -1 in x / y where a
    // forward neighbour lies there
    // (forward neighbours reach x - 1 in 8- and 26-connectivity, y - 1 in 26)
    static constexpr int BXL = (CONN % 100 == 8 || CONN == 26) ? 1 : 0;
    static constexpr int BYL = CONN == 26 ? 1 : 0;
    static constexpr int BX = TX + 1 + BXL, BY = TY + 1 + BYL, BZ = D3 ? TZ + 1 : 1;
    static constexpr int BS = BX * BY * BZ;
    static constexpr int HASH = 1024;  // shared-memory edge slots per CTA
};

inline TileGeo make_tiles(const Geo &g, int TX, int TY, int TZ)
{
    TileGeo t;
    t.TX = TX;
    t.TY = TY;
    t.TZ = TZ;
    t.ntx = (g.W + TX - 1) / TX;
    t.nty = (g.H + TY - 1) / TY;
    t.ntz = (g.D + TZ - 1) / TZ;
    t.ntiles = t.ntx * t.nty * t.ntz;
    return t;
}

template <int CONN> inline TileGeo tiles_for(const Geo &g)
{
    return make_tiles(g, TT<CONN>::TX, TT<CONN>::TY, TT<CONN>::TZ);
}

// counters[] slots in the workspace
enum { CNT_TILES = 0, CNT_ROOTS = 1, CNT_ENDS = 2, CNT_PLIST = 3 };

// 2D pipelines list every tile's plateau pixels (tile-local indices) for the
// step II / IV and jumping kernels, which then visit those pixels only.
template <int CONN> constexpr bool kPlateauList = CONN % 100 == 4 || CONN % 100 == 8;

__device__ __forceinline__ int enc_final(int g) { return -1 - g; }
__device__ __forceinline__ int dec_final(int e) { return -1 - e; }

// One image of a batch.  Images are concatenated in the workspace: pixel p
// of image i has the global index base + p, its tiles are tile0 ...
// tile0 + ntx*nty*ntz - 1 of the global tile space.
struct ImgDesc {
    int W, H, D, HW, N;
    int base;                 // first global pixel index
    int tile0;                // first global tile index
    int ntx, nty, ntz;
    int pad_[2];
    const void *grad;         // gradient samples [N]
    int32_t *out;             // NL label planes, plane stride N
    int32_t *counts;          // NL region counts (may be null)
};

// A batch: one image inline (d == nullptr), or n descriptors in device memory.
struct Batch {
    ImgDesc one;
    const ImgDesc *d;
    int n;
    int ntiles;               // tiles of all images
    int npix;                 // pixels of all images
};

__device__ __forceinline__ ImgDesc img_desc(const Batch &b, int i) { return b.d ? b.d[i] : b.one; }

// image owning global tile t / global pixel g (binary search over the batch)
__device__ __forceinline__ int img_of_tile(const Batch &b, int t)
{
    if (!b.d) return 0;
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&b.d[mid].tile0) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int img_of_pixel(const Batch &b, int g)
{
    if (!b.d) return 0;
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&b.d[mid].base) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Everything a CTA needs about the tile it works on.
struct TileCtx {
    Geo geo;                  // the image's geometry
    TileGeo tg;               // the image's tiling (tile ids local to the image)
    int base, tile0;          // global offsets of the image
    int x0, y0, z0;           // tile origin in the image
    const void *grad;
};

template <int CONN> __device__ __forceinline__ TileCtx tile_ctx(const Batch &b, int t)
{
    const ImgDesc d = img_desc(b, img_of_tile(b, t));
    TileCtx c;
    c.geo.W = d.W;
    c.geo.H = d.H;
    c.geo.D = d.D;
    c.geo.HW = d.HW;
    c.geo.N = d.N;
    c.tg.TX = TT<CONN>::TX;
    c.tg.TY = TT<CONN>::TY;
    c.tg.TZ = TT<CONN>::TZ;
    c.tg.ntx = d.ntx;
    c.tg.nty = d.nty;
    c.tg.ntz = d.ntz;
    c.tg.ntiles = d.ntx * d.nty * d.ntz;
    c.base = d.base;
    c.tile0 = d.tile0;
    const int lt = t - d.tile0;
    c.x0 = (lt % d.ntx) * TT<CONN>::TX;
    c.y0 = ((lt / d.ntx) % d.nty) * TT<CONN>::TY;
    c.z0 = (lt / (d.ntx * d.nty)) * TT<CONN>::TZ;
    c.grad = d.grad;
    return c;
}

// local tile id of pixel (x, y, z) of an image
__device__ __forceinline__ int tile_of(const TileGeo &tg, int x, int y, int z)
{
    return ((z / tg.TZ) * tg.nty + y / tg.TY) * tg.ntx + x / tg.TX;
}

// the same with the tile sizes of CONN known at compile time (shifts)
template <int CONN> __device__ __forceinline__ int tile_of_c(const TileGeo &tg, int x, int y, int z)
{
    return ((z / TT<CONN>::TZ) * tg.nty + y / TT<CONN>::TY) * tg.ntx + x / TT<CONN>::TX;
}

// state codes kept in registers by k_init
enum : int { ST0 = 0, ST1 = 1, STP = 2, STOUT = 3 };

// Optional outputs of step I (ws_step1): the state of Eq. 1 (0: a lower
// neighbour; 1: a strict minimum; 2 / 3: an equal lowest neighbour with a
// larger / smaller index) and the arrow (the lowest neighbour for states 0 and
// 2, the pixel itself for 1 and 3) of every pixel, as computed by the tiled
// step I kernels of the segmentation path.
struct StepExport {
    uint8_t *s = nullptr;
    int32_t *l = nullptr;
};

// ---------------------------------------------------------------------------
// k_init: step I + in-tile path reduction
// ---------------------------------------------------------------------------

// Shared-memory box of k_init: the tile plus a one-pixel halo in y and z and
// an x halo widened to 16 bytes on each side (the TMA alignment unit), so a
// row of the box starts on a 16-byte boundary in global memory.
template <typename T, int CONN> struct InitBox {
    using C = TC<CONN>;
    static constexpr int A = 16 / (int)sizeof(T);   // x offset of the tile inside the box
    static constexpr int RW = C::TX + 2 * A;         // row pitch (elements)
    static constexpr int ELEMS = RW * C::HY * C::HZ;
    static constexpr int BYTES = ELEMS * (int)sizeof(T);
    static constexpr int STAGE = (BYTES + 127) & ~127;
    static constexpr int LISTB = kPlateauList<CONN> ? C::NPIX * 2 : 0;   // staged plateau pixels
    static constexpr int SMEM_TMA = 2 * STAGE + C::NPIX * 4 + LISTB;   // two stages + in-tile arrows (+ list)
    static constexpr int SMEM_PLAIN = STAGE + C::NPIX * 4 + LISTB;
};

template <typename T, int CONN, bool TMA>
__device__ __forceinline__ void init_issue(const CUtensorMap *tm, T *dst, uint64_t *bar, const Batch &b, int t)
{
    using B = InitBox<T, CONN>;
    const TileCtx tc = tile_ctx<CONN>(b, t);
    mbar_arrive_expect_tx(bar, B::BYTES);
    tma_load_3d(dst, tm, tc.x0 - B::A, tc.y0 - 1, TC<CONN>::D3 ? tc.z0 - 1 : 0, bar);
}

// Step I (Eq. 1) for this thread's pixels of one tile, from the gradient box
// in shared memory: writes the in-tile arrow (local index), the path end
// (encoded global index), and the state; returns 1 if a plateau pixel was
// seen.  CHECK = false skips the neighbour bounds tests (interior tiles).
// The thread's pixels are slots k = 0..PER-1 of one column of the tile (the
// z column in 3D, every NT/TX-th row in 2D); in 3D the column and its four
// side columns are read once into registers and the z neighbours reused.
template <typename T, int CONN, bool CHECK, bool EXP>
__device__ __forceinline__ int init_step1(const T *gs, int *nx, int (&st)[TC<CONN>::PER], int tid, int x0, int y0,
                                          int z0, const Geo &geo, int base, const StepExport &ex)
{
    using C = TC<CONN>;
    using B = InitBox<T, CONN>;
    constexpr bool COL = CONN == 6 && C::NT == C::TX * C::TY;  // slot k is z = k of column tid
    int plateau = 0;
    unsigned cz[C::PER + 2];
    if (COL) {
        const int lx = tid % C::TX, ly = tid / C::TX;
        const int h0 = (ly + 1) * B::RW + lx + B::A;   // box index of (lx, ly, z = -1)
        constexpr int SZ = C::HY * B::RW;
#pragma unroll
        for (int k = 0; k < C::PER + 2; k++) cz[k] = gs[h0 + k * SZ];
    }
#pragma unroll
    for (int k = 0; k < C::PER; k++) {
        const int i = tid + k * C::NT;
        const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (CHECK && (x >= geo.W || y >= geo.H || z >= geo.D)) {
            st[k] = STOUT;
            nx[i] = enc_final(0);
            continue;
        }
        const int p = base + (z * geo.H + y) * geo.W + x;   // global index
        const int h = ((C::D3 ? lz + 1 : 0) * C::HY + ly + 1) * B::RW + lx + B::A;
        const unsigned gp = COL ? cz[k + 1] : (unsigned)gs[h];
        unsigned m = 0xffffffffu;
        int qn = -1;
#pragma unroll
        for (int n = 0; n < Nb<CONN>::n; n++) {
            if (CHECK) {
                const int xx = x + Nb<CONN>::dx(n), yy = y + Nb<CONN>::dy(n), zz = z + Nb<CONN>::dz(n);
                if (xx < 0 || xx >= geo.W || yy < 0 || yy >= geo.H || zz < 0 || zz >= geo.D) continue;
            }
            unsigned v;
            if (COL && (n == 0 || n == Nb<CONN>::n - 1)) {
                v = n == 0 ? cz[k] : cz[k + 2];   // z - 1, z + 1 from the register column
            } else {
                v = gs[h + (Nb<CONN>::dz(n) * C::HY + Nb<CONN>::dy(n)) * B::RW + Nb<CONN>::dx(n)];
            }
            if (v <= m) {  // ascending index order: ties go to the later (larger) neighbour
                m = v;
                qn = n;
            }
        }
        // the lowest neighbour (global index), when there is one
        const int q = qn < 0 ? p : p + (Nb<CONN>::dz(qn) * geo.H + Nb<CONN>::dy(qn)) * geo.W + Nb<CONN>::dx(qn);
        if (qn < 0 || m > gp) {
            st[k] = ST1;
            nx[i] = enc_final(p);
            if (EXP) {
                ex.s[p] = 1;
                ex.l[p] = p;
            }
        } else if (m < gp) {
            st[k] = ST0;
            const int lxx = lx + Nb<CONN>::dx(qn), lyy = ly + Nb<CONN>::dy(qn), lzz = lz + Nb<CONN>::dz(qn);
            if (lxx >= 0 && lxx < C::TX && lyy >= 0 && lyy < C::TY && lzz >= 0 && lzz < C::TZ)
                nx[i] = (lzz * C::TY + lyy) * C::TX + lxx;
            else
                nx[i] = enc_final(q);
            if (EXP) {
                ex.s[p] = 0;
                ex.l[p] = q;
            }
        } else {
            st[k] = STP;  // plateau pixel: resolved by step II / step IV
            nx[i] = enc_final(p);
            plateau = 1;
            if (EXP) {   // state 2 when the equal lowest neighbour comes later in index order
                ex.s[p] = (uint8_t)(q > p ? 2 : 3);
                ex.l[p] = q > p ? q : p;
            }
        }
    }
    return plateau;
}

// 26-connectivity: at most 64 registers, so that two CTAs share an SM
// EXP: also writes the states and arrows of Eq. 1 into ex (ws_step1).
template <typename T, int CONN, bool TMA, bool EXP>
__global__ void __launch_bounds__(TT<CONN>::NT, CONN == 26 ? 2 : 1)
    k_init(const __grid_constant__ CUtensorMap tm, const Batch b, int32_t *__restrict__ par,
           int32_t *__restrict__ mi, int32_t *__restrict__ dist, uint8_t *__restrict__ plat,
           uint8_t *__restrict__ act, int32_t *__restrict__ tlist, int32_t *__restrict__ roots, int32_t *counters,
           DevStatus *status, const StepExport ex, uint16_t *__restrict__ plist, int2 *__restrict__ pspan)
{
    using C = TC<CONN>;
    using B = InitBox<T, CONN>;
    constexpr bool LIST = kPlateauList<CONN>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[2];
    __shared__ int s_pc, s_pbase;   // the tile's plateau pixels, their first entry in plist
    __shared__ int s_rc, s_rbase;   // the tile's strict minima, their first entry in roots
    int *nx = (int *)(smem + (TMA ? 2 : 1) * B::STAGE);
    uint16_t *sp = (uint16_t *)(nx + C::NPIX);   // the tile's plateau pixels, staged (LIST)
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = gridDim.x;

    if (TMA) {  // a single image (b.one); two tiles in flight per CTA
        if (tid == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            mbar_fence_init();
            const int t0 = blockIdx.x;
            if (t0 < b.ntiles) init_issue<T, CONN, TMA>(&tm, (T *)smem, &bars[0], b, t0);
            if (t0 + G < b.ntiles) init_issue<T, CONN, TMA>(&tm, (T *)(smem + B::STAGE), &bars[1], b, t0 + G);
        }
        __syncthreads();
    }

    int j = 0;
    for (int t = blockIdx.x; t < b.ntiles; t += G, j++) {
        const int s = TMA ? (j & 1) : 0;
        T *gs = (T *)(smem + s * B::STAGE);
        const TileCtx tc = tile_ctx<CONN>(b, t);
        const Geo &geo = tc.geo;
        const int x0 = tc.x0, y0 = tc.y0, z0 = tc.z0, base = tc.base;
        const T *g = (const T *)tc.grad;
        if (tid == 0) {   // (ordered before the appends by the barrier below)
            s_pc = 0;
            s_rc = 0;
        }
        if (TMA) {
            const bool ok = mbar_wait(&bars[s], (unsigned)((j >> 1) & 1), status);
            if (__syncthreads_or(!ok)) return;
        } else {
            // loads are issued in batches of LB before any of them is used
            constexpr int LPT = (B::ELEMS + C::NT - 1) / C::NT;
            constexpr int LB = 12;
#pragma unroll
            for (int k0 = 0; k0 < LPT; k0 += LB) {
                unsigned v[LB];
#pragma unroll
                for (int kk = 0; kk < LB; kk++) {
                    const int i = tid + (k0 + kk) * C::NT;
                    const int hx = i % B::RW, hy = (i / B::RW) % C::HY, hz = i / (B::RW * C::HY);
                    const int x = x0 - B::A + hx, y = y0 - 1 + hy, z = C::D3 ? z0 - 1 + hz : 0;
                    v[kk] = 0;
                    if (k0 + kk < LPT && i < B::ELEMS && x >= 0 && x < geo.W && y >= 0 && y < geo.H && z >= 0 &&
                        z < geo.D)
                        v[kk] = __ldg(g + (z * geo.H + y) * geo.W + x);
                }
#pragma unroll
                for (int kk = 0; kk < LB; kk++) {
                    const int i = tid + (k0 + kk) * C::NT;
                    if (k0 + kk < LPT && i < B::ELEMS) gs[i] = (T)v[kk];
                }
            }
            __syncthreads();
        }

        int st[C::PER];
        int plateau = 0;
        // a tile whose halo lies inside the image needs no neighbour bounds checks
        const bool interior = x0 >= 1 && x0 + C::TX < geo.W && y0 >= 1 && y0 + C::TY < geo.H &&
                              (!C::D3 || (z0 >= 1 && z0 + C::TZ < geo.D));
        if (interior)
            plateau = init_step1<T, CONN, false, EXP>(gs, nx, st, tid, x0, y0, z0, geo, base, ex);
        else
            plateau = init_step1<T, CONN, true, EXP>(gs, nx, st, tid, x0, y0, z0, geo, base, ex);
        if (LIST && __any_sync(0xffffffffu, plateau)) {   // stage the tile's plateau pixels
            unsigned pm = 0;
#pragma unroll
            for (int k = 0; k < C::PER; k++) pm |= (unsigned)(st[k] == STP) << k;
            const int np = __popc(pm);
            int inc = np;   // warp scan of the counts, one shared atomic per warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            int off = 0;
            if (lane == 31) off = atomicAdd(&s_pc, inc);
            off = __shfl_sync(0xffffffffu, off, 31) + inc - np;
            for (; pm; pm &= pm - 1) sp[off++] = (uint16_t)(tid + (__ffs(pm) - 1) * C::NT);
        }
        // the strict minima are roots: the thread's place in the tile's span of
        // the root list (one global atomic per tile, taken below)
        unsigned rm = 0;
#pragma unroll
        for (int k = 0; k < C::PER; k++) rm |= (unsigned)(st[k] == ST1) << k;
        int roff = 0;
        if (__any_sync(0xffffffffu, rm)) {
            const int nr = __popc(rm);
            int inc = nr;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            int wo = 0;
            if (lane == 31) wo = atomicAdd(&s_rc, inc);
            roff = __shfl_sync(0xffffffffu, wo, 31) + inc - nr;
        }
        __syncthreads();  // the gradient box of stage s is no longer read
        if (TMA && tid == 0 && t + 2 * G < b.ntiles)
            init_issue<T, CONN, TMA>(&tm, gs, &bars[s], b, t + 2 * G);
        if (tid == 0) {   // the tile's spans (read after the next barrier)
            if (LIST && s_pc > 0) {
                s_pbase = atomicAdd(counters + CNT_PLIST, s_pc);
                pspan[t] = make_int2(s_pbase, s_pc);
            }
            if (s_rc > 0) s_rbase = atomicAdd(counters + CNT_ROOTS, s_rc);
        }

        // step III inside the tile: pointer doubling through shared memory
        // (in place: every value read is the pointer of a pixel further down
        // the same path, or the path's end), until no pointer stays in the tile.
        // No round waits for the others: each thread doubles until its own
        // pointers have left the tile (an unfinished pointer moves at least one
        // step per round down a path of fewer than NPIX steps).
        volatile int *vnx = nx;
        for (int round = 0; round < C::NPIX; round++) {
            int more = 0;
#pragma unroll
            for (int k = 0; k < C::PER; k++) {
                const int i = tid + k * C::NT;
                const int c = vnx[i];
                if (c >= 0) {
                    const int c2 = vnx[c];
                    vnx[i] = c2;
                    more |= c2 >= 0;
                }
            }
            if (!more) break;
        }
        __syncthreads();
        if (LIST)
            for (int q = tid; q < s_pc; q += C::NT) plist[s_pbase + q] = sp[q];

#pragma unroll
        for (int k = 0; k < C::PER; k++) {
            const int i = tid + k * C::NT;
            if (st[k] == STOUT) continue;
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            const int p = base + ((z0 + lz) * geo.H + y0 + ly) * geo.W + x0 + lx;
            const int e = vnx[i];
            par[p] = e < 0 ? dec_final(e) : p;  // e >= 0 does not survive the doubling
            if (st[k] != ST0) mi[p] = 0x7fffffff;
        }
        // list the strict minima in the tile's span
        for (int rp = s_rbase + roff; rm; rm &= rm - 1) {
            const int i = tid + (__ffs(rm) - 1) * C::NT;
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            roots[rp++] = base + ((z0 + lz) * geo.H + y0 + ly) * geo.W + x0 + lx;
        }
        // dist: on plateau tiles the start of step II; in 2D on every tile
        // (k_jump2 tells plateau pixels from the others by it)
        const bool pl = __syncthreads_or(plateau);
        if (pl || !C::D3) {
#pragma unroll
            for (int k = 0; k < C::PER; k++) {
                if (st[k] == STOUT) continue;
                const int i = tid + k * C::NT;
                const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
                const int p = base + ((z0 + lz) * geo.H + y0 + ly) * geo.W + x0 + lx;
                dist[p] = st[k] == ST0 ? 0 : (st[k] == ST1 ? -2 : INF_D);
            }
        }
        if (pl) {
            if (tid == 0) {
                plat[t] = 1;
                act[t] = 1;
                tlist[atomicAdd(counters + CNT_TILES, 1)] = t;
            }
        } else if (tid == 0) {
            plat[t] = 0;
        }
        // (the __syncthreads_or above also orders this tile's nx, sp, s_pc and
        // s_rbase reads before the next tile's writes)
    }
}

// ---------------------------------------------------------------------------
// k_init6: k_init for 3D 6-connectivity, one z column of the tile per thread
// ---------------------------------------------------------------------------
//
// Step I (Eq. 1) and step III inside the tile, for the 3D path (k_init6,
// k_chase, k_rag6):
//   - a pixel whose arrow leaves the tile, a minimum and a plateau pixel end
//     their in-tile paths; the ends of tile t get slots 0..n-1, ends[first +
//     slot] = (end pixel, next pixel of its path: the neighbour its arrow
//     leads to, or itself for a minimum or a plateau pixel) and tends[t] =
//     (first, n);
//   - pointer doubling (ends point at themselves; a thread's column of
//     pointers in registers, every load of a round issued before any store)
//     takes every pixel to its end: the low 13 bits of code[p] are the slot
//     of p's end (the top three, its end's lowest neighbour, are masked off
//     by every reader);
//   - only on plateau tiles, par[p] is the arrow of Eq. 1 (the lowest
//     neighbour), or p itself for a strict minimum or a plateau pixel
//     (resolved later by step II / IV); no other kernel of the path reads an
//     arrow, so the other tiles write none.
// Step I picks the lowest neighbour with one integer minimum over packed
// keys (value << 3 | 7 - n, so that ties go to the later neighbour n in
// ascending index order) and has no divergent branches.

__device__ __forceinline__ unsigned umin2(unsigned a, unsigned b) { return a < b ? a : b; }

template <typename T> struct Init6Box {
    using B = InitBox<T, 6>;
    static constexpr int NPIX = TC<6>::NPIX;
    // one gradient box, 16-bit in-tile pointers, slots: 63,872 bytes for
    // uint16, so three CTAs share an SM
    static constexpr int SMEM_TMA = B::STAGE + NPIX * 2 + NPIX * 2;
    static constexpr int SMEM_PLAIN = SMEM_TMA;
};

// Global offset of neighbour n (ascending index order: -z, -y, -x, +x, +y, +z).
__device__ __forceinline__ int go6(int n, const Geo &geo)
{
    const int a = n == 0 || n == 5 ? geo.HW : (n == 1 || n == 4 ? geo.W : 1);
    return n < 3 ? -a : a;
}

// Step I on the thread's column (z = 0..TZ-1): in-tile pointers into nx
// (ends point at themselves), the lowest neighbour n of every pixel into the
// top three bits of its slotof entry (n << 13), states into stb (two bits per
// pixel), ends into endb, strict minima into minb.  CHECK = false for a tile
// whose halo lies inside the image.  FULL also writes every pixel's arrow into
// par; when ex.s is set, the states and arrows of Eq. 1 go into ex.
template <typename T, bool CHECK, bool FULL>
__device__ __forceinline__ void init6_step1(const T *gs, uint16_t *nx, uint16_t *slotof, int32_t *par,
                                            const int *lo_tab, int tid, int lx, int ly, int h0, int p0, int x, int y,
                                            int z0, const Geo &geo, unsigned &stb, unsigned &endb, unsigned &minb,
                                            int &plateau, const StepExport &ex)
{
    using C = TC<6>;
    using B = InitBox<T, 6>;
    constexpr int SZ = C::HY * B::RW;
    const bool col_in = x < geo.W && y < geo.H;
    const bool vxm = x > 0, vxp = x + 1 < geo.W, vym = y > 0, vyp = y + 1 < geo.H;
    // bit n: neighbour n of a pixel of this column lies in the tile (z bits per k below)
    const unsigned tcol = (ly > 0 ? 2u : 0u) | (lx > 0 ? 4u : 0u) | (lx < C::TX - 1 ? 8u : 0u) |
                          (ly < C::TY - 1 ? 16u : 0u);
    unsigned cz[C::TZ + 2];
#pragma unroll
    for (int k = 0; k < C::TZ + 2; k++) cz[k] = gs[h0 + k * SZ];
#pragma unroll
    for (int k = 0; k < C::TZ; k++) {
        const int z = z0 + k, p = p0 + k * geo.HW;
        const int h = h0 + (k + 1) * SZ;
        const unsigned gp = cz[k + 1];
        unsigned k0 = cz[k] * 8u + 7u, k1 = (unsigned)gs[h - B::RW] * 8u + 6u, k2 = (unsigned)gs[h - 1] * 8u + 5u;
        unsigned k3 = (unsigned)gs[h + 1] * 8u + 4u, k4 = (unsigned)gs[h + B::RW] * 8u + 3u, k5 = cz[k + 2] * 8u + 2u;
        if (CHECK) {
            k0 = z > 0 ? k0 : 0xffffffffu;
            k1 = vym ? k1 : 0xffffffffu;
            k2 = vxm ? k2 : 0xffffffffu;
            k3 = vxp ? k3 : 0xffffffffu;
            k4 = vyp ? k4 : 0xffffffffu;
            k5 = z + 1 < geo.D ? k5 : 0xffffffffu;
        }
        const unsigned m = umin2(umin2(umin2(k0, k1), umin2(k2, k3)), umin2(k4, k5));
        const bool has = !CHECK || m != 0xffffffffu;
        const unsigned vmin = m >> 3;
        const int n = 7 - (int)(m & 7u);
        const bool in = !CHECK || (col_in && z < geo.D);
        const bool st0 = has && vmin < gp, st1 = !has || vmin > gp;
        const int state = !in ? STOUT : (st0 ? ST0 : (st1 ? ST1 : STP));
        const unsigned tin = (tcol | (k > 0 ? 1u : 0u) | (k < C::TZ - 1 ? 32u : 0u)) >> (n & 7);
        const int i = tid + k * C::NT;
        const bool follow = in && st0 && (tin & 1u);   // the arrow stays in the tile
        const int nn = has ? n : 0;
        nx[i] = (uint16_t)(follow ? i + lo_tab[nn] : i);
        if (FULL && in) par[p] = st0 ? p + go6(nn, geo) : p;
        // Only ws_step1 sets ex.s.  The uniform branch costs one instruction
        // per pixel and also keeps the compiler from interleaving all sixteen
        // pixels of the column (which runs out of registers).
        if (in && ex.s) {   // Eq. 1: state 2 when the equal lowest neighbour comes later, 3 when earlier
            const bool later = nn >= 3;
            const int q = p + go6(nn, geo);
            ex.s[p] = (uint8_t)(st0 ? 0 : (st1 ? 1 : (later ? 2 : 3)));
            ex.l[p] = st0 || (!st1 && later) ? q : p;
        }
        slotof[i] = (uint16_t)(nn << 13);
        plateau |= state == STP;
        stb |= (unsigned)state << (2 * k);
        endb |= (unsigned)(in && !follow) << k;
        minb |= (unsigned)(state == ST1) << k;
    }
}

// FULL: the variant of the step I entry points (ws_step1, ws_plateau_distance),
// which also writes every pixel's arrow into par and optionally exports the
// states and arrows.  The segmentation path writes par on plateau tiles only
// (the step II / IV kernels and k_jump2 work there); elsewhere the arrow of a
// path end travels with it in `ends`.
template <typename T, bool TMA, bool FULL>
__global__ void __launch_bounds__(TT<6>::NT, 3) k_init6(const __grid_constant__ CUtensorMap tm, const Batch b,
                                                        int32_t *__restrict__ par, int32_t *__restrict__ mi,
                                                        int32_t *__restrict__ dist, uint8_t *__restrict__ plat,
                                                        uint8_t *__restrict__ act, int32_t *__restrict__ tlist,
                                                        int32_t *__restrict__ roots, uint16_t *__restrict__ code,
                                                        int2 *__restrict__ ends, int2 *__restrict__ tends,
                                                        int32_t *counters, DevStatus *status, const StepExport ex)
{
    using C = TC<6>;
    using B = InitBox<T, 6>;
    static_assert(C::NT == C::TX * C::TY && C::TX == 32 && C::PER == C::TZ && C::NT / 32 <= 32, "column layout");
    constexpr int NW = C::NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int wbase[NW];
    __shared__ int s_first;
    __shared__ int lo_tab[6];
    uint16_t *nx = (uint16_t *)(smem + B::STAGE);
    uint16_t *slotof = nx + C::NPIX;
    const int tid = threadIdx.x, lane = tid & 31, lx = lane, ly = tid >> 5;
    const int G = gridDim.x;
    constexpr int SZ = C::HY * B::RW;              // box step of one z
    const int h0 = (ly + 1) * B::RW + lx + B::A;   // box index of (lx, ly, z = -1)
    if (tid < 6) {  // local offsets of the neighbours, ascending index order
        const int l[6] = {-C::TX * C::TY, -C::TX, -1, 1, C::TX, C::TX * C::TY};
        lo_tab[tid] = l[tid];
    }

    if (TMA) {  // a single image (b.one); the next tile's box loads while this tile's paths are doubled
        if (tid == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
            const int t0 = blockIdx.x;
            if (t0 < b.ntiles) init_issue<T, 6, TMA>(&tm, (T *)smem, &bar, b, t0);
        }
    }
    __syncthreads();

    int j = 0;
    for (int t = blockIdx.x; t < b.ntiles; t += G, j++) {
        T *gs = (T *)smem;
        const TileCtx tc = tile_ctx<6>(b, t);
        const Geo &geo = tc.geo;
        const int x0 = tc.x0, y0 = tc.y0, z0 = tc.z0, base = tc.base;
        if (TMA) {
            const bool ok = mbar_wait(&bar, (unsigned)(j & 1), status);
            if (__syncthreads_or(!ok)) return;
        } else {
            const T *g = (const T *)tc.grad;
            constexpr int LPT = (B::ELEMS + C::NT - 1) / C::NT;
            constexpr int LB = 6;
#pragma unroll
            for (int k0 = 0; k0 < LPT; k0 += LB) {
                unsigned v[LB];
#pragma unroll
                for (int kk = 0; kk < LB; kk++) {
                    const int i = tid + (k0 + kk) * C::NT;
                    const int hx = i % B::RW, hy = (i / B::RW) % C::HY, hz = i / (B::RW * C::HY);
                    const int xx = x0 - B::A + hx, yy = y0 - 1 + hy, zz = z0 - 1 + hz;
                    v[kk] = 0;
                    if (k0 + kk < LPT && i < B::ELEMS && xx >= 0 && xx < geo.W && yy >= 0 && yy < geo.H &&
                        zz >= 0 && zz < geo.D)
                        v[kk] = __ldg(g + (zz * geo.H + yy) * geo.W + xx);
                }
#pragma unroll
                for (int kk = 0; kk < LB; kk++) {
                    const int i = tid + (k0 + kk) * C::NT;
                    if (k0 + kk < LPT && i < B::ELEMS) gs[i] = (T)v[kk];
                }
            }
            __syncthreads();
        }

        // step I (Eq. 1) on the column
        const int x = x0 + lx, y = y0 + ly;
        const int HW = geo.HW;
        const bool interior = x0 >= 1 && x0 + C::TX < geo.W && y0 >= 1 && y0 + C::TY < geo.H && z0 >= 1 &&
                              z0 + C::TZ < geo.D;
        const int p0 = base + (z0 * geo.H + y) * geo.W + x;   // global index of (lx, ly, z = 0)
        unsigned stb = 0;   // pixel states, two bits each
        unsigned endb = 0;  // bit k: pixel k of the column ends its in-tile path
        unsigned minb = 0;  // bit k: pixel k of the column is a strict minimum
        int plateau = 0;
        if (interior)
            init6_step1<T, false, FULL>(gs, nx, slotof, par, lo_tab, tid, lx, ly, h0, p0, x, y, z0, geo, stb, endb,
                                        minb, plateau, ex);
        else
            init6_step1<T, true, FULL>(gs, nx, slotof, par, lo_tab, tid, lx, ly, h0, p0, x, y, z0, geo, stb, endb,
                                       minb, plateau, ex);
        // the strict minima are roots: list them (their smallest index is taken later)
        for (unsigned m = minb; m; m &= m - 1) {
            const int p = p0 + (__ffs(m) - 1) * HW;
            roots[atomicAdd(counters + CNT_ROOTS, 1)] = p;
            mi[p] = 0x7fffffff;
        }
        // number the ends: the thread's ends get consecutive slots after those
        // of the lanes before it (warp scan) and of the warps before it
        int lpre, wtot;
        {
            const int ne = __popc(endb);
            int inc = ne;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            lpre = inc - ne;
            wtot = __shfl_sync(0xffffffffu, inc, 31);
            if (lane == 31) wbase[ly] = inc;
        }
        __syncthreads();  // the gradient box is no longer read: load the next tile's
        if (TMA && tid == 0 && t + G < b.ntiles) init_issue<T, 6, TMA>(&tm, gs, &bar, b, t + G);
        int first = 0, nend = 0;
        if (ly == 0) {
            const int c = lane < NW ? wbase[lane] : 0;
            int inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            nend = __shfl_sync(0xffffffffu, inc, 31);
            if (lane < NW) wbase[lane] = inc - c;
            if (lane == 0) {
                first = atomicAdd(counters + CNT_ENDS, nend);
                s_first = first;
                tends[t] = make_int2(first, nend);
            }
        }
        __syncthreads();
        {
            // the warp's ends take the slots wbase[ly] + 0 .. wtot - 1 in lane
            // order (a lane's own ends in z order); lane j writes the warp's
            // ends j, j + 32, ...: the owner lane o of end j is the last lane
            // with lpre <= j, and the end is the (j - lpre(o))-th voxel of o's
            // column with an endb bit.  Each end's slot goes below its lowest
            // neighbour in its slotof entry; its entry of ends is (the end,
            // the next voxel of its path: the neighbour its arrow leads to out
            // of the tile, or itself for a minimum or a plateau voxel).
            const int ws0 = wbase[ly], fst = s_first + ws0;
            const int rounds = (wtot + 31) >> 5;
            for (int r = 0; r < rounds; r++) {
                const int jj = r * 32 + lane;
                int o = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int lp = __shfl_sync(0xffffffffu, lpre, o + step);
                    if (lp <= jj) o += step;
                }
                const unsigned eo = __shfl_sync(0xffffffffu, endb, o);
                const unsigned so = __shfl_sync(0xffffffffu, stb, o);
                const int lo = __shfl_sync(0xffffffffu, lpre, o);
                if (jj < wtot) {
                    // k: the voxel of the (jj - lo)-th set bit of eo
                    const int rk = jj - lo;
                    int k = 0;
#pragma unroll
                    for (int step = 8; step > 0; step >>= 1)
                        if (__popc(eo & ((1u << (k + step)) - 1u)) <= rk) k += step;
                    uint16_t *se = slotof + ly * 32 + o + k * C::NT;
                    const unsigned v = *se;
                    const int sl = ws0 + jj;
                    *se = (uint16_t)(v | (unsigned)sl);
                    const int e = p0 + (o - lane) + k * HW;
                    const int nxt = ((so >> (2 * k)) & 3u) == (unsigned)ST0 ? e + go6((int)(v >> 13), geo) : e;
                    ends[fst + jj] = make_int2(e, nxt);
                }
            }
            __syncwarp();   // the slotof entries of the warp's ends are written
        }

        // step III inside the tile: pointer doubling.  A value read while its
        // owner is updating it is the old or the new pointer of a pixel further
        // down the same path, or the path's end; so no round needs the others
        // to be done: each thread doubles until its own pixels point at their
        // ends (every round moves an unfinished pointer at least one step down
        // a path of fewer than NPIX steps, so NPIX rounds always suffice).
        int cur[C::TZ];
#pragma unroll
        for (int k = 0; k < C::TZ; k++) cur[k] = nx[tid + k * C::NT];
        volatile uint16_t *vnx = nx;
        for (int round = 0; round < C::NPIX; round++) {
            int more = 0;
#pragma unroll
            for (int h = 0; h < C::TZ; h += 8) {  // eight entries in flight
                int nxt[8];
#pragma unroll
                for (int k = 0; k < 8; k++) nxt[k] = vnx[cur[h + k]];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    vnx[tid + (h + k) * C::NT] = nxt[k];
                    more |= nxt[k] != cur[h + k];
                    cur[h + k] = nxt[k];
                }
            }
            if (!more) break;
        }
        __syncthreads();   // every pointer at its end; slotof published
#pragma unroll
        for (int k = 0; k < C::TZ; k++) {
            if (((stb >> (2 * k)) & 3u) == (unsigned)STOUT) continue;
            code[p0 + k * HW] = slotof[cur[k]];   // cur[k]: the end (the top three bits ride along)
        }
        if (__syncthreads_or(plateau)) {
            // a plateau tile: step II starts from dist, and the step II / IV
            // kernels and k_jump2 work on every pixel's arrow (rare: not unrolled)
#pragma unroll 1
            for (int k = 0; k < C::TZ; k++) {
                const unsigned sk = (stb >> (2 * k)) & 3u;
                if (sk == (unsigned)STOUT) continue;
                const int p = p0 + k * HW;
                dist[p] = sk == (unsigned)ST0 ? 0 : (sk == (unsigned)ST1 ? -2 : INF_D);
                if (!FULL) par[p] = sk == (unsigned)ST0 ? p + go6(slotof[tid + k * C::NT] >> 13, geo) : p;
                if (sk == (unsigned)STP) mi[p] = 0x7fffffff;   // a root candidate
            }
            if (tid == 0) {
                plat[t] = 1;
                act[t] = 1;
                tlist[atomicAdd(counters + CNT_TILES, 1)] = t;
            }
        } else if (tid == 0) {
            plat[t] = 0;
        }
        // (the __syncthreads_or above also orders this tile's nx, slotof,
        // wbase and s_first reads before the next tile's writes)
    }
}

// find / union in a tile-local union-find (the smaller index is the
// root; atomicCAS links a root to a smaller root)
__device__ __forceinline__ int lu_find(int *lab, int a)
{
    volatile int *v = lab;
    for (int it = 0; it < (1 << 16); it++) {
        const int b = v[a];
        if (b == a) return a;
        const int c = v[b];
        if (c == b) return b;
        v[a] = c;   // path halving
        a = c;
    }
    return a;
}

__device__ __forceinline__ void lu_union(int *lab, int a, int b)
{
    for (int it = 0; it < (1 << 16); it++) {
        a = lu_find(lab, a);
        b = lu_find(lab, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(lab + a, a, b) == a) return;
    }
}

// ---------------------------------------------------------------------------
// k_plateau2: step II distances on plateau tiles (cooperative)
// ---------------------------------------------------------------------------

template <typename T, int CONN>
__global__ void __launch_bounds__(TT<CONN>::NT) k_plateau2(const Batch b, int32_t *dist, const uint8_t *__restrict__ plat,
                                                           uint8_t *act, const int32_t *__restrict__ tlist,
                                                           const int32_t *counters, DevStatus *status, int round_cap,
                                                           unsigned long long timeout_ns,
                                                           const uint16_t *__restrict__ plist,
                                                           const int2 *__restrict__ pspan)
{
    using C = TC<CONN>;
    // 2D: the relaxation visits the tile's plateau pixels only (its span of
    // plist, staged as box indices in pl with their starting distances in po)
    constexpr bool LIST = kPlateauList<CONN>;
    extern __shared__ __align__(128) unsigned char smem[];
    int *gs = (int *)smem;
    int *ds = gs + C::HS;
    int *po = ds + C::HS;                              // (LIST) [NPIX]
    uint16_t *pl = (uint16_t *)(po + C::NPIX);         // (LIST) [NPIX]
    __shared__ int flag_s;
    const int tid = threadIdx.x;
    const int ntl = counters[CNT_TILES];
    uint8_t *act0 = act, *act1 = act + b.ntiles;

    for (int r = 0;; r++) {
        uint8_t *cur = (r & 1) ? act1 : act0;
        uint8_t *nxt = (r & 1) ? act0 : act1;
        if (blockIdx.x == 0 && tid == 0) status->changed[(r + 1) % 3] = 0;
        for (int j = blockIdx.x; j < ntl; j += gridDim.x) {
            const int t = tlist[j];
            __syncthreads();
            if (tid == 0) {
                flag_s = *(volatile uint8_t *)(cur + t);
                if (flag_s) cur[t] = 0;
            }
            __syncthreads();
            if (!flag_s) continue;
            const TileCtx tc = tile_ctx<CONN>(b, t);
            const Geo &geo = tc.geo;
            const T *g = (const T *)tc.grad;
            const int x0 = tc.x0, y0 = tc.y0, z0 = tc.z0;
            for (int i = tid; i < C::HS; i += C::NT) {
                const int hx = i % C::HX, hy = (i / C::HX) % C::HY, hz = i / (C::HX * C::HY);
                const int x = x0 - 1 + hx, y = y0 - 1 + hy, z = C::D3 ? z0 - 1 + hz : 0;
                if (x >= 0 && x < geo.W && y >= 0 && y < geo.H && z >= 0 && z < geo.D) {
                    const int q = (z * geo.H + y) * geo.W + x;
                    gs[i] = (int)g[q];
                    // a pixel of a tile without plateau pixels that is equal to a
                    // plateau neighbour has a lower neighbour: distance 0 (the
                    // tile's own pixels need no look-up: it is a plateau tile)
                    const bool own = hx >= 1 && hx <= C::TX && hy >= 1 && hy <= C::TY &&
                                     (!C::D3 || (hz >= 1 && hz <= C::TZ));
                    ds[i] = own || plat[tc.tile0 + tile_of_c<CONN>(tc.tg, x, y, z)] ? __ldcg(dist + tc.base + q) : 0;
                } else {
                    gs[i] = -1;
                    ds[i] = INF_D;
                }
            }
            int border = 0;
            if constexpr (LIST) {
                const int2 span = pspan[t];
                for (int e = tid; e < span.y; e += C::NT) {
                    const int i = plist[span.x + e];
                    pl[e] = (uint16_t)(((i / C::TX) + 1) * C::HX + i % C::TX + 1);
                }
                __syncthreads();   // the box and the list are written
                for (int e = tid; e < span.y; e += C::NT) po[e] = ds[pl[e]];
                for (int it = 0; it < 4 * C::NPIX + 8; it++) {
                    int ch = 0;
                    for (int e = tid; e < span.y; e += C::NT) {
                        const int h = pl[e];
                        const int gv = gs[h];
                        const int d = ds[h];
                        if (d <= 0) continue;
                        int best = d;
#pragma unroll
                        for (int n = 0; n < Nb<CONN>::n; n++) {
                            const int hn = h + Nb<CONN>::dy(n) * C::HX + Nb<CONN>::dx(n);
                            if (gs[hn] == gv) best = imin(best, ds[hn] + 1);
                        }
                        if (best < d) {
                            ds[h] = best;
                            ch = 1;
                        }
                    }
                    if (!__syncthreads_or(ch)) break;
                }
                for (int e = tid; e < span.y; e += C::NT) {
                    const int h = pl[e];
                    if (ds[h] == po[e]) continue;
                    const int lx = h % C::HX - 1, ly = h / C::HX - 1;
                    __stcg(dist + tc.base + (y0 + ly) * geo.W + x0 + lx, ds[h]);
                    if (lx == 0 || lx == C::TX - 1 || ly == 0 || ly == C::TY - 1) border = 1;
                }
            } else {
                __syncthreads();
                int orig[C::PER];
#pragma unroll
                for (int k = 0; k < C::PER; k++) {
                    const int i = tid + k * C::NT;
                    const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
                    orig[k] = ds[((C::D3 ? lz + 1 : 0) * C::HY + ly + 1) * C::HX + lx + 1];
                }
                for (int it = 0; it < 4 * C::NPIX + 8; it++) {
                    int ch = 0;
#pragma unroll
                    for (int k = 0; k < C::PER; k++) {
                        const int i = tid + k * C::NT;
                        const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
                        const int h = ((C::D3 ? lz + 1 : 0) * C::HY + ly + 1) * C::HX + lx + 1;
                        const int gv = gs[h];
                        const int d = ds[h];
                        if (gv < 0 || d <= 0) continue;
                        int best = d;
#pragma unroll
                        for (int n = 0; n < Nb<CONN>::n; n++) {
                            const int hn = h + (Nb<CONN>::dz(n) * C::HY + Nb<CONN>::dy(n)) * C::HX + Nb<CONN>::dx(n);
                            if (gs[hn] == gv) best = imin(best, ds[hn] + 1);
                        }
                        if (best < d) {
                            ds[h] = best;
                            ch = 1;
                        }
                    }
                    if (!__syncthreads_or(ch)) break;
                }
#pragma unroll
                for (int k = 0; k < C::PER; k++) {
                    const int i = tid + k * C::NT;
                    const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
                    const int h = ((C::D3 ? lz + 1 : 0) * C::HY + ly + 1) * C::HX + lx + 1;
                    if (ds[h] != orig[k]) {
                        __stcg(dist + tc.base + ((z0 + lz) * geo.H + y0 + ly) * geo.W + x0 + lx, ds[h]);
                        if (lx == 0 || lx == C::TX - 1 || ly == 0 || ly == C::TY - 1 ||
                            (C::D3 && (lz == 0 || lz == C::TZ - 1)))
                            border = 1;
                    }
                }
            }
            if (__syncthreads_or(border) && tid == 0) {
                const TileGeo &tg = tc.tg;
                const int lt = t - tc.tile0;
                const int tx = lt % tg.ntx, ty = (lt / tg.ntx) % tg.nty, tz = lt / (tg.ntx * tg.nty);
                for (int dz = (C::D3 ? -1 : 0); dz <= (C::D3 ? 1 : 0); dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            const int ax = tx + dx, ay = ty + dy, az = tz + dz;
                            if (ax < 0 || ax >= tg.ntx || ay < 0 || ay >= tg.nty || az < 0 || az >= tg.ntz)
                                continue;
                            const int nt = tc.tile0 + (az * tg.nty + ay) * tg.ntx + ax;
                            if (nt != t && plat[nt]) nxt[nt] = 1;
                        }
                atomicAdd(&status->changed[r % 3], 1);
            }
        }
        __threadfence();
        if (!grid_barrier(status, timeout_ns)) return;
        if (*(volatile int *)&status->changed[r % 3] == 0) {
            if (blockIdx.x == 0 && tid == 0) status->rounds_plateau = r + 1;
            return;
        }
        if (r + 1 >= round_cap) {
            if (blockIdx.x == 0 && tid == 0) record_error(status, DEV_NONCONVERGED, 2);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// k_resolve2: step II pointer choice and step IV Union on plateau tiles
// ---------------------------------------------------------------------------

// Step II pointer choice on the plateau tiles, and step IV inside each tile:
// the minimal-plateau pixels of a tile are joined in a shared-memory union-find
// and each points at its component's smallest pixel (k_union2 joins the
// components across tile borders).
template <typename T, int CONN>
__global__ void __launch_bounds__(TT<CONN>::NT) k_resolve2(const Batch b, int32_t *par, const int32_t *__restrict__ dist,
                                                           const uint8_t *__restrict__ plat,
                                                           const int32_t *__restrict__ tlist,
                                                           const int32_t *counters, DevStatus *status,
                                                           const uint16_t *__restrict__ plist,
                                                           const int2 *__restrict__ pspan)
{
    using C = TC<CONN>;
    constexpr bool LIST = kPlateauList<CONN>;
    __shared__ int lab[C::NPIX];   // tile-local union-find of the minimal-plateau pixels (-1: other pixel)
    __shared__ uint16_t sl[LIST ? C::NPIX : 1];   // (LIST) the tile's plateau pixels
    // (LIST) a plateau pixel's descent on this tile's plateau: the local index
    // of the next plateau pixel, or ~(global pixel) where it leaves them
    __shared__ int nt[LIST ? C::NPIX : 1];
    const int ntl = counters[CNT_TILES];
    for (int j = blockIdx.x; j < ntl; j += gridDim.x) {
        const int t = tlist[j];
        const TileCtx tc = tile_ctx<CONN>(b, t);
        const Geo &geo = tc.geo;
        const T *g = (const T *)tc.grad;
        // LIST: only the tile's plateau pixels can be minimal-plateau pixels or
        // point anew (the others have distance 0 or -2)
        int2 span = make_int2(0, C::NPIX);
        if (LIST) {
            for (int i = threadIdx.x; i < C::NPIX; i += C::NT) lab[i] = -1;
            __syncthreads();
            span = pspan[t];
        }
        for (int ei = threadIdx.x; ei < span.y; ei += C::NT) {
            const int i = LIST ? (int)plist[span.x + ei] : ei;
            if (LIST) sl[ei] = (uint16_t)i;
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            const int x = tc.x0 + lx, y = tc.y0 + ly, z = tc.z0 + lz;
            int l = -1;
            if (x < geo.W && y < geo.H && z < geo.D) {
                const int p = (z * geo.H + y) * geo.W + x;
                const int d = dist[tc.base + p];
                if (d >= INF_D) {
                    l = i;
                } else if (d > 0) {
                    const unsigned gp = g[p];
                    int best = -1, bestl = -1;
#pragma unroll
                    for (int n = 0; n < Nb<CONN>::n; n++) {
                        const int xx = x + Nb<CONN>::dx(n), yy = y + Nb<CONN>::dy(n), zz = z + Nb<CONN>::dz(n);
                        if (xx < 0 || xx >= geo.W || yy < 0 || yy >= geo.H || zz < 0 || zz >= geo.D) continue;
                        const int q = (zz * geo.H + yy) * geo.W + xx;
                        if (g[q] != gp) continue;
                        const int dq = plat[tc.tile0 + tile_of_c<CONN>(tc.tg, xx, yy, zz)] ? dist[tc.base + q] : 0;
                        if (dq == d - 1 && q > best) {
                            best = q;
                            const int ax = lx + Nb<CONN>::dx(n), ay = ly + Nb<CONN>::dy(n);
                            bestl = ax >= 0 && ax < C::TX && ay >= 0 && ay < C::TY ? ay * C::TX + ax : -1;
                        }
                    }
                    if (best < 0) {
                        record_error(status, DEV_NONCONVERGED, 7);
                        best = p;
                        bestl = -1;
                    }
                    if (LIST)
                        nt[i] = d > 1 && bestl >= 0 ? bestl : ~(tc.base + best);
                    else
                        par[tc.base + p] = tc.base + best;
                }
            }
            lab[i] = l;
        }
        __syncthreads();
        if (LIST) {
            // step III along the tile's plateau pixels (pointer doubling in
            // shared memory): each plateau pixel then points where its descent
            // leaves them -- a pixel at distance 0 or one of another tile
            for (int round = 0; round < C::NPIX; round++) {
                int more = 0;
                for (int ei = threadIdx.x; ei < span.y; ei += C::NT) {
                    const int i = sl[ei];
                    const int c = nt[i];
                    if (lab[i] >= 0 || c < 0) continue;
                    const int c2 = nt[c];
                    nt[i] = c2;
                    more |= c2 >= 0;
                }
                if (!__syncthreads_or(more)) break;
            }
            for (int ei = threadIdx.x; ei < span.y; ei += C::NT) {
                const int i = sl[ei];
                if (lab[i] >= 0) continue;
                const int lx = i % C::TX, ly = i / C::TX;
                par[tc.base + (tc.y0 + ly) * geo.W + tc.x0 + lx] = ~nt[i];
            }
        }
        // unions with the forward neighbours inside the tile (LIST: the
        // minimal-plateau pixels are among the listed ones)
        for (int ei = threadIdx.x; ei < span.y; ei += C::NT) {
            const int i = LIST ? (int)sl[ei] : ei;
            if (lab[i] < 0) continue;
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            const unsigned gp = g[((tc.z0 + lz) * geo.H + tc.y0 + ly) * geo.W + tc.x0 + lx];
#pragma unroll
            for (int n = Half<CONN>::first; n < Nb<CONN>::n; n++) {
                const int xx = lx + Nb<CONN>::dx(n), yy = ly + Nb<CONN>::dy(n), zz = lz + Nb<CONN>::dz(n);
                if (xx < 0 || xx >= C::TX || yy < 0 || yy >= C::TY || zz < 0 || zz >= C::TZ) continue;
                const int jn = (zz * C::TY + yy) * C::TX + xx;
                if (lab[jn] < 0) continue;
                if (g[((tc.z0 + zz) * geo.H + tc.y0 + yy) * geo.W + tc.x0 + xx] == gp) lu_union(lab, i, jn);
            }
        }
        __syncthreads();
        // every minimal-plateau pixel points at its in-tile component's smallest pixel
        for (int ei = threadIdx.x; ei < span.y; ei += C::NT) {
            const int i = LIST ? (int)sl[ei] : ei;
            if (lab[i] < 0) continue;
            const int r = lu_find(lab, i);
            const int rx = r % C::TX, ry = (r / C::TX) % C::TY, rz = r / (C::TX * C::TY);
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            par[tc.base + ((tc.z0 + lz) * geo.H + tc.y0 + ly) * geo.W + tc.x0 + lx] =
                tc.base + ((tc.z0 + rz) * geo.H + tc.y0 + ry) * geo.W + tc.x0 + rx;
        }
        __syncthreads();   // lab is reused by the next tile
    }
}

// Step IV across tile borders: every minimal-plateau pixel of a plateau tile
// is joined (global union-find, smaller index as root) with its forward
// neighbours of equal value that are minimal-plateau pixels of other tiles.
template <typename T, int CONN>
__global__ void __launch_bounds__(NTHR) k_union2(const Batch b, int32_t *par, const int32_t *__restrict__ dist,
                                               const uint8_t *__restrict__ plat, const int32_t *__restrict__ tlist,
                                               const int32_t *counters, DevStatus *status)
{
    using C = TC<CONN>;
    // 2D: the pixels with a forward neighbour outside the tile are its last
    // column, its last row and (8-connectivity) its first column; they are
    // enumerated directly (e -> (lx, ly)), 3D tests every pixel of the tile
    constexpr bool D2 = !C::D3;
    constexpr bool X0 = CONN % 100 == 8;
    constexpr int NB = D2 ? C::TY + C::TX - 1 + (X0 ? C::TY - 1 : 0) : C::NPIX;
    const int ntl = counters[CNT_TILES];
    for (int j = blockIdx.x; j < ntl; j += gridDim.x) {
        const TileCtx tc = tile_ctx<CONN>(b, tlist[j]);
        const Geo &geo = tc.geo;
        const T *g = (const T *)tc.grad;
        for (int ei = threadIdx.x; ei < NB; ei += NTHR) {
            int i = ei;
            if (D2)
                i = ei < C::TY ? ei * C::TX + C::TX - 1
                               : (ei < C::TY + C::TX - 1 ? (C::TY - 1) * C::TX + ei - C::TY
                                                         : (ei - (C::TY + C::TX - 1)) * C::TX);
            const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
            // only pixels with a forward neighbour outside the tile
            const bool border = lx == C::TX - 1 || ly == C::TY - 1 || (C::D3 && lz == C::TZ - 1) ||
                                ((CONN % 100 == 8 || CONN == 26) && lx == 0) || (CONN == 26 && ly == 0);
            if (!border) continue;
            const int x = tc.x0 + lx, y = tc.y0 + ly, z = tc.z0 + lz;
            if (x >= geo.W || y >= geo.H || z >= geo.D) continue;
            const int p = (z * geo.H + y) * geo.W + x;
            if (dist[tc.base + p] < INF_D) continue;
            const unsigned gp = g[p];
#pragma unroll
            for (int n = Half<CONN>::first; n < Nb<CONN>::n; n++) {
                const int ax = lx + Nb<CONN>::dx(n), ay = ly + Nb<CONN>::dy(n), az = lz + Nb<CONN>::dz(n);
                if (ax >= 0 && ax < C::TX && ay >= 0 && ay < C::TY && az >= 0 && az < C::TZ) continue;   // in the tile
                const int xx = x + Nb<CONN>::dx(n), yy = y + Nb<CONN>::dy(n), zz = z + Nb<CONN>::dz(n);
                if (xx < 0 || xx >= geo.W || yy < 0 || yy >= geo.H || zz < 0 || zz >= geo.D) continue;
                if (!plat[tc.tile0 + tile_of_c<CONN>(tc.tg, xx, yy, zz)]) continue;
                const int q = (zz * geo.H + yy) * geo.W + xx;
                if (dist[tc.base + q] >= INF_D && g[q] == gp) uf_union(par, tc.base + p, tc.base + q, status);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_jump2: step III on plateau tiles (cooperative), lists minimal-plateau roots
// ---------------------------------------------------------------------------

// 3D 6-connectivity (SPARSE): par holds arrows on plateau tiles only, so a
// jump stops at a pixel of another tile that is not a plateau tile (its path
// goes on through the slot codes in k_chase); at the end, every path end of a
// plateau tile takes its final pointer as the next pixel of its path in ends.
template <int CONN>
__global__ void __launch_bounds__(NTHR) k_jump2(const Batch b, int32_t *par, const int32_t *__restrict__ dist,
                                                const int32_t *__restrict__ tlist, int32_t *counters,
                                                int32_t *roots, int RR, DevStatus *status, int round_cap,
                                                unsigned long long timeout_ns, const uint8_t *__restrict__ plat,
                                                int2 *ends, const int2 *__restrict__ tends,
                                                const uint16_t *__restrict__ plist, const int2 *__restrict__ pspan)
{
    using C = TC<CONN>;
    constexpr bool SPARSE = CONN == 6;
    constexpr bool LIST = kPlateauList<CONN>;   // 2D: the tiles' plateau pixels are listed
    const int tid = threadIdx.x, lane = tid & 31;
    const int ntl = counters[CNT_TILES];
    for (int r = 0;; r++) {
        if (blockIdx.x == 0 && tid == 0) status->changed[(r + 1) % 3] = 0;
        int ch = 0;
        for (int j = blockIdx.x; j < ntl; j += gridDim.x) {   // one tile at a time per block
            const int t = tlist[j];
            const TileCtx tc = tile_ctx<CONN>(b, t);
            const int2 span = LIST ? pspan[t] : make_int2(0, C::NPIX);
            for (int ei = tid; ei < span.y; ei += NTHR) {
                const int i = LIST ? (int)plist[span.x + ei] : ei;
                const int x = tc.x0 + i % C::TX, y = tc.y0 + (i / C::TX) % C::TY, z = tc.z0 + i / (C::TX * C::TY);
                if (x >= tc.geo.W || y >= tc.geo.H || z >= tc.geo.D) continue;
                const int p = tc.base + (z * tc.geo.H + y) * tc.geo.W + x;
                // 2D: only plateau pixels jump (the listed ones), and only
                // across plateau pixels (the rest of a path is chased tile by
                // tile later; dist is valid on every tile).  3D: every pixel
                // of a plateau tile jumps.
                if (!C::D3 && !LIST && dist[p] <= 0) continue;
                const int l0 = __ldcg(par + p);
                int l = l0;
                for (int k = 0; k < RR; k++) {
                    if (!C::D3 && dist[l] <= 0) break;
                    if (SPARSE) {   // l's arrow is known only on a plateau tile
                        const int ql = l - tc.base;
                        const int zl = ql / tc.geo.HW, rl = ql - zl * tc.geo.HW, yl = rl / tc.geo.W;
                        if (!plat[tc.tile0 + tile_of_c<CONN>(tc.tg, rl - yl * tc.geo.W, yl, zl)]) break;
                    }
                    const int l2 = __ldcg(par + l);
                    if (l2 == l) break;
                    l = l2;
                }
                if (l != l0) {
                    __stcg(par + p, l);
                    ch = 1;
                }
            }
        }
        const unsigned bl = __ballot_sync(0xffffffffu, ch);
        if (lane == 0 && bl) atomicAdd(&status->changed[r % 3], 1);
        __threadfence();
        if (!grid_barrier(status, timeout_ns)) return;
        if (*(volatile int *)&status->changed[r % 3] == 0) {
            if (blockIdx.x == 0 && tid == 0) status->rounds_jump = r + 1;
            break;
        }
        if (r + 1 >= round_cap) {
            if (blockIdx.x == 0 && tid == 0) record_error(status, DEV_NONCONVERGED, 5);
            return;
        }
    }
    // roots of minimal plateaux
    for (int j = blockIdx.x; j < ntl; j += gridDim.x) {
        const TileCtx tc = tile_ctx<CONN>(b, tlist[j]);
        const int2 span = LIST ? pspan[tlist[j]] : make_int2(0, C::NPIX);
        for (int e0 = 0; e0 < span.y; e0 += NTHR) {   // warp-uniform trip count
            const int ei = e0 + tid;
            bool isr = false;
            int p = 0;
            if (ei < span.y) {
                const int i = LIST ? (int)plist[span.x + ei] : ei;
                const int x = tc.x0 + i % C::TX, y = tc.y0 + (i / C::TX) % C::TY, z = tc.z0 + i / (C::TX * C::TY);
                if (x < tc.geo.W && y < tc.geo.H && z < tc.geo.D) {
                    p = tc.base + (z * tc.geo.H + y) * tc.geo.W + x;
                    isr = dist[p] >= INF_D && __ldcg(par + p) == p;
                }
            }
            const unsigned bl = __ballot_sync(0xffffffffu, isr);
            if (!bl) continue;
            int rb = 0;
            if (lane == 0) rb = atomicAdd(counters + CNT_ROOTS, __popc(bl));
            rb = __shfl_sync(0xffffffffu, rb, 0);
            if (isr) roots[rb + __popc(bl & ((1u << lane) - 1u))] = p;
        }
        if (SPARSE) {   // the path ends of the tile continue where their pointers now lead
            const int2 te = tends[tlist[j]];
            for (int i = tid; i < te.y; i += NTHR) {
                int2 c = ends[te.x + i];
                c.y = __ldcg(par + c.x);
                ends[te.x + i] = c;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_label: final roots, smallest index per basin, pass values (Alg. 5 step V)
// ---------------------------------------------------------------------------

// Insert (key, h) into the CTA's edge hash (min of h per key).  The slot is
// read before any atomic: lanes that find their key already present with a
// pass value <= h issue no atomic at all.  A crowded CTA table sends the pair
// straight to the sink.
template <bool HASHED>
static __device__ __noinline__ void smem_edge_insert(unsigned a, unsigned b, unsigned h, unsigned long long *hk,
                                                     unsigned *hv, int nslots, const EdgeSink L, DevStatus *status)
{
    const unsigned long long key = ((unsigned long long)a << 32) | b;
    unsigned s = (a * 0x9E3779B1u) ^ (b * 0x85EBCA77u);
    s = (s ^ (s >> 15)) & (unsigned)(nslots - 1);
    for (int probe = 0; probe < 32; probe++) {
        unsigned long long k = hk[s];
        if (k == EMPTY_KEY) {
            k = atomicCAS(hk + s, EMPTY_KEY, key);
            if (k == EMPTY_KEY) k = key;
        }
        if (k == key) {
            if (h < hv[s]) atomicMin(hv + s, h);
            return;
        }
        s = (s + 1) & (unsigned)(nslots - 1);
    }
    sink_put1<HASHED>(L, a, b, h, status);
}

// Shared-memory layout of k_label: the CTA's edge hash, then the path-end /
// root box and the gradient box of the tile's forward neighbourhood, each
// row widened to start on a 16-byte boundary.
template <typename T, int CONN> struct LabelBox {
    using C = TC<CONN>;
    static constexpr int AP = 4;                        // int32 per 16 bytes
    static constexpr int RWP = C::TX + 2 * AP;          // par box: x from x0 - 4
    static constexpr int AG = 16 / (int)sizeof(T);
    static constexpr int RWG = C::TX + 2 * AG;          // grad box: x from x0 - AG
    static constexpr int PBYTES = RWP * C::BY * C::BZ * 4;
    static constexpr int GBYTES = RWG * C::BY * C::BZ * (int)sizeof(T);
    // distinct path ends per tile (dedupe table): a 2D tile's box holds about 2,100 pixels whose paths
    // end at a few hundred pixels; a 3D box (26-connectivity) about 9,500
    static constexpr int DSLOTS = C::D3 ? 4096 : 1024;
    static constexpr int RBYTES = DSLOTS * 8 > C::HASH * 12 ? DSLOTS * 8 : C::HASH * 12;
    static constexpr int OFF_P = (RBYTES + 127) & ~127; // region R (dedupe, then edge hash) first
    static constexpr int OFF_G = OFF_P + ((PBYTES + 127) & ~127);
    static constexpr int SMEM = OFF_G + ((GBYTES + 127) & ~127);
};

// Slot of `key` in the CTA's table of distinct path ends (inserted if new);
// -1 when the table is crowded.
__device__ __forceinline__ int dedupe_slot(int *dk, int key, int nslots)
{
    volatile int *vk = dk;
    // the top log2(nslots) bits of a multiplicative hash (nslots a power of two)
    unsigned s = ((unsigned)key * 0x9E3779B1u) >> (33 - __ffs(nslots));
    s &= (unsigned)(nslots - 1);
    for (int probe = 0; probe < 64; probe++) {
        const int k = vk[s];
        if (k == key) return (int)s;
        if (k == -1) {
            const int old = atomicCAS(dk + s, -1, key);
            if (old == -1 || old == key) return (int)s;
        }
        s = (s + 1) & (unsigned)(nslots - 1);
    }
    return -1;
}

template <typename T, int CONN, bool TMA>
__global__ void __launch_bounds__(TT<CONN>::NT) k_label(const __grid_constant__ CUtensorMap tmp,
                                                        const __grid_constant__ CUtensorMap tmg, const Batch b,
                                                        int32_t *par, int32_t *mi, int do_rag, const EdgeSink L,
                                                        DevStatus *status)
{
    using C = TC<CONN>;
    using B = LabelBox<T, CONN>;
    constexpr bool HASHED = !kPlateauList<CONN>;   // 2D: the edge list; 26-connectivity: the region table
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    unsigned long long *hk = (unsigned long long *)smem;   // edge hash (after the root phase)
    unsigned *hv = (unsigned *)(hk + C::HASH);
    int *dk = (int *)smem;                                  // distinct path ends (root phase)
    int *dr = dk + B::DSLOTS;                               // their roots
    int *pb = (int *)(smem + B::OFF_P);
    T *gb = (T *)(smem + B::OFF_G);
    const int tid = threadIdx.x, lane = tid & 31;
    const TileCtx tc = tile_ctx<CONN>(b, blockIdx.x);   // TMA: a single image (b.one)
    const Geo &geo = tc.geo;
    const T *g = (const T *)tc.grad;
    const int x0 = tc.x0, y0 = tc.y0, z0 = tc.z0, base = tc.base;
    if (TMA) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
            mbar_arrive_expect_tx(&bar, B::PBYTES + (do_rag ? B::GBYTES : 0));
            tma_load_3d(pb, &tmp, x0 - B::AP, y0 - C::BYL, z0, &bar);
            if (do_rag) tma_load_3d(gb, &tmg, x0 - B::AG, y0 - C::BYL, z0, &bar);
        }
    }
    for (int i = tid; i < B::DSLOTS; i += C::NT) dk[i] = -1;
    // Roots of the tile and of its forward halo.  Many pixels of a tile share
    // the end of their in-tile path (parallel paths leave the tile through the
    // same face pixels), so the ends are first deduplicated in shared memory,
    // each distinct end is chased to its root once (in lock step, LPD chases
    // in flight per thread), and the pixels take the root of their end.
    {
        // box entries: -1 outside the image, -2 - slot for a deduplicated end,
        // the end itself (>= 0) when the table had no room (chased directly)
        constexpr int LPB = (C::BS + C::NT - 1) / C::NT;
        constexpr int LPD = B::DSLOTS / C::NT;
        __syncthreads();  // the dedupe table is cleared (and the barrier initialised)
        if (TMA) {
            const bool ok = mbar_wait(&bar, 0, status);
            if (__syncthreads_or(!ok)) return;
        }
#pragma unroll 4
        for (int k = 0; k < LPB; k++) {
            const int i = tid + k * C::NT;
            if (i >= C::BS) break;
            const int bx = i % C::BX, by = (i / C::BX) % C::BY, bz = i / (C::BX * C::BY);
            const int x = x0 - C::BXL + bx, y = y0 - C::BYL + by, z = z0 + bz;
            const int pos = (bz * C::BY + by) * B::RWP + bx + B::AP - C::BXL;
            int r = -1;
            if (x >= 0 && x < geo.W && y >= 0 && y < geo.H && z < geo.D) {
                if (TMA) {
                    r = pb[pos];
                } else {
                    const int q = (z * geo.H + y) * geo.W + x;
                    r = par[base + q];
                    if (do_rag) gb[(bz * C::BY + by) * B::RWG + bx + B::AG - C::BXL] = g[q];
                }
                const int sl = dedupe_slot(dk, r, B::DSLOTS);
                if (sl >= 0) r = -2 - sl;
            }
            pb[pos] = r;
        }
        __syncthreads();
        // chase the distinct ends to their roots, LPD chases in flight per thread
        {
            int e[LPD];
            unsigned live = 0;
#pragma unroll
            for (int m = 0; m < LPD; m++) {
                e[m] = dk[tid + m * C::NT];
                live |= (e[m] >= 0 ? 1u : 0u) << m;
            }
            for (int hop = 0; live && hop < (1 << 22); hop++) {
                int u[LPD];
#pragma unroll
                for (int m = 0; m < LPD; m++) u[m] = (live >> m) & 1u ? par[e[m]] : e[m];
#pragma unroll
                for (int m = 0; m < LPD; m++) {
                    if (u[m] == e[m]) live &= ~(1u << m);
                    e[m] = u[m];
                }
            }
            if (live) record_error(status, DEV_NONCONVERGED, 9);
#pragma unroll
            for (int m = 0; m < LPD; m++) dr[tid + m * C::NT] = e[m];
        }
        __syncthreads();
        // every box entry takes its root
#pragma unroll 4
        for (int k = 0; k < LPB; k++) {
            const int i = tid + k * C::NT;
            if (i >= C::BS) break;
            const int bx = i % C::BX, by = (i / C::BX) % C::BY, bz = i / (C::BX * C::BY);
            const int pos = (bz * C::BY + by) * B::RWP + bx + B::AP - C::BXL;
            int r = pb[pos];
            if (r < -1) {
                r = dr[-2 - r];
            } else if (r >= 0) {  // crowded table: chase this end alone
                int guard = 0;
                for (int u = par[r]; u != r && guard < (1 << 22); u = par[r], guard++) r = u;
                if (guard >= (1 << 22)) record_error(status, DEV_NONCONVERGED, 9);
            }
            pb[pos] = r;
        }
    }
    __syncthreads();   // the dedupe table is dead: region R becomes the edge hash
    if (do_rag)
        for (int i = tid; i < C::HASH; i += C::NT) {
            hk[i] = EMPTY_KEY;
            hv[i] = 0xffffffffu;
        }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < C::PER; k++) {
        const int i = tid + k * C::NT;
        const int lx = i % C::TX, ly = (i / C::TX) % C::TY, lz = i / (C::TX * C::TY);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        const bool in = x < geo.W && y < geo.H && z < geo.D;
        const int bp = (lz * C::BY + ly + C::BYL) * B::RWP + lx + B::AP;
        const int bg = (lz * C::BY + ly + C::BYL) * B::RWG + lx + B::AG;
        const int r = in ? pb[bp] : -1;
        const int p = in ? base + (z * geo.H + y) * geo.W + x : 0;
        if (in) par[p] = r;
        // smallest pixel index of each basin: lanes are consecutive x of one
        // row, so the first lane of every run of equal roots holds the run's
        // smallest index (a basin met in several runs takes several atomics)
        const int rprev = __shfl_up_sync(0xffffffffu, r, 1);
        if (in && (lane == 0 || rprev != r)) atomicMin(mi + r, p);
        if (!do_rag || !in) continue;
        const unsigned gp = gb[bg];
        // neighbours in the same other basin follow each other: merge each run
        // of equal roots in registers (lowest height) and insert once per run
        int rl = -1;
        unsigned hl = 0;
#pragma unroll
        for (int n = Half<CONN>::first; n < Nb<CONN>::n; n++) {
            const int dn = Nb<CONN>::dz(n) * C::BY + Nb<CONN>::dy(n);
            const int xx = x + Nb<CONN>::dx(n), yy = y + Nb<CONN>::dy(n), zz = z + Nb<CONN>::dz(n);
            if (xx < 0 || xx >= geo.W || yy < 0 || yy >= geo.H || zz >= geo.D) continue;
            const int rq = pb[bp + dn * B::RWP + Nb<CONN>::dx(n)];
            if (rq == r) continue;
            const unsigned gq = gb[bg + dn * B::RWG + Nb<CONN>::dx(n)];
            const unsigned h = gp > gq ? gp : gq;
            if (rq == rl) {
                hl = h < hl ? h : hl;
                continue;
            }
            if (rl >= 0)
                smem_edge_insert<HASHED>((unsigned)(r < rl ? r : rl), (unsigned)(r < rl ? rl : r), hl, hk, hv,
                                         C::HASH, L, status);
            rl = rq;
            hl = h;
        }
        if (rl >= 0)
            smem_edge_insert<HASHED>((unsigned)(r < rl ? r : rl), (unsigned)(r < rl ? rl : r), hl, hk, hv, C::HASH, L,
                                     status);
    }
    if (!do_rag) return;
    __syncthreads();
    static_assert(C::HASH % C::NT == 0, "warp-uniform flush");
    if (HASHED) {
        for (int i0 = 0; i0 < C::HASH; i0 += C::NT) {
            const int i = i0 + tid;
            const unsigned long long k = hk[i];
            sink_put_warp<true>(L, k != EMPTY_KEY, (unsigned)(k >> 32), (unsigned)k, hv[i], status);
        }
        return;
    }
    // the list: the tile's pairs take one span of it (one global atomic per
    // tile; each warp's entries are placed by a shared atomic per pass)
    constexpr int NP = C::HASH / C::NT;
    __shared__ int s_n, s_base;
    if (tid == 0) s_n = 0;
    __syncthreads();
    int off[NP];
    unsigned msk[NP];
#pragma unroll
    for (int u = 0; u < NP; u++) {
        msk[u] = __ballot_sync(0xffffffffu, hk[u * C::NT + tid] != EMPTY_KEY);
        int o = 0;
        if (lane == 0 && msk[u]) o = atomicAdd(&s_n, __popc(msk[u]));
        off[u] = __shfl_sync(0xffffffffu, o, 0) + __popc(msk[u] & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (tid == 0) s_base = s_n ? atomicAdd(L.n, s_n) : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NP; u++) {
        if (!((msk[u] >> lane) & 1u)) continue;
        const int i = u * C::NT + tid;
        const unsigned long long k = hk[i];
        list_put(L, s_base + off[u], (unsigned)(k >> 32), (unsigned)k, hv[i], status);
    }
}

// ---------------------------------------------------------------------------
// k_chase, k_rag6: roots and region adjacency of the 3D path
// ---------------------------------------------------------------------------

// Global tile of pixel g (3D tiling of its image).
__device__ __forceinline__ int tile_of_pixel(const Batch &b, int g)
{
    const ImgDesc d = img_desc(b, img_of_pixel(b, g));
    const int q = g - d.base;
    const int z = q / d.HW, r = q - z * d.HW, y = r / d.W, x = r - y * d.W;
    return d.tile0 + ((z / TT<6>::TZ) * d.nty + y / TT<6>::TY) * d.ntx + x / TT<6>::TX;
}

// Root of every listed in-tile path end, in place.  ends[j] = (e, q): e the
// end pixel, q the next pixel of its path (in a neighbouring tile, or given
// by step II / IV on a plateau tile), or q == e for a root.  q's own in-tile
// end is the entry first-of-q's-tile + code[q]; repeat until a root, then
// ends[j] = (root, root).  An entry read while another thread rewrites it
// holds pixels of the same path in either field, so every walk ends at the
// same root.
static __global__ void __launch_bounds__(NTHR) k_chase(const Batch b, int2 *ends, const int2 *__restrict__ tends,
                                                       const uint16_t *__restrict__ code, const int32_t *counters,
                                                       DevStatus *status)
{
    const int n = counters[CNT_ENDS];
    const int npix = b.npix;
    for (int j = blockIdx.x * NTHR + threadIdx.x; j < n; j += gridDim.x * NTHR) {
        const int2 c0 = ends[j];
        int e = c0.x, q = c0.y;
        bool ok = (unsigned)e < (unsigned)npix;
        for (int hop = 0; ok && q != e; hop++) {
            if ((unsigned)q >= (unsigned)npix || hop >= (1 << 22)) {
                ok = false;
                break;
            }
            const int2 te = __ldg(tends + tile_of_pixel(b, q));
            const int s = __ldg(code + q) & (TC<6>::NPIX - 1);
            if (s >= te.y) {
                ok = false;
                break;
            }
            const int2 c = ends[te.x + s];
            e = c.x;
            q = c.y;
            if ((unsigned)e >= (unsigned)npix) ok = false;
        }
        if (!ok) {  // only after an earlier device error
            record_error(status, DEV_NONCONVERGED, 12);
            ends[j] = make_int2(0, 0);
            continue;
        }
        if (e != c0.x || q != c0.y) ends[j] = make_int2(e, e);
    }
}

// Shared-memory layout of k_rag6: the roots (then basin ids) of the +x, +y,
// +z face pixels of the neighbouring tiles, the tile's basin list and its
// hash, the smallest index per basin; one region that holds first the basin
// id of every slot of the tile, then the basin-pair pass matrix (or the edge
// hash of a crowded tile); the packed ids of every column; then the
// slot-code box (later the warps' lists of boundary pixels) and the gradient
// box of the tile and its forward faces (x from x0, rows padded to 16-byte
// multiples).  74,752 bytes for uint16 (three CTAs per SM).
template <typename T> struct Rag6Box {
    using C = TC<6>;
    static constexpr int BY = C::TY + 1, BZ = C::TZ + 1;
    static constexpr int CW = C::TX + 8;                                  // uint16 code row: x0 .. x0 + 39
    static constexpr int GW = sizeof(T) == 1 ? C::TX + 16 : C::TX + 8;    // gradient row
    static constexpr int CBYTES = CW * BY * BZ * 2;
    static constexpr int GBYTES = GW * BY * BZ * (int)sizeof(T);
    static constexpr int HX = C::TY * C::TZ, HY = C::TX * C::TZ, HZ = C::TX * C::TY, NH = HX + HY + HZ;
    static constexpr int RB = 253;        // basins a tile can number (ids 0..RB-1)
    static constexpr int RH = 512;        // basin hash slots
    static constexpr int RM = 64;         // basins of the pass matrix
    static constexpr int PMN = 2048;      // pass matrix entries: pairs a < c of RM ids (2016), padded
    static constexpr int EH = 512;        // edge hash slots (tiles with more than RM basins)
    static constexpr int WL = C::TX * C::TZ;                  // boundary items per warp (every pixel)
    static constexpr int WLBYTES = (C::NT / 32) * WL * 2;
    static constexpr int OFF_HR = 0;                          // int32 [NH]
    static constexpr int OFF_RL = OFF_HR + NH * 4;            // int32 [256]
    static constexpr int OFF_RHK = OFF_RL + 256 * 4;          // int32 [RH]
    static constexpr int OFF_RHV = OFF_RHK + RH * 4;          // int32 [RH]
    static constexpr int OFF_RMIN = OFF_RHV + RH * 4;         // int32 [256]
    // uint8 [NPIX] slot ids, then uint32 [PMN] pass matrix or (uint64 [EH], uint32 [EH]) edge hash
    static constexpr int OFF_U = OFF_RMIN + 256 * 4;
    static constexpr int UBYTES = C::NPIX > PMN * 4 ? (C::NPIX > EH * 12 ? C::NPIX : EH * 12)
                                                    : (PMN * 4 > EH * 12 ? PMN * 4 : EH * 12);
    static constexpr int OFF_COL = OFF_U + UBYTES;            // uint4 [NT]: packed basin ids of each column
    static constexpr int OFF_XF = OFF_COL + C::NT * 16;       // uint8 [TY][TZ]: ids of the +x face
    static constexpr int OFF_YF = OFF_XF + C::TY * C::TZ;     // uint8 [TX][TZ]: ids of the +y face
    static constexpr int OFF_C = (OFF_YF + C::TX * C::TZ + 127) & ~127;   // code box, then uint16 [NT / 32][WL]
    static constexpr int OFF_G = OFF_C + (((CBYTES > WLBYTES ? CBYTES : WLBYTES) + 127) & ~127);
    static constexpr int SMEM = OFF_G + ((GBYTES + 127) & ~127);
    static_assert(OFF_U % 8 == 0, "edge keys are 8-byte words");
    static_assert(RM * (RM - 1) / 2 <= PMN && PMN % C::NT == 0 && EH % C::NT == 0, "warp-uniform flush");
};

// Bit 7 of byte k set where byte k of a and b differ (no carry crosses a
// byte: the low seven bits of each byte plus 0x7f stay inside it).
__device__ __forceinline__ unsigned ne4(unsigned a, unsigned b)
{
    const unsigned x = a ^ b;
    return (((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
}

// Entry of the pass matrix for basin ids a < c.
__device__ __forceinline__ int pm_index(int a, int c) { return (c * (c - 1) >> 1) + a; }

// root of slot c of a neighbouring tile whose span of the end list is e,
// -1 if invalid
__device__ __forceinline__ int face_root(bool valid, int c, int2 e, const int2 *ends, DevStatus *status)
{
    if (!valid) return -1;
    if (c >= e.y) {  // only after an earlier device error
        record_error(status, DEV_NONCONVERGED, 13);
        return -1;
    }
    return __ldg(&ends[e.x + c].x);
}

// Per 3D tile, one z column per thread: the smallest pixel index per basin,
// and with do_rag Alg. 5 step V on the
// +x, +y, +z pixel pairs: the pass value max(G(p), G(q)) of every pair of
// different basins, min-reduced per pair.
//   - The tile's basins (of its slots and of the forward faces) get 8-bit
//     ids through a shared hash.  A thread packs its column's ids four to a
//     register; the +z, +x (next lane) and +y (next warp, through shared
//     memory) comparisons, and the -x, -y, -z ones for the smallest index,
//     run four pixels per byte-SIMD instruction, and only the few pixels
//     they flag are visited one by one.
//   - With at most RM basins a pair's pass value goes straight into a
//     shared RM x RM matrix by atomic min; tiles with more basins use the
//     shared edge hash; tiles with more than RB basins take a per-pixel path
//     that compares roots read from the global end list.
//   - Smallest index: only a pixel with no pixel of its basin at -x, -y or
//     -z inside the tile can hold the tile's smallest index of that basin;
//     those candidates take a shared atomic min per basin id.
template <typename T, bool TMA>
__global__ void __launch_bounds__(TT<6>::NT, 3) k_rag6(const __grid_constant__ CUtensorMap tmc,
                                                       const __grid_constant__ CUtensorMap tmg, const Batch b,
                                                       const uint16_t *__restrict__ code,
                                                       const int2 *__restrict__ ends,
                                                       const int2 *__restrict__ tends, int32_t *mi,
                                                       int do_rag, const EdgeSink L, DevStatus *status)
{
    using C = TC<6>;
    using B = Rag6Box<T>;
    static_assert(C::NT == C::TX * C::TY && C::TX == 32 && C::TY == 16 && C::TZ == 16, "column layout");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int s_nr, s_full;
    int *hr = (int *)(smem + B::OFF_HR);
    int *hxr = hr, *hyr = hr + B::HX, *hzr = hyr + B::HY;
    uint8_t *ss = smem + B::OFF_U;
    int *rl = (int *)(smem + B::OFF_RL);
    int *rhk = (int *)(smem + B::OFF_RHK);
    int *rhv = (int *)(smem + B::OFF_RHV);
    int *rmin = (int *)(smem + B::OFF_RMIN);
    unsigned *pm = (unsigned *)(smem + B::OFF_U);
    uint4 *colw = (uint4 *)(smem + B::OFF_COL);
    uint8_t *xfb = smem + B::OFF_XF, *yfb = smem + B::OFF_YF;
    unsigned long long *hk = (unsigned long long *)(smem + B::OFF_U);
    unsigned *hv = (unsigned *)(smem + B::OFF_U + B::EH * 8);
    uint16_t *cb = (uint16_t *)(smem + B::OFF_C);
    T *gb = (T *)(smem + B::OFF_G);
    const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
    const int t = blockIdx.x;
    const TileCtx tc = tile_ctx<6>(b, t);
    const Geo &geo = tc.geo;
    const int x0 = tc.x0, y0 = tc.y0, z0 = tc.z0, base = tc.base;
    constexpr int SZ = B::BY * B::CW, GZ = B::BY * B::GW;
    if (TMA && tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&bar, B::CBYTES + (do_rag ? B::GBYTES : 0));
        tma_load_3d(cb, &tmc, x0, y0, z0, &bar);
        if (do_rag) tma_load_3d(gb, &tmg, x0, y0, z0, &bar);
    }
    const int2 te = __ldg(tends + t);
    const int ntx = tc.tg.ntx, nty = tc.tg.nty;
    for (int i = tid; i < B::RH; i += C::NT) rhk[i] = -1;
    if (tid < 256) rmin[tid] = 0x7fffffff;
    if (tid == 0) {
        s_nr = 0;
        s_full = 0;
    }
    if (!TMA) {
        const T *g = (const T *)tc.grad;
        for (int i = tid; i < B::CW * B::BY * B::BZ; i += C::NT) {
            const int bx = i % B::CW, by = (i / B::CW) % B::BY, bz = i / (B::CW * B::BY);
            const int xx = x0 + bx, yy = y0 + by, zz = z0 + bz;
            const bool in = xx < geo.W && yy < geo.H && zz < geo.D;
            const int q = (zz * geo.H + yy) * geo.W + xx;
            cb[i] = in ? code[base + q] : (uint16_t)0;
            if (do_rag && bx < B::GW) gb[(bz * B::BY + by) * B::GW + bx] = in ? g[q] : (T)0;
        }
        constexpr int XW = B::GW > B::CW ? B::GW - B::CW : 1;   // gradient columns beyond the code box
        if (do_rag && B::GW > B::CW)
            for (int i = tid; i < XW * B::BY * B::BZ; i += C::NT) {
                const int bx = B::CW + i % XW, by = (i / XW) % B::BY, bz = i / (XW * B::BY);
                const int xx = x0 + bx, yy = y0 + by, zz = z0 + bz;
                const bool in = xx < geo.W && yy < geo.H && zz < geo.D;
                gb[(bz * B::BY + by) * B::GW + bx] = in ? g[(zz * geo.H + yy) * geo.W + xx] : (T)0;
            }
    }
    __syncthreads();   // tables cleared (and the barrier initialised)

    const int x = x0 + lane, y = y0 + ly;
    const bool col_in = x < geo.W && y < geo.H;
    // number the tile's basins: its slots' roots and its forward faces' roots
    auto rh_insert = [&](int r) {
        if (r < 0) return;
        volatile int *vk = rhk;
        unsigned h = ((unsigned)r * 0x9E3779B1u) >> 23;   // 9 bits: RH == 512
        for (int probe = 0; probe < B::RH; probe++) {
            int k = vk[h];
            if (k == -1) {
                k = atomicCAS(rhk + h, -1, r);
                if (k == -1) return;
            }
            if (k == r) return;
            h = (h + 1) & (B::RH - 1);
        }
        s_full = 1;   // more than RH basins
    };
    auto rh_find = [&](int r) -> int {
        if (r < 0) return 0xff;
        unsigned h = ((unsigned)r * 0x9E3779B1u) >> 23;
        for (int probe = 0; probe < B::RH; probe++) {
            const int k = rhk[h];
            if (k == r) return rhv[h];
            if (k == -1) break;
            h = (h + 1) & (B::RH - 1);
        }
        return B::RB;   // not numbered
    };
    // Neither the roots of this tile's slots nor those of its forward face
    // pixels need the boxes: their codes are read from global memory, so all
    // of it goes before the wait.  The thread's first slot root stays in a
    // register for the ids below.
    const bool hasx = x0 + C::TX < geo.W, hasy = y0 + C::TY < geo.H, hasz = z0 + C::TZ < geo.D;
    const int rown = tid < te.y ? __ldg(&ends[te.x + tid].x) : -1;
    int fzr = -1, fyr = -1, fxr = -1;   // roots of the face pixels (lane, ly, TZ), (lane, TY, ly), (TX, fy, fz)
    if (do_rag) {
        const int fy = tid % C::TY, fz = tid / C::TY;
        const bool vz = col_in && hasz, vy = x < geo.W && hasy && z0 + ly < geo.D;
        const bool vx = tid < B::HX && hasx && y0 + fy < geo.H && z0 + fz < geo.D;
        const int2 tez = vz ? __ldg(tends + t + ntx * nty) : make_int2(0, 0);
        const int2 tey = vy ? __ldg(tends + t + ntx) : make_int2(0, 0);
        const int2 tex = vx ? __ldg(tends + t + 1) : make_int2(0, 0);
        constexpr int CM = C::NPIX - 1;   // slot bits of a code
        const int cz = vz ? __ldg(code + base + ((z0 + C::TZ) * geo.H + y) * geo.W + x) & CM : 0;
        const int cy = vy ? __ldg(code + base + ((z0 + ly) * geo.H + y0 + C::TY) * geo.W + x) & CM : 0;
        const int cx = vx ? __ldg(code + base + ((z0 + fz) * geo.H + y0 + fy) * geo.W + x0 + C::TX) & CM : 0;
        fzr = face_root(vz, cz, tez, ends, status);
        fyr = face_root(vy, cy, tey, ends, status);
        fxr = face_root(vx, cx, tex, ends, status);
    }
    rh_insert(rown);
    for (int i = tid + C::NT; i < te.y; i += C::NT) rh_insert(__ldg(&ends[te.x + i].x));
    rh_insert(fzr);
    rh_insert(fyr);
    rh_insert(fxr);
    if (TMA) {
        const bool ok = mbar_wait(&bar, 0, status);
        if (__syncthreads_or(!ok)) return;
    } else {
        __syncthreads();
    }
    for (int i = tid; i < B::RH; i += C::NT)
        if (rhk[i] >= 0) {
            const int id = atomicAdd(&s_nr, 1);
            rhv[i] = id < B::RB ? id : B::RB;
            if (id < B::RB) rl[id] = rhk[i];
        }
    __syncthreads();
    const int nr = s_nr;
    const int mode = (s_full || nr > B::RB) ? 2 : (nr > B::RM ? 1 : 0);   // uniform in the CTA
    // the pass matrix or the edge hash shares its words with the slot ids:
    // cleared once those are read (modes 0, 1) or right away (mode 2, which
    // numbers no slots)
    auto clear_pairs = [&]() {
        if (mode == 0)
            for (int i = tid; i < B::PMN; i += C::NT) pm[i] = 0xffffffffu;
        else
            for (int i = tid; i < B::EH; i += C::NT) {
                hk[i] = EMPTY_KEY;
                hv[i] = 0xffffffffu;
            }
    };
    if (do_rag && mode == 2) clear_pairs();
    const int first = te.x;

    auto edge = [&](int ida, int idb, unsigned h) {   // ids (mode 0, 1) or roots (mode 2)
        if (mode == 0) {
            const int a = ida < idb ? ida : idb, c2 = ida < idb ? idb : ida;
            atomicMin(pm + pm_index(a, c2), h);
        } else {
            const int ra = mode < 2 ? rl[ida] : ida, rb = mode < 2 ? rl[idb] : idb;
            smem_edge_insert<true>((unsigned)(ra < rb ? ra : rb), (unsigned)(ra < rb ? rb : ra), h, hk, hv, B::EH, L,
                             status);
        }
    };
    const int p0 = base + (z0 * geo.H + y) * geo.W + x;   // global index of (lane, ly, z = 0)
    const int nz = geo.D - z0 < C::TZ ? geo.D - z0 : C::TZ;

    if (do_rag) {   // the face roots (mode 2 compares roots)
        hzr[tid] = fzr;
        hyr[tid] = fyr;
        if (tid < B::HX) hxr[tid] = fxr;
    }
    if (mode < 2) {
        if (tid < te.y) ss[tid] = (uint8_t)rh_find(rown);
        for (int i = tid + C::NT; i < te.y; i += C::NT) ss[i] = (uint8_t)rh_find(__ldg(&ends[te.x + i].x));
        if (do_rag) {   // ids of the forward faces
            const int iz = rh_find(hzr[tid]);
            hzr[tid] = iz;
            yfb[lane * C::TZ + ly] = (uint8_t)rh_find(hyr[tid]);
            if (tid < B::HX) xfb[(tid % C::TY) * C::TZ + tid / C::TY] = (uint8_t)rh_find(hxr[tid]);
        }
        __syncthreads();
        // this column's ids, four to a register (byte k & 3 of word k >> 2;
        // 0xff outside the image)
        unsigned P[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
            unsigned v = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int k = 4 * w + q;
                const unsigned id = (col_in && k < nz) ? (unsigned)ss[cb[ly * B::CW + lane + k * SZ] & (C::NPIX - 1)]
                                                       : 0xffu;
                v |= id << (8 * q);
            }
            P[w] = v;
        }
        colw[tid] = make_uint4(P[0], P[1], P[2], P[3]);
        const unsigned P4 = do_rag ? ((unsigned)hzr[tid] & 0xffu) : 0xffu;   // +z face pixel
        __syncthreads();   // slot ids read; the code box is read no more
        if (do_rag) clear_pairs();
        // smallest index: candidates differ from their -z, -y, -x neighbours
        {
            const uint4 ym = ly > 0 ? colw[tid - 32] : make_uint4(~0u, ~0u, ~0u, ~0u);
            const unsigned YM[4] = {ym.x, ym.y, ym.z, ym.w};
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const unsigned zm = __funnelshift_l(w > 0 ? P[w - 1] : ~0u, P[w], 8);   // bytes k - 1
                unsigned xm = __shfl_up_sync(0xffffffffu, P[w], 1);
                if (lane == 0) xm = ~0u;
                unsigned cand = ne4(P[w], zm) & ne4(P[w], YM[w]) & ne4(P[w], xm) & ne4(P[w], 0xffffffffu);
                while (cand) {
                    const int q = (__ffs(cand) - 1) >> 3;
                    cand &= ~(0xffu << (8 * q));
                    const int k = 4 * w + q;
                    atomicMin(rmin + ((P[w] >> (8 * q)) & 0xffu), p0 + k * geo.HW);
                }
            }
        }
        if (do_rag) {
            __syncthreads();   // pass matrix / edge hash cleared
            // pass values of the +x, +y, +z pairs of different basins
            const unsigned *ynw = ly + 1 < C::TY ? (const unsigned *)(colw + tid + 32) : (const unsigned *)yfb + 4 * lane;
            const unsigned *xfw = (const unsigned *)xfb + 4 * ly;
            const uint8_t *colb = (const uint8_t *)colw;   // byte k of column c: colb[c * 16 + k]
            uint16_t *wlst = (uint16_t *)(smem + B::OFF_C) + ly * B::WL;   // the code box is read no more
            auto pass = [&](auto matrix) {
                constexpr bool MATRIX = decltype(matrix)::value;
                auto note = [&](int ida, int idb, unsigned h) {
                    const int a = ida < idb ? ida : idb, c2 = ida < idb ? idb : ida;
                    if (MATRIX) {
                        unsigned *e = pm + pm_index(a, c2);
                        if (h < *e) atomicMin(e, h);
                    } else {
                        const int ra = rl[a], rb = rl[c2];
                        smem_edge_insert<true>((unsigned)(ra < rb ? ra : rb), (unsigned)(ra < rb ? rb : ra), h, hk, hv,
                                         B::EH, L, status);
                    }
                };
                // 0x00 / 0xff bytes -> bits 0..3
                auto bits = [](unsigned m) { return ((((m >> 7) & 0x01010101u) * 0x01020408u) >> 24) & 0xfu; };
                // flag the column's pixels with a boundary in +x, +y or +z (bit k)
                unsigned fx = 0, fy = 0, fz = 0;
#pragma unroll
                for (int w = 0; w < 4; w++) {
                    const unsigned zn = __funnelshift_r(P[w], w < 3 ? P[w + 1] : P4, 8);   // bytes k + 1
                    unsigned xn = __shfl_down_sync(0xffffffffu, P[w], 1);
                    if (lane == 31) xn = xfw[w];
                    const unsigned yn = ynw[w];
                    const unsigned own = ne4(P[w], 0xffffffffu);
                    fz |= bits(ne4(P[w], zn) & own & ne4(zn, 0xffffffffu)) << (4 * w);
                    fy |= bits(ne4(P[w], yn) & own & ne4(yn, 0xffffffffu)) << (4 * w);
                    fx |= bits(ne4(P[w], xn) & own & ne4(xn, 0xffffffffu)) << (4 * w);
                }
                // compact them into the warp's list: (directions, k, lane)
                unsigned fa = fx | fy | fz;
                const int cnt = __popc(fa);
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += v;
                }
                const int total = __shfl_sync(0xffffffffu, inc, 31);
                int pos = inc - cnt;
                while (fa) {
                    const int k = __ffs(fa) - 1;
                    fa &= fa - 1;
                    const unsigned d = ((fx >> k) & 1u) | (((fy >> k) & 1u) << 1) | (((fz >> k) & 1u) << 2);
                    wlst[pos++] = (uint16_t)((d << 9) | (k << 5) | lane);
                }
                __syncwarp();
                // pass values of the listed pairs, every lane busy
                for (int e = lane; e < total; e += 32) {
                    const int it = wlst[e];
                    const int ls = it & 31, k = (it >> 5) & 15, d = it >> 9;
                    const int ts = ly * 32 + ls;
                    const int id = colb[ts * 16 + k];
                    const int gpos = (k * B::BY + ly) * B::GW + ls;
                    const unsigned gp = gb[gpos];
                    if (d & 1) {
                        const int nid = ls < 31 ? colb[(ts + 1) * 16 + k] : xfb[ly * C::TZ + k];
                        const unsigned gq = gb[gpos + 1];
                        note(id, nid, gp > gq ? gp : gq);
                    }
                    if (d & 2) {
                        const int nid = ly + 1 < C::TY ? colb[(ts + 32) * 16 + k] : yfb[ls * C::TZ + k];
                        const unsigned gq = gb[gpos + B::GW];
                        note(id, nid, gp > gq ? gp : gq);
                    }
                    if (d & 4) {
                        const int nid = k + 1 < C::TZ ? colb[ts * 16 + k + 1] : (hzr[ts] & 0xff);
                        const unsigned gq = gb[gpos + GZ];
                        note(id, nid, gp > gq ? gp : gq);
                    }
                }
            };
            if (mode == 0)
                pass(std::true_type{});
            else
                pass(std::false_type{});
        }
    } else {
        __syncthreads();   // edge hash cleared
        // more than RB basins in the tile: per-pixel loop over roots read from
        // the global end list
        auto root_at = [&](bool valid, int c) -> int {
            return valid ? __ldg(&ends[first + (c & (C::NPIX - 1))].x) : -1;
        };
        const bool vy = y + 1 < geo.H;
        int pid = -1;
        const int pcol = ly * B::CW + lane, gcol = ly * B::GW + lane;
        int iz = root_at(col_in && nz > 0, cb[pcol]);
#pragma unroll 1
        for (int k = 0; k < nz; k++) {   // trip count uniform in the CTA
            const int pos = pcol + k * SZ, p = p0 + k * geo.HW;
            const int id = iz;
            if (k + 1 < C::TZ) iz = root_at(col_in && k + 1 < nz, cb[pos + SZ]);
            else iz = do_rag ? hzr[tid] : -1;
            const int ixm = __shfl_up_sync(0xffffffffu, id, 1);
            const int iym = ly > 0 ? root_at(col_in, cb[pos - B::CW]) : -1;
            if (id >= 0 && id != pid && id != iym && (lane == 0 || id != ixm)) atomicMin(mi + id, p);
            pid = id;
            if (!do_rag) continue;
            int ix = __shfl_down_sync(0xffffffffu, id, 1);
            if (lane == 31) ix = hxr[ly + C::TY * k];
            const int iy = ly + 1 < C::TY ? root_at(vy, cb[pos + B::CW]) : hyr[lane + C::TX * k];
            if (id < 0) continue;
            const int gpos = gcol + k * GZ;
            const unsigned gp = gb[gpos];
            if (ix >= 0 && ix != id) {
                const unsigned gq = gb[gpos + 1];
                edge(id, ix, gp > gq ? gp : gq);
            }
            if (iy >= 0 && iy != id) {
                const unsigned gq = gb[gpos + B::GW];
                edge(id, iy, gp > gq ? gp : gq);
            }
            if (iz >= 0 && iz != id) {
                const unsigned gq = gb[gpos + GZ];
                edge(id, iz, gp > gq ? gp : gq);
            }
        }
    }
    __syncthreads();
    if (mode < 2 && tid < nr && tid < B::RB && rmin[tid] != 0x7fffffff) atomicMin(mi + rl[tid], rmin[tid]);
    if (!do_rag) return;
    if (mode == 0) {
        for (int e = tid; e < B::PMN; e += C::NT) {
            const unsigned h = pm[e];
            const bool have = h != 0xffffffffu;
            unsigned lo = 0, hi = 0;
            if (have) {   // the basin list is read for the few pairs present only
                // the ids (a, c) of entry e = c (c - 1) / 2 + a, a < c
                int c = (int)((1.0f + __fsqrt_rn(1.0f + 8.0f * (float)e)) * 0.5f);
                while (pm_index(0, c) > e) c--;
                while (pm_index(0, c + 1) <= e) c++;
                const int ra = rl[e - pm_index(0, c)], rb = rl[c];
                lo = (unsigned)(ra < rb ? ra : rb);
                hi = (unsigned)(ra < rb ? rb : ra);
            }
            sink_put_warp<true>(L, have, lo, hi, h, status);
        }
    } else {
        for (int i = tid; i < B::EH; i += C::NT) {
            const unsigned long long k = hk[i];
            sink_put_warp<true>(L, k != EMPTY_KEY, (unsigned)(k >> 32), (unsigned)k, hv[i], status);
        }
    }
}

// ---------------------------------------------------------------------------
// canonical ids by rank of each basin's smallest pixel index
// ---------------------------------------------------------------------------

static __global__ void __launch_bounds__(NTHR) k_rank_mark(int N, const int32_t *__restrict__ roots,
                                                           const int32_t *counters, const int32_t *__restrict__ mi,
                                                           int32_t *__restrict__ rootm, unsigned *bitmap,
                                                           DevStatus *status)
{
    const int n = counters[CNT_ROOTS];
    for (int j = blockIdx.x * NTHR + threadIdx.x; j < n; j += gridDim.x * NTHR) {
        const int m = mi[roots[j]];
        if (m < 0 || m >= N) {  // only after an earlier device error
            rootm[j] = -1;
            record_error(status, DEV_NONCONVERGED, 10);
            continue;
        }
        rootm[j] = m;
        atomicOr(bitmap + (m >> 5), 1u << (m & 31));
    }
}

// popcount of each group of 32 bitmap words (1024 pixel indices) -> gcnt
static __global__ void __launch_bounds__(NTHR) k_rank_groups(const unsigned *__restrict__ bitmap, int nwords,
                                                             int32_t *__restrict__ gcnt, int ngroups)
{
    const int gi = blockIdx.x * (NTHR / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (gi >= ngroups) return;
    const int w = gi * 32 + lane;
    int c = w < nwords ? __popc(bitmap[w]) : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) gcnt[gi] = c;
}

// id[root] = number of basins whose smallest index is below this basin's
static __global__ void __launch_bounds__(NTHR) k_rank_assign(const int32_t *__restrict__ roots,
                                                             const int32_t *counters,
                                                             const int32_t *__restrict__ rootm,
                                                             const unsigned *__restrict__ bitmap,
                                                             const int32_t *__restrict__ gpre, int32_t *idmap)
{
    const int n = counters[CNT_ROOTS];
    for (int j = blockIdx.x * NTHR + threadIdx.x; j < n; j += gridDim.x * NTHR) {
        const int m = rootm[j];
        if (m < 0) {
            idmap[roots[j]] = -1;
            continue;
        }
        const int w = m >> 5, gi = w >> 5;
        int rank = gpre[gi];
        for (int u = gi * 32; u < w; u++) rank += __popc(bitmap[u]);
        rank += __popc(bitmap[w] & ((1u << (m & 31)) - 1u));
        idmap[roots[j]] = rank;
    }
}

static __global__ void __launch_bounds__(NTHR) k_rank_clear(const int32_t *counters, const int32_t *__restrict__ rootm,
                                                            unsigned *bitmap)
{
    const int n = counters[CNT_ROOTS];
    for (int j = blockIdx.x * NTHR + threadIdx.x; j < n; j += gridDim.x * NTHR)
        if (rootm[j] >= 0) bitmap[rootm[j] >> 5] = 0u;
}

// Canonical id of a root; ids outside [0, K0) can only come from an earlier
// device error and are written as -1 instead of being used as an index.
__device__ __forceinline__ int safe_id(const int32_t *__restrict__ idmap, int r, int K0)
{
    const int c = idmap[r];
    return (unsigned)c < (unsigned)K0 ? c : -1;
}

__device__ __forceinline__ int level_id(const int32_t *__restrict__ gm, int c) { return c >= 0 ? gm[c] : -1; }

// rbase[i] = number of basins (of the whole batch) whose smallest pixel index
// lies below image i's first pixel, i.e. the global id of image i's first
// basin; rbase[n] = total.  Image i's canonical ids are global ids - rbase[i].
static __global__ void __launch_bounds__(NTHR) k_rank_bases(const Batch b, const unsigned *__restrict__ bitmap,
                                                            const int32_t *__restrict__ gpre, const int32_t *counters,
                                                            int32_t *rbase)
{
    for (int i = blockIdx.x * NTHR + threadIdx.x; i <= b.n; i += gridDim.x * NTHR) {
        if (i == b.n) {
            rbase[i] = counters[CNT_ROOTS];
            continue;
        }
        const int m = img_desc(b, i).base;
        const int w = m >> 5, gi = w >> 5;
        int rank = gpre[gi];
        for (int u = gi * 32; u < w; u++) rank += __popc(bitmap[u]);
        rank += __popc(bitmap[w] & ((1u << (m & 31)) - 1u));
        rbase[i] = rank;
    }
}

// Batched level write: pixel g of the batch belongs to image i; its level-0
// id is its basin's global id minus rbase[i], its level-k id the global
// level-k id minus that of image i's first basin (regions never span images,
// and global ids are ordered image by image).
static __global__ void __launch_bounds__(NTHR) k_write_batch(const Batch b, const int32_t *__restrict__ par,
                                                             const int32_t *__restrict__ idmap,
                                                             const int32_t *__restrict__ gmap, size_t kstride, int NL,
                                                             const int32_t *__restrict__ rbase,
                                                             const int32_t *__restrict__ k0_ptr)
{
    const int K0 = *k0_ptr;
    int cur = -1, lo = 0, hi = -1;   // cached image of the previous pixel
    ImgDesc d{};
    int rb = 0;
    // each CTA writes one contiguous range of the batch's pixels, so that a
    // thread's next pixel is almost always in the image of its last one
    const int chunk = (int)(((long long)b.npix + gridDim.x - 1) / gridDim.x);
    const int g0 = blockIdx.x * chunk, g1 = (int)min((long long)b.npix, (long long)g0 + chunk);
    for (int g = g0 + threadIdx.x; g < g1; g += NTHR) {
        if (g < lo || g > hi) {
            cur = img_of_pixel(b, g);
            d = img_desc(b, cur);
            lo = d.base;
            hi = d.base + d.N - 1;
            rb = rbase[cur];
        }
        const int p = g - d.base;
        const int c = safe_id(idmap, par[g], K0);
        d.out[p] = c >= 0 ? c - rb : -1;
        for (int k = 1; k < NL; k++) {
            const int32_t *gm = gmap + (size_t)(k - 1) * kstride;
            d.out[(size_t)k * d.N + p] = c >= 0 ? gm[c] - gm[rb] : -1;
        }
    }
}


// 3D label write, one CTA per tile: every voxel's canonical id and its id on
// each waterfall level, from its 16-bit end slot and a per-tile table (slot
// -> root, after k_chase, in ends; root -> id through idmap; id -> level
// ids through gmap), one plane per level.  A tile with more slots than the
// table holds maps each voxel through the global arrays.  Batched calls:
// rbase holds each image's first basin id (single image: nullptr).
static constexpr int kWrite6Tab = 12288;   // level ids held in shared memory per tile

static __global__ void __launch_bounds__(TT<6>::NT, 3) k_write6(const Batch b, const uint16_t *__restrict__ code,
                                                             const int2 *__restrict__ ends,
                                                             const int2 *__restrict__ tends,
                                                             const int32_t *__restrict__ idmap,
                                                             const int32_t *__restrict__ gmap, size_t kstride,
                                                             int NL, const int32_t *__restrict__ rbase,
                                                             const int32_t *__restrict__ k0_ptr)
{
    using C = TC<6>;
    constexpr int GX = C::TX / 4;                  // groups of four x per row
    constexpr int G = C::NPIX / 4 / C::NT;         // groups per thread
    static_assert(C::NPIX % (4 * C::NT) == 0, "whole groups per thread");
    __shared__ int lv[kWrite6Tab];   // lv[k * n + slot]: id of the slot's basin on level k
    const int tid = threadIdx.x;
    const int t = blockIdx.x;
    const int ii = img_of_tile(b, t);
    const ImgDesc d = img_desc(b, ii);
    const TileCtx tc = tile_ctx<6>(b, t);
    const int2 te = tends[t];
    // the voxels' end slots first (their loads overlap the table build):
    // thread group g covers x = x0 + 4 (tid % GX) .. + 3 of row tid / GX + g * NT / GX
    const int gx = tc.x0 + 4 * (tid % GX);
    const bool vec = (d.W % 4 == 0) && (d.base % 4 == 0) && (((uintptr_t)d.out & 15) == 0);
    int q[G];
    uint2 cv[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int row = tid / GX + g * (C::NT / GX);   // (y, z) row of the tile
        const int y = tc.y0 + row % C::TY, z = tc.z0 + row / C::TY;
        q[g] = (y < d.H && z < d.D && gx < d.W) ? (z * d.H + y) * d.W + gx : -1;
        cv[g] = make_uint2(0, 0);
        if (q[g] >= 0) {
            if (vec) {
                cv[g] = __ldg(reinterpret_cast<const uint2 *>(code + d.base + q[g]));
            } else {
                unsigned c4[4] = {0, 0, 0, 0};
                for (int u = 0; u < 4; u++)
                    if (gx + u < d.W) c4[u] = code[d.base + q[g] + u];
                cv[g] = make_uint2(c4[0] | (c4[1] << 16), c4[2] | (c4[3] << 16));
            }
        }
    }
    const int K0 = *k0_ptr;
    const int rb = rbase ? rbase[ii] : 0;
    const int n = te.y;
    const bool tab = n * NL <= kWrite6Tab;
    auto level_of = [&](int s, int k) -> int {   // level-k id of slot s's basin
        const int c = safe_id(idmap, ends[te.x + s].x, K0);
        if (c < 0) return -1;
        if (k == 0) return c - rb;
        const int32_t *gm = gmap + (size_t)(k - 1) * kstride;
        return gm[c] - (rbase ? gm[rb] : 0);
    };
    if (tab) {
        for (int s = tid; s < n; s += C::NT) {
            const int c = safe_id(idmap, ends[te.x + s].x, K0);
            lv[s] = c >= 0 ? c - rb : -1;
            for (int k = 1; k < NL; k++) {
                const int32_t *gm = gmap + (size_t)(k - 1) * kstride;
                lv[k * n + s] = c >= 0 ? gm[c] - (rbase ? gm[rb] : 0) : -1;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (q[g] < 0) continue;
        const int s0 = cv[g].x & 0x1fff, s1 = (cv[g].x >> 16) & 0x1fff, s2 = cv[g].y & 0x1fff,
                  s3 = (cv[g].y >> 16) & 0x1fff;
        for (int l = 0; l < NL; l++) {
            int4 o;
            if (tab) {
                o = make_int4(lv[l * n + s0], lv[l * n + s1], lv[l * n + s2], lv[l * n + s3]);
            } else {
                o = make_int4(level_of(s0, l), level_of(s1, l), level_of(s2, l), level_of(s3, l));
            }
            int32_t *dst = d.out + (size_t)l * d.N + q[g];
            if (vec && gx + 3 < d.W) {
                __stcs(reinterpret_cast<int4 *>(dst), o);
            } else {
                const int ov[4] = {o.x, o.y, o.z, o.w};
                for (int u = 0; u < 4; u++)
                    if (gx + u < d.W) __stcs(dst + u, ov[u]);
            }
        }
    }
}

// Per-image region counts of every level (batched calls).  Level-k ids are
// contiguous per image and ordered image by image; image i's smallest level-k
// id is that of its first basin, so its count is the next image's smallest
// id (or the level's total, ktot[k]) minus its own.
static __global__ void __launch_bounds__(NTHR) k_counts_batch(const Batch b, const int32_t *__restrict__ gmap,
                                                              size_t kstride, int NL, const int32_t *__restrict__ rbase,
                                                              const int32_t *__restrict__ ktot)
{
    for (int i = blockIdx.x * NTHR + threadIdx.x; i < b.n; i += gridDim.x * NTHR) {
        const ImgDesc d = img_desc(b, i);
        if (!d.counts) continue;
        d.counts[0] = rbase[i + 1] - rbase[i];
        for (int k = 1; k < NL; k++) {
            const int32_t *gm = gmap + (size_t)(k - 1) * kstride;
            const int next = i + 1 < b.n ? gm[rbase[i + 1]] : ktot[k];
            d.counts[k] = next - gm[rbase[i]];
        }
    }
}

// Step II distances as ws_plateau_distance reports them: 0 for state-0
// pixels, the distance for reached plateau pixels, -1 otherwise.
static __global__ void __launch_bounds__(NTHR) k_dist_out2(Geo geo, TileGeo tg, const int32_t *__restrict__ par,
                                                           const int32_t *__restrict__ dist,
                                                           const uint8_t *__restrict__ plat, int32_t *__restrict__ out)
{
    for (int p = blockIdx.x * NTHR + threadIdx.x; p < geo.N; p += gridDim.x * NTHR) {
        const int z = p / geo.HW, r = p - z * geo.HW, y = r / geo.W, x = r - y * geo.W;
        int v;
        if (plat[tile_of(tg, x, y, z)]) {
            v = dist[p];
            if (v >= INF_D || v < 0) v = -1;
        } else {
            v = par[p] == p ? -1 : 0;   // a minimum, or a pixel with a lower neighbour
        }
        out[p] = v;
    }
}

// ---------------------------------------------------------------------------
// k_write: one pass writing the canonical level-0 id and every waterfall level
// ---------------------------------------------------------------------------

static __global__ void __launch_bounds__(NTHR) k_write_vec(int N, const int32_t *__restrict__ par,
                                                           const int32_t *__restrict__ idmap,
                                                           const int32_t *__restrict__ gmap, size_t kstride, int NL,
                                                           const int32_t *__restrict__ k0_ptr,
                                                           int32_t *__restrict__ out)
{
    constexpr int U = 4;   // int4 vectors per thread per iteration (loads issued together)
    const int n4 = N >> 2;
    const int K0 = *k0_ptr;
    const int stride = gridDim.x * NTHR;
    for (int v0 = blockIdx.x * NTHR + threadIdx.x; v0 < n4; v0 += stride * U) {
        int4 c[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int v = v0 + u * stride;
            c[u] = v < n4 ? __ldcs(reinterpret_cast<const int4 *>(par) + v) : make_int4(0, 0, 0, 0);
        }
        // lanes past the end (v >= n4) gather nothing and store nothing
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (v0 + u * stride < n4) {
                c[u].x = safe_id(idmap, c[u].x, K0);
                c[u].y = safe_id(idmap, c[u].y, K0);
                c[u].z = safe_id(idmap, c[u].z, K0);
                c[u].w = safe_id(idmap, c[u].w, K0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int v = v0 + u * stride;
            if (v < n4) __stcs(reinterpret_cast<int4 *>(out) + v, c[u]);
        }
        for (int k = 1; k < NL; k++) {
            const int32_t *gm = gmap + (size_t)(k - 1) * kstride;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int v = v0 + u * stride;
                if (v >= n4) continue;
                int4 o;
                o.x = level_id(gm, c[u].x);
                o.y = level_id(gm, c[u].y);
                o.z = level_id(gm, c[u].z);
                o.w = level_id(gm, c[u].w);
                __stcs(reinterpret_cast<int4 *>(out + (size_t)k * N) + v, o);
            }
        }
    }
}

static __global__ void __launch_bounds__(NTHR) k_write_scalar(int N, const int32_t *__restrict__ par,
                                                              const int32_t *__restrict__ idmap,
                                                              const int32_t *__restrict__ gmap, size_t kstride,
                                                              int NL, const int32_t *__restrict__ k0_ptr,
                                                              int32_t *__restrict__ out)
{
    const int K0 = *k0_ptr;
    for (int p = blockIdx.x * NTHR + threadIdx.x; p < N; p += gridDim.x * NTHR) {
        const int c = safe_id(idmap, par[p], K0);
        out[p] = c;
        for (int k = 1; k < NL; k++) out[(size_t)k * N + p] = level_id(gmap + (size_t)(k - 1) * kstride, c);
    }
}

}  // namespace ws
