// ws_static.cu -- ws_watershed_static: the watershed for callers that cannot
// allocate device memory.
//
// Some callers own every byte of device memory they touch: frameworks that
// reserve the GPU's memory up front for their own pool, or latency-critical
// loops where the implicit device-wide synchronisation of cudaMalloc and
// cudaFree is not acceptable.  They cannot create a ws_context (which
// allocates its workspace on first use).  This entry point runs the same
// watershed pipeline as ws_watershed, but every scratch array it needs lives
// in one file-scope device array, ws_static_scratch, of fixed size: images up
// to WS_STATIC_MAX_PIXELS pixels.  The array is part of the library image, so
// every GPU that loads the library holds it until the process exits.
//
// Host code cannot take the address of a __device__ array directly (the
// symbol seen by host code is a host-side stand-in): the first call on each
// device looks the device address up with cudaGetSymbolAddress while that
// device is current, and keeps it.
#include <mutex>

#include "ws_tiles.cuh"

using namespace ws;

namespace {

constexpr size_t kMaxPixels = (size_t)WS_STATIC_MAX_PIXELS;
// tiles of an image of at most kMaxPixels pixels: at most kMaxPixels / 16 + 1
// (a 3D image one voxel wide and high has one 16-voxel-deep tile per 16 voxels)
constexpr size_t kMaxTiles = kMaxPixels / 16 + 4;
constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr size_t kRmax = kMaxPixels / 2 + 2;
constexpr size_t kWords = (kMaxPixels + 31) / 32, kGroups = (kWords + 31) / 32, kChunks = (kGroups + 2047) / 2048;
constexpr size_t OFF_PAR = 0;
constexpr size_t OFF_AUX = OFF_PAR + a256(kMaxPixels * 4);
constexpr size_t OFF_DIST = OFF_AUX + a256(kMaxPixels * 4);
constexpr size_t OFF_ROOTS = OFF_DIST + a256(kMaxPixels * 4);
constexpr size_t OFF_ROOTM = OFF_ROOTS + a256(kRmax * 4);
constexpr size_t OFF_BITMAP = OFF_ROOTM + a256(kRmax * 4);
constexpr size_t OFF_GCNT = OFF_BITMAP + a256(kWords * 4);
constexpr size_t OFF_CSUM = OFF_GCNT + a256((kGroups + 1) * 4);
constexpr size_t OFF_PLAT = OFF_CSUM + a256((kChunks + 1) * 4);
constexpr size_t OFF_ACT = OFF_PLAT + a256(kMaxTiles);
constexpr size_t OFF_TLIST = OFF_ACT + a256(kMaxTiles * 2);
constexpr size_t OFF_COUNTERS = OFF_TLIST + a256(kMaxTiles * 4);
constexpr size_t OFF_STATUS = OFF_COUNTERS + 256;
constexpr size_t OFF_KCOUNT = OFF_STATUS + a256(sizeof(DevStatus));
constexpr size_t OFF_CODE = OFF_KCOUNT + 256;                  // 3D path: slot code per pixel
constexpr size_t OFF_ENDS = OFF_CODE + a256(kMaxPixels * 2);   // 3D path: (end, next), then (root, root)
constexpr size_t OFF_TENDS = OFF_ENDS + a256(kMaxPixels * 8);  // 3D path: slot span per tile
constexpr size_t OFF_PLIST = OFF_TENDS + a256(kMaxTiles * 8); // 2D path: plateau pixels per tile
constexpr size_t OFF_PSPAN = OFF_PLIST + a256(kMaxPixels * 2); // 2D path: their span per tile
constexpr size_t kScratchBytes = OFF_PSPAN + a256(kMaxTiles * 8);
static_assert(kScratchBytes == (size_t)WS_STATIC_SCRATCH_BYTES, "WS_STATIC_SCRATCH_BYTES must match the layout");

}  // namespace

// All scratch of ws_watershed_static.  Zero at load; every call leaves the
// bitmap and the status word zero again and clears the rest itself.
static __device__ __align__(256) unsigned char ws_static_scratch[kScratchBytes];

namespace {

// Reports a device-side error of the call through the count output (-1) and
// returns the status word to zero.
__global__ void k_static_finish(int32_t *count)
{
    DevStatus *s = reinterpret_cast<DevStatus *>(ws_static_scratch + OFF_STATUS);
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (s->code != 0) *count = -1;
        s->code = 0;
        s->where = 0;
        s->abort = 0;
    }
}

struct Slot {
    bool ready = false;
    ws_context ctx;  // never owns memory: its workspace points into the scratch array (each call copies it)
};
constexpr int kMaxDevices = 64;
Slot g_slots[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: the device address of the
// scratch array, carved into the workspace of a context that never allocates.
// *out receives a copy, so that host threads calling at the same time share
// no host state.
ws_status setup(int dev, ws_context *out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    Slot &sl = g_slots[dev];
    if (!sl.ready) {
        unsigned char *base = nullptr;
        if (cudaGetSymbolAddress((void **)&base, ws_static_scratch) != cudaSuccess || !base) {
            cudaGetLastError();
            return WS_ERR_CUDA;
        }
        ws_context &c = sl.ctx;
        c.device = dev;
        if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return WS_ERR_CUDA;
        }
        c.status = reinterpret_cast<DevStatus *>(base + OFF_STATUS);
        Workspace &w = c.w;
        w.N = kMaxPixels;
        w.par = reinterpret_cast<int32_t *>(base + OFF_PAR);
        w.aux = reinterpret_cast<int32_t *>(base + OFF_AUX);
        w.dist = reinterpret_cast<int32_t *>(base + OFF_DIST);
        w.rmax = kRmax;
        w.roots = reinterpret_cast<int32_t *>(base + OFF_ROOTS);
        w.rootm = reinterpret_cast<int32_t *>(base + OFF_ROOTM);
        w.nwords = kWords;
        w.ngroups = kGroups;
        w.nchunks = kChunks;
        w.bitmap = reinterpret_cast<uint32_t *>(base + OFF_BITMAP);
        w.gcnt = reinterpret_cast<int32_t *>(base + OFF_GCNT);
        w.csum = reinterpret_cast<int32_t *>(base + OFF_CSUM);
        w.ntiles = kMaxTiles;
        w.plat = base + OFF_PLAT;
        w.act = base + OFF_ACT;
        w.tlist = reinterpret_cast<int32_t *>(base + OFF_TLIST);
        w.counters = reinterpret_cast<int32_t *>(base + OFF_COUNTERS);
        w.kcount = reinterpret_cast<int32_t *>(base + OFF_KCOUNT);
        w.ncode = kMaxPixels;
        w.code = reinterpret_cast<uint16_t *>(base + OFF_CODE);
        w.ends = reinterpret_cast<int2 *>(base + OFF_ENDS);
        w.ntends = kMaxTiles;
        w.tends = reinterpret_cast<int2 *>(base + OFF_TENDS);
        w.nplist = kMaxPixels;
        w.plist = reinterpret_cast<uint16_t *>(base + OFF_PLIST);
        w.npspan = kMaxTiles;
        w.pspan = reinterpret_cast<int2 *>(base + OFF_PSPAN);
        sl.ready = true;
    }
    *out = sl.ctx;
    return WS_OK;
}

}  // namespace

extern "C" ws_status ws_watershed_static(const void *grad_d, ws_dtype dtype, const ws_shape *shape, int connectivity,
                                         int32_t *labels_d, int32_t *count_d, ws_stream_t stream)
{
    if (!grad_d || !labels_d || !count_d || !shape) return WS_ERR_INVALID;
    if (dtype != WS_U8 && dtype != WS_U16) return WS_ERR_INVALID;
    if (shape->ndim != 2 && shape->ndim != 3) return WS_ERR_INVALID;
    const int64_t W = shape->dims[0], H = shape->dims[1], D = shape->ndim == 3 ? shape->dims[2] : 1;
    if (W < 1 || H < 1 || D < 1) return WS_ERR_INVALID;
    if (W > (int64_t)kMaxPixels || H > (int64_t)kMaxPixels || D > (int64_t)kMaxPixels ||
        W * H * D > (int64_t)kMaxPixels)
        return WS_ERR_INVALID;  // larger than WS_STATIC_MAX_PIXELS: use ws_watershed
    const bool ok2 = shape->ndim == 2 && (connectivity == 4 || connectivity == 8);
    const bool ok3 = shape->ndim == 3 && (connectivity == 6 || connectivity == 26);
    if (!ok2 && !ok3) return WS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return WS_ERR_CUDA;
    }
    ws_context local;
    ws_status st = setup(dev, &local);
    if (st != WS_OK) return st;
    ws_context *c = &local;
    Geo g;
    g.W = (int)W;
    g.H = (int)H;
    g.D = (int)D;
    g.HW = (int)(W * H);
    g.N = (int)(W * H * D);
    const TileGeo tg = shape->ndim == 2 ? tiles_for<4>(g) : tiles_for<6>(g);
    if ((size_t)tg.ntiles > kMaxTiles) return WS_ERR_INVALID;
    const Launchers *L = launchers(dtype, connectivity);
    if (!L) return WS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    // clear the error state an earlier call that failed on the host side may
    // have left (its k_static_finish never ran)
    if (cudaMemsetAsync(c->status, 0, offsetof(DevStatus, bar_count), s) != cudaSuccess) {
        cudaGetLastError();
        return WS_ERR_CUDA;
    }
    st = L->watershed(c, grad_d, g, labels_d, count_d, s);
    if (st != WS_OK) return st;
    k_static_finish<<<1, 32, 0, s>>>(count_d);
    return cudaGetLastError() == cudaSuccess ? WS_OK : WS_ERR_CUDA;
}
