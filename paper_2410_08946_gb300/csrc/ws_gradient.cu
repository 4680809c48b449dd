// ws_gradient.cu -- pipeline steps 1-2 of Sec. 1 (minimal smoothing, then
// gradient magnitude; optional per Fig. 2) for images and volumes, and a
// label-count helper.
//
// One CTA produces a 32 x 16 tile of the gradient:
//   1. the 38 x 22 input window (3-pixel halo, replicated border) is staged
//      in shared memory;
//   2. the 5x5 binomial blur [1 4 6 4 1]^2, (sum + 128) >> 8, is evaluated
//      at the 34 x 18 positions the Sobel stencil reads; a position outside
//      the image takes the blur of the nearest border pixel (the blurred
//      image's border is replicated, not re-blurred);
//   3. 3x3 integer Sobel, exact floor square root of gx^2 + gy^2 (sqrtf
//      estimate corrected by integer comparisons), clip to 255, >> shift.
#include "ws_internal.h"

namespace ws {

namespace {

constexpr int GTW = 32, GTH = 16;
constexpr int GIW = GTW + 6, GIH = GTH + 6;   // input window
constexpr int GBW = GTW + 2, GBH = GTH + 2;   // blur window

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// floor(sqrt(v)) for 0 <= v < 2^24: float estimate, then exact integer fix-up.
__device__ __forceinline__ unsigned isqrt_exact(unsigned v)
{
    unsigned r = (unsigned)sqrtf((float)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

__global__ void __launch_bounds__(256) k_gradient(const uint8_t *__restrict__ img, int W, int H, int shift,
                                                  uint8_t *__restrict__ out)
{
    __shared__ uint8_t in[GIH][GIW];
    __shared__ int bl[GBH][GBW];
    const int x0 = blockIdx.x * GTW, y0 = blockIdx.y * GTH;
    for (int i = threadIdx.x; i < GIH * GIW; i += 256) {
        int iy = i / GIW, ix = i % GIW;
        int y = clampi(y0 - 3 + iy, 0, H - 1), x = clampi(x0 - 3 + ix, 0, W - 1);
        in[iy][ix] = img[(size_t)y * W + x];
    }
    __syncthreads();
    const int w5[5] = {1, 4, 6, 4, 1};
    for (int i = threadIdx.x; i < GBH * GBW; i += 256) {
        int by = i / GBW, bx = i % GBW;
        int cy = clampi(y0 - 1 + by, 0, H - 1), cx = clampi(x0 - 1 + bx, 0, W - 1);
        int iy = cy - (y0 - 3), ix = cx - (x0 - 3);
        int s = 0;
#pragma unroll
        for (int a = 0; a < 5; a++) {
            int row = 0;
#pragma unroll
            for (int b = 0; b < 5; b++) row += w5[b] * in[iy - 2 + a][ix - 2 + b];
            s += w5[a] * row;
        }
        bl[by][bx] = (s + 128) >> 8;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GTW * GTH; i += 256) {
        int oy = i / GTW, ox = i % GTW;
        int y = y0 + oy, x = x0 + ox;
        if (y >= H || x >= W) continue;
        int by = oy + 1, bx = ox + 1;
        int gx = (bl[by - 1][bx + 1] + 2 * bl[by][bx + 1] + bl[by + 1][bx + 1]) -
                 (bl[by - 1][bx - 1] + 2 * bl[by][bx - 1] + bl[by + 1][bx - 1]);
        int gy = (bl[by + 1][bx - 1] + 2 * bl[by + 1][bx] + bl[by + 1][bx + 1]) -
                 (bl[by - 1][bx - 1] + 2 * bl[by - 1][bx] + bl[by - 1][bx + 1]);
        unsigned m = isqrt_exact((unsigned)(gx * gx + gy * gy));
        if (m > 255) m = 255;
        out[(size_t)y * W + x] = (uint8_t)(m >> shift);
    }
}

// ---------------------------------------------------------------------------
// 3D: one CTA streams a 32 x 16 column of the volume along z
// ---------------------------------------------------------------------------
// A CTA owns the outputs (x0..x0+31, y0..y0+15, z0..z0+ZC-1), one thread per
// (x, y), and walks the input planes in z order, so that every input voxel
// of the column (with its 3-voxel x-y halo) is read once:
//   1. the plane's 38 x 22 window (replicated border) goes to shared memory
//      (the next plane's values are loaded into registers meanwhile);
//   2. the 5-tap binomial x-pass, then y-pass, give the plane's x-y blurred
//      sums at the 34 x 18 positions the Sobel reads, kept in a ring of the
//      last five planes;
//   3. once a plane has its two successors, the z-pass over the ring gives
//      its 5x5x5 blur, rounded once: (sum + 2048) >> 12 (sums below 2^29);
//   4. each thread turns its 3x3 neighbourhood of that plane into the
//      plane's x difference dx and y difference dy (each smoothed [1 2 1]
//      across) and its [1 2 1]^2 sum sm, and keeps them for three planes:
//      gx = [1 2 1]_z of dx, gy = [1 2 1]_z of dy, gz = sm(z + 1) - sm(z - 1);
//      exact floor square root of gx^2 + gy^2 + gz^2 (float estimate
//      corrected by 64-bit integer comparisons), >> shift, clip.
// A blur position outside the volume takes the blur of the nearest border
// voxel, in x, y and z alike (the blurred volume's border is replicated).
constexpr int ZX = 32, ZY = 16, ZT = ZX * ZY;                 // output tile, one thread per (x, y)
constexpr int ZIX = ZX + 6, ZIY = ZY + 6, ZBX = ZX + 2, ZBY = ZY + 2;
constexpr int ZIN = ZIX * ZIY, ZXS = ZBX * ZIY, ZBS = ZBX * ZBY;
constexpr int ZC = 64;                                        // output planes per CTA
static_assert(ZIN <= 2 * ZT, "two window loads per thread");

__device__ __forceinline__ unsigned isqrt64_exact(unsigned long long v)
{
    unsigned long long r = (unsigned long long)sqrtf((float)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return (unsigned)r;
}

struct Sob {   // one blurred plane's x and y differences and its 3x3 sum at a thread's (x, y)
    int dx, dy, sm;
};

template <typename V>
__global__ void __launch_bounds__(ZT) k_gradient3d(const V *__restrict__ img, int W, int H, int D, int shift,
                                                   uint16_t *__restrict__ out)
{
    __shared__ unsigned inp[ZIN];       // the input plane's window
    __shared__ unsigned xs[ZXS];        // its x-pass
    __shared__ unsigned ring[5][ZBS];   // x-y blurred sums of the last five input planes (slot: plane mod 5)
    __shared__ unsigned bz[ZBS];        // the blurred plane
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * ZX, y0 = blockIdx.y * ZY, z0 = blockIdx.z * ZC;
    const int z1 = min(z0 + ZC, D);                             // outputs z0 .. z1 - 1
    const int zlo = max(z0 - 1, 0), zhi = min(z1, D - 1);       // the blurred planes they read
    const size_t HW = (size_t)H * W;
    // this thread's two slots of the window, as offsets within a plane (clamped), or -1
    auto slot = [&](int l) -> long long {
        if (l >= ZIN) return -1;
        const int ix = l % ZIX, iy = l / ZIX;
        return (long long)clampi(y0 - 3 + iy, 0, H - 1) * W + clampi(x0 - 3 + ix, 0, W - 1);
    };
    const long long a0 = slot(tid), a1 = slot(tid + ZT);
    auto fetch = [&](int zi, unsigned &v0, unsigned &v1) {
        const size_t pz = (size_t)clampi(zi, 0, D - 1) * HW;
        v0 = a0 >= 0 ? (unsigned)img[pz + a0] : 0u;
        v1 = a1 >= 0 ? (unsigned)img[pz + a1] : 0u;
    };
    unsigned v0, v1;
    fetch(zlo - 2, v0, v1);
    const int ox = tid % ZX, oy = tid / ZX;
    const int x = x0 + ox, y = y0 + oy;
    const bool mine = x < W && y < H;
    Sob A{0, 0, 0}, B{0, 0, 0};   // planes zb - 2, zb - 1
    auto emit = [&](int z, const Sob &m, const Sob &c, const Sob &p) {
        const long long gxs = m.dx + 2 * c.dx + p.dx, gys = m.dy + 2 * c.dy + p.dy, gzs = p.sm - m.sm;
        const unsigned long long s2 =
            (unsigned long long)(gxs * gxs) + (unsigned long long)(gys * gys) + (unsigned long long)(gzs * gzs);
        const unsigned mg = isqrt64_exact(s2) >> shift;
        out[(size_t)z * HW + (size_t)y * W + x] = (uint16_t)(mg > 65535u ? 65535u : mg);
    };
    for (int zi = zlo - 2; zi <= zhi + 2; zi++) {
        if (a0 >= 0) inp[tid] = v0;
        if (a1 >= 0) inp[tid + ZT] = v1;
        __syncthreads();
        if (zi < zhi + 2) fetch(zi + 1, v0, v1);   // in flight while this plane is blurred
        // x-pass at X = clamp(x0 - 1 + bx)
        for (int e = tid; e < ZXS; e += ZT) {
            const int bx = e % ZBX, iy = e / ZBX;
            const unsigned *r = inp + iy * ZIX + clampi(x0 - 1 + bx, 0, W - 1) - (x0 - 3);
            xs[e] = r[-2] + 4u * r[-1] + 6u * r[0] + 4u * r[1] + r[2];
        }
        __syncthreads();
        // y-pass at Y = clamp(y0 - 1 + by), into the ring
        unsigned *rs = ring[(zi + 10) % 5];
        for (int e = tid; e < ZBS; e += ZT) {
            const int bx = e % ZBX, by = e / ZBX;
            const unsigned *c = xs + (clampi(y0 - 1 + by, 0, H - 1) - (y0 - 3)) * ZBX + bx;
            rs[e] = c[-2 * ZBX] + 4u * c[-ZBX] + 6u * c[0] + 4u * c[ZBX] + c[2 * ZBX];
        }
        __syncthreads();
        const int zb = zi - 2;   // the blurred plane whose five input planes are in the ring
        if (zb < zlo) continue;
        // z-pass: planes zb - 2 .. zb + 2 are the ring's input planes zi - 4 .. zi
        // (clamped into the volume when they were loaded)
        for (int e = tid; e < ZBS; e += ZT) {
            const unsigned sum = ring[(zi + 6) % 5][e] + 4u * ring[(zi + 7) % 5][e] + 6u * ring[(zi + 8) % 5][e] +
                                 4u * ring[(zi + 9) % 5][e] + ring[(zi + 10) % 5][e];
            bz[e] = (sum + 2048u) >> 12;
        }
        __syncthreads();
        const unsigned *pl = bz + oy * ZBX + ox;   // (y - 1, x - 1) of this plane
        int v[3][3];
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) v[j][i] = (int)pl[j * ZBX + i];
        Sob T;
        T.dx = (v[0][2] - v[0][0]) + 2 * (v[1][2] - v[1][0]) + (v[2][2] - v[2][0]);
        T.dy = (v[2][0] - v[0][0]) + 2 * (v[2][1] - v[0][1]) + (v[2][2] - v[0][2]);
        T.sm = (v[0][0] + 2 * v[0][1] + v[0][2]) + 2 * (v[1][0] + 2 * v[1][1] + v[1][2]) +
               (v[2][0] + 2 * v[2][1] + v[2][2]);
        if (mine) {
            // output z = zb - 1 reads planes zb - 2 (clamped at 0), zb - 1, zb
            if (zb > zlo && zb - 1 >= z0 && zb - 1 < z1) emit(zb - 1, zb >= 2 ? A : B, B, T);
            // the volume's last plane reads itself in place of plane D
            if (zb == D - 1 && zb >= z0 && zb < z1) emit(zb, zb > zlo ? B : T, T, T);
        }
        A = B;
        B = T;
    }
}

__global__ void k_max_label(const int32_t *__restrict__ L, int N, int32_t *kcount)
{
    int m = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) m = max(m, L[p] + 1);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(kcount, m);
}

}  // namespace

ws_status launch_gradient(ws_context *c, const uint8_t *img, int W, int H, int shift, uint8_t *grad,
                          cudaStream_t s)
{
    dim3 grid((W + GTW - 1) / GTW, (H + GTH - 1) / GTH);
    PhaseScope ps(c, PH_GRADIENT, s);
    k_gradient<<<grid, 256, 0, s>>>(img, W, H, shift, grad);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "gradient launch");
}

ws_status launch_gradient3d(ws_context *c, const void *vol, int bps, int W, int H, int D, int shift,
                            uint16_t *grad, cudaStream_t s)
{
    dim3 grid((W + ZX - 1) / ZX, (H + ZY - 1) / ZY, (D + ZC - 1) / ZC);
    PhaseScope ps(c, PH_GRADIENT, s);
    if (bps == 1)
        k_gradient3d<uint8_t><<<grid, ZT, 0, s>>>((const uint8_t *)vol, W, H, D, shift, grad);
    else
        k_gradient3d<uint16_t><<<grid, ZT, 0, s>>>((const uint16_t *)vol, W, H, D, shift, grad);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "gradient3d launch");
}

ws_status launch_count_labels(ws_context *c, const int32_t *labels, int N, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(c->w.kcount, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
    int grid = c->num_sms * 8;
    k_max_label<<<grid, 256, 0, s>>>(labels, N, c->w.kcount);
    c->launches += 1;
    e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "count launch");
}

}  // namespace ws
