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
// 3D: one CTA produces a 32 x 8 x 8 tile of the gradient of a volume
// ---------------------------------------------------------------------------
//   1. the 38 x 14 x 14 input window (3-voxel halo, replicated border) is
//      staged in shared memory;
//   2. the 5x5x5 binomial blur is taken as three exact integer passes (x, y,
//      z; sums below 2^29, rounded once: (sum + 2048) >> 12) at the 34 x 10 x
//      10 positions the Sobel stencil reads, each a 5-tap window sliding in
//      registers; a position outside the volume takes the blur of the nearest
//      border voxel, like the 2D kernel;
//   3. 3x3x3 Sobel from per-plane 3x3 sums sliding along z, exact floor square
//      root of gx^2 + gy^2 + gz^2 (float estimate corrected by 64-bit integer
//      comparisons), >> shift, clip.
constexpr int G3X = 32, G3Y = 8, G3Z = 8;
constexpr int I3X = G3X + 6, I3Y = G3Y + 6, I3Z = G3Z + 6;   // input window
constexpr int B3X = G3X + 2, B3Y = G3Y + 2, B3Z = G3Z + 2;   // blur window
constexpr int S3A = I3Z * I3Y * I3X;   // input window, then the x-y sums  (>= I3Z * B3Y * B3X)
constexpr int S3B = I3Z * I3Y * B3X;   // x sums, then the blur            (>= B3Z * B3Y * B3X)
constexpr int G3_SMEM = (S3A + S3B) * 4;

__device__ __forceinline__ unsigned isqrt64_exact(unsigned long long v)
{
    unsigned long long r = (unsigned long long)sqrtf((float)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return (unsigned)r;
}

// One line of a blur pass: out[k * os] = the 5-tap binomial sum of `line` at
// position P0 + k clamped to [0, L - 1] (so positions beyond the border repeat
// the border's sum), for k < n; line[u * is] is the input at coordinate u
// (only coordinates clamped into [0, L - 1] are read).  In the interior the
// window slides: one new load per output.  ROUND: (sum + 2048) >> 12.
template <bool ROUND>
__device__ __forceinline__ void blur_line(const unsigned *line, int is, unsigned *out, int os, int P0, int n, int L)
{
    auto at = [&](int u) { return line[clampi(u, 0, L - 1) * is]; };
    auto put = [&](int k, unsigned sum) { out[k * os] = ROUND ? (sum + 2048u) >> 12 : sum; };
    int k = 0;
    for (; k < n && P0 + k < 0; k++) put(k, at(-2) + 4u * at(-1) + 6u * at(0) + 4u * at(1) + at(2));   // = position 0
    if (k < n && P0 + k < L) {
        int X = P0 + k;
        unsigned w0 = at(X - 2), w1 = at(X - 1), w2 = at(X), w3 = at(X + 1);
        for (; k < n && X < L; k++, X++) {
            const unsigned w4 = at(X + 2);
            put(k, w0 + 4u * w1 + 6u * w2 + 4u * w3 + w4);
            w0 = w1;
            w1 = w2;
            w2 = w3;
            w3 = w4;
        }
    }
    if (k < n) {   // beyond the far border: the sum at L - 1
        const unsigned e = at(L - 3) + 4u * at(L - 2) + 6u * at(L - 1) + 4u * at(L) + at(L + 1);
        for (; k < n; k++) put(k, e);
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_gradient3d(const V *__restrict__ img, int W, int H, int D, int shift,
                                                    uint16_t *__restrict__ out)
{
    extern __shared__ unsigned g3s[];
    unsigned *A = g3s, *B = g3s + S3A;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * G3X, y0 = blockIdx.y * G3Y, z0 = blockIdx.z * G3Z;
    for (int i = tid; i < S3A; i += 256) {
        const int ix = i % I3X, iy = (i / I3X) % I3Y, iz = i / (I3X * I3Y);
        const int gx = clampi(x0 - 3 + ix, 0, W - 1), gy = clampi(y0 - 3 + iy, 0, H - 1);
        const int gz = clampi(z0 - 3 + iz, 0, D - 1);
        A[i] = img[((size_t)gz * H + gy) * W + gx];
    }
    __syncthreads();
    // Each pass slides a 5-tap window along its axis in registers: one thread
    // per row / column / pillar reads every input once.
    // x: B[iz][iy][bx] = sum_t w_t A[iz][iy][clamp(X + t)], X = clamp(x0 - 1 + bx)
    for (int r = tid; r < I3Z * I3Y; r += 256)
        blur_line<false>(A + r * I3X - (x0 - 3), 1, B + r * B3X, 1, x0 - 1, B3X, W);
    __syncthreads();
    // y: A[iz][by][bx] = sum_t w_t B[iz][clamp(Y + t)][bx], Y = clamp(y0 - 1 + by)
    for (int c = tid; c < I3Z * B3X; c += 256) {
        const int bx = c % B3X, iz = c / B3X;
        blur_line<false>(B + iz * I3Y * B3X - (y0 - 3) * B3X + bx, B3X, A + iz * B3Y * B3X + bx, B3X, y0 - 1, B3Y,
                         H);
    }
    __syncthreads();
    // z: B[bz][by][bx] = (sum_t w_t A[clamp(Z + t)][by][bx] + 2048) >> 12, Z = clamp(z0 - 1 + bz)
    for (int c = tid; c < B3Y * B3X; c += 256)
        blur_line<true>(A - (z0 - 3) * (B3Y * B3X) + c, B3Y * B3X, B + c, B3Y * B3X, z0 - 1, B3Z, D);
    __syncthreads();
    // Sobel (positions beyond the border hold the border's blur).  Per blurred
    // plane the thread's 3x3 (y, x) neighbourhood gives dx = [1 2 1]_y of the
    // x difference, dy = [1 2 1]_x of the y difference and sm = [1 2 1]^2 of
    // the values; then gx = [1 2 1]_z of dx, gy = [1 2 1]_z of dy and
    // gz = sm(z + 1) - sm(z - 1).
    const int lx = tid & 31, ly = tid >> 5;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    int dxm = 0, dym = 0, smm = 0, dx0 = 0, dy0 = 0, sm0 = 0;
    for (int bz = 0; bz < B3Z; bz++) {
        const unsigned *pl = B + (bz * B3Y + ly) * B3X + lx;   // (y - 1, x - 1) of this plane
        int v[3][3];
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) v[j][i] = (int)pl[j * B3X + i];
        const int dx = (v[0][2] - v[0][0]) + 2 * (v[1][2] - v[1][0]) + (v[2][2] - v[2][0]);
        const int dy = (v[2][0] - v[0][0]) + 2 * (v[2][1] - v[0][1]) + (v[2][2] - v[0][2]);
        const int sm = (v[0][0] + 2 * v[0][1] + v[0][2]) + 2 * (v[1][0] + 2 * v[1][1] + v[1][2]) +
                       (v[2][0] + 2 * v[2][1] + v[2][2]);
        if (bz >= 2) {   // output plane z = z0 + bz - 2 (its blurred planes are bz - 2 .. bz)
            const int z = z0 + bz - 2;
            if (z >= D) break;
            const int gxs = dxm + 2 * dx0 + dx, gys = dym + 2 * dy0 + dy, gzs = sm - smm;
            const unsigned long long s2 = (unsigned long long)((long long)gxs * gxs) +
                                          (unsigned long long)((long long)gys * gys) +
                                          (unsigned long long)((long long)gzs * gzs);
            const unsigned m = isqrt64_exact(s2) >> shift;
            out[((size_t)z * H + y) * W + x] = (uint16_t)(m > 65535u ? 65535u : m);
        }
        dxm = dx0; dym = dy0; smm = sm0;
        dx0 = dx; dy0 = dy; sm0 = sm;
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
    dim3 grid((W + G3X - 1) / G3X, (H + G3Y - 1) / G3Y, (D + G3Z - 1) / G3Z);
    cudaError_t e = bps == 1 ? cudaFuncSetAttribute(k_gradient3d<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    G3_SMEM)
                             : cudaFuncSetAttribute(k_gradient3d<uint16_t>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, G3_SMEM);
    if (e != cudaSuccess) return set_cuda_error(c, e, "smem attribute");
    PhaseScope ps(c, PH_GRADIENT, s);
    if (bps == 1)
        k_gradient3d<uint8_t><<<grid, 256, G3_SMEM, s>>>((const uint8_t *)vol, W, H, D, shift, grad);
    else
        k_gradient3d<uint16_t><<<grid, 256, G3_SMEM, s>>>((const uint16_t *)vol, W, H, D, shift, grad);
    c->launches += 1;
    e = cudaGetLastError();
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
