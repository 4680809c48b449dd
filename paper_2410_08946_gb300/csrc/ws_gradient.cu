// ws_gradient.cu -- pipeline steps 1-2 of Sec. 1 (minimal smoothing, then
// gradient magnitude; optional per Fig. 2), and a label-count helper.
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
