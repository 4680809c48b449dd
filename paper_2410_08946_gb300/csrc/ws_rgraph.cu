// ws_rgraph.cu -- export of the region graph of one labelling.  Sec. 6 uses the
// regions of a waterfall level in place of superpixels as the graph of a graph
// network; here every region id 0..K-1 of a labelling is a node and two regions
// share an edge when a pixel of one is a neighbour (Sec. 3.1, N(p)) of a pixel
// of the other.  The edge weight is pass(A, B) of Alg. 5 step V (the smallest
// max(G(p), G(q)) over those pixel pairs); the node features are the pixel
// count and the per-channel sums of a value image.
//
//   k_label_range    the largest id (K = largest + 1), and a flag for negative ids
//   k_region_stats   pixel count and value sums per region: runs of equal ids
//                    in each thread's 8 pixels, the last run combined across
//                    the warp (match_any, reduce_add) before its atomic
//   k_rag            (shared with ws_waterfall) the distinct region pairs with
//                    their smallest pixel-pair height, into the region table;
//   k_edges_compact  the table to a dense list of (a < b, pass)
//   k_dir_keys       both directions of every edge as 64-bit sort keys
//                    (row << s | col), pass values alongside
//   k_radix_hist /   stable least-significant-digit radix sort of the keys,
//   k_radix_scatter  8-bit digits over the 2s key bits: per-tile digit counts,
//                    a device-wide scan (digit-major), then a stable scatter
//                    that ranks equal digits in index order inside the tile
//   k_csr_rows       row starts from the sorted keys (no atomics)
//   k_csr_out        the caller's CSR arrays and the means (sum / count)
// The sort makes the CSR deterministic: row A lists its neighbours in
// increasing id order, whatever order the pairs were found in.
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int RT = 4096;             // keys per radix tile (256 threads x 16)
constexpr int RPT = RT / NTHR;       // keys per thread
static_assert(NTHR == 256, "one thread per radix digit");

__global__ void k_label_range(const int32_t *__restrict__ L, long long N, int32_t *misc)
{
    int m = 0, neg = 0;   // largest id (misc[0] starts at 0), any id < 0
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int l = L[p];
        m = max(m, l);
        neg |= l < 0;
    }
    m = __reduce_max_sync(0xffffffffu, m);
    neg = __reduce_or_sync(0xffffffffu, neg);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(misc + 0, m);
        if (neg) atomicOr(misc + 1, 1);
    }
}

__global__ void k_put_int(int32_t *p, int v)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *p = v;
}

// Each thread takes 8 consecutive pixels and adds up runs of equal ids; a run
// that ends inside the 8 goes to global memory at once, the thread's last run
// is first combined across the warp (lanes with the same id: match_any,
// reduce_add), so a region that covers whole warps costs one atomic per 256
// pixels.  VEC: 16-byte label loads and one vector load of values per channel
// (pointers 16-byte aligned, N a multiple of 8).
constexpr int SPIX = 8;

template <typename V, bool VEC>
__global__ void __launch_bounds__(NTHR) k_region_stats(const int32_t *__restrict__ L, const V *__restrict__ vals,
                                                       long long N, int C, unsigned long long *size,
                                                       unsigned long long *sum)
{
    const int lane = threadIdx.x & 31;
    const long long nch = (N + SPIX - 1) / SPIX;
    for (long long q0 = (long long)blockIdx.x * NTHR; q0 < nch; q0 += (long long)gridDim.x * NTHR) {
        const long long p0 = (q0 + threadIdx.x) * SPIX;
        const bool full = p0 + SPIX <= N;
        int lab[SPIX];
        if (VEC && full) {
            const int4 u = *reinterpret_cast<const int4 *>(L + p0);
            const int4 w = *reinterpret_cast<const int4 *>(L + p0 + 4);
            lab[0] = u.x; lab[1] = u.y; lab[2] = u.z; lab[3] = u.w;
            lab[4] = w.x; lab[5] = w.y; lab[6] = w.z; lab[7] = w.w;
        } else {
#pragma unroll
            for (int j = 0; j < SPIX; j++) lab[j] = p0 + j < N ? L[p0 + j] : -1;
        }
        // sizes
        int cur = lab[0];
        unsigned cnt = 0;
#pragma unroll
        for (int j = 0; j < SPIX; j++) {
            if (lab[j] != cur) {
                if (cur >= 0) atomicAdd(size + cur, (unsigned long long)cnt);
                cur = lab[j];
                cnt = 0;
            }
            cnt += lab[j] >= 0;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, cur);
        const bool lead = cur >= 0 && lane == __ffs(grp) - 1;
        const unsigned tot = __reduce_add_sync(grp, cnt);
        if (lead) atomicAdd(size + cur, (unsigned long long)tot);
        // value sums, channel by channel (the same runs)
        for (int c = 0; c < C; c++) {
            const V *vp = vals + (size_t)c * N + p0;
            unsigned v[SPIX];
            if (VEC && full) {
                if constexpr (sizeof(V) == 2) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(vp);
                    const unsigned w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        v[2 * j] = w4[j] & 0xffffu;
                        v[2 * j + 1] = w4[j] >> 16;
                    }
                } else {
                    const uint2 u = *reinterpret_cast<const uint2 *>(vp);
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        v[j] = (u.x >> (8 * j)) & 0xffu;
                        v[4 + j] = (u.y >> (8 * j)) & 0xffu;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < SPIX; j++) v[j] = p0 + j < N ? (unsigned)vp[j] : 0u;
            }
            int cr = lab[0];
            unsigned sm = 0;
#pragma unroll
            for (int j = 0; j < SPIX; j++) {
                if (lab[j] != cr) {
                    if (cr >= 0) atomicAdd(sum + (size_t)cr * C + c, (unsigned long long)sm);
                    cr = lab[j];
                    sm = 0;
                }
                sm += v[j];   // 0 past the end
            }
            const unsigned st = __reduce_add_sync(grp, sm);   // <= 32 * 8 * 65535
            if (lead) atomicAdd(sum + (size_t)cur * C + c, (unsigned long long)st);
        }
    }
}

__global__ void __launch_bounds__(NTHR) k_dir_keys(const Edge *__restrict__ e, int E, int s,
                                                   unsigned long long *key, uint32_t *val)
{
    for (int i = blockIdx.x * NTHR + threadIdx.x; i < E; i += gridDim.x * NTHR) {
        const Edge ed = e[i];
        const unsigned long long a = (unsigned)ed.a, b = (unsigned)ed.b;
        key[2 * i] = a << s | b;
        key[2 * i + 1] = b << s | a;
        val[2 * i] = ed.h;
        val[2 * i + 1] = ed.h;
    }
}

// Digit counts of one 4096-key tile, digit-major: hist[d * ntl + tile].
__global__ void __launch_bounds__(NTHR) k_radix_hist(const unsigned long long *__restrict__ key, int n, int shift,
                                                     int ntl, int32_t *hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * RT;
#pragma unroll 4
    for (int j = 0; j < RPT; j++) {
        const int i = t0 + j * NTHR + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(int)(key[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[threadIdx.x * ntl + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: warp w of the tile owns keys [w*512, w*512+512) in 16 rounds
// of 32; a key's destination is the scanned offset of (digit, tile), plus the
// keys of that digit in the tile's earlier warps, earlier rounds of its warp
// and lower lanes of its round -- i.e. its rank in index order.
__global__ void __launch_bounds__(NTHR) k_radix_scatter(const unsigned long long *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin, int n, int shift, int ntl,
                                                        const int32_t *__restrict__ hist,
                                                        unsigned long long *__restrict__ kout,
                                                        uint32_t *__restrict__ vout)
{
    constexpr int NW = NTHR / 32;
    __shared__ int wcnt[NW][256];
    __shared__ int gofs[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < NW * 256; d += NTHR) (&wcnt[0][0])[d] = 0;
    gofs[threadIdx.x] = hist[threadIdx.x * ntl + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int i0 = blockIdx.x * RT + w * (RT / NW);
    unsigned long long k[RPT];
    int rk[RPT];
#pragma unroll
    for (int r = 0; r < RPT; r++) {
        const int i = i0 + r * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? kin[i] : 0ull;
        const int d = valid ? (int)(k[r] >> shift) & 255 : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int base = 0;
        if (valid) base = wcnt[w][d];
        rk[r] = base + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[w][d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive prefix over the warps, per digit
        const int d = threadIdx.x;
        int run = 0;
        for (int q = 0; q < NW; q++) {
            const int c = wcnt[q][d];
            wcnt[q][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; r++) {
        const int i = i0 + r * 32 + lane;
        if (i < n) {
            const int d = (int)(k[r] >> shift) & 255;
            const int pos = gofs[d] + wcnt[w][d] + rk[r];
            kout[pos] = k[r];
            vout[pos] = vin[i];
        }
    }
}

// row[r] = first sorted entry of row r (row[K] = n): entry i starts every row
// after the previous entry's row up to its own.
__global__ void __launch_bounds__(NTHR) k_csr_rows(const unsigned long long *__restrict__ key, int n, int s, int K,
                                                   int32_t *row)
{
    for (int i = blockIdx.x * NTHR + threadIdx.x; i <= n; i += gridDim.x * NTHR) {
        const long long cur = i < n ? (long long)(key[i] >> s) : (long long)K;
        const long long prev = i > 0 ? (long long)(key[i - 1] >> s) : -1;
        for (long long r = prev + 1; r <= cur && r <= K; r++) row[r] = i;
    }
}

__global__ void __launch_bounds__(NTHR) k_csr_out(const int32_t *__restrict__ row, int K,
                                                  const unsigned long long *__restrict__ key,
                                                  const uint32_t *__restrict__ val, int n, int s,
                                                  const unsigned long long *__restrict__ size,
                                                  const unsigned long long *__restrict__ sum, int C,
                                                  int64_t *row_ptr, int32_t *col, uint32_t *pass, int64_t *size_out,
                                                  uint64_t *sum_out, double *mean)
{
    const unsigned long long cmask = (1ull << s) - 1ull;
    const long long gs = (long long)gridDim.x * NTHR;
    const long long t = (long long)blockIdx.x * NTHR + threadIdx.x;
    if (row_ptr)
        for (long long r = t; r <= K; r += gs) row_ptr[r] = row[r];
    for (long long i = t; i < n; i += gs) {
        if (col) col[i] = (int32_t)(key[i] & cmask);
        if (pass) pass[i] = val[i];
    }
    if (size_out)
        for (long long r = t; r < K; r += gs) size_out[r] = (int64_t)size[r];
    const long long ns = (long long)K * C;
    for (long long j = t; j < ns; j += gs) {
        if (sum_out) sum_out[j] = sum[j];
        if (mean) {
            const unsigned long long z = size[j / C];
            mean[j] = z ? (double)sum[j] / (double)z : 0.0;
        }
    }
}

int grid_for(const ws_context *c, long long work)
{
    long long g = (work + NTHR - 1) / NTHR;
    const long long cap = (long long)c->num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <typename T, int CONN> void launch_rag(ws_context *c, const void *grad, const Geo &geo, const int32_t *L,
                                                cudaStream_t s)
{
    Workspace &w = c->w;
    k_rag<T, CONN><<<grid_for(c, geo.N), NTHR, 0, s>>>((const T *)grad, geo, L, w.keys, w.vals, w.slots, w.ecount,
                                                       (unsigned long long)(w.edge_cap - 1), c->status);
}

template <typename T> bool launch_rag_conn(ws_context *c, const void *grad, const Geo &geo, int conn,
                                           const int32_t *L, cudaStream_t s)
{
    switch (conn) {
    case 4: launch_rag<T, 4>(c, grad, geo, L, s); return true;
    case 8: launch_rag<T, 8>(c, grad, geo, L, s); return true;
    case 6: launch_rag<T, 6>(c, grad, geo, L, s); return true;
    case 26: launch_rag<T, 26>(c, grad, geo, L, s); return true;
    }
    return false;
}

}  // namespace

ws_status region_graph_build(ws_context *c, const int32_t *L, const void *grad, int dtype, const Geo &geo, int conn,
                             const void *values, int vdtype, int C, long long *Kout, long long *nnz_out,
                             cudaStream_t s)
{
    Workspace &w = c->w;
    Workspace::RGraph &r = w.rg;
    r.valid = 0;
    ws_status st;
    if ((st = ensure_rgraph(c, 1, 1, 1)) != WS_OK) return st;
    const long long N = geo.N;
    int32_t h[4] = {0, 0, 0, 0};
    cudaError_t e;
    {
        PhaseScope ps(c, PH_EXPORT, s);
        e = cudaMemsetAsync(r.misc, 0, 16, s);
        if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
        k_label_range<<<grid_for(c, N), NTHR, 0, s>>>(L, N, r.misc);
        c->launches += 1;
        e = cudaMemcpyAsync(h, r.misc, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_cuda_error(c, e, "label range");
    }
    if (h[1]) return set_error_msg(c, WS_ERR_INVALID, "labels must be >= 0");
    const long long K = (long long)h[0] + 1;
    if (K > N) return set_error_msg(c, WS_ERR_INVALID, "label ids must be below the pixel count");
    // region table: the same sizing as the waterfall's (load factor <= 1/2)
    if ((st = ensure_edges(c, edge_slots((size_t)N, conn, c), s)) != WS_OK) return st;
    if ((st = ensure_rgraph(c, (size_t)K, (size_t)K * C, 1)) != WS_OK) return st;
    {
        PhaseScope ps(c, PH_EXPORT, s);
        k_put_int<<<1, 32, 0, s>>>(r.misc + 3, (int)K);   // the id bound of k_edges_compact
        e = cudaMemsetAsync(r.size, 0, (size_t)K * 8, s);
        if (e == cudaSuccess && C > 0) e = cudaMemsetAsync(r.sum, 0, (size_t)K * C * 8, s);
        if (e != cudaSuccess) return set_cuda_error(c, e, "memset");
        const bool vec = ((uintptr_t)L & 15) == 0 && ((uintptr_t)values & 15) == 0 && N % SPIX == 0;
        const int sg = grid_for(c, (N + SPIX - 1) / SPIX);
        if (vdtype == WS_U16) {
            const uint16_t *vv = (const uint16_t *)values;
            if (vec) k_region_stats<uint16_t, true><<<sg, NTHR, 0, s>>>(L, vv, N, C, r.size, r.sum);
            else k_region_stats<uint16_t, false><<<sg, NTHR, 0, s>>>(L, vv, N, C, r.size, r.sum);
        } else {
            const uint8_t *vv = (const uint8_t *)values;
            if (vec) k_region_stats<uint8_t, true><<<sg, NTHR, 0, s>>>(L, vv, N, C, r.size, r.sum);
            else k_region_stats<uint8_t, false><<<sg, NTHR, 0, s>>>(L, vv, N, C, r.size, r.sum);
        }
        const bool ok = dtype == WS_U16 ? launch_rag_conn<uint16_t>(c, grad, geo, conn, L, s)
                                        : launch_rag_conn<uint8_t>(c, grad, geo, conn, L, s);
        if (!ok) return set_error_msg(c, WS_ERR_UNSUPPORTED, "connectivity");
        k_edges_compact<<<c->num_sms * 8, NTHR, 0, s>>>(w.keys, w.vals, w.slots, w.ecount, nullptr, r.misc + 3,
                                                        (Edge *)w.ea, nullptr, c->status);
        k_edges_reset<<<1, 32, 0, s>>>(w.ecount, r.misc + 2, 1);
        c->launches += 5;
        e = cudaMemcpyAsync(h + 2, r.misc + 2, 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return set_cuda_error(c, e, "edge count");
    }
    if ((st = ws_context_check(c, (ws_stream_t)s)) != WS_OK) return st;  // synchronises; table full, ...
    const long long E = h[2];
    const long long n = 2 * E;
    if (n >= 0x7fffffffLL) return set_error_msg(c, WS_ERR_UNSUPPORTED, "more than 2^30 region pairs");
    if ((st = ensure_rgraph(c, (size_t)K, (size_t)K * C, (size_t)(n > 0 ? n : 1))) != WS_OK) return st;
    int sh = 1;
    while ((1LL << sh) < K) sh++;
    int cur = 0;
    {
        PhaseScope ps(c, PH_EXPORT, s);
        if (n > 0) {
            k_dir_keys<<<grid_for(c, E), NTHR, 0, s>>>((const Edge *)w.ea, (int)E, sh, r.key[0], r.val[0]);
            c->launches += 1;
            const int ntl = (int)((n + RT - 1) / RT);
            const int m = 256 * ntl;
            const int nch = (m + SCAN_CHUNK - 1) / SCAN_CHUNK;
            for (int shift = 0; shift < 2 * sh; shift += 8) {
                k_radix_hist<<<ntl, NTHR, 0, s>>>(r.key[cur], (int)n, shift, ntl, r.hist);
                k_scan_chunks<<<nch, NTHR, 0, s>>>(r.hist, m, r.hsum);
                if (nch > 1) {   // one chunk is already scanned
                    k_scan<<<1, 1024, 0, s>>>(r.hsum, nch, nullptr);
                    k_scan_add<<<nch, NTHR, 0, s>>>(r.hist, m, r.hsum);
                    c->launches += 2;
                }
                k_radix_scatter<<<ntl, NTHR, 0, s>>>(r.key[cur], r.val[cur], (int)n, shift, ntl, r.hist,
                                                     r.key[cur ^ 1], r.val[cur ^ 1]);
                c->launches += 3;
                cur ^= 1;
            }
        }
        k_csr_rows<<<grid_for(c, n + 1), NTHR, 0, s>>>(r.key[cur], (int)n, sh, (int)K, r.row);
        c->launches += 1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(c, e, "region graph launch");
    r.K = K;
    r.nnz = n;
    r.C = C;
    r.sorted = cur;
    r.shift = sh;
    r.valid = 1;
    if (Kout) *Kout = K;
    if (nnz_out) *nnz_out = n;
    return WS_OK;
}

ws_status region_graph_read(ws_context *c, int64_t *row_ptr, int32_t *col, uint32_t *pass, int64_t *size,
                            uint64_t *sum, double *mean, cudaStream_t s)
{
    const Workspace::RGraph &r = c->w.rg;
    if (!r.valid) return set_error_msg(c, WS_ERR_INVALID, "no region graph has been built in this context");
    long long work = r.nnz > r.K + 1 ? r.nnz : r.K + 1;
    if (r.K * r.C > work) work = r.K * r.C;
    PhaseScope ps(c, PH_EXPORT, s);
    k_csr_out<<<grid_for(c, work), NTHR, 0, s>>>(r.row, (int)r.K, r.key[r.sorted], r.val[r.sorted], (int)r.nnz,
                                                 r.shift, r.size, r.sum, r.C, row_ptr, col, pass, size, sum, mean);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WS_OK : set_cuda_error(c, e, "region graph read");
}

}  // namespace ws
