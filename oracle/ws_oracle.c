/*
 * ws_oracle.c -- sequential CPU oracle for the watershed (steps I-IV) and the
 * graph-form waterfall of "Parallel Watershed Partitioning: GPU-Based
 * Hierarchical Image Segmentation" (Yeghiazaryan, Gabrielyan, Voiculescu,
 * arXiv 2410.08946).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and it never calls into it.
 *
 * Style: plain, single-threaded, obviously-correct C.  Each function computes
 * the *defined* result directly (breadth-first search, root chasing, sorting)
 * rather than emulating the parallel iterations of the paper's kernels.
 *
 * Conventions (shared with the paper's statement of the problem, Sec. 3.1):
 *   - pixels are numbered in row-major order, x fastest:
 *       2D  p = y*W + x,     3D  p = (z*H + y)*W + x;
 *   - N(p) is the set of in-image pixels at unit distance (Sec. 3.1, the
 *     definition of the neighbourhood): no padding, no wrap-around;
 *   - connectivity 4 / 8 in 2D (von Neumann / Moore), 6 / 26 in 3D;
 *   - gradient samples are 8-bit (bytes_per_sample = 1) or 16-bit (2).
 *
 * Readings taken where the paper is silent (each repeated at its function):
 *   R1  empty neighbourhood (a 1x1 image): the pixel is a minimum (state 1);
 *   R2  step II pointer choice when several equal neighbours one step closer to
 *       the plateau border qualify: the one with the largest index, mirroring
 *       the tie-break of Eq. 1;
 *   R3  labels are canonical: region ids 0..K-1 ordered by each region's
 *       smallest pixel index;
 *   R4  the waterfall is the graph form: level k+1 joins every pair of level-k
 *       regions whose lowest pass (Alg. 5 step V) is the lowest pass of one of
 *       the two; NL counts level 0 (Sec. 4, the NL definition).
 *   R12 the 3D gradient: the 2D operators of orc_gradient2d extended to a
 *       third axis (the paper names no operator for volumes either);
 *   R11 the paper-literal waterfall (Alg. 4 with Alg. 5's reconstruction):
 *       the constant M of step V is the sample type's maximum (255 / 65535),
 *       so a region without neighbours is raised to that maximum;
 *   R10 the region graph handed to a graph network (Sec. 6, waterfall regions
 *       in place of superpixels): one node per region id 0..K-1 of a labelling,
 *       an edge between two regions exactly when a pixel of one has a pixel of
 *       the other in N(p), weighted by pass(A,B) of Alg. 5 step V; node
 *       features are the pixel count and, per channel of a value image, the sum
 *       and the mean (sum / count; 0 for an id no pixel carries).
 *
 * Parity pins (tests/test_oracle_*.py): the worked examples of Sec. 3.3 and
 * Sec. 3.4 (tests/golden/), exhaustive tiny images against a literal
 * simulation of Alg. 1 / Alg. 3 and against Floyd-Warshall distances, the
 * 1D property of Sec. 3.1, invariants, closed forms for the gradient.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* ------------------------------------------------------------------------ */
/* image geometry                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t W, H, D;   /* D = 1 for 2D images */
    int64_t N;
    int conn;
    /* neighbour offsets (dx, dy, dz) of the chosen connectivity */
    int noff;
    int off[26][3];
} geom_t;

static int geom_init(geom_t *g, int ndim, const int64_t *dims, int conn)
{
    if (ndim != 2 && ndim != 3) return ORC_EINVAL;
    g->W = dims[0];
    g->H = dims[1];
    g->D = (ndim == 3) ? dims[2] : 1;
    if (g->W < 1 || g->H < 1 || g->D < 1) return ORC_EINVAL;
    g->N = g->W * g->H * g->D;
    g->conn = conn;
    g->noff = 0;
    if (ndim == 2 && conn != 4 && conn != 8) return ORC_EINVAL;
    if (ndim == 3 && conn != 6 && conn != 26) return ORC_EINVAL;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int l1 = abs(dx) + abs(dy) + abs(dz);
                if (l1 == 0) continue;
                if (ndim == 2 && dz != 0) continue;
                /* von Neumann: unit L1 distance; Moore: unit L-infinity distance */
                if ((conn == 4 || conn == 6) && l1 != 1) continue;
                g->off[g->noff][0] = dx;
                g->off[g->noff][1] = dy;
                g->off[g->noff][2] = dz;
                g->noff++;
            }
    return ORC_OK;
}

/* Writes the in-image neighbours of p into nb[] and returns how many. */
static int neighbours(const geom_t *g, int64_t p, int64_t *nb)
{
    int64_t x = p % g->W;
    int64_t y = (p / g->W) % g->H;
    int64_t z = p / (g->W * g->H);
    int n = 0;
    for (int i = 0; i < g->noff; i++) {
        int64_t xx = x + g->off[i][0], yy = y + g->off[i][1], zz = z + g->off[i][2];
        if (xx < 0 || xx >= g->W || yy < 0 || yy >= g->H || zz < 0 || zz >= g->D) continue;
        nb[n++] = (zz * g->H + yy) * g->W + xx;
    }
    return n;
}

static inline uint32_t sample(const void *img, int bps, int64_t p)
{
    return bps == 1 ? ((const uint8_t *)img)[p] : ((const uint16_t *)img)[p];
}

/* ------------------------------------------------------------------------ */
/* exact integer square root, classical digit-by-digit (binary) method        */
/* ------------------------------------------------------------------------ */

uint32_t orc_isqrt_u64(uint64_t v)
{
    uint64_t res = 0;
    uint64_t bit = (uint64_t)1 << 62;
    while (bit > v) bit >>= 2;
    while (bit != 0) {
        if (v >= res + bit) {
            v -= res + bit;
            res = (res >> 1) + bit;
        } else {
            res >>= 1;
        }
        bit >>= 2;
    }
    return (uint32_t)res;
}

/* ------------------------------------------------------------------------ */
/* a0: gradient magnitude of a smoothed 2D image                              */
/* ------------------------------------------------------------------------ */

static inline int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/*
 * Pipeline steps 1-2 of Sec. 1 (smooth minimally, then take the gradient
 * magnitude; Fig. 2 marks both optional).  The paper names no operators, so
 * the ones used are: 5x5 binomial blur [1 4 6 4 1] x [1 4 6 4 1] with
 * round-half-up (sum + 128) >> 8, 3x3 integer Sobel, exact floor square root
 * of gx^2 + gy^2, clipped to 255, then shifted right by quant_shift (a
 * monotone quantisation).  Borders replicate the edge pixel.
 * Parity pinned by closed forms (ramps, impulses, symmetry) only.
 */
int orc_gradient2d(const uint8_t *img, int64_t W, int64_t H, int quant_shift, uint8_t *grad)
{
    static const int w[5] = {1, 4, 6, 4, 1};
    if (W < 1 || H < 1 || quant_shift < 0 || quant_shift > 7) return ORC_EINVAL;
    int32_t *blur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(W * H));
    if (!blur) return ORC_ENOMEM;
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
            int64_t s = 0;
            for (int i = -2; i <= 2; i++)
                for (int j = -2; j <= 2; j++)
                    s += (int64_t)w[i + 2] * w[j + 2] *
                         img[clampi(y + i, 0, H - 1) * W + clampi(x + j, 0, W - 1)];
            blur[y * W + x] = (int32_t)((s + 128) >> 8);
        }
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
#define B(yy, xx) ((int64_t)blur[clampi((yy), 0, H - 1) * W + clampi((xx), 0, W - 1)])
            int64_t gx = (B(y - 1, x + 1) + 2 * B(y, x + 1) + B(y + 1, x + 1)) -
                         (B(y - 1, x - 1) + 2 * B(y, x - 1) + B(y + 1, x - 1));
            int64_t gy = (B(y + 1, x - 1) + 2 * B(y + 1, x) + B(y + 1, x + 1)) -
                         (B(y - 1, x - 1) + 2 * B(y - 1, x) + B(y - 1, x + 1));
#undef B
            uint32_t mag = orc_isqrt_u64((uint64_t)(gx * gx + gy * gy));
            if (mag > 255) mag = 255;
            grad[y * W + x] = (uint8_t)(mag >> quant_shift);
        }
    free(blur);
    return ORC_OK;
}

/*
 * The same two steps for a volume (reading R12: the 3D counterparts of the
 * 2D operators): 5x5x5 binomial blur [1 4 6 4 1]^3 with round-half-up
 * (sum + 2048) >> 12, 3x3x3 Sobel (central difference [-1 0 1] along one axis,
 * [1 2 1] smoothing along the other two), exact floor square root of
 * gx^2 + gy^2 + gz^2, shifted right by shift and clipped to 65535.  Borders
 * replicate the edge voxel, for the blur and for the blurred volume.
 * img: bps = 1 or 2 bytes per voxel, [D][H][W]; grad: uint16 [D][H][W].
 */
int orc_gradient3d(const void *img, int bps, int64_t W, int64_t H, int64_t D, int shift, uint16_t *grad)
{
    static const int w[5] = {1, 4, 6, 4, 1};
    static const int sw[3] = {1, 2, 1};
    if (W < 1 || H < 1 || D < 1 || shift < 0 || shift > 31 || (bps != 1 && bps != 2)) return ORC_EINVAL;
    const int64_t N = W * H * D;
    int64_t *blur = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!blur) return ORC_ENOMEM;
#define IDX(z, y, x) ((clampi((z), 0, D - 1) * H + clampi((y), 0, H - 1)) * W + clampi((x), 0, W - 1))
    for (int64_t z = 0; z < D; z++)
        for (int64_t y = 0; y < H; y++)
            for (int64_t x = 0; x < W; x++) {
                int64_t acc = 0;
                for (int k = -2; k <= 2; k++)
                    for (int j = -2; j <= 2; j++)
                        for (int i = -2; i <= 2; i++)
                            acc += (int64_t)w[k + 2] * w[j + 2] * w[i + 2] *
                                   (int64_t)sample(img, bps, IDX(z + k, y + j, x + i));
                blur[(z * H + y) * W + x] = (acc + 2048) >> 12;
            }
    for (int64_t z = 0; z < D; z++)
        for (int64_t y = 0; y < H; y++)
            for (int64_t x = 0; x < W; x++) {
                int64_t gx = 0, gy = 0, gz = 0;
                for (int a = -1; a <= 1; a++)
                    for (int b = -1; b <= 1; b++) {
                        const int64_t wt = (int64_t)sw[a + 1] * sw[b + 1];
                        /* d/dx: (a, b) range over (z, y); d/dy: over (z, x); d/dz: over (y, x) */
                        gx += wt * (blur[IDX(z + a, y + b, x + 1)] - blur[IDX(z + a, y + b, x - 1)]);
                        gy += wt * (blur[IDX(z + a, y + 1, x + b)] - blur[IDX(z + a, y - 1, x + b)]);
                        gz += wt * (blur[IDX(z + 1, y + a, x + b)] - blur[IDX(z - 1, y + a, x + b)]);
                    }
                uint64_t mag = orc_isqrt_u64((uint64_t)(gx * gx + gy * gy + gz * gz)) >> shift;
                grad[(z * H + y) * W + x] = (uint16_t)(mag > 65535 ? 65535 : mag);
            }
#undef IDX
    free(blur);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* step I: states and arrows (Alg. 1 step I, Eq. 1)                           */
/* ------------------------------------------------------------------------ */

/*
 * q = the neighbour of lowest value, the largest index among equal lowest
 * values (Eq. 1).  State 0: q is lower than p (arrow p -> q).  State 1: every
 * neighbour is higher (p is a strict minimum; arrow p -> p).  State 2: q has
 * the same value and a larger index (arrow p -> q).  State 3: q has the same
 * value and a smaller index (arrow p -> p).  Reading R1: an empty
 * neighbourhood makes p a minimum.
 */
int orc_step1(const void *grad, int bps, int ndim, const int64_t *dims, int conn,
              uint8_t *S, int32_t *L)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2)) return ORC_EINVAL;
    int64_t nb[26];
    for (int64_t p = 0; p < g.N; p++) {
        int n = neighbours(&g, p, nb);
        int64_t q = -1;
        uint32_t m = 0;
        for (int i = 0; i < n; i++) {
            uint32_t v = sample(grad, bps, nb[i]);
            if (q < 0 || v < m || (v == m && nb[i] > q)) {
                m = v;
                q = nb[i];
            }
        }
        uint32_t gp = sample(grad, bps, p);
        if (q < 0 || m > gp) {
            S[p] = 1;
            L[p] = (int32_t)p;
        } else if (m < gp) {
            S[p] = 0;
            L[p] = (int32_t)q;
        } else if (q > p) {
            S[p] = 2;
            L[p] = (int32_t)q;
        } else {
            S[p] = 3;
            L[p] = (int32_t)p;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* plateaux: connected components of equal value                              */
/* ------------------------------------------------------------------------ */

/* comp[p] = index of the smallest pixel of p's plateau (the connected set of
 * equal-valued pixels containing p, Sec. 3.1 state description).  BFS. */
static int plateau_components(const geom_t *g, const void *grad, int bps, int64_t *comp)
{
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)g->N);
    if (!queue) return ORC_ENOMEM;
    for (int64_t p = 0; p < g->N; p++) comp[p] = -1;
    int64_t nb[26];
    for (int64_t s = 0; s < g->N; s++) {
        if (comp[s] >= 0) continue;
        uint32_t v = sample(grad, bps, s);
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        comp[s] = s; /* s is the first unvisited pixel, hence the smallest */
        while (head < tail) {
            int64_t p = queue[head++];
            int n = neighbours(g, p, nb);
            for (int i = 0; i < n; i++) {
                int64_t q = nb[i];
                if (comp[q] < 0 && sample(grad, bps, q) == v) {
                    comp[q] = s;
                    queue[tail++] = q;
                }
            }
        }
    }
    free(queue);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* step II: distances inside non-minimal plateaux                             */
/* ------------------------------------------------------------------------ */

/*
 * Alg. 1 step II (synchronous, with the S' buffer of Sec. 3.3) turns a
 * plateau pixel into state 0 at the iteration equal to its distance from the
 * pixels of its plateau that have a lower neighbour; Alg. 3 stores the same
 * distance as -S at its fixpoint (the 14x1 example of Sec. 3.4).  This
 * function computes that distance directly: a multi-source BFS over
 * equal-valued neighbours, sources = the state-0 pixels, reaching only
 * pixels of state >= 2.
 *   dist[p] = 0           if S[p] == 0
 *   dist[p] = BFS length  if S[p] >= 2 and p is reached (non-minimal plateau)
 *   dist[p] = -1          otherwise (state 1, or a minimal plateau)
 */
int orc_plateau_distance(const void *grad, int bps, int ndim, const int64_t *dims, int conn,
                         const uint8_t *S, int32_t *dist)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2)) return ORC_EINVAL;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)g.N);
    if (!queue) return ORC_ENOMEM;
    int64_t head = 0, tail = 0;
    for (int64_t p = 0; p < g.N; p++) {
        dist[p] = (S[p] == 0) ? 0 : -1;
        if (S[p] == 0) queue[tail++] = p;
    }
    int64_t nb[26];
    while (head < tail) {
        int64_t p = queue[head++];
        uint32_t v = sample(grad, bps, p);
        int n = neighbours(&g, p, nb);
        for (int i = 0; i < n; i++) {
            int64_t q = nb[i];
            if (S[q] >= 2 && dist[q] < 0 && sample(grad, bps, q) == v) {
                dist[q] = dist[p] + 1;
                queue[tail++] = q;
            }
        }
    }
    free(queue);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* canonical relabelling (reading R3)                                         */
/* ------------------------------------------------------------------------ */

/* Rewrites raw[] (arbitrary ids in [0, idspace)) into 0..K-1 in order of first
 * appearance in a row-major scan, i.e. ordered by each region's smallest
 * pixel index.  Returns K, or a negative error. */
static int64_t canonical_relabel(int64_t N, const int64_t *raw, int64_t idspace, int32_t *out)
{
    int64_t *map = (int64_t *)malloc(sizeof(int64_t) * (size_t)(idspace > 0 ? idspace : 1));
    if (!map) return ORC_ENOMEM;
    for (int64_t i = 0; i < idspace; i++) map[i] = -1;
    int64_t K = 0;
    for (int64_t p = 0; p < N; p++) {
        if (map[raw[p]] < 0) map[raw[p]] = K++;
        out[p] = (int32_t)map[raw[p]];
    }
    free(map);
    return K;
}

/* ------------------------------------------------------------------------ */
/* W0: the watershed, steps I-IV                                              */
/* ------------------------------------------------------------------------ */

/*
 * labels[p] = canonical id of p's catchment basin; *K = number of basins.
 * Optional debug outputs (may be NULL): S1 = states after step I, dist = step
 * II distances (orc_plateau_distance), ptr = arrows after step II (state-0
 * pixels point down their steepest descent or towards the plateau border;
 * minimal-plateau and minimum pixels keep their step I arrow).
 *
 * Steps:
 *   I    states and arrows (orc_step1, Eq. 1);
 *   II   each non-minimal plateau pixel (state >= 2, distance d > 0) points to
 *        an equal-valued neighbour at distance d-1; reading R2 takes the
 *        largest index among those;
 *   III  root(p) = the end of the arrow chain from p: a pixel whose arrow is a
 *        self-loop (state 1, or state 3 inside a minimal plateau), Sec. 3.1;
 *   IV   every pixel of one minimal plateau belongs to one basin (the
 *        Union-Find merge of Sec. 3.1), so basin(p) = the minimal plateau that
 *        contains root(p);
 *   then the canonical relabelling R3.
 */
int orc_watershed(const void *grad, int bps, int ndim, const int64_t *dims, int conn,
                  int32_t *labels, int32_t *K_out, uint8_t *S1_out, int32_t *dist_out,
                  int32_t *ptr_out)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2)) return ORC_EINVAL;
    if (g.N >= ((int64_t)1 << 31)) return ORC_EINVAL;
    int64_t N = g.N;
    int rc = ORC_ENOMEM;
    uint8_t *S = (uint8_t *)malloc((size_t)N);
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *comp = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!S || !L || !dist || !comp || !root || !stack) goto out;

    /* step I */
    orc_step1(grad, bps, ndim, dims, conn, S, L);
    if (S1_out) memcpy(S1_out, S, (size_t)N);

    /* step II */
    if ((rc = orc_plateau_distance(grad, bps, ndim, dims, conn, S, dist)) != ORC_OK) goto out;
    int64_t nb[26];
    for (int64_t p = 0; p < N; p++) {
        if (S[p] < 2 || dist[p] <= 0) continue;
        uint32_t v = sample(grad, bps, p);
        int n = neighbours(&g, p, nb);
        int64_t best = -1;
        for (int i = 0; i < n; i++) {
            int64_t q = nb[i];
            if (sample(grad, bps, q) == v && dist[q] == dist[p] - 1 && q > best) best = q;
        }
        /* a BFS predecessor always exists */
        L[p] = (int32_t)best;
    }
    for (int64_t p = 0; p < N; p++)
        if (S[p] >= 2 && dist[p] > 0) S[p] = 0;
    if (dist_out) memcpy(dist_out, dist, sizeof(int32_t) * (size_t)N);
    if (ptr_out) memcpy(ptr_out, L, sizeof(int32_t) * (size_t)N);

    /* step III: chase every arrow chain to its self-loop (memoised) */
    for (int64_t p = 0; p < N; p++) root[p] = -1;
    for (int64_t p = 0; p < N; p++) {
        if (root[p] >= 0) continue;
        int64_t top = 0, c = p;
        while (root[c] < 0 && L[c] != c) {
            stack[top++] = c;
            c = L[c];
        }
        int64_t r = (root[c] >= 0) ? root[c] : c;
        root[c] = r;
        while (top > 0) root[stack[--top]] = r;
    }

    /* step IV: basin = minimal plateau of the root */
    if ((rc = plateau_components(&g, grad, bps, comp)) != ORC_OK) goto out;
    for (int64_t p = 0; p < N; p++) stack[p] = comp[root[p]];
    int64_t K = canonical_relabel(N, stack, N, labels);
    if (K < 0) {
        rc = (int)K;
        goto out;
    }
    *K_out = (int32_t)K;
    rc = ORC_OK;
out:
    free(S);
    free(L);
    free(dist);
    free(comp);
    free(root);
    free(stack);
    return rc;
}

/* Steps I-III only (no minimal-plateau merge): raw root index per pixel.  Used
 * to check the 1D property of Sec. 3.1 (in 1D, I-III already give the
 * watershed). */
int orc_roots_without_merge(const void *grad, int bps, int ndim, const int64_t *dims, int conn,
                            int32_t *roots)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK) return ORC_EINVAL;
    int64_t N = g.N;
    int32_t *ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t K;
    if (!ptr || !lab) {
        free(ptr);
        free(lab);
        return ORC_ENOMEM;
    }
    int rc = orc_watershed(grad, bps, ndim, dims, conn, lab, &K, NULL, NULL, ptr);
    if (rc == ORC_OK) {
        for (int64_t p = 0; p < N; p++) {
            int64_t c = p;
            while (ptr[c] != c) c = ptr[c];
            roots[p] = (int32_t)c;
        }
    }
    free(ptr);
    free(lab);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* W: graph-form waterfall (reading R4)                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t a, b;
    uint32_t h;
} pair_t;

static int cmp_pair(const void *x, const void *y)
{
    const pair_t *u = (const pair_t *)x, *v = (const pair_t *)y;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    if (u->b != v->b) return u->b < v->b ? -1 : 1;
    if (u->h != v->h) return u->h < v->h ? -1 : 1;
    return 0;
}

static int64_t uf_find(int64_t *par, int64_t a)
{
    while (par[a] != a) a = par[a];
    return a;
}

/*
 * One waterfall level, from the pixels (Alg. 5 step V definitions):
 *   height(p,q) = max(G(p), G(q)) for adjacent p, q in different regions;
 *   pass(A,B)   = the smallest height over adjacent pixel pairs of A and B;
 *   newmin(A)   = min over B of pass(A,B)   (the lowest pass of A).
 * Level k+1 = connected components of the region graph that keeps (A,B)
 * exactly when pass(A,B) equals newmin(A) or newmin(B); then canonical
 * relabelling.  A region with no neighbour stays as it is.
 */
static int64_t waterfall_level(const geom_t *g, const void *grad, int bps, const int32_t *Lk,
                               int64_t Kk, int32_t *Lnext)
{
    int64_t N = g->N;
    int64_t cap = 1024, np = 0;
    pair_t *pairs = (pair_t *)malloc(sizeof(pair_t) * (size_t)cap);
    uint32_t *newmin = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(Kk > 0 ? Kk : 1));
    int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)(Kk > 0 ? Kk : 1));
    int64_t *raw = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t K = ORC_ENOMEM;
    if (!pairs || !newmin || !par || !raw) goto out;

    /* every unordered adjacent pixel pair once (q > p) */
    int64_t nb[26];
    for (int64_t p = 0; p < N; p++) {
        int n = neighbours(g, p, nb);
        for (int i = 0; i < n; i++) {
            int64_t q = nb[i];
            if (q <= p || Lk[p] == Lk[q]) continue;
            uint32_t gp = sample(grad, bps, p), gq = sample(grad, bps, q);
            if (np == cap) {
                cap *= 2;
                pair_t *t = (pair_t *)realloc(pairs, sizeof(pair_t) * (size_t)cap);
                if (!t) goto out;
                pairs = t;
            }
            pairs[np].a = Lk[p] < Lk[q] ? Lk[p] : Lk[q];
            pairs[np].b = Lk[p] < Lk[q] ? Lk[q] : Lk[p];
            pairs[np].h = gp > gq ? gp : gq;
            np++;
        }
    }
    /* pass(A,B): sort, keep the first (smallest h) record of each (A,B) */
    qsort(pairs, (size_t)np, sizeof(pair_t), cmp_pair);
    int64_t ne = 0;
    for (int64_t i = 0; i < np; i++)
        if (ne == 0 || pairs[ne - 1].a != pairs[i].a || pairs[ne - 1].b != pairs[i].b)
            pairs[ne++] = pairs[i];
    /* newmin */
    for (int64_t A = 0; A < Kk; A++) newmin[A] = UINT32_MAX;
    for (int64_t e = 0; e < ne; e++) {
        if (pairs[e].h < newmin[pairs[e].a]) newmin[pairs[e].a] = pairs[e].h;
        if (pairs[e].h < newmin[pairs[e].b]) newmin[pairs[e].b] = pairs[e].h;
    }
    /* components of the kept edges */
    for (int64_t A = 0; A < Kk; A++) par[A] = A;
    for (int64_t e = 0; e < ne; e++) {
        if (pairs[e].h != newmin[pairs[e].a] && pairs[e].h != newmin[pairs[e].b]) continue;
        int64_t ra = uf_find(par, pairs[e].a), rb = uf_find(par, pairs[e].b);
        if (ra != rb) par[ra > rb ? ra : rb] = ra < rb ? ra : rb;
    }
    for (int64_t p = 0; p < N; p++) raw[p] = uf_find(par, Lk[p]);
    K = canonical_relabel(N, raw, Kk, Lnext);
out:
    free(pairs);
    free(newmin);
    free(par);
    free(raw);
    return K;
}

/*
 * Hierarchy (Alg. 4, graph form): given level-0 labels L0 (canonical, K0
 * regions), writes levels 1..NL-1 into levels[(k-1)*N ...] and the region
 * count of every level 0..NL-1 into counts[].
 */
int orc_waterfall(const int32_t *L0, const void *grad, int bps, int ndim, const int64_t *dims,
                  int conn, int NL, int32_t *levels, int32_t *counts)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2) || NL < 1)
        return ORC_EINVAL;
    int64_t N = g.N;
    int64_t K0 = 0;
    for (int64_t p = 0; p < N; p++)
        if (L0[p] + 1 > K0) K0 = L0[p] + 1;
    counts[0] = (int32_t)K0;
    const int32_t *prev = L0;
    int64_t Kk = K0;
    for (int k = 1; k < NL; k++) {
        int32_t *cur = levels + (int64_t)(k - 1) * N;
        int64_t Kn = waterfall_level(&g, grad, bps, prev, Kk, cur);
        if (Kn < 0) return (int)Kn;
        counts[k] = (int32_t)Kn;
        prev = cur;
        Kk = Kn;
    }
    return ORC_OK;
}

/* Convenience: watershed + waterfall; levels holds NL planes (level 0 first). */
int orc_segment(const void *grad, int bps, int ndim, const int64_t *dims, int conn, int NL,
                int32_t *levels, int32_t *counts)
{
    if (NL < 1) return ORC_EINVAL;
    int32_t K;
    int rc = orc_watershed(grad, bps, ndim, dims, conn, levels, &K, NULL, NULL, NULL);
    if (rc != ORC_OK) return rc;
    geom_t g;
    geom_init(&g, ndim, dims, conn);
    return orc_waterfall(levels, grad, bps, ndim, dims, conn, NL, levels + g.N, counts);
}

/* ------------------------------------------------------------------------ */
/* G: region graph of one labelling (reading R10)                             */
/* ------------------------------------------------------------------------ */

/*
 * Region adjacency of the labelling L (ids in [0, K)) as a symmetric CSR:
 * row A lists, in increasing order, every region B != A with a pixel in N(p)
 * of a pixel p of A, and pass[] holds pass(A,B) = the smallest
 * max(G(p), G(q)) over those pixel pairs (Alg. 5 step V).  col/pass have room
 * for cap entries; *nnz_out gets the number written (twice the edges).
 * size[A] = pixels of A; with C > 0 channels of values (channel-major planes
 * of N samples, vbps bytes each), sum[A*C + c] and mean[A*C + c] =
 * sum / size (0 when size is 0).
 */
int orc_region_graph(const int32_t *L, const void *grad, int bps, int ndim, const int64_t *dims, int conn,
                     const void *values, int vbps, int C, int64_t K, int64_t *row_ptr, int32_t *col,
                     uint32_t *pass, int64_t cap, int64_t *nnz_out, int64_t *size, uint64_t *sum, double *mean)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2) || K < 1 || C < 0 ||
        (C > 0 && vbps != 1 && vbps != 2))
        return ORC_EINVAL;
    int64_t N = g.N;
    for (int64_t p = 0; p < N; p++)
        if (L[p] < 0 || L[p] >= K) return ORC_EINVAL;

    /* node features: plain counting */
    for (int64_t A = 0; A < K; A++) size[A] = 0;
    for (int64_t i = 0; i < K * C; i++) sum[i] = 0;
    for (int64_t p = 0; p < N; p++) {
        size[L[p]]++;
        for (int c = 0; c < C; c++) sum[(int64_t)L[p] * C + c] += sample(values, vbps, (int64_t)c * N + p);
    }
    for (int64_t A = 0; A < K; A++)
        for (int c = 0; c < C; c++)
            mean[A * C + c] = size[A] ? (double)sum[A * C + c] / (double)size[A] : 0.0;

    /* one record (L[p], L[q], max(G(p), G(q))) per ordered neighbour pair of
       different regions, so both directions of every edge are present */
    int64_t np = 0, pcap = 1024;
    pair_t *pairs = (pair_t *)malloc(sizeof(pair_t) * (size_t)pcap);
    if (!pairs) return ORC_ENOMEM;
    int64_t nb[26];
    for (int64_t p = 0; p < N; p++) {
        int n = neighbours(&g, p, nb);
        for (int i = 0; i < n; i++) {
            int64_t q = nb[i];
            if (L[p] == L[q]) continue;
            if (np == pcap) {
                pcap *= 2;
                pair_t *t = (pair_t *)realloc(pairs, sizeof(pair_t) * (size_t)pcap);
                if (!t) {
                    free(pairs);
                    return ORC_ENOMEM;
                }
                pairs = t;
            }
            uint32_t gp = sample(grad, bps, p), gq = sample(grad, bps, q);
            pairs[np].a = L[p];
            pairs[np].b = L[q];
            pairs[np].h = gp > gq ? gp : gq;
            np++;
        }
    }
    /* sorted by (A, B, height): the first record of each (A, B) holds pass(A,B) */
    qsort(pairs, (size_t)np, sizeof(pair_t), cmp_pair);
    for (int64_t A = 0; A <= K; A++) row_ptr[A] = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < np; i++) {
        if (i > 0 && pairs[i].a == pairs[i - 1].a && pairs[i].b == pairs[i - 1].b) continue;
        if (nnz == cap) {
            free(pairs);
            return ORC_ENOMEM;
        }
        col[nnz] = (int32_t)pairs[i].b;
        pass[nnz] = pairs[i].h;
        row_ptr[pairs[i].a + 1]++;
        nnz++;
    }
    for (int64_t A = 0; A < K; A++) row_ptr[A + 1] += row_ptr[A];
    *nnz_out = nnz;
    free(pairs);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* P: paper-literal waterfall by image reconstruction (reading R11)          */
/* ------------------------------------------------------------------------ */

/*
 * Hierarchy of Alg. 4 with the image reconstruction of Alg. 5: level 0 is the
 * watershed of I = G; while a next level is wanted,
 *   step V:  newmin(A) = the smallest height(p, q) = max(I(p), I(q)) over
 *            pixels p of A and neighbours q of p in another region (M, the
 *            sample type's maximum, when A has no such pair);
 *   step VI: I(p) = newmin(L(p)) wherever I(p) < newmin(L(p));
 * and level n+1 is the watershed of the raised image.  levels holds NL planes
 * (level 0 first), counts the region count of each.  Unlike the graph form,
 * a level need not be a union of regions of the level below.
 */
int orc_waterfall_reconstruct(const void *grad, int bps, int ndim, const int64_t *dims, int conn, int NL,
                              int32_t *levels, int32_t *counts)
{
    geom_t g;
    if (geom_init(&g, ndim, dims, conn) != ORC_OK || (bps != 1 && bps != 2) || NL < 1) return ORC_EINVAL;
    const int64_t N = g.N;
    const uint32_t M = bps == 1 ? 0xffu : 0xffffu;
    void *img = malloc((size_t)N * (size_t)bps);
    uint32_t *newmin = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    int rc = ORC_ENOMEM;
    if (!img || !newmin) goto out;
    memcpy(img, grad, (size_t)N * (size_t)bps);
    for (int n = 0; n < NL; n++) {
        int32_t *L = levels + (int64_t)n * N;
        int32_t K;
        rc = orc_watershed(img, bps, ndim, dims, conn, L, &K, NULL, NULL, NULL);
        if (rc != ORC_OK) goto out;
        counts[n] = K;
        if (n == NL - 1) break;
        /* step V */
        for (int64_t A = 0; A < K; A++) newmin[A] = M;
        int64_t nb[26];
        for (int64_t p = 0; p < N; p++) {
            int m = neighbours(&g, p, nb);
            for (int i = 0; i < m; i++) {
                int64_t q = nb[i];
                if (L[q] == L[p]) continue;
                uint32_t a = sample(img, bps, p), b = sample(img, bps, q);
                uint32_t h = a > b ? a : b;
                if (h < newmin[L[p]]) newmin[L[p]] = h;
            }
        }
        /* step VI */
        for (int64_t p = 0; p < N; p++) {
            uint32_t v = sample(img, bps, p);
            if (v < newmin[L[p]]) {
                if (bps == 1)
                    ((uint8_t *)img)[p] = (uint8_t)newmin[L[p]];
                else
                    ((uint16_t *)img)[p] = (uint16_t)newmin[L[p]];
            }
        }
    }
    rc = ORC_OK;
out:
    free(img);
    free(newmin);
    return rc;
}
