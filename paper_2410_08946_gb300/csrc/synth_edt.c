/*
 * synth_edt.c -- seeded synthetic 3D input: distance to the nearest of a set
 * of seed points, scaled to 16 bits, plus uniform integer noise.
 *
 * This is an INPUT GENERATOR, not part of the watershed method: it holds none
 * of the method's arithmetic and is used identically by the tests, the bench
 * and the oracle's callers.  Output definition (all integer, exact):
 *
 *   d2(v)   = min over seeds s of |v - s|^2           (exact squared EDT)
 *   base(v) = floor(sqrt(floor(d2(v) * 65535^2 / d2max)))   (d2max = max d2)
 *   out(v)  = min(65535, base(v) + noise(v)),  noise(v) = splitmix64(key + v) % 65
 *
 * The EDT is the separable lower-envelope method of Felzenszwalb and
 * Huttenlocher ("Distance Transforms of Sampled Functions", 2012), run along
 * x, then y, then z; lines are split across POSIX threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_INF 0x3fffffffu

static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* floor(sqrt(v)) for v < 2^62, by the digit-by-digit binary method */
static uint64_t isqrt64(uint64_t v)
{
    uint64_t res = 0, bit = (uint64_t)1 << 62;
    while (bit > v) bit >>= 2;
    while (bit) {
        if (v >= res + bit) {
            v -= res + bit;
            res = (res >> 1) + bit;
        } else {
            res >>= 1;
        }
        bit >>= 2;
    }
    return res;
}

/* 1D squared distance transform of f[0..n) into d[0..n); scratch v, z. */
static void dt1d(const uint32_t *f, uint32_t *d, int64_t n, int64_t *v, double *z)
{
    int64_t k = 0;
    int64_t first = -1;
    for (int64_t q = 0; q < n; q++)
        if (f[q] < SYN_INF) {
            first = q;
            break;
        }
    if (first < 0) {
        for (int64_t q = 0; q < n; q++) d[q] = SYN_INF;
        return;
    }
    v[0] = first;
    z[0] = -INFINITY;
    z[1] = INFINITY;
    for (int64_t q = first + 1; q < n; q++) {
        if (f[q] >= SYN_INF) continue; /* not a parabola */
        double s;
        for (;;) { /* z[0] = -inf, so k never drops below 0 */
            int64_t r = v[k];
            s = ((double)f[q] + (double)q * q - (double)f[r] - (double)r * r) / (2.0 * (double)(q - r));
            if (s > z[k]) break;
            k--;
        }
        k++;
        v[k] = q;
        z[k] = s;
        z[k + 1] = INFINITY;
    }
    k = 0;
    for (int64_t q = 0; q < n; q++) {
        while (z[k + 1] < (double)q) k++;
        int64_t r = v[k];
        uint64_t val = (uint64_t)f[r] + (uint64_t)((q - r) * (q - r));
        d[q] = val >= SYN_INF ? SYN_INF : (uint32_t)val;
    }
}

typedef struct {
    uint32_t *buf;
    int64_t W, H, D;
    int axis;
    int64_t l0, l1; /* line range */
} job_t;

static void *run_lines(void *arg)
{
    job_t *j = (job_t *)arg;
    int64_t n = j->axis == 0 ? j->W : (j->axis == 1 ? j->H : j->D);
    uint32_t *f = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int64_t *v = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    for (int64_t l = j->l0; l < j->l1; l++) {
        int64_t base, stride;
        if (j->axis == 0) { /* lines along x: l = z*H + y */
            base = l * j->W;
            stride = 1;
        } else if (j->axis == 1) { /* lines along y: l = z*W + x */
            int64_t zz = l / j->W, xx = l % j->W;
            base = zz * j->H * j->W + xx;
            stride = j->W;
        } else { /* lines along z: l = y*W + x */
            base = l;
            stride = j->W * j->H;
        }
        for (int64_t i = 0; i < n; i++) f[i] = j->buf[base + i * stride];
        dt1d(f, d, n, v, z);
        for (int64_t i = 0; i < n; i++) j->buf[base + i * stride] = d[i];
    }
    free(f);
    free(d);
    free(v);
    free(z);
    return NULL;
}

static void pass(uint32_t *buf, int64_t W, int64_t H, int64_t D, int axis, int nthreads)
{
    int64_t lines = axis == 0 ? H * D : (axis == 1 ? W * D : W * H);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].buf = buf;
        jobs[t].W = W;
        jobs[t].H = H;
        jobs[t].D = D;
        jobs[t].axis = axis;
        jobs[t].l0 = lines * t / nthreads;
        jobs[t].l1 = lines * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, run_lines, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* Exact squared EDT of the seed set into d2 (uint32, W*H*D). */
int synth_edt3d(int64_t W, int64_t H, int64_t D, const int64_t *seeds, int64_t nseeds,
                uint32_t *d2, int nthreads)
{
    int64_t N = W * H * D;
    for (int64_t i = 0; i < N; i++) d2[i] = SYN_INF;
    for (int64_t s = 0; s < nseeds; s++) {
        int64_t x = seeds[3 * s], y = seeds[3 * s + 1], z = seeds[3 * s + 2];
        if (x < 0 || x >= W || y < 0 || y >= H || z < 0 || z >= D) return -1;
        d2[(z * H + y) * W + x] = 0;
    }
    pass(d2, W, H, D, 0, nthreads);
    pass(d2, W, H, D, 1, nthreads);
    pass(d2, W, H, D, 2, nthreads);
    return 0;
}

typedef struct {
    const uint32_t *d2;
    uint16_t *out;
    int64_t i0, i1;
    uint64_t d2max, key;
    int noise_levels;
    uint64_t local_max;
} conv_t;

static void *run_max(void *arg)
{
    conv_t *c = (conv_t *)arg;
    uint64_t m = 0;
    for (int64_t i = c->i0; i < c->i1; i++)
        if (c->d2[i] > m) m = c->d2[i];
    c->local_max = m;
    return NULL;
}

static void *run_convert(void *arg)
{
    conv_t *c = (conv_t *)arg;
    const uint64_t full = 65535ull * 65535ull;
    for (int64_t i = c->i0; i < c->i1; i++) {
        uint64_t base = isqrt64((uint64_t)c->d2[i] * full / c->d2max);
        uint64_t nz = c->noise_levels > 0 ? splitmix64(c->key + (uint64_t)i) % (uint64_t)c->noise_levels : 0;
        uint64_t v = base + nz;
        c->out[i] = (uint16_t)(v > 65535 ? 65535 : v);
    }
    return NULL;
}

/* Full volume generator (definition at the top of this file). */
int synth_distance_volume(int64_t W, int64_t H, int64_t D, const int64_t *seeds, int64_t nseeds,
                          uint64_t noise_key, int noise_levels, uint16_t *out, int nthreads)
{
    int64_t N = W * H * D;
    uint32_t *d2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    if (!d2) return -2;
    int rc = synth_edt3d(W, H, D, seeds, nseeds, d2, nthreads);
    if (rc) {
        free(d2);
        return rc;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    conv_t jobs[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].d2 = d2;
        jobs[t].out = out;
        jobs[t].i0 = N * t / nthreads;
        jobs[t].i1 = N * (t + 1) / nthreads;
        jobs[t].key = noise_key;
        jobs[t].noise_levels = noise_levels;
        pthread_create(&th[t], NULL, run_max, &jobs[t]);
    }
    uint64_t d2max = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        if (jobs[t].local_max > d2max) d2max = jobs[t].local_max;
    }
    if (d2max == 0) d2max = 1;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].d2max = d2max;
        pthread_create(&th[t], NULL, run_convert, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(d2);
    return 0;
}
