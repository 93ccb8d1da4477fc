/*
 * synth.c - seeded synthetic inputs shared by the CUDA path's tests/bench and the
 * FP64 oracle's tests.
 *
 * This module holds none of the membrane-classification arithmetic. It only makes
 * inputs: EM-like uint8 slices (a stand-in for the Kasthuri S1 stack the paper
 * measures on, Sec. 2 and Sec. 2.2) and He-normal network parameters.
 *
 * Generator recipe (one slice, every step seeded and deterministic):
 *   1. n cells: n = round(120 * H * W / 65536) uniform points in [0,W) x [0,H)
 *      (about 120 cells per 256x256 area).
 *   2. For each pixel centre, the nearest seed s1 and second-nearest s2
 *      (Euclidean; ties broken by the lower seed index).
 *   3. The pixel is membrane when its distance to the bisector of s1 and s2,
 *      (d2^2 - d1^2) / (2 |s1 - s2|), is below half a per-pair width drawn
 *      uniformly in [2, 3) from a hash of the (unordered) pair.
 *   4. Intensity: membrane N(60, 15^2), interior N(170, 20^2), iid per pixel.
 *   5. Separable Gaussian blur, sigma 1, radius 3, normalised taps,
 *      reflect-101 border.
 *   6. Round half to even, clip to [0, 255].
 * Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) for streams and
 * its output finaliser as a counter hash; normals by the Box-Muller transform.
 *
 * Compile with -ffp-contract=off so results do not depend on FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_OK 0
#define SYNTH_ERR_ARG 1
#define SYNTH_ERR_OOM 2

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t sm64_next(uint64_t* s) {
    *s += 0x9E3779B97F4A7C15ULL;
    return mix64(*s);
}

/* uniform in [0, 1) with 53 random bits */
static double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
/* uniform in (0, 1] */
static double u01_open0(uint64_t x) { return (double)((x >> 11) + 1) * 0x1.0p-53; }

static double box_muller(uint64_t a, uint64_t b) {
    const double two_pi = 6.283185307179586476925286766559;
    return sqrt(-2.0 * log(u01_open0(a))) * cos(two_pi * u01(b));
}

static double stream_normal(uint64_t* s) {
    uint64_t a = sm64_next(s);
    uint64_t b = sm64_next(s);
    return box_muller(a, b);
}

static int64_t refl101(int64_t t, int64_t n) {
    if (t < 0) t = -t;
    if (t >= n) t = 2 * (n - 1) - t;
    return t;
}

int64_t synth_default_cells(int64_t h, int64_t w) {
    double n = 120.0 * (double)h * (double)w / 65536.0;
    int64_t k = (int64_t)llround(n);
    return k < 2 ? 2 : k;
}

/* Seed of slice z of block b under base seed s: SplitMix64 finaliser of s ^ (b << 32) ^ z. */
uint64_t synth_slice_seed(uint64_t base, uint64_t block, uint64_t z) {
    return mix64(base ^ (block << 32) ^ z);
}

/*
 * One EM-like slice. out[y * pitch + x], 0 <= y < h, 0 <= x < w.
 * n_cells <= 0 selects the default density. Needs h, w >= 4 (blur radius 3).
 * truth (may be NULL): the generator's own membrane flag of step 3 per pixel (0/1, same layout),
 * i.e. the ground truth a membrane classifier is meant to recover.
 */
int synth_em_slice_truth(uint64_t seed, int64_t h, int64_t w, int64_t n_cells, uint8_t* out, int64_t pitch,
                         uint8_t* truth) {
    if (!out || h < 4 || w < 4 || pitch < w) return SYNTH_ERR_ARG;
    int64_t n = n_cells > 0 ? n_cells : synth_default_cells(h, w);
    if (n < 2) n = 2;

    double* px = (double*)malloc(sizeof(double) * (size_t)n);
    double* py = (double*)malloc(sizeof(double) * (size_t)n);
    double* img = (double*)malloc(sizeof(double) * (size_t)(h * w));
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(h * w));
    if (!px || !py || !img || !tmp) {
        free(px); free(py); free(img); free(tmp);
        return SYNTH_ERR_OOM;
    }
    uint64_t st = mix64(seed ^ 0x5EED5EED5EED5EEDULL);
    for (int64_t i = 0; i < n; ++i) {
        px[i] = u01(sm64_next(&st)) * (double)w;
        py[i] = u01(sm64_next(&st)) * (double)h;
    }

    /* bucket grid for the nearest-two search */
    int64_t G = (int64_t)sqrt((double)h * (double)w / (double)n);
    if (G < 8) G = 8;
    int64_t gx = (w + G - 1) / G, gy = (h + G - 1) / G;
    int64_t* bstart = (int64_t*)calloc((size_t)(gx * gy + 1), sizeof(int64_t));
    int64_t* bitems = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* bfill = (int64_t*)calloc((size_t)(gx * gy), sizeof(int64_t));
    if (!bstart || !bitems || !bfill) {
        free(px); free(py); free(img); free(tmp); free(bstart); free(bitems); free(bfill);
        return SYNTH_ERR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t bx = (int64_t)(px[i] / (double)G), by = (int64_t)(py[i] / (double)G);
        if (bx >= gx) bx = gx - 1;
        if (by >= gy) by = gy - 1;
        bstart[by * gx + bx + 1]++;
    }
    for (int64_t b = 0; b < gx * gy; ++b) bstart[b + 1] += bstart[b];
    for (int64_t i = 0; i < n; ++i) {
        int64_t bx = (int64_t)(px[i] / (double)G), by = (int64_t)(py[i] / (double)G);
        if (bx >= gx) bx = gx - 1;
        if (by >= gy) by = gy - 1;
        int64_t b = by * gx + bx;
        bitems[bstart[b] + bfill[b]++] = i; /* ascending index within a bucket */
    }

    const uint64_t noise_key = mix64(seed ^ 0x0123456789ABCDEFULL);
    const uint64_t width_key = mix64(seed ^ 0x0FEDCBA987654321ULL);

#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t y = 0; y < h; ++y) {
        for (int64_t x = 0; x < w; ++x) {
            double xc = (double)x + 0.5, yc = (double)y + 0.5;
            int64_t cx = x / G, cy = y / G;
            double b1 = INFINITY, b2 = INFINITY;
            int64_t i1 = -1, i2 = -1;
            int64_t rmax = gx > gy ? gx : gy;
            for (int64_t r = 0; r <= rmax; ++r) {
                for (int64_t by = cy - r; by <= cy + r; ++by) {
                    if (by < 0 || by >= gy) continue;
                    for (int64_t bx = cx - r; bx <= cx + r; ++bx) {
                        if (bx < 0 || bx >= gx) continue;
                        int64_t ax = bx - cx < 0 ? cx - bx : bx - cx;
                        int64_t ay = by - cy < 0 ? cy - by : by - cy;
                        if ((ax > ay ? ax : ay) != r) continue;
                        int64_t b = by * gx + bx;
                        for (int64_t k = bstart[b]; k < bstart[b + 1]; ++k) {
                            int64_t i = bitems[k];
                            double dx = px[i] - xc, dy = py[i] - yc;
                            double d = dx * dx + dy * dy;
                            if (d < b1 || (d == b1 && i < i1)) {
                                b2 = b1; i2 = i1; b1 = d; i1 = i;
                            } else if (d < b2 || (d == b2 && i < i2)) {
                                b2 = d; i2 = i;
                            }
                        }
                    }
                }
                double lim = (double)(r * G);
                if (i2 >= 0 && b2 < lim * lim) break;
            }
            double sx = px[i1] - px[i2], sy = py[i1] - py[i2];
            double sep = sqrt(sx * sx + sy * sy);
            double dist = sep > 0.0 ? (b2 - b1) / (2.0 * sep) : 0.0;
            uint64_t lo = (uint64_t)(i1 < i2 ? i1 : i2), hi = (uint64_t)(i1 < i2 ? i2 : i1);
            double width = 2.0 + u01(mix64(width_key ^ (lo * 0x9E3779B97F4A7C15ULL) ^ (hi << 21) ^ hi));
            int membrane = dist < 0.5 * width;
            if (truth) truth[y * pitch + x] = (uint8_t)membrane;
            uint64_t ctr = noise_key + 2ULL * (uint64_t)(y * w + x);
            double z = box_muller(mix64(ctr), mix64(ctr + 1ULL));
            img[y * w + x] = membrane ? 60.0 + 15.0 * z : 170.0 + 20.0 * z;
        }
    }

    double g[7], gs = 0.0;
    for (int t = -3; t <= 3; ++t) { g[t + 3] = exp(-0.5 * (double)(t * t)); gs += g[t + 3]; }
    for (int t = 0; t < 7; ++t) g[t] /= gs;

#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < h; ++y)
        for (int64_t x = 0; x < w; ++x) {
            double a = 0.0;
            for (int t = -3; t <= 3; ++t) a += g[t + 3] * img[y * w + refl101(x + t, w)];
            tmp[y * w + x] = a;
        }
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < h; ++y)
        for (int64_t x = 0; x < w; ++x) {
            double a = 0.0;
            for (int t = -3; t <= 3; ++t) a += g[t + 3] * tmp[refl101(y + t, h) * w + x];
            double q = nearbyint(a); /* default rounding mode: half to even */
            if (q < 0.0) q = 0.0;
            if (q > 255.0) q = 255.0;
            out[y * pitch + x] = (uint8_t)q;
        }

    free(px); free(py); free(img); free(tmp); free(bstart); free(bitems); free(bfill);
    return SYNTH_OK;
}

int synth_em_slice(uint64_t seed, int64_t h, int64_t w, int64_t n_cells, uint8_t* out, int64_t pitch) {
    return synth_em_slice_truth(seed, h, w, n_cells, out, pitch, NULL);
}

/* z slices of one block; slice zi uses synth_slice_seed(base, block, zi). */
int synth_em_volume(uint64_t base, uint64_t block, int64_t z, int64_t h, int64_t w, int64_t n_cells,
                    uint8_t* out, int64_t pitch, int64_t slice_pitch) {
    if (!out || z < 0) return SYNTH_ERR_ARG;
    for (int64_t zi = 0; zi < z; ++zi) {
        int rc = synth_em_slice(synth_slice_seed(base, block, (uint64_t)zi), h, w, n_cells,
                                out + zi * slice_pitch, pitch);
        if (rc) return rc;
    }
    return SYNTH_OK;
}

/*
 * He-normal parameters of one layer: w[i] ~ N(0, 2 / fan_in), b[i] ~ N(0, bias_std^2),
 * drawn in that order from one SplitMix64 stream seeded by `seed`, stored as FP32.
 */
int synth_he_normal(uint64_t seed, int64_t fan_in, int64_t n_w, float* w, int64_t n_b, float* b,
                    double bias_std) {
    if (fan_in <= 0 || n_w < 0 || n_b < 0 || (n_w && !w) || (n_b && !b)) return SYNTH_ERR_ARG;
    uint64_t st = mix64(seed);
    double sd = sqrt(2.0 / (double)fan_in);
    for (int64_t i = 0; i < n_w; ++i) w[i] = (float)(sd * stream_normal(&st));
    for (int64_t i = 0; i < n_b; ++i) b[i] = (float)(bias_std * stream_normal(&st));
    return SYNTH_OK;
}

/* n integers uniform in [lo, hi] (inclusive) from one SplitMix64 stream. */
int synth_uniform_ints(uint64_t seed, int64_t n, int64_t lo, int64_t hi, int64_t* out) {
    if (!out || n < 0 || hi < lo) return SYNTH_ERR_ARG;
    uint64_t st = mix64(seed);
    uint64_t span = (uint64_t)(hi - lo) + 1ULL;
    for (int64_t i = 0; i < n; ++i) out[i] = lo + (int64_t)(u01(sm64_next(&st)) * (double)span);
    return SYNTH_OK;
}

/* n FP32 values uniform in [lo, hi) from one SplitMix64 stream (test fixtures). */
int synth_uniform_floats(uint64_t seed, int64_t n, double lo, double hi, float* out) {
    if (!out || n < 0) return SYNTH_ERR_ARG;
    uint64_t st = mix64(seed);
    for (int64_t i = 0; i < n; ++i) out[i] = (float)(lo + (hi - lo) * u01(sm64_next(&st)));
    return SYNTH_OK;
}
