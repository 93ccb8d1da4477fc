/*
 * oracle.c - plain, slow FP64 CPU oracle of dense membrane-probability inference.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the bench's CPU
 * baseline leg may load this library. It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes (all in FP64, direct loops, no blocking or fusion):
 *  - Sec. 2.1 (membrane classification): every pixel of an EM slice gets the probability that
 *    it lies on a membrane. The network is a stack of valid cross-correlations with bias and
 *    ReLU, 2x2 stride-1 max-filters and a 1x1 head followed by a sigmoid.
 *  - Sec. 2.2, "Accelerating dense computation": dense computation gives every pixel the same
 *    value as evaluating the network on that pixel's own field-of-view patch (the patch
 *    calculation); max-pooling is replaced by stride-1 max-filtering. oracle_forward_region
 *    is the dense form, oracle_patch_pixel the patch form.
 *  - The border is mirror-padded (reflect-101: t -> -t below 0, t -> 2(n-1)-t above n-1) by
 *    the network's radius, so the output has the input's size.
 *  - The distilled student (conv3x3 1->16 ReLU, conv3x3 16->16 ReLU, conv1x1 16->1 sigmoid):
 *    forward, mean-squared-error loss against teacher maps, and the analytic weight gradient.
 *  - Adam (Kingma and Ba, 2014) with bias correction.
 *
 * FastMemb (Sec. 2.2, "A lightweight network architecture"; "Accelerating dense computation"):
 *    its dense form is the stride-1 network in which every stride-2 max-pool becomes a 2x2
 *    max-filter and every later layer is dilated by the accumulated stride (dilated cross-
 *    correlation y[i][j] = b + sum W[ky][kx] x[i + d ky][j + d kx]); max-out keeps the maximum
 *    over groups of feature maps (output channel c = max_g of conv channel c*G + g); the 2-class
 *    softmax head outputs p = exp(z1) / (exp(z0) + exp(z1)).
 * MaskExtend (Sec. 3.2): the same max-out family with a 12-map input stack, five 4x4 convs with
 *    max-out (32, 40, 48, 56, 64 features, dilations 1..16 in dense form) and a 1x1 head to 3
 *    classes with a softmax over all of them (OR_SOFTMAXN: every class probability is output);
 *    J (smoothing and thresholding) is a 3x3 mean with reflect-101 borders followed by >= thr.
 *
 * Conventions: activations are [c][y][x] row-major; parameters per parameterised layer are
 * W[cout*G][cin][k][k] followed by b[cout*G] (G = max-out groups, 1 without max-out); the input
 * pixel value is u / 255. A layer description is 7 ints {kind, k, cin, cout, relu, dilation, G}.
 * Compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2

/* layer kinds of a layer description: {kind, k, cin, cout, relu, dilation, maxout} per layer */
#define OR_CONV 0
#define OR_MAXF 1
#define OR_HEAD 2
#define OR_SOFTMAX 3
#define OR_SOFTMAXN 4
#define OR_DW 7

/* reflect-101 index map for n >= 2 (one reflection suffices when |overhang| < n) */
int64_t oracle_reflect101(int64_t t, int64_t n) {
    if (t < 0) t = -t;
    if (t >= n) t = 2 * (n - 1) - t;
    return t;
}

/*
 * Valid cross-correlation with dilation d: y[co][i][j] = b[co] + sum_ci sum_ky sum_kx
 * W[co][ci][ky][kx] * x[ci][i + d ky][j + d kx], then max(0, .) when relu. x is cin x h x w, y is
 * cout x (h - (k-1)d) x (w - (k-1)d). Each output element accumulates its terms in the order
 * (ci, ky, kx), starting from the bias.
 */
int oracle_conv_dil(const double* x, int64_t cin, int64_t h, int64_t w, const double* W, const double* b,
                    int64_t cout, int64_t k, int64_t dil, int relu, double* y) {
    if (!x || !W || !b || !y || cin < 1 || cout < 1 || k < 1 || dil < 1) return OR_ERR_ARG;
    const int64_t span = (k - 1) * dil;
    if (h <= span || w <= span) return OR_ERR_ARG;
    int64_t oh = h - span, ow = w - span;
#pragma omp parallel for schedule(static)
    for (int64_t co = 0; co < cout; ++co) {
        double* yc = y + co * oh * ow;
        for (int64_t i = 0; i < oh * ow; ++i) yc[i] = b[co];
        for (int64_t ci = 0; ci < cin; ++ci)
            for (int64_t ky = 0; ky < k; ++ky)
                for (int64_t kx = 0; kx < k; ++kx) {
                    double wt = W[((co * cin + ci) * k + ky) * k + kx];
                    const double* xs = x + (ci * h + ky * dil) * w + kx * dil;
                    for (int64_t i = 0; i < oh; ++i)
                        for (int64_t j = 0; j < ow; ++j) yc[i * ow + j] += wt * xs[i * w + j];
                }
        if (relu)
            for (int64_t i = 0; i < oh * ow; ++i) yc[i] = yc[i] > 0.0 ? yc[i] : 0.0;
    }
    return OR_OK;
}

/* Valid cross-correlation without dilation (see oracle_conv_dil). */
int oracle_conv(const double* x, int64_t cin, int64_t h, int64_t w, const double* W, const double* b,
                int64_t cout, int64_t k, int relu, double* y) {
    return oracle_conv_dil(x, cin, h, w, W, b, cout, k, 1, relu, y);
}

/* 2x2 stride-1 max-filter with dilation d, valid: y[c][i][j] = max of x[c][i + {0,d}][j + {0,d}];
 * y is c x (h-d) x (w-d). */
int oracle_maxfilter2_dil(const double* x, int64_t c, int64_t h, int64_t w, int64_t d, double* y) {
    if (!x || !y || c < 1 || d < 1 || h <= d || w <= d) return OR_ERR_ARG;
    int64_t oh = h - d, ow = w - d;
    for (int64_t ch = 0; ch < c; ++ch)
        for (int64_t i = 0; i < oh; ++i)
            for (int64_t j = 0; j < ow; ++j) {
                const double* p = x + (ch * h + i) * w + j;
                double m = p[0];
                if (p[d] > m) m = p[d];
                if (p[d * w] > m) m = p[d * w];
                if (p[d * w + d] > m) m = p[d * w + d];
                y[(ch * oh + i) * ow + j] = m;
            }
    return OR_OK;
}

int oracle_maxfilter2(const double* x, int64_t c, int64_t h, int64_t w, double* y) {
    return oracle_maxfilter2_dil(x, c, h, w, 1, y);
}

/* Max-out: y[c] = max over g < G of x[c*G + g]; x has c_out*G channels, y has c_out. */
int oracle_maxout(const double* x, int64_t c_out, int64_t G, int64_t hw, double* y) {
    if (!x || !y || c_out < 1 || G < 1 || hw < 1) return OR_ERR_ARG;
    for (int64_t c = 0; c < c_out; ++c)
        for (int64_t i = 0; i < hw; ++i) {
            double m = x[(c * G) * hw + i];
            for (int64_t g = 1; g < G; ++g)
                if (x[(c * G + g) * hw + i] > m) m = x[(c * G + g) * hw + i];
            y[c * hw + i] = m;
        }
    return OR_OK;
}

/* Head: z = b + sum_c wv[c] x[c][i][j]; p = 1 / (1 + exp(-z)). */
int oracle_head_sigmoid(const double* x, int64_t c, int64_t h, int64_t w, const double* wv, double b,
                        double* p) {
    if (!x || !wv || !p || c < 1 || h < 1 || w < 1) return OR_ERR_ARG;
    for (int64_t i = 0; i < h * w; ++i) {
        double z = b;
        for (int64_t ch = 0; ch < c; ++ch) z += wv[ch] * x[ch * h * w + i];
        p[i] = 1.0 / (1.0 + exp(-z));
    }
    return OR_OK;
}

static int64_t dil_of(const int32_t* d) { return d[5] > 0 ? d[5] : 1; }
static int64_t groups_of(const int32_t* d) { return d[6] > 0 ? d[6] : 1; }

/* Sum over layers of the size each one removes: (k - 1) d for convs and max-filters. */
static int64_t net_shrink(const int32_t* desc, int n_layers) {
    int64_t s = 0;
    for (int l = 0; l < n_layers; ++l) s += (int64_t)(desc[OR_DW * l + 1] - 1) * dil_of(desc + OR_DW * l);
    return s;
}

int64_t oracle_net_radius(const int32_t* desc, int n_layers) {
    int64_t s = net_shrink(desc, n_layers);
    return (s % 2) ? -1 : s / 2;
}

int64_t oracle_param_count(const int32_t* desc, int n_layers) {
    int64_t n = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int32_t* d = desc + OR_DW * l;
        const int64_t co = (int64_t)d[3] * groups_of(d);
        if (d[0] == OR_CONV || d[0] == OR_HEAD || d[0] == OR_SOFTMAX || d[0] == OR_SOFTMAXN)
            n += co * d[2] * d[1] * d[1] + co;
    }
    return n;
}

/*
 * Mirror-padded, normalised input region: xp[r][c] = u8[refl(y0 - R + r)][refl(x0 - R + c)] / 255
 * for r < h + 2R, c < wd + 2R.
 */
int oracle_pad_region(const uint8_t* in, int64_t H, int64_t W, int64_t pitch, int64_t y0, int64_t x0,
                      int64_t h, int64_t wd, int64_t R, double* xp) {
    if (!in || !xp || H < 2 || W < 2 || R < 0 || R >= H || R >= W) return OR_ERR_ARG;
    int64_t ph = h + 2 * R, pw = wd + 2 * R;
    for (int64_t r = 0; r < ph; ++r)
        for (int64_t c = 0; c < pw; ++c) {
            int64_t yy = oracle_reflect101(y0 - R + r, H), xx = oracle_reflect101(x0 - R + c, W);
            xp[r * pw + c] = (double)in[yy * pitch + xx] / 255.0;
        }
    return OR_OK;
}

/*
 * Run the layer stack on an already padded single-channel input xp (ph x pw); writes the
 * (ph - shrink) x (pw - shrink) probability map to p. Returns OR_OK or an error.
 */
int oracle_run_layers_mc(const int32_t* desc, int n_layers, const double* params, const double* xp, int64_t cin0,
                         int64_t ph, int64_t pw, double* p) {
    if (!desc || !params || !xp || !p || n_layers < 1 || cin0 < 1) return OR_ERR_ARG;
    int64_t c = cin0, h = ph, w = pw;
    double* cur = (double*)malloc(sizeof(double) * (size_t)(c * h * w));
    if (!cur) return OR_ERR_OOM;
    memcpy(cur, xp, sizeof(double) * (size_t)(c * h * w));
    const double* prm = params;
    int rc = OR_OK;
    for (int l = 0; l < n_layers && rc == OR_OK; ++l) {
        const int32_t* d = desc + OR_DW * l;
        const int64_t k = d[1], cin = d[2], cout = d[3], dl = dil_of(d), G = groups_of(d);
        const int last = l == n_layers - 1;
        if (d[0] == OR_CONV || d[0] == OR_SOFTMAX || d[0] == OR_SOFTMAXN) {
            const int64_t span = (k - 1) * dl, cg = cout * G;
            if (cin != c || h <= span || w <= span) { rc = OR_ERR_ARG; break; }
            if (d[0] == OR_SOFTMAX && (cout != 2 || G != 1 || !last)) { rc = OR_ERR_ARG; break; }
            if (d[0] == OR_SOFTMAXN && (cout < 2 || G != 1 || !last)) { rc = OR_ERR_ARG; break; }
            int64_t oh = h - span, ow = w - span;
            double* full = (double*)malloc(sizeof(double) * (size_t)(cg * oh * ow));
            if (!full) { rc = OR_ERR_OOM; break; }
            rc = oracle_conv_dil(cur, cin, h, w, prm, prm + cg * cin * k * k, cg, k, dl, d[4], full);
            prm += cg * cin * k * k + cg;
            free(cur);
            if (rc == OR_OK && d[0] == OR_SOFTMAX) {
                for (int64_t i = 0; i < oh * ow; ++i) p[i] = 1.0 / (1.0 + exp(full[i] - full[oh * ow + i]));
                free(full);
                cur = NULL;
                c = 1; h = oh; w = ow;
                continue;
            }
            if (rc == OR_OK && d[0] == OR_SOFTMAXN) {
                /* p[class][i] = exp(z_class - max) / sum_j exp(z_j - max) */
                for (int64_t i = 0; i < oh * ow; ++i) {
                    double m = full[i];
                    for (int64_t j = 1; j < cout; ++j)
                        if (full[j * oh * ow + i] > m) m = full[j * oh * ow + i];
                    double den = 0.0;
                    for (int64_t j = 0; j < cout; ++j) den += exp(full[j * oh * ow + i] - m);
                    for (int64_t j = 0; j < cout; ++j) p[j * oh * ow + i] = exp(full[j * oh * ow + i] - m) / den;
                }
                free(full);
                cur = NULL;
                c = cout; h = oh; w = ow;
                continue;
            }
            if (rc == OR_OK && G > 1) {
                double* mo = (double*)malloc(sizeof(double) * (size_t)(cout * oh * ow));
                if (!mo) { free(full); rc = OR_ERR_OOM; cur = NULL; break; }
                rc = oracle_maxout(full, cout, G, oh * ow, mo);
                free(full);
                full = mo;
            }
            cur = full; c = cout; h = oh; w = ow;
        } else if (d[0] == OR_MAXF) {
            if (k != 2 || h <= dl || w <= dl) { rc = OR_ERR_ARG; break; }
            double* nxt = (double*)malloc(sizeof(double) * (size_t)(c * (h - dl) * (w - dl)));
            if (!nxt) { rc = OR_ERR_OOM; break; }
            rc = oracle_maxfilter2_dil(cur, c, h, w, dl, nxt);
            free(cur); cur = nxt; h -= dl; w -= dl;
        } else if (d[0] == OR_HEAD) {
            if (cin != c || cout != 1 || k != 1 || !last) { rc = OR_ERR_ARG; break; }
            rc = oracle_head_sigmoid(cur, c, h, w, prm, prm[c], p);
            prm += c + 1;
        } else {
            rc = OR_ERR_ARG;
        }
    }
    {
        const int kind = desc[OR_DW * (n_layers - 1)];
        if (rc == OR_OK && kind != OR_HEAD && kind != OR_SOFTMAX && kind != OR_SOFTMAXN) rc = OR_ERR_ARG;
    }
    free(cur);
    return rc;
}

/* Single-channel input (the membrane networks). */
int oracle_run_layers(const int32_t* desc, int n_layers, const double* params, const double* xp,
                      int64_t ph, int64_t pw, double* p) {
    return oracle_run_layers_mc(desc, n_layers, params, xp, 1, ph, pw, p);
}

/*
 * J of the MaskExtend transfer (Sec. 3.2): smoothing by the 3x3 mean (reflect-101 at the borders)
 * and thresholding: mask[i][j] = 1 if mean of p over (i-1..i+1, j-1..j+1) >= thr, else 0.
 */
int oracle_smooth_threshold(const double* p, int64_t h, int64_t w, double thr, uint8_t* mask) {
    if (!p || !mask || h < 2 || w < 2) return OR_ERR_ARG;
    for (int64_t i = 0; i < h; ++i)
        for (int64_t j = 0; j < w; ++j) {
            double s = 0.0;
            for (int64_t a = -1; a <= 1; ++a)
                for (int64_t b = -1; b <= 1; ++b) s += p[oracle_reflect101(i + a, h) * w + oracle_reflect101(j + b, w)];
            mask[i * w + j] = (s / 9.0 >= thr) ? 1 : 0;
        }
    return OR_OK;
}

/*
 * Dense form: probabilities of the h x wd output region at (y0, x0) of a slice H x W, with
 * mirror padding only at the slice borders (true context elsewhere).
 */
int oracle_forward_region(const int32_t* desc, int n_layers, const double* params, const uint8_t* in,
                          int64_t H, int64_t W, int64_t pitch, int64_t y0, int64_t x0, int64_t h,
                          int64_t wd, double* p) {
    int64_t R = oracle_net_radius(desc, n_layers);
    if (R < 0 || h < 1 || wd < 1 || y0 < 0 || x0 < 0 || y0 + h > H || x0 + wd > W) return OR_ERR_ARG;
    int64_t ph = h + 2 * R, pw = wd + 2 * R;
    double* xp = (double*)malloc(sizeof(double) * (size_t)(ph * pw));
    if (!xp) return OR_ERR_OOM;
    int rc = oracle_pad_region(in, H, W, pitch, y0, x0, h, wd, R, xp);
    if (rc == OR_OK) rc = oracle_run_layers(desc, n_layers, params, xp, ph, pw, p);
    free(xp);
    return rc;
}

/*
 * Patch form for one output pixel (i, j): cut that pixel's (2R+1) x (2R+1) field of view out
 * of the mirror-padded slice and evaluate the network on it alone.
 */
int oracle_patch_pixel(const int32_t* desc, int n_layers, const double* params, const uint8_t* in,
                       int64_t H, int64_t W, int64_t pitch, int64_t i, int64_t j, double* p) {
    int64_t R = oracle_net_radius(desc, n_layers);
    if (R < 0 || i < 0 || j < 0 || i >= H || j >= W) return OR_ERR_ARG;
    int64_t n = 2 * R + 1;
    double* patch = (double*)malloc(sizeof(double) * (size_t)(n * n));
    if (!patch) return OR_ERR_OOM;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t c = 0; c < n; ++c) {
            int64_t yy = oracle_reflect101(i - R + r, H), xx = oracle_reflect101(j - R + c, W);
            patch[r * n + c] = (double)in[yy * pitch + xx] / 255.0;
        }
    int rc = oracle_run_layers(desc, n_layers, params, patch, n, n, p);
    free(patch);
    return rc;
}

/*
 * Per-channel maximum of the activations after the network's max-filter layers (the inputs of
 * the 2nd and 3rd convolutions of the stand-in net) over a region: amax[m * C + c] for the m-th
 * max-filter. Used for FP8 activation calibration checks.
 */
int oracle_maxfilter_amax(const int32_t* desc, int n_layers, const double* params, const uint8_t* in,
                          int64_t H, int64_t W, int64_t pitch, int64_t y0, int64_t x0, int64_t h,
                          int64_t wd, double* amax, int64_t amax_len) {
    int64_t R = oracle_net_radius(desc, n_layers);
    if (R < 0 || !amax) return OR_ERR_ARG;
    int64_t ph = h + 2 * R, pw = wd + 2 * R;
    double* cur = (double*)malloc(sizeof(double) * (size_t)(ph * pw));
    if (!cur) return OR_ERR_OOM;
    int rc = oracle_pad_region(in, H, W, pitch, y0, x0, h, wd, R, cur);
    int64_t c = 1, hh = ph, ww = pw, m = 0;
    const double* prm = params;
    for (int l = 0; l < n_layers && rc == OR_OK; ++l) {
        const int32_t* d = desc + OR_DW * l;
        int64_t k = d[1], cin = d[2], cout = d[3];
        if (dil_of(d) != 1 || groups_of(d) != 1) { rc = OR_ERR_ARG; break; }
        if (d[0] == OR_CONV) {
            int64_t oh = hh - k + 1, ow = ww - k + 1;
            double* nxt = (double*)malloc(sizeof(double) * (size_t)(cout * oh * ow));
            if (!nxt) { rc = OR_ERR_OOM; break; }
            rc = oracle_conv(cur, cin, hh, ww, prm, prm + cout * cin * k * k, cout, k, d[4], nxt);
            prm += cout * cin * k * k + cout;
            free(cur); cur = nxt; c = cout; hh = oh; ww = ow;
        } else if (d[0] == OR_MAXF) {
            double* nxt = (double*)malloc(sizeof(double) * (size_t)(c * (hh - 1) * (ww - 1)));
            if (!nxt) { rc = OR_ERR_OOM; break; }
            rc = oracle_maxfilter2(cur, c, hh, ww, nxt);
            free(cur); cur = nxt; hh -= 1; ww -= 1;
            if ((m + 1) * c > amax_len) { rc = OR_ERR_ARG; break; }
            for (int64_t ch = 0; ch < c; ++ch) {
                double a = 0.0;
                for (int64_t t = 0; t < hh * ww; ++t) {
                    double v = fabs(cur[ch * hh * ww + t]);
                    if (v > a) a = v;
                }
                amax[m * c + ch] = a;
            }
            ++m;
        } else {
            break;
        }
    }
    free(cur);
    return rc;
}

/*
 * Student loss and weight gradient for n slices (each H x W, pitch `pitch`, slice stride
 * `spitch`) against FP64-promoted target maps t (same layout, n x H x W contiguous).
 * The network must be conv / conv / head (no max-filters). Loss L = (1/N) sum (p - t)^2 over
 * all N = n*H*W output pixels. grad has the parameter layout. Backward, per the chain rule:
 *   dL/dz = (2/N)(p - t) p (1 - p)
 *   head:  dW[c] = sum dz h[c];  db = sum dz;  dh[c] = dz W[c]
 *   conv:  dy = dh * [y > 0] (ReLU subgradient 0 at 0)
 *          dW[co][ci][ky][kx] = sum_{i,j} dy[co][i][j] x[ci][i+ky][j+kx];  db[co] = sum dy[co]
 *          dx[ci][i+ky][j+kx] += dy[co][i][j] W[co][ci][ky][kx]
 */
int oracle_student_loss_grad(const int32_t* desc, int n_layers, const double* params, const uint8_t* in,
                             int64_t n, int64_t H, int64_t W, int64_t pitch, int64_t spitch,
                             const double* t, double* loss, double* grad) {
    if (!desc || !params || !in || !t || !loss || !grad || n < 1 || n_layers < 2 || n_layers > 16)
        return OR_ERR_ARG;
    int64_t R = oracle_net_radius(desc, n_layers);
    if (R < 0) return OR_ERR_ARG;
    for (int l = 0; l < n_layers; ++l) {
        int kind = desc[OR_DW * l];
        if (kind == OR_MAXF || dil_of(desc + OR_DW * l) != 1 || groups_of(desc + OR_DW * l) != 1) return OR_ERR_ARG;
        if (kind == OR_HEAD && l != n_layers - 1) return OR_ERR_ARG;
    }
    if (desc[OR_DW * (n_layers - 1)] != OR_HEAD) return OR_ERR_ARG;
    int64_t np = oracle_param_count(desc, n_layers);
    memset(grad, 0, sizeof(double) * (size_t)np);
    double N = (double)(n * H * W);
    double lsum = 0.0;
    int rc = OR_OK;

    /* per-layer parameter offsets */
    int64_t off[16];
    {
        int64_t o = 0;
        for (int l = 0; l < n_layers; ++l) {
            off[l] = o;
            const int32_t* d = desc + OR_DW * l;
            o += (int64_t)d[3] * d[2] * d[1] * d[1] + d[3];
        }
    }

    for (int64_t s = 0; s < n && rc == OR_OK; ++s) {
        /* forward, keeping every layer's input and pre-activation */
        double* acts[17];
        double* pre[17];
        int64_t ac[17], ah[17], aw[17];
        memset(acts, 0, sizeof(acts));
        memset(pre, 0, sizeof(pre));
        ah[0] = H + 2 * R; aw[0] = W + 2 * R; ac[0] = 1;
        acts[0] = (double*)malloc(sizeof(double) * (size_t)(ah[0] * aw[0]));
        if (!acts[0]) { rc = OR_ERR_OOM; break; }
        oracle_pad_region(in + s * spitch, H, W, pitch, 0, 0, H, W, R, acts[0]);
        for (int l = 0; l < n_layers - 1 && rc == OR_OK; ++l) {
            const int32_t* d = desc + OR_DW * l;
            int64_t k = d[1], cin = d[2], cout = d[3];
            int64_t oh = ah[l] - k + 1, ow = aw[l] - k + 1;
            pre[l] = (double*)malloc(sizeof(double) * (size_t)(cout * oh * ow));
            acts[l + 1] = (double*)malloc(sizeof(double) * (size_t)(cout * oh * ow));
            if (!pre[l] || !acts[l + 1]) { rc = OR_ERR_OOM; break; }
            rc = oracle_conv(acts[l], cin, ah[l], aw[l], params + off[l],
                             params + off[l] + cout * cin * k * k, cout, k, 0, pre[l]);
            for (int64_t q = 0; q < cout * oh * ow; ++q)
                acts[l + 1][q] = (d[4] && pre[l][q] < 0.0) ? 0.0 : pre[l][q];
            ac[l + 1] = cout; ah[l + 1] = oh; aw[l + 1] = ow;
        }
        int L = n_layers - 1; /* head index */
        if (rc == OR_OK && (ah[L] != H || aw[L] != W || ac[L] != desc[OR_DW * L + 2])) rc = OR_ERR_ARG;
        double* dcur = NULL;
        if (rc == OR_OK) {
            int64_t C = ac[L];
            const double* hw = params + off[L];
            double hb = hw[C];
            dcur = (double*)calloc((size_t)(C * H * W), sizeof(double));
            if (!dcur) rc = OR_ERR_OOM;
            for (int64_t q = 0; q < H * W && rc == OR_OK; ++q) {
                double z = hb;
                for (int64_t c = 0; c < C; ++c) z += hw[c] * acts[L][c * H * W + q];
                double p = 1.0 / (1.0 + exp(-z));
                double tv = t[s * H * W + q];
                lsum += (p - tv) * (p - tv);
                double dz = (2.0 / N) * (p - tv) * p * (1.0 - p);
                for (int64_t c = 0; c < C; ++c) {
                    grad[off[L] + c] += dz * acts[L][c * H * W + q];
                    dcur[c * H * W + q] = dz * hw[c];
                }
                grad[off[L] + C] += dz;
            }
        }
        for (int l = L - 1; l >= 0 && rc == OR_OK; --l) {
            const int32_t* d = desc + OR_DW * l;
            int64_t k = d[1], cin = d[2], cout = d[3];
            int64_t ih = ah[l], iw = aw[l], oh = ah[l + 1], ow = aw[l + 1];
            const double* Wl = params + off[l];
            double* gW = grad + off[l];
            double* gb = grad + off[l] + cout * cin * k * k;
            for (int64_t q = 0; q < cout * oh * ow; ++q)
                if (d[4] && !(pre[l][q] > 0.0)) dcur[q] = 0.0;
            double* dprev = NULL;
            if (l > 0) {
                dprev = (double*)calloc((size_t)(cin * ih * iw), sizeof(double));
                if (!dprev) { rc = OR_ERR_OOM; break; }
            }
            for (int64_t co = 0; co < cout; ++co) {
                for (int64_t i = 0; i < oh; ++i)
                    for (int64_t j = 0; j < ow; ++j) gb[co] += dcur[(co * oh + i) * ow + j];
                for (int64_t ci = 0; ci < cin; ++ci)
                    for (int64_t ky = 0; ky < k; ++ky)
                        for (int64_t kx = 0; kx < k; ++kx) {
                            double a = 0.0;
                            double wt = Wl[((co * cin + ci) * k + ky) * k + kx];
                            for (int64_t i = 0; i < oh; ++i)
                                for (int64_t j = 0; j < ow; ++j) {
                                    double dy = dcur[(co * oh + i) * ow + j];
                                    a += dy * acts[l][(ci * ih + i + ky) * iw + j + kx];
                                    if (dprev) dprev[(ci * ih + i + ky) * iw + j + kx] += dy * wt;
                                }
                            gW[((co * cin + ci) * k + ky) * k + kx] += a;
                        }
            }
            free(dcur);
            dcur = dprev;
        }
        free(dcur);
        for (int l = 0; l < 17; ++l) { free(acts[l]); free(pre[l]); }
    }
    *loss = lsum / N;
    return rc;
}

/*
 * One Adam step (Kingma and Ba, 2014) at step number `step` (1-based):
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   mhat = m / (1 - b1^step);  vhat = v / (1 - b2^step);  w -= lr mhat / (sqrt(vhat) + eps)
 */
int oracle_adam_step(double* w, double* m, double* v, const double* g, int64_t n, int64_t step, double lr,
                     double b1, double b2, double eps) {
    if (!w || !m || !v || !g || n < 0 || step < 1) return OR_ERR_ARG;
    double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
    return OR_OK;
}
