/*
 * FP64 CPU oracle of the per-frame panoramic stitching path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (paper Sec. 4.3, Alg. 4 step 1 "cut and transformed" and
 * step 6 "transform the video and blend it into a panoramic video"; Sec. 1,
 * contribution 3, "multi band fusion" to remove seams).  The paper gives no
 * formulas for any of these steps; the definitions below are the textbook
 * Burt-Adelson multiresolution spline with the readings listed in the design
 * notes (C1-C17).  Everything is evaluated literally in double precision:
 *
 *  S1 warp:   A_i = M_i^-1 scaled by 1/|a33| (a positive factor, so the sign of w, which
 *             tells points in front of the camera from points behind it, is kept; a33 = +-1).
 *             For canvas pixel (x, y):
 *             (nu, nv, w) = A_i (x, y, 1); u = nu/w, v = nv/w.
 *             Cylindrical canvas (focal length f, centre (cx, cy); a canvas column is an angle):
 *             the camera's 3x3 matrix P_i (= K_i R_i) is used as given, A_i = P_i, on the ray
 *             (sin t, (y - cy)/f, cos t) with t = (x - cx)/f instead of (x, y, 1).
 *             I_i = gain_i * bilinear(frame_i, clamp(u), clamp(v)) / 255,
 *             coordinates clamped to [0, W-1] x [0, H-1]; I_i = 0 where w <= 0.
 *             valid_i = w > 0 and -0.5 <= u < W-0.5 and -0.5 <= v < H-0.5.
 *  S2 weight: w_i = valid_i * max(0, min(u+0.5, v+0.5, W-0.5-u, H-0.5-v)),
 *             What_i = w_i / sum_j w_j where the sum is > 0, else 0 (feather weights).
 *             Seam weights (binary masks of the Burt-Adelson multiresolution spline, the
 *             "multi band fusion" of Sec. 1): What_i = 1 for the owner of the pixel, the
 *             lowest-index camera with w_i > 0 and w_i >= (1 - 1e-9) max_j w_j, 0 for the
 *             others (no owner: all 0).
 *  S3 REDUCE: G^{l+1}(k, j) = sum_{m,n=-2..2} w(m) w(n) G^l(r(2k+m), r(2j+n)),
 *             w = [1,4,6,4,1]/16, r = reflect-101 on the finer grid, size ceil(n/2).
 *  S4 EXPAND: E(x, y) = sum_{k,j} 2w(x-2k) 2w(y-2j) G(r(k), r(j)), r = reflect-101
 *             on the coarser grid; L^l = G^l - E(G^{l+1}), L^{L-1} = G^{L-1}.
 *  S5 blend:  N^l = sum_i G^l(What_i) L^l(I_i), S^l = sum_i G^l(What_i),
 *             B^l = N^l / S^l where S^l > 1e-12, else 0.
 *  S6 collapse: R^{L-1} = B^{L-1}, R^l = B^l + E(R^{l+1});
 *             out = clamp(R^0, 0, 1) where sum_i w_i > 0, else 0;
 *             out_u8 = round-half-even(255 * out).
 *  S7 loss:   sum over canvas pixels of sum_{i<j} valid_i valid_j |I_i - I_j|^2
 *             and its analytic gradient with respect to (a11..a32, gain) of each
 *             camera, validity masks held constant.
 *
 * Output windows: the forward pass evaluates the definition on the smallest
 * per-level rectangles that the requested output window depends on (reflect-101
 * folds every index back into the level, so the rectangles are computed by
 * enumerating the folded indices).  For a window equal to the canvas this is
 * the whole-canvas definition; for a sub-window the values are bit-identical
 * to the whole-canvas run because every needed value is computed by the same
 * expression from the same inputs.
 */
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

static const double W5[5] = {1.0 / 16.0, 4.0 / 16.0, 6.0 / 16.0, 4.0 / 16.0, 1.0 / 16.0};

/* reflect-101 index folding (..., 2, 1, 0, 1, 2, ..., n-2, n-1, n-2, ...); size 1 clamps. */
static int reflect101(int i, int n) {
    if (n <= 1) return 0;
    int p = 2 * (n - 1);
    i %= p;
    if (i < 0) i += p;
    if (i >= n) i = p - i;
    return i;
}

/* ------------------------------------------------------------------------------------------ */
/* homography inverse                                                                          */

/* A = M^-1 / |(M^-1)_33|, so a33 = +1 or -1.  Only a positive factor is applied: for a canvas
 * point x = M p / w_c(p) the third component of M^-1 x is 1 / w_c(p), positive exactly when the
 * camera point p is in front, and that sign must survive the scaling (a33 = -1 happens when the
 * canvas origin lies behind the camera).  Returns 0, or -1 when M is singular or a33 == 0. */
int oracle_invert_h(const double* M, double* A) {
    double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], k = M[8];
    double C00 = e * k - f * h, C01 = -(d * k - f * g), C02 = d * h - e * g;
    double det = a * C00 + b * C01 + c * C02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return -1;
    double inv[9];
    inv[0] = C00 / det;
    inv[1] = -(b * k - c * h) / det;
    inv[2] = (b * f - c * e) / det;
    inv[3] = C01 / det;
    inv[4] = (a * k - c * g) / det;
    inv[5] = -(a * f - c * d) / det;
    inv[6] = C02 / det;
    inv[7] = -(a * h - b * g) / det;
    inv[8] = (a * e - b * d) / det;
    double s = fabs(inv[8]);
    if (!(s > 0.0)) return -1;
    for (int i = 0; i < 9; ++i) A[i] = inv[i] / s;
    A[8] = inv[8] > 0.0 ? 1.0 : -1.0;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* cameras and sampling                                                                        */

typedef struct {
    int W, H;
    double A[9];
    double gain;
    const uint8_t* px;
    int64_t pitch;
    int cyl;             /* cylindrical canvas */
    double cf, ccx, ccy; /* its focal length and centre */
} ocam;

static inline double texel(const ocam* c, int x, int y, int ch) {
    return (double)c->px[(int64_t)y * c->pitch + 3 * (int64_t)x + ch];
}

/* S1 + S2 at one canvas point.  rgb gets I_i, *wraw the un-normalised feather weight,
 * *dist the distance (source px) to the border of the validity rectangle, or DBL_MAX when w<=0. */
static void cam_sample(const ocam* c, double x, double y, double rgb[3], double* wraw, double* dist) {
    const double* A = c->A;
    double X = x, Y = y, Z = 1.0;
    if (c->cyl) {
        const double t = (x - c->ccx) / c->cf;
        X = sin(t);
        Y = (y - c->ccy) / c->cf;
        Z = cos(t);
    }
    double nu = A[0] * X + A[1] * Y + A[2] * Z;
    double nv = A[3] * X + A[4] * Y + A[5] * Z;
    double w = A[6] * X + A[7] * Y + A[8] * Z;
    if (!(w > 0.0)) {
        rgb[0] = rgb[1] = rgb[2] = 0.0;
        *wraw = 0.0;
        if (dist) *dist = DBL_MAX;
        return;
    }
    double u = nu / w, v = nv / w;
    /* bilinear with coordinates clamped to the image (reading C2) */
    double uc = u < 0.0 ? 0.0 : (u > c->W - 1 ? (double)(c->W - 1) : u);
    double vc = v < 0.0 ? 0.0 : (v > c->H - 1 ? (double)(c->H - 1) : v);
    int i0 = (int)floor(uc), j0 = (int)floor(vc);
    double fx = uc - i0, fy = vc - j0;
    int i1 = i0 + 1 < c->W ? i0 + 1 : i0;
    int j1 = j0 + 1 < c->H ? j0 + 1 : j0;
    for (int ch = 0; ch < 3; ++ch) {
        double top = (1.0 - fx) * texel(c, i0, j0, ch) + fx * texel(c, i1, j0, ch);
        double bot = (1.0 - fx) * texel(c, i0, j1, ch) + fx * texel(c, i1, j1, ch);
        rgb[ch] = c->gain * ((1.0 - fy) * top + fy * bot) / 255.0;
    }
    int valid = (u >= -0.5) && (u < c->W - 0.5) && (v >= -0.5) && (v < c->H - 0.5);
    double m = u + 0.5;
    if (v + 0.5 < m) m = v + 0.5;
    if (c->W - 0.5 - u < m) m = c->W - 0.5 - u;
    if (c->H - 0.5 - v < m) m = c->H - 0.5 - v;
    *wraw = valid ? (m > 0.0 ? m : 0.0) : 0.0;
    if (dist) {
        double dx = fmax(fmax(-0.5 - u, u - (c->W - 0.5)), 0.0);
        double dy = fmax(fmax(-0.5 - v, v - (c->H - 0.5)), 0.0);
        if (dx == 0.0 && dy == 0.0)
            *dist = fmin(fmin(u + 0.5, c->W - 0.5 - u), fmin(v + 0.5, c->H - 0.5 - v));
        else
            *dist = hypot(dx, dy);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* index intervals and level images                                                            */

typedef struct {
    int lo, hi; /* inclusive; empty when lo > hi */
} ivl;

static ivl ivl_union(ivl a, ivl b) {
    if (a.lo > a.hi) return b;
    if (b.lo > b.hi) return a;
    ivl r = {a.lo < b.lo ? a.lo : b.lo, a.hi > b.hi ? a.hi : b.hi};
    return r;
}

/* finer-grid indices read by REDUCE outputs k in `c` (finer size n) */
static ivl reduce_support(ivl c, int n) {
    ivl r = {INT_MAX, INT_MIN};
    for (int k = c.lo; k <= c.hi; ++k)
        for (int m = -2; m <= 2; ++m) {
            int i = reflect101(2 * k + m, n);
            if (i < r.lo) r.lo = i;
            if (i > r.hi) r.hi = i;
        }
    return r;
}

/* coarser-grid indices read by EXPAND outputs x in `f` (coarser size n) */
static ivl expand_support(ivl f, int n) {
    ivl r = {INT_MAX, INT_MIN};
    for (int x = f.lo; x <= f.hi; ++x)
        for (int k = x / 2 - 2; k <= x / 2 + 2; ++k) {
            int d = x - 2 * k;
            if (d < -2 || d > 2) continue;
            int i = reflect101(k, n);
            if (i < r.lo) r.lo = i;
            if (i > r.hi) r.hi = i;
        }
    return r;
}

typedef struct {
    int x0, y0, w, h, ch;
    double* d;
} limg; /* image on a rectangle of one level, addressed by level coordinates */

static int limg_alloc(limg* im, ivl xs, ivl ys, int ch) {
    im->x0 = xs.lo;
    im->y0 = ys.lo;
    im->w = xs.hi - xs.lo + 1;
    im->h = ys.hi - ys.lo + 1;
    im->ch = ch;
    im->d = (double*)calloc((size_t)im->w * im->h * ch, sizeof(double));
    return im->d ? 0 : -1;
}

static inline double* limg_at(const limg* im, int x, int y) {
    int lx = x - im->x0, ly = y - im->y0;
    if (lx < 0 || ly < 0 || lx >= im->w || ly >= im->h) {
        fprintf(stderr, "oracle: level access (%d,%d) outside [%d,%d)x[%d,%d)\n", x, y, im->x0,
                im->x0 + im->w, im->y0, im->y0 + im->h);
        abort();
    }
    return im->d + ((size_t)ly * im->w + lx) * im->ch;
}

/* S3: REDUCE of `in` (finer level of size nxf x nyf) onto out's rectangle, all channels */
static void reduce_into(const limg* in, int nxf, int nyf, limg* out) {
#pragma omp parallel for schedule(static)
    for (int j = out->y0; j < out->y0 + out->h; ++j)
        for (int k = out->x0; k < out->x0 + out->w; ++k) {
            double* o = limg_at(out, k, j);
            for (int c = 0; c < out->ch; ++c) o[c] = 0.0;
            for (int n = -2; n <= 2; ++n) {
                int yy = reflect101(2 * j + n, nyf);
                for (int m = -2; m <= 2; ++m) {
                    int xx = reflect101(2 * k + m, nxf);
                    const double* s = limg_at(in, xx, yy);
                    double wt = W5[m + 2] * W5[n + 2];
                    for (int c = 0; c < out->ch; ++c) o[c] += wt * s[c];
                }
            }
        }
}

/* S4: EXPAND of coarse image `in` (level size nxc x nyc) at fine (x, y); first `ch` channels */
static void expand_at(const limg* in, int nxc, int nyc, int x, int y, int ch, double* o) {
    for (int c = 0; c < ch; ++c) o[c] = 0.0;
    for (int j = y / 2 - 2; j <= y / 2 + 2; ++j) {
        int dy = y - 2 * j;
        if (dy < -2 || dy > 2) continue;
        int jj = reflect101(j, nyc);
        for (int k = x / 2 - 2; k <= x / 2 + 2; ++k) {
            int dx = x - 2 * k;
            if (dx < -2 || dx > 2) continue;
            int kk = reflect101(k, nxc);
            const double* s = limg_at(in, kk, jj);
            double wt = (2.0 * W5[dx + 2]) * (2.0 * W5[dy + 2]);
            for (int c = 0; c < ch; ++c) o[c] += wt * s[c];
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* whole-image REDUCE / EXPAND (used by the pin tests)                                         */

int oracle_reduce(const double* in, int w, int h, int ch, double* out) {
    if (w < 1 || h < 1 || ch < 1) return OR_EINVAL;
    int wc = (w + 1) / 2, hc = (h + 1) / 2;
    limg a = {0, 0, w, h, ch, (double*)in}, b = {0, 0, wc, hc, ch, out};
    reduce_into(&a, w, h, &b);
    return OR_OK;
}

int oracle_expand(const double* in, int wc, int hc, int ch, int w, int h, double* out) {
    if (w < 1 || h < 1 || ch < 1 || wc != (w + 1) / 2 || hc != (h + 1) / 2) return OR_EINVAL;
    limg a = {0, 0, wc, hc, ch, (double*)in};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) expand_at(&a, wc, hc, x, y, ch, out + ((size_t)y * w + x) * ch);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* forward                                                                                     */

/* cyl: NULL for the planar canvas, else {f, cx, cy} of the cylindrical canvas (matrices are then
 * the cameras' P = K R, used as given). */
static int setup_cams(int n, const int32_t* Ws, const int32_t* Hs, const double* Ms, const double* gains,
                      const uint8_t* const* frames, const int64_t* pitches, const double* cyl, ocam* cams) {
    if (cyl && !(cyl[0] > 0.0)) return OR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (Ws[i] < 1 || Hs[i] < 1 || !frames[i] || pitches[i] < 3LL * Ws[i]) return OR_EINVAL;
        cams[i].W = Ws[i];
        cams[i].H = Hs[i];
        cams[i].cyl = cyl != NULL;
        cams[i].cf = cyl ? cyl[0] : 0.0;
        cams[i].ccx = cyl ? cyl[1] : 0.0;
        cams[i].ccy = cyl ? cyl[2] : 0.0;
        if (cyl) memcpy(cams[i].A, Ms + 9 * i, 9 * sizeof(double));
        else if (oracle_invert_h(Ms + 9 * i, cams[i].A) != 0) return OR_EINVAL;
        cams[i].gain = gains ? gains[i] : 1.0;
        cams[i].px = frames[i];
        cams[i].pitch = pitches[i];
    }
    return OR_OK;
}

/* Per-level rectangles of the forward pass for an output window: X_l (output dependency)
 * and Y_l (pyramid region).  Arrays of length L, level coordinates, inclusive bounds. */
static void forward_regions(int Wc, int Hc, int L, int wx0, int wy0, int ww, int wh, int* nx, int* ny,
                            ivl* Xx, ivl* Xy, ivl* Yx, ivl* Yy) {
    nx[0] = Wc;
    ny[0] = Hc;
    for (int l = 1; l < L; ++l) {
        nx[l] = (nx[l - 1] + 1) / 2;
        ny[l] = (ny[l - 1] + 1) / 2;
    }
    Xx[0].lo = wx0; Xx[0].hi = wx0 + ww - 1;
    Xy[0].lo = wy0; Xy[0].hi = wy0 + wh - 1;
    for (int l = 0; l + 1 < L; ++l) {
        Xx[l + 1] = expand_support(Xx[l], nx[l + 1]);
        Xy[l + 1] = expand_support(Xy[l], ny[l + 1]);
    }
    Yx[L - 1] = Xx[L - 1];
    Yy[L - 1] = Xy[L - 1];
    for (int l = L - 2; l >= 0; --l) {
        Yx[l] = ivl_union(Xx[l], reduce_support(Yx[l + 1], nx[l]));
        Yy[l] = ivl_union(Xy[l], reduce_support(Yy[l + 1], ny[l]));
    }
}

/* Rectangles (x0, x1_exclusive, y0, y1_exclusive) of X_l and Y_l for each level: 8*L ints. */
int oracle_regions(int Wc, int Hc, int L, int wx0, int wy0, int ww, int wh, int32_t* out) {
    if (L < 1 || L > 24 || Wc < 1 || Hc < 1 || ww < 1 || wh < 1 || wx0 < 0 || wy0 < 0 || wx0 + ww > Wc ||
        wy0 + wh > Hc)
        return OR_EINVAL;
    int nx[24], ny[24];
    ivl Xx[24], Xy[24], Yx[24], Yy[24];
    forward_regions(Wc, Hc, L, wx0, wy0, ww, wh, nx, ny, Xx, Xy, Yx, Yy);
    for (int l = 0; l < L; ++l) {
        int32_t* o = out + 8 * l;
        o[0] = Xx[l].lo; o[1] = Xx[l].hi + 1; o[2] = Xy[l].lo; o[3] = Xy[l].hi + 1;
        o[4] = Yx[l].lo; o[5] = Yx[l].hi + 1; o[6] = Yy[l].lo; o[7] = Yy[l].hi + 1;
    }
    return OR_OK;
}

/*
 * The whole stitching path (S1-S6) on the output window [wx0, wx0+ww) x [wy0, wy0+wh).
 *   out      ww*wh*3 doubles, [0,1] canvas after mask and clamp (may be NULL)
 *   out_u8   ww*wh*3 bytes (may be NULL)
 *   mindist  ww*wh doubles: min over cameras of the distance (source px) from (u, v) to the
 *            border of the validity rectangle (may be NULL)
 *   dbg_S, dbg_B  optional arrays of L pointers; level l receives S^l (1 ch) / B^l (3 ch) on
 *            the X_l rectangle reported by oracle_regions.
 */
int oracle_forward(int n, const int32_t* Ws, const int32_t* Hs, const double* Ms, const double* gains,
                   const uint8_t* const* frames, const int64_t* pitches, int Wc, int Hc, int L, int wx0,
                   int wy0, int ww, int wh, double* out, uint8_t* out_u8, double* mindist, double** dbg_S,
                   double** dbg_B, int seam, const double* cyl) {
    if (n < 1 || n > 64 || L < 1 || L > 24 || Wc < 1 || Hc < 1 || ww < 1 || wh < 1 || wx0 < 0 || wy0 < 0 ||
        wx0 + ww > Wc || wy0 + wh > Hc || (seam != 0 && seam != 1))
        return OR_EINVAL;
    ocam cams[64];
    int rc = setup_cams(n, Ws, Hs, Ms, gains, frames, pitches, cyl, cams);
    if (rc) return rc;

    int nx[24], ny[24];
    ivl Xx[24], Xy[24], Yx[24], Yy[24];
    forward_regions(Wc, Hc, L, wx0, wy0, ww, wh, nx, ny, Xx, Xy, Yx, Yy);

    limg Nl[24], Sl[24], G[24], wsum;
    memset(Nl, 0, sizeof(Nl));
    memset(Sl, 0, sizeof(Sl));
    memset(G, 0, sizeof(G));
    memset(&wsum, 0, sizeof(wsum));
    rc = OR_ENOMEM;
    for (int l = 0; l < L; ++l)
        if (limg_alloc(&Nl[l], Xx[l], Xy[l], 3) || limg_alloc(&Sl[l], Xx[l], Xy[l], 1) ||
            limg_alloc(&G[l], Yx[l], Yy[l], 4))
            goto done;
    if (limg_alloc(&wsum, Yx[0], Yy[0], 1)) goto done;

    /* S2 denominator: sum of raw feather weights at level 0; with seam weights, 1 + the index of
     * the pixel's owner (0: none), so that the coverage test "> 0" of S6 reads both alike */
#pragma omp parallel for schedule(static)
    for (int y = Yy[0].lo; y <= Yy[0].hi; ++y)
        for (int x = Yx[0].lo; x <= Yx[0].hi; ++x) {
            double s = 0.0, rgb[3], wr, wv[64], wmax = 0.0;
            for (int i = 0; i < n; ++i) {
                cam_sample(&cams[i], x, y, rgb, &wr, NULL);
                s += wr;
                wv[i] = wr;
                if (wr > wmax) wmax = wr;
            }
            if (seam) {
                int owner = -1;
                for (int i = 0; i < n && owner < 0; ++i)
                    if (wv[i] > 0.0 && wv[i] >= (1.0 - 1e-9) * wmax) owner = i;
                s = (double)(owner + 1);
            }
            *limg_at(&wsum, x, y) = s;
        }

    for (int i = 0; i < n; ++i) {
        /* S1 + S2: level 0 of camera i (image and normalised weight) */
#pragma omp parallel for schedule(static)
        for (int y = Yy[0].lo; y <= Yy[0].hi; ++y)
            for (int x = Yx[0].lo; x <= Yx[0].hi; ++x) {
                double rgb[3], wr;
                cam_sample(&cams[i], x, y, rgb, &wr, NULL);
                double s = *limg_at(&wsum, x, y);
                double* g = limg_at(&G[0], x, y);
                g[0] = rgb[0];
                g[1] = rgb[1];
                g[2] = rgb[2];
                if (seam) g[3] = (s == (double)(i + 1)) ? 1.0 : 0.0;
                else g[3] = s > 0.0 ? wr / s : 0.0;
            }
        /* S3: Gaussian pyramids of image and weight */
        for (int l = 0; l + 1 < L; ++l) reduce_into(&G[l], nx[l], ny[l], &G[l + 1]);
        /* S4 + S5 numerator and denominator */
        for (int l = 0; l < L; ++l) {
#pragma omp parallel for schedule(static)
            for (int y = Xy[l].lo; y <= Xy[l].hi; ++y)
                for (int x = Xx[l].lo; x <= Xx[l].hi; ++x) {
                    const double* g = limg_at(&G[l], x, y);
                    double lap[3] = {g[0], g[1], g[2]};
                    if (l + 1 < L) {
                        double e[3];
                        expand_at(&G[l + 1], nx[l + 1], ny[l + 1], x, y, 3, e);
                        for (int c = 0; c < 3; ++c) lap[c] -= e[c];
                    }
                    double* nn = limg_at(&Nl[l], x, y);
                    for (int c = 0; c < 3; ++c) nn[c] += g[3] * lap[c];
                    *limg_at(&Sl[l], x, y) += g[3];
                }
        }
    }

    /* S5: B^l = N^l / S^l (kept in Nl), then S6 collapse from the coarsest level (kept in Nl) */
    for (int l = 0; l < L; ++l) {
        if (dbg_S && dbg_S[l]) memcpy(dbg_S[l], Sl[l].d, sizeof(double) * (size_t)Sl[l].w * Sl[l].h);
#pragma omp parallel for schedule(static)
        for (int y = Xy[l].lo; y <= Xy[l].hi; ++y)
            for (int x = Xx[l].lo; x <= Xx[l].hi; ++x) {
                double s = *limg_at(&Sl[l], x, y);
                double* nn = limg_at(&Nl[l], x, y);
                for (int c = 0; c < 3; ++c) nn[c] = s > 1e-12 ? nn[c] / s : 0.0;
            }
        if (dbg_B && dbg_B[l]) memcpy(dbg_B[l], Nl[l].d, sizeof(double) * 3 * (size_t)Nl[l].w * Nl[l].h);
    }
    for (int l = L - 2; l >= 0; --l) {
#pragma omp parallel for schedule(static)
        for (int y = Xy[l].lo; y <= Xy[l].hi; ++y)
            for (int x = Xx[l].lo; x <= Xx[l].hi; ++x) {
                double e[3];
                expand_at(&Nl[l + 1], nx[l + 1], ny[l + 1], x, y, 3, e);
                double* r = limg_at(&Nl[l], x, y);
                for (int c = 0; c < 3; ++c) r[c] += e[c];
            }
    }

    /* output: mask by coverage, clamp, quantise */
#pragma omp parallel for schedule(static)
    for (int y = wy0; y < wy0 + wh; ++y)
        for (int x = wx0; x < wx0 + ww; ++x) {
            size_t o = (size_t)(y - wy0) * ww + (x - wx0);
            int covered = *limg_at(&wsum, x, y) > 0.0;
            const double* r = limg_at(&Nl[0], x, y);
            for (int c = 0; c < 3; ++c) {
                double v = covered ? (r[c] < 0.0 ? 0.0 : (r[c] > 1.0 ? 1.0 : r[c])) : 0.0;
                if (out) out[3 * o + c] = v;
                if (out_u8) out_u8[3 * o + c] = (uint8_t)nearbyint(255.0 * v);
            }
            if (mindist) {
                double md = DBL_MAX, rgb[3], wr, d;
                for (int i = 0; i < n; ++i) {
                    cam_sample(&cams[i], x, y, rgb, &wr, &d);
                    if (d < md) md = d;
                }
                mindist[o] = md;
            }
        }
    rc = OR_OK;
done:
    for (int l = 0; l < L; ++l) {
        free(Nl[l].d);
        free(Sl[l].d);
        free(G[l].d);
    }
    free(wsum.d);
    return rc;
}

/*
 * Level 0 of one camera on the whole canvas: I_i (3 ch), raw feather weight and validity.
 * img: Hc*Wc*3 doubles, wraw: Hc*Wc doubles (either may be NULL).
 */
int oracle_warp(int W, int H, const double* M, double gain, const uint8_t* frame, int64_t pitch, int Wc,
                int Hc, double* img, double* wraw, const double* cyl) {
    ocam c;
    int32_t Ws = W, Hs = H;
    if (setup_cams(1, &Ws, &Hs, M, &gain, &frame, &pitch, cyl, &c)) return OR_EINVAL;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Hc; ++y)
        for (int x = 0; x < Wc; ++x) {
            double rgb[3], wr;
            cam_sample(&c, x, y, rgb, &wr, NULL);
            size_t o = (size_t)y * Wc + x;
            if (img) {
                img[3 * o] = rgb[0];
                img[3 * o + 1] = rgb[1];
                img[3 * o + 2] = rgb[2];
            }
            if (wraw) wraw[o] = wr;
        }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* S7: overlap photometric loss and its analytic gradient                                      */

typedef struct {
    double I[3], dIu[3], dIv[3], u, v, w, B[3];
    int ok;
} gsample;

/* I = gain * bilinear / 255 with clamped coordinates, and dI/du, dI/dv (zero on a clamped axis). */
static void grad_sample(const int W, const int H, const uint8_t* px, int64_t pitch, const double* p, double a33,
                        double x, double y, gsample* s) {
    double nu = p[0] * x + p[1] * y + p[2];
    double nv = p[3] * x + p[4] * y + p[5];
    double w = p[6] * x + p[7] * y + a33;
    memset(s, 0, sizeof(*s));
    if (!(w > 0.0)) return;
    s->ok = 1;
    s->w = w;
    s->u = nu / w;
    s->v = nv / w;
    int cu = s->u < 0.0 || s->u > W - 1, cv = s->v < 0.0 || s->v > H - 1;
    double uc = s->u < 0.0 ? 0.0 : (s->u > W - 1 ? (double)(W - 1) : s->u);
    double vc = s->v < 0.0 ? 0.0 : (s->v > H - 1 ? (double)(H - 1) : s->v);
    int i0 = (int)floor(uc), j0 = (int)floor(vc);
    double fx = uc - i0, fy = vc - j0;
    int i1 = i0 + 1 < W ? i0 + 1 : i0;
    int j1 = j0 + 1 < H ? j0 + 1 : j0;
    double g = p[8];
    for (int c = 0; c < 3; ++c) {
        double p00 = px[(int64_t)j0 * pitch + 3 * i0 + c], p01 = px[(int64_t)j0 * pitch + 3 * i1 + c];
        double p10 = px[(int64_t)j1 * pitch + 3 * i0 + c], p11 = px[(int64_t)j1 * pitch + 3 * i1 + c];
        double top = (1.0 - fx) * p00 + fx * p01, bot = (1.0 - fx) * p10 + fx * p11;
        s->B[c] = ((1.0 - fy) * top + fy * bot) / 255.0;
        s->I[c] = g * s->B[c];
        s->dIu[c] = cu ? 0.0 : g * ((1.0 - fy) * (p01 - p00) + fy * (p11 - p10)) / 255.0;
        s->dIv[c] = cv ? 0.0 : g * ((1.0 - fx) * (p10 - p00) + fx * (p11 - p01)) / 255.0;
    }
}

static int mask_valid(int W, int H, const double* p, double a33, double x, double y) {
    double nu = p[0] * x + p[1] * y + p[2];
    double nv = p[3] * x + p[4] * y + p[5];
    double w = p[6] * x + p[7] * y + a33;
    if (!(w > 0.0)) return 0;
    double u = nu / w, v = nv / w;
    return (u >= -0.5) && (u < W - 0.5) && (v >= -0.5) && (v < H - 0.5);
}

/*
 * params: n*9 doubles per camera (a11 a12 a13 a21 a22 a23 a31 a32 gain) of the canvas->camera map
 * A whose a33 is given per camera in a33 (+1 or -1, NULL: all +1).  mask_params: same layout,
 * used only for the validity masks (NULL: params).
 * Window [x0,x0+w) x [y0,y0+h) of the canvas.  loss: 1 double; grad: n*9 doubles (may be NULL).
 * Rows are summed independently and then added in row order, so the result does not depend on
 * the number of threads.
 */
int oracle_loss_grad(int n, const int32_t* Ws, const int32_t* Hs, const double* params, const double* mask_params,
                     const double* a33, const uint8_t* const* frames, const int64_t* pitches, int x0, int y0, int w,
                     int h, double* loss, double* grad) {
    if (n < 1 || n > 64 || w < 0 || h < 0 || !loss) return OR_EINVAL;
    for (int i = 0; i < n; ++i)
        if (Ws[i] < 1 || Hs[i] < 1 || !frames[i] || pitches[i] < 3LL * Ws[i]) return OR_EINVAL;
    const double* mp = mask_params ? mask_params : params;
    int stride = 1 + 9 * n;
    double* rows = (double*)calloc((size_t)(h > 0 ? h : 1) * stride, sizeof(double));
    if (!rows) return OR_ENOMEM;
#pragma omp parallel for schedule(dynamic, 4)
    for (int yy = 0; yy < h; ++yy) {
        double* acc = rows + (size_t)yy * stride;
        double y = (double)(y0 + yy);
        gsample s[64];
        int val[64];
        for (int xx = 0; xx < w; ++xx) {
            double x = (double)(x0 + xx);
            int k = 0;
            for (int i = 0; i < n; ++i) {
                val[i] = mask_valid(Ws[i], Hs[i], mp + 9 * i, a33 ? a33[i] : 1.0, x, y);
                k += val[i];
            }
            if (k < 2) continue;
            for (int i = 0; i < n; ++i)
                if (val[i])
                    grad_sample(Ws[i], Hs[i], frames[i], pitches[i], params + 9 * i, a33 ? a33[i] : 1.0, x, y, &s[i]);
            for (int i = 0; i < n; ++i) {
                if (!val[i]) continue;
                for (int j = i + 1; j < n; ++j) {
                    if (!val[j]) continue;
                    for (int c = 0; c < 3; ++c) {
                        double d = s[i].I[c] - s[j].I[c];
                        acc[0] += d * d;
                    }
                }
                if (!grad || !s[i].ok) continue;
                double gu = 0.0, gv = 0.0, gg = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double r = 0.0;
                    for (int j = 0; j < n; ++j)
                        if (j != i && val[j]) r += s[i].I[c] - s[j].I[c];
                    gu += 2.0 * r * s[i].dIu[c];
                    gv += 2.0 * r * s[i].dIv[c];
                    gg += 2.0 * r * s[i].B[c];
                }
                double iw = 1.0 / s[i].w;
                double* gi = acc + 1 + 9 * i;
                gi[0] += gu * x * iw;
                gi[1] += gu * y * iw;
                gi[2] += gu * iw;
                gi[3] += gv * x * iw;
                gi[4] += gv * y * iw;
                gi[5] += gv * iw;
                double q = gu * s[i].u + gv * s[i].v;
                gi[6] += -q * x * iw;
                gi[7] += -q * y * iw;
                gi[8] += gg;
            }
        }
    }
    double L = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 9 * (size_t)n);
    for (int yy = 0; yy < h; ++yy) {
        const double* acc = rows + (size_t)yy * stride;
        L += acc[0];
        if (grad)
            for (int k = 0; k < 9 * n; ++k) grad[k] += acc[1 + k];
    }
    *loss = L;
    free(rows);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* L-ORB feature extraction (Sec. 4.1, Algorithms 1 and 2), all in exact integer arithmetic     */
/*                                                                                            */
/* Readings (the paper fixes the steps, not their constants):                                 */
/*  L1 gray = (77 R + 150 G + 29 B + 128) >> 8.                                               */
/*  L2 candidates: pixels inside one of the m detection areas (Algorithm 2, step 1) and at     */
/*     least LORB_MARGIN px from the image border (room for every neighbourhood below).       */
/*  L3 FAST (Algorithm 1, step 4): FAST-9 on the 16-pixel circle of radius 3, threshold t:    */
/*     a corner when 9 contiguous circle pixels are all > I(p) + t or all < I(p) - t.         */
/*  L4 gradients (step 1): Ix = I(x+1, y) - I(x-1, y), Iy = I(x, y+1) - I(x, y-1).           */
/*  L5 Gaussian weighting with sigma = 1 (step 3): the binomial [1,4,6,4,1] in x and y        */
/*     (variance exactly 1), unnormalised: A = sum b b Ix^2, B = sum b b Iy^2, C = sum b b IxIy.*/
/*  L6 Harris response with alpha = 0.04 (step 5): R' = 25 (AB - C^2) - (A + B)^2 = 25 R;      */
/*     kept when R' > harris_t.                                                               */
/*  L7 non-maximum suppression (step 6) over the 8-neighbourhood, ties to the lower index     */
/*     y W + x; the N (= P) strongest (step 7, Algorithm 2 step 3): R' descending, index      */
/*     ascending.                                                                             */
/*  L8 BRIEF (Sec. 4.1.2, Algorithm 2 step 4): smoothed image S = binomial 5x5 of gray        */
/*     (unnormalised); n_d = 256 point pairs (p_k, q_k) of offsets in [-15, 15]^2 (an input);  */
/*     bit k = [S(x + p_k) > S(x + q_k)], stored LSB-first in 32 bytes.                       */
/* ------------------------------------------------------------------------------------------ */

#define LORB_MARGIN 18
#define LORB_ND 256

static const int fast_dx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
static const int fast_dy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};
static const int binom5[5] = {1, 4, 6, 4, 1};

static int fast9(const uint8_t* g, int W, int x, int y, int t) {
    const int p = g[(int64_t)y * W + x];
    int run_b = 0, run_d = 0;
    /* walk the circle twice so that arcs wrapping past the start are seen */
    for (int k = 0; k < 32; ++k) {
        const int c = g[(int64_t)(y + fast_dy[k & 15]) * W + x + fast_dx[k & 15]];
        run_b = c > p + t ? run_b + 1 : 0;
        run_d = c < p - t ? run_d + 1 : 0;
        if (run_b >= 9 || run_d >= 9) return 1;
    }
    return 0;
}

typedef struct {
    int64_t r;
    int32_t idx;
} lorb_cand;

static int lorb_better(const lorb_cand* a, const lorb_cand* b) {
    return a->r > b->r || (a->r == b->r && a->idx < b->idx);
}

static int lorb_cmp(const void* pa, const void* pb) {
    const lorb_cand* a = (const lorb_cand*)pa;
    const lorb_cand* b = (const lorb_cand*)pb;
    if (lorb_better(a, b)) return -1;
    if (lorb_better(b, a)) return 1;
    return 0;
}

/*
 * frame: W x H RGB8 (pitch bytes); areas: n_areas x (x0, y0, x1, y1), half-open image
 * rectangles; pattern: LORB_ND x (px, py, qx, qy).  Outputs (up to max_points): out_xy
 * (x, y), out_resp (R'), out_desc (32 bytes each); *out_count the number written.  dbg_resp
 * (optional, W*H): R' of every candidate that is a FAST corner with R' > harris_t, INT64_MIN
 * elsewhere (before non-maximum suppression).
 */
int oracle_lorb(int W, int H, const uint8_t* frame, int64_t pitch, const int32_t* areas, int n_areas, int fast_t,
                int64_t harris_t, int max_points, const int8_t* pattern, int32_t* out_xy, int64_t* out_resp,
                uint8_t* out_desc, int32_t* out_count, int64_t* dbg_resp) {
    if (W < 1 || H < 1 || !frame || pitch < 3LL * W || n_areas < 0 || (n_areas > 0 && !areas) || fast_t < 0 ||
        max_points < 0 || !pattern || !out_count)
        return OR_EINVAL;
    for (int k = 0; k < LORB_ND; ++k)
        for (int j = 0; j < 4; ++j)
            if (pattern[4 * k + j] < -15 || pattern[4 * k + j] > 15) return OR_EINVAL;
    const int64_t N = (int64_t)W * H;
    uint8_t* gray = (uint8_t*)malloc((size_t)N);
    int64_t* resp = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    uint8_t* mask = (uint8_t*)calloc((size_t)N, 1);
    lorb_cand* cand = (lorb_cand*)malloc(sizeof(lorb_cand) * (size_t)N);
    if (!gray || !resp || !mask || !cand) {
        free(gray); free(resp); free(mask); free(cand);
        return OR_ENOMEM;
    }
    /* L1 */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t* q = frame + (int64_t)y * pitch + 3 * (int64_t)x;
            gray[(int64_t)y * W + x] = (uint8_t)((77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8);
        }
    /* L2: candidate mask */
    for (int a = 0; a < n_areas; ++a) {
        int x0 = areas[4 * a], y0 = areas[4 * a + 1], x1 = areas[4 * a + 2], y1 = areas[4 * a + 3];
        if (x0 < LORB_MARGIN) x0 = LORB_MARGIN;
        if (y0 < LORB_MARGIN) y0 = LORB_MARGIN;
        if (x1 > W - LORB_MARGIN) x1 = W - LORB_MARGIN;
        if (y1 > H - LORB_MARGIN) y1 = H - LORB_MARGIN;
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) mask[(int64_t)y * W + x] = 1;
    }
    /* L3-L6 */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t o = (int64_t)y * W + x;
            resp[o] = INT64_MIN;
            if (!mask[o] || !fast9(gray, W, x, y, fast_t)) continue;
            int64_t A = 0, B = 0, C = 0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    const int64_t q = (int64_t)(y + dy) * W + (x + dx);
                    const int ix = (int)gray[q + 1] - (int)gray[q - 1];
                    const int iy = (int)gray[q + W] - (int)gray[q - W];
                    const int64_t w = binom5[dx + 2] * binom5[dy + 2];
                    A += w * ix * ix;
                    B += w * iy * iy;
                    C += w * ix * iy;
                }
            const int64_t r = 25 * (A * B - C * C) - (A + B) * (A + B);
            if (r > harris_t) resp[o] = r;
        }
    if (dbg_resp) memcpy(dbg_resp, resp, sizeof(int64_t) * (size_t)N);
    /* L7 */
    int64_t nc = 0;
    for (int y = 1; y < H - 1; ++y)
        for (int x = 1; x < W - 1; ++x) {
            const int64_t o = (int64_t)y * W + x;
            if (resp[o] == INT64_MIN) continue;
            lorb_cand me = {resp[o], (int32_t)o};
            int keep = 1;
            for (int dy = -1; dy <= 1 && keep; ++dy)
                for (int dx = -1; dx <= 1 && keep; ++dx) {
                    if (!dx && !dy) continue;
                    const int64_t q = o + (int64_t)dy * W + dx;
                    if (resp[q] == INT64_MIN) continue;
                    lorb_cand other = {resp[q], (int32_t)q};
                    if (!lorb_better(&me, &other)) keep = 0;
                }
            if (keep) cand[nc++] = me;
        }
    qsort(cand, (size_t)nc, sizeof(lorb_cand), lorb_cmp);
    const int n = nc < max_points ? (int)nc : max_points;
    /* L8 */
    for (int k = 0; k < n; ++k) {
        const int x = cand[k].idx % W, y = cand[k].idx / W;
        if (out_xy) {
            out_xy[2 * k] = x;
            out_xy[2 * k + 1] = y;
        }
        if (out_resp) out_resp[k] = cand[k].r;
        if (!out_desc) continue;
        uint8_t* d = out_desc + 32 * (int64_t)k;
        memset(d, 0, 32);
        for (int b = 0; b < LORB_ND; ++b) {
            int64_t s[2];
            for (int e = 0; e < 2; ++e) {
                const int px = x + pattern[4 * b + 2 * e], py = y + pattern[4 * b + 2 * e + 1];
                int64_t acc = 0;
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx)
                        acc += binom5[dx + 2] * binom5[dy + 2] * gray[(int64_t)(py + dy) * W + px + dx];
                s[e] = acc;
            }
            if (s[0] > s[1]) d[b >> 3] |= (uint8_t)(1u << (b & 7));
        }
    }
    *out_count = n;
    free(gray);
    free(resp);
    free(mask);
    free(cand);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Feature matching and homography estimation (Sec. 4.2, Algorithm 3)                         */
/*                                                                                            */
/* Readings:                                                                                  */
/*  M1 Multi-Probe LSH (Sec. 4.2.1): L tables, each hashing a descriptor to k of its 256 bits  */
/*     (positions given); a query probes its own bucket and the k buckets at Hamming distance  */
/*     1 of every table.  Among the probed descriptors of image B the nearest (Hamming, ties to  */
/*     the lower index) is the match when its distance is <= max_dist and passes the ratio     */
/*     test ratio_den * d1 < ratio_num * d2 (d2: nearest other probed index; none: passes).    */
/*  M2 quality order (Algorithm 3, step 1): distance ascending, then query index ascending.    */
/*  M3 PROSAC (Sec. 4.2.2, Algorithm 3, step 2): the growth schedule of Chum and Matas with     */
/*     m = 4 and T_N = 200000 (its increments evaluated exactly in integers); iteration t samples the newest of the top n and 3 others from    */
/*     the top n - 1 (or 4 from the top n once t exceeds T'_n); samples are drawn without        */
/*     replacement from given random words (4 per iteration).  Hypothesis: the homography with  */
/*     h33 = 1 through the 4 pairs (8x8 Gaussian elimination, partial pivoting, ties to the     */
/*     lower row; |pivot| < 1e-12 rejects the sample), fitted in coordinates normalised per     */
/*     image (centre and half-extent of the matched points' bounding box, as Hartley's          */
/*     normalisation).  Inlier: in front (w > 0) and squared transfer error < inlier_px^2 (in   */
/*     normalised units of image B).  Best: most inliers, ties to the earlier iteration; then   */
/*     least squares on its inliers (normal equations summed in quality order, same solver),    */
/*     returned in pixel coordinates with h33 = 1.                                              */
/*  Geometry in IEEE double without contractions, so that a device implementation in the    */
/*  same operation order takes the same decisions.                                            */
/* ------------------------------------------------------------------------------------------ */

static int hamming256(const uint8_t* a, const uint8_t* b) {
    int d = 0;
    for (int k = 0; k < 32; ++k) d += __builtin_popcount((unsigned)(a[k] ^ b[k]));
    return d;
}

static uint32_t lsh_key(const uint8_t* d, const uint8_t* bits, int k) {
    uint32_t key = 0;
    for (int j = 0; j < k; ++j) key |= (uint32_t)((d[bits[j] >> 3] >> (bits[j] & 7)) & 1u) << j;
    return key;
}

/* solve the 8x8 system M h = r in place (row-major M), partial pivoting; returns 0 when singular */
static int solve8(double M[8][8], double r[8], double h[8]) {
    for (int c = 0; c < 8; ++c) {
        int p = c;
        for (int i = c + 1; i < 8; ++i)
            if (fabs(M[i][c]) > fabs(M[p][c])) p = i;
        if (!(fabs(M[p][c]) >= 1e-12)) return 0;
        if (p != c) {
            for (int j = 0; j < 8; ++j) {
                const double t = M[c][j];
                M[c][j] = M[p][j];
                M[p][j] = t;
            }
            const double t = r[c];
            r[c] = r[p];
            r[p] = t;
        }
        for (int i = c + 1; i < 8; ++i) {
            const double f = M[i][c] / M[c][c];
            for (int j = c; j < 8; ++j) M[i][j] = M[i][j] - f * M[c][j];
            r[i] = r[i] - f * r[c];
        }
    }
    for (int c = 7; c >= 0; --c) {
        double s = r[c];
        for (int j = c + 1; j < 8; ++j) s = s - M[c][j] * h[j];
        h[c] = s / M[c][c];
    }
    return 1;
}

static int homography4(const double* ax, const double* ay, const double* bx, const double* by, double h[8]) {
    double M[8][8], r[8];
    for (int k = 0; k < 4; ++k) {
        const double x = ax[k], y = ay[k], u = bx[k], v = by[k];
        double* m0 = M[2 * k];
        double* m1 = M[2 * k + 1];
        m0[0] = x; m0[1] = y; m0[2] = 1.0; m0[3] = 0.0; m0[4] = 0.0; m0[5] = 0.0; m0[6] = -(u * x); m0[7] = -(u * y);
        m1[0] = 0.0; m1[1] = 0.0; m1[2] = 0.0; m1[3] = x; m1[4] = y; m1[5] = 1.0; m1[6] = -(v * x); m1[7] = -(v * y);
        r[2 * k] = u;
        r[2 * k + 1] = v;
    }
    return solve8(M, r, h);
}

static int is_inlier(const double h[8], double x, double y, double u, double v, double t2) {
    const double w = h[6] * x + h[7] * y + 1.0;
    if (!(w > 0.0)) return 0;
    const double pu = (h[0] * x + h[1] * y + h[2]) / w - u;
    const double pv = (h[3] * x + h[4] * y + h[5]) / w - v;
    return pu * pu + pv * pv < t2;
}

/* PROSAC growth schedule (m = 4, T_N = 200000): T_n = T_N C(n, m) / C(N, m) is the expected
 * number of the T_N samples drawn from the top n; the top n grows to n + 1 at iteration T'_n, with
 * T'_m = 1 and T'_{n+1} = T'_n + ceil(T_{n+1} - T_n).  The increment is evaluated exactly:
 * T_{n+1} - T_n = T_N m n (n-1) (n-2) / (N (N-1) (N-2) (N-3)), an integer ceiling division.
 * Output for t = 1..T: n(t), and whether the schedule has passed (T'_n < t: sample uniformly
 * from the top n). */
static void prosac_schedule(int N, int T, int* nt, uint8_t* uni) {
    const long long Q = (long long)N * (N - 1) * (N - 2) * (N - 3);
    int n = 4;
    long long Tp = 1;
    for (int t = 1; t <= T; ++t) {
        if (t == Tp && n < N) {
            const long long num = 800000LL * n * (n - 1) * (n - 2);
            Tp += (num + Q - 1) / Q;
            n = n + 1;
        }
        nt[t - 1] = n;
        uni[t - 1] = Tp < t ? 1 : 0;
    }
}

int oracle_prosac_schedule(int N, int T, int32_t* nt, uint8_t* uni) {
    if (N < 4 || N > 65536 || T < 0 || (T > 0 && (!nt || !uni))) return OR_EINVAL;
    prosac_schedule(N, T, nt, uni);
    return OR_OK;
}

/* the j-th smallest element of {0..n-1} not in chosen[0..c) */
static int nth_free(int j, const int* chosen, int c) {
    int s[4];
    for (int i = 0; i < c; ++i) s[i] = chosen[i];
    for (int i = 1; i < c; ++i)
        for (int k = i; k > 0 && s[k - 1] > s[k]; --k) {
            const int tmp = s[k];
            s[k] = s[k - 1];
            s[k - 1] = tmp;
        }
    for (int i = 0; i < c; ++i)
        if (s[i] <= j) ++j;
    return j;
}

/* the 4 sample indices (into the quality order) of iteration t */
static void prosac_sample(int n, int uniform, const uint32_t* rnd, int* idx) {
    if (uniform) {
        for (int k = 0; k < 4; ++k) idx[k] = nth_free((int)(rnd[k] % (uint32_t)(n - k)), idx, k);
    } else {
        idx[0] = n - 1;
        int chosen[3];
        for (int k = 0; k < 3; ++k) {
            chosen[k] = nth_free((int)(rnd[k] % (uint32_t)(n - 1 - k)), chosen, k);
            idx[k + 1] = chosen[k];
        }
    }
}

int oracle_prosac_sample(int n, int uniform, const uint32_t* rnd, int32_t* idx) {
    if (n < 4 || !rnd || !idx) return OR_EINVAL;
    int v[4];
    prosac_sample(n, uniform, rnd, v);
    for (int k = 0; k < 4; ++k) idx[k] = v[k];
    return OR_OK;
}

/*
 * xy_a, desc_a (na points), xy_b, desc_b (nb points); bits: L x k bit positions.  rnd: iters x 4
 * random words.  Outputs: matches (up to na, quality order) as (index a, index b, distance),
 * *n_matches; H (9, h33 = 1, maps image-A points to image B), *n_inliers (0: no model), inlier
 * flags per match (optional).
 */
int oracle_match_prosac(int na, const int32_t* xy_a, const uint8_t* desc_a, int nb, const int32_t* xy_b,
                        const uint8_t* desc_b, int L, int k, const uint8_t* bits, int max_dist, int ratio_num,
                        int ratio_den, double inlier_px, int iters, const uint32_t* rnd, int32_t* matches,
                        int32_t* n_matches, double* H, int32_t* n_inliers, uint8_t* inlier) {
    if (na < 0 || nb < 0 || L < 1 || L > 32 || k < 1 || k > 20 || !bits || iters < 0 || (iters > 0 && !rnd) ||
        !matches || !n_matches || !H || !n_inliers || ratio_den < 1 || ratio_num < 1)
        return OR_EINVAL;
    for (int i = 0; i < L * k; ++i)
        if (bits[i] > 255) return OR_EINVAL;
    /* M1: tables as (key, index) sorted by key, index */
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)L * (nb > 0 ? nb : 1));
    int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * (size_t)L * (nb > 0 ? nb : 1));
    int32_t* mt = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(na > 0 ? na : 1));
    if (!keys || !ord || !mt) {
        free(keys); free(ord); free(mt);
        return OR_ENOMEM;
    }
    for (int l = 0; l < L; ++l) {
        for (int i = 0; i < nb; ++i) {
            keys[(size_t)l * nb + i] = lsh_key(desc_b + 32 * (size_t)i, bits + l * k, k);
            ord[(size_t)l * nb + i] = i;
        }
        /* insertion sort by (key, index): small tables */
        uint32_t* kk = keys + (size_t)l * nb;
        int32_t* oo = ord + (size_t)l * nb;
        for (int i = 1; i < nb; ++i)
            for (int j = i; j > 0 && kk[j - 1] > kk[j]; --j) {
                const uint32_t tk = kk[j]; kk[j] = kk[j - 1]; kk[j - 1] = tk;
                const int32_t to = oo[j]; oo[j] = oo[j - 1]; oo[j - 1] = to;
            }
    }
    int nm = 0;
    for (int a = 0; a < na; ++a) {
        const uint8_t* da = desc_a + 32 * (size_t)a;
        int b1 = -1, d1 = 1 << 30, b2 = -1, d2 = 1 << 30;
        for (int l = 0; l < L; ++l) {
            const uint32_t q0 = lsh_key(da, bits + l * k, k);
            for (int p = -1; p < k; ++p) {
                const uint32_t q = p < 0 ? q0 : (q0 ^ (1u << p));
                /* bucket range by binary search */
                int lo = 0, hi = nb;
                while (lo < hi) {
                    const int mid = (lo + hi) / 2;
                    if (keys[(size_t)l * nb + mid] < q) lo = mid + 1; else hi = mid;
                }
                for (int i = lo; i < nb && keys[(size_t)l * nb + i] == q; ++i) {
                    const int b = ord[(size_t)l * nb + i];
                    const int d = hamming256(da, desc_b + 32 * (size_t)b);
                    if (d < d1 || (d == d1 && b < b1)) {
                        if (b != b1) { d2 = d1; b2 = b1; }
                        d1 = d; b1 = b;
                    } else if (b != b1 && (d < d2 || (d == d2 && b < b2))) {
                        d2 = d; b2 = b;
                    }
                }
            }
        }
        (void)b2;
        if (b1 >= 0 && d1 <= max_dist && (d2 == (1 << 30) || (long long)ratio_den * d1 < (long long)ratio_num * d2)) {
            mt[3 * nm] = a;
            mt[3 * nm + 1] = b1;
            mt[3 * nm + 2] = d1;
            ++nm;
        }
    }
    /* M2: quality order (insertion sort: distance, then query index; stable in a) */
    for (int i = 1; i < nm; ++i)
        for (int j = i; j > 0 && mt[3 * (j - 1) + 2] > mt[3 * j + 2]; --j)
            for (int e = 0; e < 3; ++e) {
                const int32_t t = mt[3 * j + e]; mt[3 * j + e] = mt[3 * (j - 1) + e]; mt[3 * (j - 1) + e] = t;
            }
    memcpy(matches, mt, sizeof(int32_t) * 3 * (size_t)nm);
    *n_matches = nm;
    /* M3 */
    for (int i = 0; i < 9; ++i) H[i] = i % 4 == 0 ? 1.0 : 0.0;
    *n_inliers = 0;
    if (inlier) memset(inlier, 0, (size_t)nm);
    int best_t = -1, best_c = -1;
    double best_h[8];
    /* normalisation of each image's matched points: centre and scale of their bounding box */
    double ca[2] = {0.0, 0.0}, cb[2] = {0.0, 0.0}, sa = 1.0, sb = 1.0;
    if (nm > 0) {
        int mn[2][2], mx[2][2];
        for (int e = 0; e < 2; ++e) {
            const int32_t* xy = e == 0 ? xy_a : xy_b;
            for (int c = 0; c < 2; ++c) mn[e][c] = mx[e][c] = xy[2 * mt[e] + c];
            for (int i = 1; i < nm; ++i)
                for (int c = 0; c < 2; ++c) {
                    const int v = xy[2 * mt[3 * i + e] + c];
                    if (v < mn[e][c]) mn[e][c] = v;
                    if (v > mx[e][c]) mx[e][c] = v;
                }
        }
        for (int c = 0; c < 2; ++c) {
            ca[c] = 0.5 * ((double)mn[0][c] + (double)mx[0][c]);
            cb[c] = 0.5 * ((double)mn[1][c] + (double)mx[1][c]);
        }
        int ra = mx[0][0] - mn[0][0], rb = mx[1][0] - mn[1][0];
        if (mx[0][1] - mn[0][1] > ra) ra = mx[0][1] - mn[0][1];
        if (mx[1][1] - mn[1][1] > rb) rb = mx[1][1] - mn[1][1];
        sa = 2.0 / (double)(ra > 1 ? ra : 1);
        sb = 2.0 / (double)(rb > 1 ? rb : 1);
    }
#define NAX(i) (((double)xy_a[2 * mt[3 * (i)]] - ca[0]) * sa)
#define NAY(i) (((double)xy_a[2 * mt[3 * (i)] + 1] - ca[1]) * sa)
#define NBX(i) (((double)xy_b[2 * mt[3 * (i) + 1]] - cb[0]) * sb)
#define NBY(i) (((double)xy_b[2 * mt[3 * (i) + 1] + 1] - cb[1]) * sb)
    if (nm >= 4 && iters > 0) {
        int* nt = (int*)malloc(sizeof(int) * (size_t)iters);
        uint8_t* uni = (uint8_t*)malloc((size_t)iters);
        if (!nt || !uni) {
            free(nt); free(uni); free(keys); free(ord); free(mt);
            return OR_ENOMEM;
        }
        prosac_schedule(nm, iters, nt, uni);
        const double tn = inlier_px * sb;
        const double t2 = tn * tn;
        for (int t = 0; t < iters; ++t) {
            int idx[4];
            prosac_sample(nt[t], uni[t], rnd + 4 * (size_t)t, idx);
            double ax[4], ay[4], bx[4], by[4], h[8];
            for (int q = 0; q < 4; ++q) {
                ax[q] = NAX(idx[q]);
                ay[q] = NAY(idx[q]);
                bx[q] = NBX(idx[q]);
                by[q] = NBY(idx[q]);
            }
            if (!homography4(ax, ay, bx, by, h)) continue;
            int c = 0;
            for (int i = 0; i < nm; ++i) c += is_inlier(h, NAX(i), NAY(i), NBX(i), NBY(i), t2);
            if (c > best_c) {
                best_c = c;
                best_t = t;
                memcpy(best_h, h, sizeof(best_h));
            }
        }
        free(nt);
        free(uni);
        if (best_t >= 0 && best_c >= 4) {
            /* least squares on the inliers: normal equations in quality order */
            double M[8][8], r[8], h[8];
            memset(M, 0, sizeof(M));
            memset(r, 0, sizeof(r));
            for (int i = 0; i < nm; ++i) {
                const double x = NAX(i), y = NAY(i), u = NBX(i), v = NBY(i);
                if (!is_inlier(best_h, x, y, u, v, t2)) continue;
                if (inlier) inlier[i] = 1;
                const double row0[8] = {x, y, 1.0, 0.0, 0.0, 0.0, -(u * x), -(u * y)};
                const double row1[8] = {0.0, 0.0, 0.0, x, y, 1.0, -(v * x), -(v * y)};
                for (int p = 0; p < 8; ++p) {
                    for (int q = 0; q < 8; ++q) M[p][q] = M[p][q] + row0[p] * row0[q] + row1[p] * row1[q];
                    r[p] = r[p] + row0[p] * u + row1[p] * v;
                }
            }
            const double* hn = solve8(M, r, h) ? h : best_h;
            /* back to pixels: H = Tb^-1 Hn Ta, Ta = [[sa, 0, -sa ca0], [0, sa, -sa ca1], [0, 0, 1]] */
            const double Hn[9] = {hn[0], hn[1], hn[2], hn[3], hn[4], hn[5], hn[6], hn[7], 1.0};
            const double Ta[9] = {sa, 0.0, -(sa * ca[0]), 0.0, sa, -(sa * ca[1]), 0.0, 0.0, 1.0};
            const double Tbi[9] = {1.0 / sb, 0.0, cb[0], 0.0, 1.0 / sb, cb[1], 0.0, 0.0, 1.0};
            double P[9], Q[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    P[3 * i + j] = Hn[3 * i] * Ta[j] + Hn[3 * i + 1] * Ta[3 + j] + Hn[3 * i + 2] * Ta[6 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Q[3 * i + j] = Tbi[3 * i] * P[j] + Tbi[3 * i + 1] * P[3 + j] + Tbi[3 * i + 2] * P[6 + j];
            for (int i = 0; i < 9; ++i) H[i] = Q[i] / Q[8];
            *n_inliers = best_c;
        }
    }
#undef NAX
#undef NAY
#undef NBX
#undef NBY
    free(keys);
    free(ord);
    free(mt);
    return OR_OK;
}
