/*
 * Seeded synthetic scene and camera-view renderer.
 *
 * This file produces INPUT DATA only: camera frames rendered from a procedural
 * scene through a known camera->canvas homography.  It holds none of the
 * stitching arithmetic (no resampling of images, no pyramids, no blending):
 * every view pixel is a point evaluation of an analytic scene function, so
 * neither the oracle nor the CUDA path shares any code with it.
 *
 * Scene (defined on the canvas plane, in canvas pixel units):
 *   - smooth value noise: integer lattice of spacing `lattice` px, cubic fade
 *     3t^2 - 2t^3, 4 octaves (spacing halves, amplitude halves), one
 *     independent lattice per colour channel, lattice values from a
 *     counter-based hash (splitmix64 finaliser) of (seed, octave, channel, ix, iy);
 *   - axis-aligned rectangles drawn in order over the noise, each solid,
 *     horizontally or vertically striped, or checkered, with two colours.
 * Frame t of a sequence shows the scene translated by +shift_x * t px in x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double x0, y0, x1, y1; /* [x0,x1) x [y0,y1) in scene px */
    int32_t kind;          /* 0 solid, 1 horizontal stripes, 2 vertical stripes, 3 checker */
    int32_t period;        /* stripe / checker period in px (>= 2) */
    double ca[3], cb[3];   /* two colours in [0,1] */
} synth_rect;

static inline uint64_t splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double lattice_value(uint64_t seed, int oct, int ch, int64_t ix, int64_t iy) {
    uint64_t h = splitmix(seed ^ ((uint64_t)oct << 56) ^ ((uint64_t)ch << 48));
    h = splitmix(h ^ (uint64_t)(uint32_t)(int32_t)ix);
    h = splitmix(h ^ ((uint64_t)(uint32_t)(int32_t)iy << 21));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static inline double fade(double t) { return t * t * (3.0 - 2.0 * t); }

static void noise_rgb(uint64_t seed, double lattice, double X, double Y, double out[3]) {
    double amp = 1.0, norm = 0.0;
    out[0] = out[1] = out[2] = 0.0;
    double s = lattice;
    for (int oct = 0; oct < 4; ++oct) {
        double gx = X / s, gy = Y / s;
        double fx0 = floor(gx), fy0 = floor(gy);
        int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
        double tx = fade(gx - fx0), ty = fade(gy - fy0);
        for (int c = 0; c < 3; ++c) {
            double v00 = lattice_value(seed, oct, c, ix, iy);
            double v10 = lattice_value(seed, oct, c, ix + 1, iy);
            double v01 = lattice_value(seed, oct, c, ix, iy + 1);
            double v11 = lattice_value(seed, oct, c, ix + 1, iy + 1);
            double a = v00 + (v10 - v00) * tx;
            double b = v01 + (v11 - v01) * tx;
            out[c] += amp * (a + (b - a) * ty);
        }
        norm += amp;
        amp *= 0.5;
        s *= 0.5;
    }
    for (int c = 0; c < 3; ++c) out[c] /= norm;
}

/* Coarse bins of rectangle indices so each point only tests nearby rectangles. */
typedef struct {
    double bx0, by0, cell;
    int nbx, nby;
    int32_t* start; /* nbx*nby+1 */
    int32_t* idx;
} rect_bins;

static int bins_build(const synth_rect* r, int n, double cell, rect_bins* b) {
    double minx = 0, miny = 0, maxx = 1, maxy = 1;
    for (int i = 0; i < n; ++i) {
        if (i == 0 || r[i].x0 < minx) minx = r[i].x0;
        if (i == 0 || r[i].y0 < miny) miny = r[i].y0;
        if (i == 0 || r[i].x1 > maxx) maxx = r[i].x1;
        if (i == 0 || r[i].y1 > maxy) maxy = r[i].y1;
    }
    b->bx0 = minx; b->by0 = miny; b->cell = cell;
    b->nbx = (int)((maxx - minx) / cell) + 1;
    b->nby = (int)((maxy - miny) / cell) + 1;
    int nb = b->nbx * b->nby;
    int32_t* cnt = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
    if (!cnt) return -1;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            b->start = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
            for (int k = 0; k < nb; ++k) b->start[k + 1] = b->start[k] + cnt[k];
            b->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(b->start[nb] + 1));
            memset(cnt, 0, sizeof(int32_t) * (size_t)nb);
        }
        for (int i = 0; i < n; ++i) {
            int cx0 = (int)((r[i].x0 - minx) / cell), cx1 = (int)((r[i].x1 - minx) / cell);
            int cy0 = (int)((r[i].y0 - miny) / cell), cy1 = (int)((r[i].y1 - miny) / cell);
            for (int cy = cy0; cy <= cy1 && cy < b->nby; ++cy)
                for (int cx = cx0; cx <= cx1 && cx < b->nbx; ++cx) {
                    int k = cy * b->nbx + cx;
                    if (pass == 0) cnt[k]++;
                    else b->idx[b->start[k] + cnt[k]++] = i; /* ascending i: draw order */
                }
        }
    }
    free(cnt);
    return 0;
}

static void scene_eval(uint64_t seed, double lattice, const synth_rect* r, const rect_bins* b,
                       double X, double Y, double out[3]) {
    noise_rgb(seed, lattice, X, Y, out);
    int cx = (int)floor((X - b->bx0) / b->cell), cy = (int)floor((Y - b->by0) / b->cell);
    if (cx < 0 || cy < 0 || cx >= b->nbx || cy >= b->nby) return;
    int k = cy * b->nbx + cx;
    for (int j = b->start[k]; j < b->start[k + 1]; ++j) {
        const synth_rect* q = &r[b->idx[j]];
        if (X < q->x0 || X >= q->x1 || Y < q->y0 || Y >= q->y1) continue;
        int sel = 0;
        double p = (double)q->period;
        if (q->kind == 1) sel = ((int64_t)floor((Y - q->y0) / p)) & 1;
        else if (q->kind == 2) sel = ((int64_t)floor((X - q->x0) / p)) & 1;
        else if (q->kind == 3) sel = (((int64_t)floor((X - q->x0) / p)) + ((int64_t)floor((Y - q->y0) / p))) & 1;
        const double* c = sel ? q->cb : q->ca;
        out[0] = c[0]; out[1] = c[1]; out[2] = c[2];
    }
}

/*
 * Render one camera view.  Pixel (u, v) of the view (centre at integer
 * coordinates) shows the scene at canvas point M * (u, v, 1) (projected),
 * translated to scene coordinates by (off_x, off_y).  Quantised with
 * round-half-even of 255 * value after clamping to [0, 1].
 * Returns 0, or -1 when a pixel maps behind the camera (w <= 0).
 */
int synth_render_view(uint64_t seed, double lattice, const synth_rect* rects, int n_rects,
                      const double* M, int W, int H, double off_x, double off_y,
                      uint8_t* out, int64_t pitch) {
    rect_bins b;
    memset(&b, 0, sizeof(b));
    if (bins_build(rects, n_rects, 64.0, &b) != 0) return -2;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int v = 0; v < H; ++v) {
        uint8_t* row = out + (int64_t)v * pitch;
        for (int u = 0; u < W; ++u) {
            double xw = M[0] * u + M[1] * v + M[2];
            double yw = M[3] * u + M[4] * v + M[5];
            double ww = M[6] * u + M[7] * v + M[8];
            if (!(ww > 0.0)) { bad |= 1; row[3 * u] = row[3 * u + 1] = row[3 * u + 2] = 0; continue; }
            double X = xw / ww + off_x, Y = yw / ww + off_y;
            double c[3];
            scene_eval(seed, lattice, rects, &b, X, Y, c);
            for (int k = 0; k < 3; ++k) {
                double t = c[k] < 0.0 ? 0.0 : (c[k] > 1.0 ? 1.0 : c[k]);
                row[3 * u + k] = (uint8_t)nearbyint(255.0 * t);
            }
        }
    }
    free(b.start);
    free(b.idx);
    return bad ? -1 : 0;
}

/*
 * Render one camera view of a scene laid on a cylindrical canvas (focal length f, centre
 * (cx, cy)).  Pixel (u, v) of the view looks along the ray Pinv * (u, v, 1) = (X, Y, Z), which
 * meets the canvas at x = cx + f atan2(X, Z), y = cy + f Y / hypot(X, Z); the scene is evaluated
 * there, translated by (off_x, off_y).  Returns 0, or -1 when a ray points backwards (Z <= 0 and
 * X = 0) so that its canvas column is undefined.
 */
int synth_render_view_cyl(uint64_t seed, double lattice, const synth_rect* rects, int n_rects,
                          const double* Pinv, int W, int H, double f, double cx, double cy, double off_x,
                          double off_y, uint8_t* out, int64_t pitch) {
    rect_bins b;
    memset(&b, 0, sizeof(b));
    if (bins_build(rects, n_rects, 64.0, &b) != 0) return -2;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int v = 0; v < H; ++v) {
        uint8_t* row = out + (int64_t)v * pitch;
        for (int u = 0; u < W; ++u) {
            double X = Pinv[0] * u + Pinv[1] * v + Pinv[2];
            double Y = Pinv[3] * u + Pinv[4] * v + Pinv[5];
            double Z = Pinv[6] * u + Pinv[7] * v + Pinv[8];
            double r = hypot(X, Z);
            if (!(r > 0.0)) { bad |= 1; row[3 * u] = row[3 * u + 1] = row[3 * u + 2] = 0; continue; }
            double xs = cx + f * atan2(X, Z) + off_x, ys = cy + f * Y / r + off_y;
            double c[3];
            scene_eval(seed, lattice, rects, &b, xs, ys, c);
            for (int k = 0; k < 3; ++k) {
                double t = c[k] < 0.0 ? 0.0 : (c[k] > 1.0 ? 1.0 : c[k]);
                row[3 * u + k] = (uint8_t)nearbyint(255.0 * t);
            }
        }
    }
    free(b.start);
    free(b.idx);
    return bad ? -1 : 0;
}

/* Render the scene itself on an axis-aligned grid (scene px), for inspection. */
int synth_render_scene(uint64_t seed, double lattice, const synth_rect* rects, int n_rects,
                       double x0, double y0, int W, int H, uint8_t* out) {
    rect_bins b;
    memset(&b, 0, sizeof(b));
    if (bins_build(rects, n_rects, 64.0, &b) != 0) return -2;
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double c[3];
            scene_eval(seed, lattice, rects, &b, x0 + u, y0 + v, c);
            for (int k = 0; k < 3; ++k) {
                double t = c[k] < 0.0 ? 0.0 : (c[k] > 1.0 ? 1.0 : c[k]);
                out[((int64_t)v * W + u) * 3 + k] = (uint8_t)nearbyint(255.0 * t);
            }
        }
    free(b.start);
    free(b.idx);
    return 0;
}
