// Internal declarations shared by the libstitch translation units (device structs, planner
// output, launch helpers).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "stitch.h"

#define MAXL STITCH_MAX_LEVELS
#define MAXC STITCH_MAX_CAMERAS

// Half-open rectangle of one pyramid level, in that level's canvas coordinates.
struct Rect {
    int x0, x1, y0, y1;
    __host__ __device__ int w() const { return x1 - x0; }
    __host__ __device__ int h() const { return y1 - y0; }
    __host__ __device__ bool empty() const { return x1 <= x0 || y1 <= y0; }
    __host__ __device__ bool contains(int x, int y) const { return x >= x0 && x < x1 && y >= y0 && y < y1; }
    __host__ __device__ long long area() const { return empty() ? 0 : (long long)w() * h(); }
};

// Per-camera descriptor, resident in device memory for the life of a rig.
struct CamDev {
    double A[9];     // canvas -> camera homography, a33 = +1 or -1
    int W, H;        // source frame size
    float gain;
    int visible;     // 0 when the camera's footprint misses the canvas
    Rect V;          // level-0 bounding box of the validity region (empty when !visible)
    Rect Om[MAXL];   // Omega^l: region on which the camera's pyramid is evaluated
    Rect Z[MAXL];    // Z^l: region where the camera's weight pyramid can be non-zero
    // plain path buffers
    float4* G[MAXL];   // Gaussian pyramid (r, g, b, weight) on Om[l], row pitch Om[l].w()
    float4* Lp[MAXL];  // (Laplacian r, g, b, weight) on Z[l] for l < L-1, row pitch Z[l].w()
    // fused path buffers
    void* FG[MAXL];    // Gaussian pyramid (r, g, b, weight) on Om[l] for l >= 1 (FP32 or FP16)
};

// Rig-wide sizes passed by value to kernels.
struct RigGeom {
    int ncam, levels;
    int seam;  // level-0 weights: 0 feather, 1 seam owner masks
    int cyl;   // canvas: 0 planar (homographies), 1 cylindrical (focal length cf, centre ccx, ccy)
    double cf, ccx, ccy;
    int nx[MAXL], ny[MAXL];  // canvas size of every level (nx[l+1] = ceil(nx[l] / 2))
};

// Device frame pointers of one call, passed by value.
struct FramePtrs {
    const uint8_t* p[MAXC];
    long long pitch[MAXC];
};

// Output descriptor of one call.
struct OutDesc {
    void* ptr;
    long long pitch;  // bytes
    int is_float;
};

// ------------------------------------------------------------------------------------------------
// debug build (STITCH_DEBUG): index checks that record the first failure in a device word of the
// translation unit and let the caller skip the access (no trap, so the context stays usable), and
// guard bands around every rig allocation.  Release builds compile the checks to `true`.

#ifdef STITCH_DEBUG
constexpr bool kStitchDebug = true;
#define STITCH_DCHECK(cond, code, val) ((cond) ? true : (stitch_dcheck_fail((code), (long long)(val)), false))
#else
constexpr bool kStitchDebug = false;
#define STITCH_DCHECK(cond, code, val) true
#endif

// Guard band around each rig allocation in the debug build: this many bytes before and after,
// filled with the quiet-NaN word kGuardWord.
constexpr size_t kGuardBytes = 256;
constexpr uint32_t kGuardWord = 0x7FC0DEADu;

// ------------------------------------------------------------------------------------------------
// small device helpers

// reflect-101 border folding on a grid of n samples: ... 2 1 | 0 1 2 ... n-1 | n-2 n-3 ...
__host__ __device__ __forceinline__ int fold101(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (n == 1) return 0;
    const int period = 2 * n - 2;
    int r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - r;
}

// Accurate per-tile parameterisation of a homography.  With (X, Y) the tile anchor and
// U0 = round(u(X, Y)), the offset u - U0 = (pu0 + pu1 dx + pu2 dy) / (q0 + q1 dx + q2 dy) is
// small, so single precision keeps ~1e-5 px accuracy anywhere on a 24000-px canvas; the
// coefficients are formed in double precision once per tile.
struct TileMap {
    int U0, V0;
    float pu0, pu1, pu2, pv0, pv1, pv2, q0, q1, q2;
};

__host__ __device__ __forceinline__ TileMap make_tile_map(const double* A, int X, int Y) {
    const double x = (double)X, y = (double)Y;
    const double n0 = A[0] * x + A[1] * y + A[2];
    const double m0 = A[3] * x + A[4] * y + A[5];
    const double d0 = A[6] * x + A[7] * y + A[8];
    double u0 = n0 / d0, v0 = m0 / d0;
    u0 = fmin(fmax(u0, -1.0e8), 1.0e8);
    v0 = fmin(fmax(v0, -1.0e8), 1.0e8);
    const double U = rint(u0), V = rint(v0);
    TileMap t;
    t.U0 = (int)U;
    t.V0 = (int)V;
    t.pu0 = (float)(n0 - U * d0);
    t.pu1 = (float)(A[0] - U * A[6]);
    t.pu2 = (float)(A[1] - U * A[7]);
    t.pv0 = (float)(m0 - V * d0);
    t.pv1 = (float)(A[3] - V * A[6]);
    t.pv2 = (float)(A[4] - V * A[7]);
    t.q0 = (float)d0;
    t.q1 = (float)A[6];
    t.q2 = (float)A[7];
    return t;
}

// Source position of canvas point (anchor + (dx, dy)) as integer part + fraction in [0, 1).
struct SrcPos {
    int iu, iv;
    float fu, fv;
    float den;
};

__device__ __forceinline__ SrcPos map_point(const TileMap& t, float dx, float dy) {
    SrcPos s;
    s.den = fmaf(t.q2, dy, fmaf(t.q1, dx, t.q0));
    // approximate reciprocal (2 ulp): the offsets it scales are below ~100 px, so the error in
    // the source position stays near 1e-5 px
    const float rden = __fdividef(1.0f, s.den);
    float ru = fmaf(t.pu2, dy, fmaf(t.pu1, dx, t.pu0)) * rden;
    float rv = fmaf(t.pv2, dy, fmaf(t.pv1, dx, t.pv0)) * rden;
    ru = fminf(fmaxf(ru, -1.0e7f), 1.0e7f);
    rv = fminf(fmaxf(rv, -1.0e7f), 1.0e7f);
    const float flu = floorf(ru), flv = floorf(rv);
    s.iu = t.U0 + (int)flu;
    s.iv = t.V0 + (int)flv;
    s.fu = ru - flu;
    s.fv = rv - flv;
    return s;
}

// Raw feather weight: distance (source px) to the nearest border of the validity rectangle
// [-0.5, W-0.5) x [-0.5, H-0.5), zero outside it or behind the camera.
__device__ __forceinline__ float feather_weight(const SrcPos& s, int W, int H) {
    if (!(s.den > 0.0f)) return 0.0f;
    const bool okx = (s.iu >= 0 || (s.iu == -1 && s.fu >= 0.5f)) && (s.iu <= W - 2 || (s.iu == W - 1 && s.fu < 0.5f));
    const bool oky = (s.iv >= 0 || (s.iv == -1 && s.fv >= 0.5f)) && (s.iv <= H - 2 || (s.iv == H - 1 && s.fv < 0.5f));
    if (!(okx && oky)) return 0.0f;
    const float u = (float)s.iu + s.fu, v = (float)s.iv + s.fv;
    float m = fminf(fminf(u + 0.5f, v + 0.5f), fminf(((float)W - 0.5f) - u, ((float)H - 0.5f) - v));
    return fmaxf(m, 0.0f);
}

// The canvas point (x, y) as the vector the camera matrix A acts on: (x, y, 1) on the planar
// canvas; on the cylindrical canvas the ray (sin t, (y - cy)/f, cos t) with t = (x - cx)/f.
__host__ __device__ inline void canvas_ray(const RigGeom& g, double x, double y, double r[3]) {
    if (g.cyl) {
        const double t = (x - g.ccx) / g.cf;
        r[0] = sin(t);
        r[1] = (y - g.ccy) / g.cf;
        r[2] = cos(t);
    } else {
        r[0] = x;
        r[1] = y;
        r[2] = 1.0;
    }
}

// Source point of canvas point (x, y) in camera c, FP64: (u, v) and w (> 0 in front).
__host__ __device__ inline double source_point64(const CamDev& c, const RigGeom& g, double x, double y, double* u,
                                                 double* v) {
    double r[3];
    canvas_ray(g, x, y, r);
    const double w = c.A[6] * r[0] + c.A[7] * r[1] + c.A[8] * r[2];
    *u = (c.A[0] * r[0] + c.A[1] * r[1] + c.A[2] * r[2]) / w;
    *v = (c.A[3] * r[0] + c.A[4] * r[1] + c.A[5] * r[2]) / w;
    return w;
}

// S2 feather weight of camera c at canvas point (x, y) in FP64: distance from the source point to
// the border of the pixel-edge rectangle [-0.5, W-0.5) x [-0.5, H-0.5), 0 outside it or behind
// the camera.
__host__ __device__ inline double feather_weight64(const CamDev& c, const RigGeom& g, double x, double y) {
    double u, v;
    const double w = source_point64(c, g, x, y, &u, &v);
    if (!(w > 0.0)) return 0.0;
    if (!(u >= -0.5 && u < c.W - 0.5 && v >= -0.5 && v < c.H - 0.5)) return 0.0;
    const double m = fmin(fmin(u + 0.5, v + 0.5), fmin(c.W - 0.5 - u, c.H - 0.5 - v));
    return m > 0.0 ? m : 0.0;
}

// SrcPos of canvas pixel (x, y) in camera c from the FP64 map (see map_pos64).
__device__ inline SrcPos map_point64(const CamDev& c, const RigGeom& g, int x, int y) {
    double u, v;
    const double w = source_point64(c, g, (double)x, (double)y, &u, &v);
    u = fmin(fmax(u, -1.0e7), 1.0e7);
    v = fmin(fmax(v, -1.0e7), 1.0e7);
    const double fu = floor(u), fv = floor(v);
    SrcPos s;
    s.iu = (int)fu;
    s.iv = (int)fv;
    s.fu = (float)(u - fu);
    s.fv = (float)(v - fv);
    s.den = w > 0.0 ? 1.0f : -1.0f;
    return s;
}

// Seam owner of canvas point (x, y) among n cameras given in ascending camera order by cam_at(k)
// (which must include every camera whose validity box contains the point): the first position k
// whose feather weight is > 0 and >= (1 - 1e-9) times the largest, -1 when no weight is > 0.
// Decided in FP64, so that the binary masks do not depend on the FP32 tile anchoring.
template <class CamAt>
__device__ inline int seam_owner(const RigGeom& g, int n, const CamAt& cam_at, int x, int y) {
    double wmax = 0.0;
    for (int k = 0; k < n; ++k) {
        const CamDev& c = cam_at(k);
        if (c.V.contains(x, y)) wmax = fmax(wmax, feather_weight64(c, g, (double)x, (double)y));
    }
    if (!(wmax > 0.0)) return -1;
    for (int k = 0; k < n; ++k) {
        const CamDev& c = cam_at(k);
        if (!c.V.contains(x, y)) continue;
        const double w = feather_weight64(c, g, (double)x, (double)y);
        if (w > 0.0 && w >= (1.0 - 1e-9) * wmax) return k;
    }
    return -1;
}

// Clamped texel coordinates and fractions of a bilinear sample.
struct Tap {
    int i0, i1, j0, j1;
    float fx, fy;
};

__device__ __forceinline__ Tap clamp_tap(const SrcPos& s, int W, int H) {
    Tap t;
    if (s.iu < 0) { t.i0 = 0; t.fx = 0.0f; }
    else if (s.iu >= W - 1) { t.i0 = W - 1; t.fx = 0.0f; }
    else { t.i0 = s.iu; t.fx = s.fu; }
    if (s.iv < 0) { t.j0 = 0; t.fy = 0.0f; }
    else if (s.iv >= H - 1) { t.j0 = H - 1; t.fy = 0.0f; }
    else { t.j0 = s.iv; t.fy = s.fv; }
    t.i1 = min(t.i0 + 1, W - 1);
    t.j1 = min(t.j0 + 1, H - 1);
    return t;
}

// Bilinear RGB sample of an 8-bit frame, scaled by `scale` (= gain / 255).
__device__ __forceinline__ float3 bilinear_rgb(const uint8_t* __restrict__ px, long long pitch, const Tap& t,
                                               float scale) {
    const uint8_t* r0 = px + (long long)t.j0 * pitch;
    const uint8_t* r1 = px + (long long)t.j1 * pitch;
    float3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p00 = __ldg(r0 + 3 * t.i0 + c), p01 = __ldg(r0 + 3 * t.i1 + c);
        const float p10 = __ldg(r1 + 3 * t.i0 + c), p11 = __ldg(r1 + 3 * t.i1 + c);
        const float top = fmaf(t.fx, p01 - p00, p00);
        const float bot = fmaf(t.fx, p11 - p10, p10);
        const float v = fmaf(t.fy, bot - top, top) * scale;
        if (c == 0) o.x = v; else if (c == 1) o.y = v; else o.z = v;
    }
    return o;
}

// Anchor for a camera's tile map: the tile origin clamped into the camera's validity box, where
// w > 0 is guaranteed by the planner.
__host__ __device__ __forceinline__ void tile_anchor(const Rect& V, int X, int Y, int* ax, int* ay) {
    *ax = min(max(X, V.x0), V.x1 - 1);
    *ay = min(max(Y, V.y0), V.y1 - 1);
}

// ------------------------------------------------------------------------------------------------
// lean per-sample helpers used by the fused kernels

// Exact float of an 8-bit value with one integer OR and one add: the bits 0x4B000000 | b encode
// 2^23 + b, so subtracting 2^23 leaves b (IEEE-754 single precision, no rounding).
__device__ __forceinline__ float u8_to_f(uint32_t b) { return __int_as_float(0x4B000000u | b) - 8388608.0f; }

// One camera's mapping of canvas point anchor + (dx, dy): fraction-exact source position,
// float source coordinates for the weight, and the sign of w.
struct Pos {
    int iu, iv;    // floor of the source coordinates
    float fu, fv;  // fractions in [0, 1)
    float u, v;    // source coordinates (for validity and weight)
    float den;     // w, positive in front of the camera
};

// map_pos with the column terms (the anchored numerators and denominator at row dy = 0) given:
// fmaf(t.pu1, dx, t.pu0) etc. on the planar canvas, a host-built column table on the cylindrical
// canvas (where a column is an angle); t.pu2, t.pv2, t.q2 are the per-row slopes on both.
__device__ __forceinline__ Pos map_pos_col(const TileMap& t, float fU0, float fV0, float nuc, float nvc, float dqc,
                                           float dy) {
    Pos p;
    p.den = fmaf(t.q2, dy, dqc);
    const float rden = __fdividef(1.0f, p.den);
    float ru = fmaf(t.pu2, dy, nuc) * rden;
    float rv = fmaf(t.pv2, dy, nvc) * rden;
    ru = fminf(fmaxf(ru, -1.0e7f), 1.0e7f);
    rv = fminf(fmaxf(rv, -1.0e7f), 1.0e7f);
    const float flu = floorf(ru), flv = floorf(rv);
    p.iu = t.U0 + (int)flu;
    p.iv = t.V0 + (int)flv;
    p.fu = ru - flu;
    p.fv = rv - flv;
    p.u = fU0 + ru;
    p.v = fV0 + rv;
    return p;
}

// Position of canvas pixel (x, y) in camera c from the FP64 map (paths that are not per-frame
// hot: GENERAL tiles and the plain path on the cylindrical canvas).
__device__ inline Pos map_pos64(const CamDev& c, const RigGeom& g, int x, int y) {
    double u, v;
    const double w = source_point64(c, g, (double)x, (double)y, &u, &v);
    Pos p;
    u = fmin(fmax(u, -1.0e7), 1.0e7);
    v = fmin(fmax(v, -1.0e7), 1.0e7);
    const double fu = floor(u), fv = floor(v);
    p.iu = (int)fu;
    p.iv = (int)fv;
    p.fu = (float)(u - fu);
    p.fv = (float)(v - fv);
    p.u = (float)u;
    p.v = (float)v;
    p.den = w > 0.0 ? 1.0f : -1.0f;
    return p;
}

__device__ __forceinline__ Pos map_pos(const TileMap& t, float fU0, float fV0, float dx, float dy) {
    Pos p;
    p.den = fmaf(t.q2, dy, fmaf(t.q1, dx, t.q0));
    const float rden = __fdividef(1.0f, p.den);
    float ru = fmaf(t.pu2, dy, fmaf(t.pu1, dx, t.pu0)) * rden;
    float rv = fmaf(t.pv2, dy, fmaf(t.pv1, dx, t.pv0)) * rden;
    ru = fminf(fmaxf(ru, -1.0e7f), 1.0e7f);
    rv = fminf(fmaxf(rv, -1.0e7f), 1.0e7f);
    const float flu = floorf(ru), flv = floorf(rv);
    p.iu = t.U0 + (int)flu;
    p.iv = t.V0 + (int)flv;
    p.fu = ru - flu;
    p.fv = rv - flv;
    p.u = fU0 + ru;
    p.v = fV0 + rv;
    return p;
}

// Raw feather weight from float source coordinates; Wm = W - 0.5, Hm = H - 0.5.  Within ~1e-4 px
// of a validity border the float test may differ from the exact one (those pixels are the
// coverage-boundary set that parity excludes); everywhere else it is the same decision.
__device__ __forceinline__ float weight_of(const Pos& p, float Wm, float Hm) {
    const float m = fminf(fminf(p.u + 0.5f, p.v + 0.5f), fminf(Wm - p.u, Hm - p.v));
    const bool ok = (p.den > 0.0f) & (p.u >= -0.5f) & (p.u < Wm) & (p.v >= -0.5f) & (p.v < Hm);
    return ok ? fmaxf(m, 0.0f) : 0.0f;
}

// Bilinear RGB sample with clamped coordinates, scaled by `scale` (= gain / 255).
__device__ __forceinline__ float3 sample_rgb(const uint8_t* __restrict__ px, long long pitch, const Pos& p, int W,
                                             int H, float scale) {
    int i0, j0;
    float fx, fy;
    if (p.iu < 0) { i0 = 0; fx = 0.0f; }
    else if (p.iu >= W - 1) { i0 = W - 1; fx = 0.0f; }
    else { i0 = p.iu; fx = p.fu; }
    if (p.iv < 0) { j0 = 0; fy = 0.0f; }
    else if (p.iv >= H - 1) { j0 = H - 1; fy = 0.0f; }
    else { j0 = p.iv; fy = p.fv; }
    const int di = (i0 + 1 < W) ? 3 : 0;
    const long long dj = (j0 + 1 < H) ? pitch : 0;
    const uint8_t* a = px + (long long)j0 * pitch + 3 * i0;
    const uint8_t* b = a + dj;
    float3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p00 = u8_to_f(__ldg(a + c)), p01 = u8_to_f(__ldg(a + di + c));
        const float p10 = u8_to_f(__ldg(b + c)), p11 = u8_to_f(__ldg(b + di + c));
        const float top = fmaf(fx, p01 - p00, p00);
        const float bot = fmaf(fx, p11 - p10, p10);
        const float v = fmaf(fy, bot - top, top) * scale;
        if (c == 0) o.x = v; else if (c == 1) o.y = v; else o.z = v;
    }
    return o;
}

// Bilinear RGB sample of a position known to lie in [0, W-1) x [0, H-1) (no clamping needed).
__device__ __forceinline__ float3 sample_rgb_inside(const uint8_t* __restrict__ px, long long pitch, const Pos& p,
                                                    float scale) {
    const uint8_t* a = px + (long long)p.iv * pitch + 3 * p.iu;
    const uint8_t* b = a + pitch;
    float3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p00 = u8_to_f(__ldg(a + c)), p01 = u8_to_f(__ldg(a + 3 + c));
        const float p10 = u8_to_f(__ldg(b + c)), p11 = u8_to_f(__ldg(b + 3 + c));
        const float top = fmaf(p.fu, p01 - p00, p00);
        const float bot = fmaf(p.fu, p11 - p10, p10);
        const float v = fmaf(p.fv, bot - top, top) * scale;
        if (c == 0) o.x = v; else if (c == 1) o.y = v; else o.z = v;
    }
    return o;
}

__device__ __forceinline__ unsigned char quantize_u8(float v) {
    // v already clamped to [0, 1]: 2^23 + 255 v rounded once to nearest even in the addition of one
    // fused multiply-add, whose low byte is round-half-even(255 v)
    return (unsigned char)(__float_as_uint(fmaf(v, 255.0f, 8388608.0f)) & 0xffu);
}

// ------------------------------------------------------------------------------------------------
// index-range planning on one axis (host)

struct Span {
    int lo, hi;  // half-open [lo, hi); empty when lo >= hi
    bool empty() const { return hi <= lo; }
};

inline Span span_union(Span a, Span b) {
    if (a.empty()) return b;
    if (b.empty()) return a;
    return {std::min(a.lo, b.lo), std::max(a.hi, b.hi)};
}

// finer-level samples read by REDUCE outputs in `c` (finer level of size n)
inline Span reduce_reads(Span c, int n) {
    if (c.empty()) return {0, 0};
    int lo = n, hi = -1;
    for (int k = c.lo; k < c.hi; ++k)
        for (int m = -2; m <= 2; ++m) {
            const int i = fold101(2 * k + m, n);
            lo = std::min(lo, i);
            hi = std::max(hi, i);
        }
    return {lo, hi + 1};
}

// coarser-level samples read by EXPAND outputs in `f` (coarser level of size n)
inline Span expand_reads(Span f, int n) {
    if (f.empty()) return {0, 0};
    int lo = n, hi = -1;
    for (int x = f.lo; x < f.hi; ++x) {
        const int k0 = (x % 2 == 0) ? x / 2 - 1 : (x - 1) / 2;
        const int k1 = (x % 2 == 0) ? x / 2 + 1 : (x + 1) / 2;
        for (int k = k0; k <= k1; ++k) {
            const int i = fold101(k, n);
            lo = std::min(lo, i);
            hi = std::max(hi, i);
        }
    }
    return {lo, hi + 1};
}

// coarser-level outputs (level size nc) whose REDUCE support meets the finer span `f` (size nf)
inline Span reduce_touch(Span f, int nf, int nc) {
    if (f.empty()) return {0, 0};
    int lo = nc, hi = -1;
    for (int k = 0; k < nc; ++k) {
        bool hit = false;
        for (int m = -2; m <= 2 && !hit; ++m) {
            const int i = fold101(2 * k + m, nf);
            hit = i >= f.lo && i < f.hi;
        }
        if (hit) {
            lo = std::min(lo, k);
            hi = std::max(hi, k);
        }
    }
    return hi < lo ? Span{0, 0} : Span{lo, hi + 1};
}

inline Rect make_rect(Span x, Span y) {
    if (x.empty() || y.empty()) return Rect{0, 0, 0, 0};
    return Rect{x.lo, x.hi, y.lo, y.hi};
}


// ------------------------------------------------------------------------------------------------
// host side

struct KernelStat {
    const char* name;
    double ms;
    long long launches;
};

struct ProfMark {
    const char* name;  // kernel that starts at this event (nullptr: end marker)
    cudaEvent_t ev;
};

struct stitch_rig {
    int device = 0;
    stitch_rig_desc desc{};
    std::vector<stitch_camera> cams;
    RigGeom geom{};
    CamDev hcam[MAXC]{};
    CamDev* dcam = nullptr;
    float4* Bl[MAXL]{};  // plain path: blended band / collapse buffer per level (full level grid)
    std::vector<void*> allocs;
    std::vector<std::pair<uint32_t*, size_t>> guards;  // debug build: guard bands (words)
    long long scratch_bytes = 0;
    long long roi_pixels = 0;
    int kernels_per_frame = 0;

    // fused path state
    void* fused = nullptr;

    // backward state
    void* bw = nullptr;

    // host staging for stitch_frames_host, and the overlapped pipeline of stitch_frames_host_async
    uint8_t* stage_frames[MAXC]{};
    void* stage_out = nullptr;
    void* pipe = nullptr;

    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfMark> marks;
    std::vector<KernelStat> stats;
};

// Validate one camera and plan its regions; adds its level-0 region area to *roi.
stitch_status plan_camera_geometry(const stitch_camera& c, const RigGeom& g, CamDev& d, long long* roi);

// Record a profiling mark before a launch (name) or at the end of a call (nullptr).
void prof_mark(stitch_rig* r, const char* name, cudaStream_t s);

// Device allocation owned by the rig.
void* rig_alloc(stitch_rig* r, size_t bytes);

// Path entry points (one translation unit each).
stitch_status plain_plan(stitch_rig* r);
stitch_status plain_frames(stitch_rig* r, const FramePtrs& fp, const OutDesc& od, cudaStream_t s);
stitch_status fused_plan(stitch_rig* r);
stitch_status fused_frames(stitch_rig* r, const FramePtrs& fp, const OutDesc& od, cudaStream_t s);
void fused_release(stitch_rig* r);
void fused_tile_counts(const stitch_rig* r, int counts[8]);
stitch_status backward_plan(stitch_rig* r);
stitch_status backward_run(stitch_rig* r, const FramePtrs& fp, const double* params, double* loss, double* grad,
                           cudaStream_t s);
void backward_release(stitch_rig* r);
void pipeline_release(stitch_rig* r);
stitch_status fused_precompute(stitch_rig* r);  // geometry-only tables, after the camera upload
stitch_status fused_batch_create(stitch_rig* const* rigs, int n, void** out);
stitch_status fused_batch_frames(void* b, const uint8_t* const* const* frames, const int64_t* const* pitches,
                                 void* const* outs, const int64_t* out_pitches, cudaStream_t s);
void fused_batch_destroy(void* b);
stitch_status fused_batch_info(void* b, int32_t* order, int32_t* grid, int64_t* ntasks);
stitch_status fused_batch_wait_test(void* b, int spin_limit, int rig);
stitch_status fused_batch_status(void* b);
// debug build: the fused path's first failed index check (code << 48 | value), 0 when none; reset
long long fused_debug_take(int device);

#define STITCH_CUDA_TRY(expr)                         \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return STITCH_ECUDA;   \
    } while (0)

static inline stitch_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? STITCH_OK : STITCH_ECUDA;
}
