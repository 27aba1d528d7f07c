// Fused forward path: the per-frame step of Algorithm 4 (step 6: transform every camera's video and
// blend it into the panorama; step 1: the transform follows the pre-corrected parameters), with
// the multi-band fusion that removes the seams (Sec. 1, contribution 3), as S1-S6 below.
//
// Data that crosses HBM per frame: the source frames (read once, by `down1`), the Gaussian
// level 1 of every camera (written by `down1`, read by `reduce` and `up_full`), the level-0
// samples of the blended (FULL) canvas tiles (written by `down1` into one slot per tile and
// camera, read by `up_full`), the small levels >= 2 and the output canvas.  The collapsed level 1
// never leaves the chip.
//
//   down1    per camera tile: the source footprint staged in shared memory, warp + feather weights
//            (S1, S2) of a level-0 tile and its halo, both separable REDUCE passes on chip (S3),
//            write G^1 (r, g, b, weight); SOLO canvas tiles get their output here, FULL ones their
//            level-0 slot.
//   reduce   G^{l+1} = REDUCE(G^l) for l >= 1, every camera in one launch.
//   coarse   levels L-1 .. 2: Laplacian (S4) + normalised blend (S5) + collapse step (S6) fused,
//            writing R^l on the canvas grid of level l.
//   up_full  per FULL canvas tile: level 1 bands of every contributing camera, blend and collapse
//            to R^1 in shared memory; then level 0 from the cameras' slots: Laplacian against
//            EXPAND(G^1_i), blend, add EXPAND(R^1), mask, clamp, quantise and write the output.
//   up_simple / up_general  ZERO tiles (output 0) / tiles with more than 4 cameras (one camera at
//            a time, warping level 0 itself).
//
// down1, reduce and up_full each prefetch into L2 the inputs of the tile one resident wave later
// (thread blocks start in index order as resident ones finish).
//
// The per-level blend and collapse are evaluated in the equivalent form
//   R^l = sum_i a_i (G^l_i + EXPAND(R^{l+1} - G^{l+1}_i)),  a_i = G^l(What_i) / S^l,
// which follows from B^l = sum_i a_i (G^l_i - EXPAND(G^{l+1}_i)) and sum_i a_i = 1 wherever
// S^l > 1e-12 (elsewhere R^l = EXPAND(R^{l+1})); it needs one EXPAND per camera and level.
// At level 0, a_i = w_i / sum_j w_j with the raw feather weights.
//
// Canvas tiles of `up` are classified when the rig is created:
//   ZERO   no camera's validity box meets the tile: the output is 0;
//   SOLO   one camera c is valid with weight > 0 on every level-0 pixel that the tile's outputs
//          depend on (the whole pyramid cone) and no other camera's validity box meets that
//          region.  Then every weight pyramid of c is exactly 1 there, every other one exactly 0,
//          B^l = L^l_c at every level and the collapse telescopes to G^0_c: the output is the
//          clamped warp of camera c, with no pyramid work;
//   FULL   up to 2 or 4 contributing cameras, everything in shared memory;
//   GENERAL more cameras: a slower kernel that streams one camera at a time.
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>

#include "stitch_internal.cuh"

#ifdef STITCH_DEBUG
// debug build: the first failed index check of this translation unit (code << 48 | value)
static __device__ unsigned long long g_dcheck;
__device__ __noinline__ void stitch_dcheck_fail(int code, long long val) {
    atomicCAS(&g_dcheck, 0ull, ((unsigned long long)code << 48) | ((unsigned long long)val & 0xFFFFFFFFFFFFull));
}
#endif

long long fused_debug_take(int device) {
#ifdef STITCH_DEBUG
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_dcheck, sizeof(v)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_dcheck, &zero, sizeof(zero)) != cudaSuccess) {
        cudaGetLastError();
        v = ~0ull;
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return (long long)v;
#else
    (void)device;
    return 0;
#endif
}

namespace {

// ------------------------------------------------------------------------------------------------
// storage of pyramid data between kernels: FP32 (float4) or FP16 (four halves)

struct __align__(8) half4 {
    __half2 a, b;
};

// Pyramid data is read through L2 (ld.global.cg): in the batched persistent kernel it is written
// by other blocks of the same launch, which the non-coherent read-only path would not see.
__device__ __forceinline__ float4 ld(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld(const half4* p) {
    const uint2 u = __ldcg(reinterpret_cast<const uint2*>(p));
    __half2 a = *reinterpret_cast<const __half2*>(&u.x), b = *reinterpret_cast<const __half2*>(&u.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void st(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st(half4* p, float4 v) {
    half4 h;
    h.a = __floats2half2_rn(v.x, v.y);
    h.b = __floats2half2_rn(v.z, v.w);
    *p = h;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ float4 f4fma(float s, float4 v, float4 acc) {
    return make_float4(fmaf(s, v.x, acc.x), fmaf(s, v.y, acc.y), fmaf(s, v.z, acc.z), fmaf(s, v.w, acc.w));
}

__constant__ float c_w5[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};

// Tile of work of the reduce kernel: camera and origin in level coordinates.
struct Tile {
    int cam, x0, y0, pad;
};

// A camera taking part in a tile, with its homography anchored near the tile (host-built).  For
// the cameras blended at level 0 of a FULL canvas tile, g0 is the slot of the tile's level-0
// samples written by the camera's down1 tile (-1 otherwise).
struct CamRef {
    TileMap tm;
    int cam, ax, ay, g0;
};

// down1 tile: camera, level-1 origin, the camera's CamRef anchored at the tile, the tile's block in
// the table of normalised level-0 weights (-1 for INTERIOR tiles, whose weight is 1 everywhere),
// and the source-image footprint of its samples staged in shared memory (fx0 | fy0 << 16,
// fw | fh << 16; fwh = 0 when the footprint does not fit and samples are read from the frame).
struct D1Tile {
    int cam, k0, j0, ref, wtab, flags, fxy, fwh, g0;  // g0: slot of the level-0 samples (D1_G0_OUT)
    int coltab;                                       // cylindrical canvas: the tile's column table
    // the staging inputs of the tile one resident wave later (footprint as fxy/fwh, camera and
    // weight block as cam | (wtab + 1) << 8; pf_fwh = 0: none), prefetched into L2 by this tile
    int pf_fxy, pf_fwh, pf_cw;
    int wsel;  // weight table the samples take: wtab, or the table of ones for INTERIOR tiles
};

// Cameras (CamRef range, in camera order) whose validity box meets a down1 tile's level-0 inputs,
// and the position of the tile's own camera among them: the weight normalisation of the tile.
struct D1Cams {
    int first, count, self, pad;
};
constexpr int D1_INTERIOR = 1;  // inputs solidly inside the camera, no other camera: weight 1
constexpr int D1_SOLO_OUT = 2;  // the canvas tile under this tile is SOLO for this camera
constexpr int D1_G0_OUT = 4;    // the canvas tile under this tile is FULL: write its level-0 samples
constexpr int D1_NOCLAMP = 8;   // every input maps at least 0.01 px inside the image: no coordinate clamping
constexpr int D1_G1_OUT = 16;   // some of the tile's level-1 outputs are read: REDUCE and store G^1

// up tile: level-0 origin and the contributing cameras (CamRef range), in camera order.
struct UpTile {
    int x0, y0, first, count;
};

// ------------------------------------------------------------------------------------------------
// packed single-precision pairs (f32x2: two IEEE binary32 lanes, each rounded exactly as the
// scalar operation), used where the path computes on pairs of channels

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a + (-1) b: the product is exact, so this is the rounded difference, bit for bit
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add_rm(float2 a, float2 b) { return __fadd2_rd(a, b); }  // toward -infinity

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// (r, g, b, weight) as two pairs
struct V4 {
    float2 a, b;
};
__device__ __forceinline__ V4 v4_mul(float2 w, V4 s) { return {f2mul(w, s.a), f2mul(w, s.b)}; }
__device__ __forceinline__ V4 v4_fma(float2 w, V4 s, V4 acc) { return {f2fma(w, s.a, acc.a), f2fma(w, s.b, acc.b)}; }
__device__ __forceinline__ V4 v4_of(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 f4_of(V4 v) { return make_float4(v.a.x, v.a.y, v.b.x, v.b.y); }

// ------------------------------------------------------------------------------------------------
// down1
//
// One block of 64 threads per tile of 32 x 8 level-1 outputs of one camera, on the global grid.
// The tile's level-0 virtual region is 67 x 19 samples (columns 2 k0 - 2 .. 2 k0 + 64, rows
// 2 j0 - 2 .. 2 j0 + 16, folded at the canvas borders).  Thread c takes virtual column c < 64 and
// sweeps its 19 rows: it warps every sample (S1, S2) and feeds it straight into the vertical
// REDUCE pass (S3), whose three running sums stay in registers; each finished level-1 row goes to
// shared memory.  The last three columns are one sample per thread.  The horizontal REDUCE pass
// then reads the 8 x 67 vertically reduced values and writes G^1.  The source footprint of the
// tile's samples is staged in shared memory as one 32-bit word per texel (R, G, B bytes), so a
// bilinear tap is four 32-bit shared loads.

constexpr int D1_TX = 32, D1_TY = 8;                         // level-1 outputs per tile
constexpr int D1_SX = 2 * D1_TX + 3, D1_SY = 2 * D1_TY + 3;  // level-0 virtual region (67 x 19)
constexpr int D1_THREADS = 64;                               // one thread per virtual column 0..63
constexpr int D1_XC = D1_SX - D1_THREADS;                    // the last 3 columns: one sample per thread

constexpr int D1_NSAMP = D1_SX * D1_SY;                      // level-0 samples of a tile's region
// a FULL canvas tile's level-0 slot (64 x 32 samples per blended camera), written by the camera's
// two down1 tiles over it (rows 0..15 and 16..31)
constexpr int D1_SLOT = (2 * D1_TX) * (4 * D1_TY);
// A slot element: the sample's R, G, B and normalised weight a as 16-bit codes, R | G << 16 and
// B | a << 16.  Colours go in steps of 1/256 of an 8-bit level (a bilinear sample of 8-bit texels
// rounds to within 1/512 of a level), the weight in steps of 1/65535; the blend divides by the sum
// of the weights, so their codes enter it as they are.  Both band precisions use this format.
using Slot = uint2;
constexpr float SLOT_RGB = 256.0f;  // codes per 8-bit level
constexpr float SLOT_A = 65535.0f;  // codes per unit weight
// Footprint capacity in texels (one 32-bit word each; rows padded to a multiple of 4 texels).  The
// kernel comes in two capacities: 2048 texels with 12 resident blocks per SM, and 1536 with 13.  A
// rig takes the smaller one when at most 2 % of its staged tiles need more (those then read their
// taps from the frame): one more block per SM beats that (8 x 4K: 315 of 76 350 tiles).
constexpr int D1_FOOT = 2048;        // the larger capacity (planning, the batched kernels)
constexpr int D1_FOOT_SMALL = 1536;
// Vertically reduced values: per level-1 row, the even columns at slots 0..33 and the odd columns
// at slots 36..68 (float4), so that a warp's 128-bit stores of 32 consecutive columns and the
// horizontal pass's loads of consecutive even (odd) columns are free of bank conflicts.
constexpr int D1_VODD = 36, D1_VROW = 70;
constexpr int D1_SM_V = 16 * D1_VROW * D1_TY;
constexpr int D1_SM_X = 16 * D1_XC * D1_SY;
constexpr int D1_SM_ROW = 8 * ((D1_SY + 1) & ~1);            // (dy, dy) per row
// shared memory of a block with footprint capacity CAP: footprint, vertically reduced rows, the
// last three columns' samples, (dy, dy) per row
template <int CAP>
struct D1Cap {
    static constexpr int SM_FOOT = 4 * CAP;
    static constexpr size_t SMEM = SM_FOOT + D1_SM_V + D1_SM_X + D1_SM_ROW;
    static constexpr int BLOCKS = CAP > D1_FOOT_SMALL ? 12 : 13;  // resident blocks per SM
    static constexpr int SG = (CAP / 4 + D1_THREADS - 1) / D1_THREADS;  // staging groups per thread (at most)
    static_assert(CAP % 16 == 0, "whole groups of 4 texels, 16-byte aligned parts");
};
constexpr size_t D1_SMEM = D1Cap<D1_FOOT>::SMEM;  // the larger capacity's
static_assert(D1_SX == 67 && D1_THREADS == 64 && D1_XC == 3, "column-per-thread sweep of a 67-column region");
static_assert(D1_SM_V % 16 == 0 && D1_SM_X % 16 == 0, "16-byte aligned parts");

__device__ __forceinline__ int d1_vslot(int c) { return (c & 1) * D1_VODD + (c >> 1); }

// REDUCE taps [1, 4, 6, 4, 1] / 16 as pairs
__device__ __forceinline__ float2 d1_w(int n) { return f2(n == 0 || n == 4 ? 0.0625f : n == 2 ? 0.375f : 0.25f); }

// Normalised feather weights of the level-0 samples of a down1 tile (S2: w_i / sum_j w_j over the
// cameras whose validity box contains the sample), or -1 for samples outside the camera's pyramid
// region Omega^0_i.  They depend on the geometry only, so the rig computes them once at creation
// (the paper's pre-corrected parameters, Algorithm 4, and start-up preallocation, Sec. 4.3.2), one
// block per tile; down1 then warps only its own camera.
constexpr int D1W_THREADS = 256;
__global__ void __launch_bounds__(D1W_THREADS) k_d1_weights(const CamDev* __restrict__ cams, RigGeom g,
                                                           const D1Tile* __restrict__ tiles,
                                                           const D1Cams* __restrict__ tcams,
                                                           const CamRef* __restrict__ refs, float* __restrict__ d1w) {
    const D1Tile tl = tiles[blockIdx.x];
    const D1Cams tc = tcams[blockIdx.x];
    if (tl.wtab < 0) return;
    const Rect o0 = cams[tl.cam].Om[0];
    const int vx0 = 2 * tl.k0 - 2, vy0 = 2 * tl.j0 - 2;
    float* out = d1w + (long long)tl.wtab * D1_NSAMP;
    for (int q = threadIdx.x; q < D1_NSAMP; q += D1W_THREADS) {
        const int r = q / D1_SX, c = q % D1_SX;
        const int x = fold101(vx0 + c, g.nx[0]), y = fold101(vy0 + r, g.ny[0]);
        if (!o0.contains(x, y)) {
            out[q] = -1.f;
            continue;
        }
        if (g.seam) {
            const int own = seam_owner(g, tc.count, [&](int k) -> const CamDev& { return cams[refs[tc.first + k].cam]; }, x, y);
            out[q] = own == tc.self ? 1.f : 0.f;
            continue;
        }
        if (g.cyl) {
            double ws = 0.0, wself = 0.0;
            for (int a = 0; a < tc.count; ++a) {
                const CamDev& cj = cams[refs[tc.first + a].cam];
                if (!cj.V.contains(x, y)) continue;
                const double w = feather_weight64(cj, g, (double)x, (double)y);
                ws += w;
                if (a == tc.self) wself = w;
            }
            out[q] = ws > 0.0 ? (float)(wself / ws) : 0.f;
            continue;
        }
        float ws = 0.f, wself = 0.f;
        for (int a = 0; a < tc.count; ++a) {
            const CamRef ref = refs[tc.first + a];
            const CamDev& cj = cams[ref.cam];
            if (!cj.V.contains(x, y)) continue;
            const Pos p = map_pos(ref.tm, (float)ref.tm.U0, (float)ref.tm.V0, (float)(x - ref.ax), (float)(y - ref.ay));
            const float w = weight_of(p, (float)cj.W - 0.5f, (float)cj.H - 0.5f);
            ws += w;
            if (a == tc.self) wself = w;
        }
        out[q] = ws > 0.f ? __fdividef(wself, ws) : 0.f;
    }
}


// Copy the footprint [fx0, fx0 + fw) x [fy0, fy0 + fh) of an RGB8 frame into shared memory, one
// word per texel (bytes R, G, B, and one unused byte), rows of S = fw rounded up to 4 texels.  A
// thread takes groups of 4 texels (12 bytes: three aligned 32-bit words, since fx0 is a multiple of
// 4), issues the loads of all its groups before repacking, and writes the 4 texel words with one
// 16-byte store.  Frames whose base or pitch is not a multiple of 4 bytes are read byte by byte.

template <int CAP>
__device__ __forceinline__ void stage_footprint(uint32_t* __restrict__ foot, const uint8_t* __restrict__ px,
                                                long long pitch, int W, int fx0, int fy0, int fw, int fh, int t) {
    const int gpr = (fw + 3) >> 2, ng = gpr * fh;  // groups per row = S / 4
    if (!STITCH_DCHECK(ng <= CAP / 4, 2, ng)) return;
    if (((reinterpret_cast<uintptr_t>(px) | (uintptr_t)pitch) & 3) != 0) {
        for (int q = t; q < 4 * ng; q += D1_THREADS) {
            const int rr = q / (4 * gpr), u = q - rr * 4 * gpr;
            uint32_t w = 0u;
            if (u < fw) {
                const uint8_t* src = px + (long long)(fy0 + rr) * pitch + 3 * (fx0 + u);
                w = (uint32_t)__ldg(src) | ((uint32_t)__ldg(src + 1) << 8) | ((uint32_t)__ldg(src + 2) << 16);
            }
            foot[q] = w;
        }
        return;
    }
    constexpr int SG = D1Cap<CAP>::SG;
    uint32_t w[SG][3];
#pragma unroll
    for (int k = 0; k < SG; ++k) {
        const int q = t + k * D1_THREADS;
        w[k][0] = w[k][1] = w[k][2] = 0u;
        if (q < ng) {
            const int rr = q / gpr, gx = q - rr * gpr;
            const int u0 = fx0 + 4 * gx;
            const uint8_t* src = px + (long long)(fy0 + rr) * pitch + 3 * u0;
            if (u0 + 4 <= W) {
                const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
                w[k][0] = __ldg(s32);
                w[k][1] = __ldg(s32 + 1);
                w[k][2] = __ldg(s32 + 2);
            } else {
                // the image's last texels: only the bytes of texels < W exist
                const int nb = 3 * (W - u0);
#pragma unroll
                for (int j = 0; j < 12; ++j)
                    if (j < nb) w[k][j >> 2] |= (uint32_t)__ldg(src + j) << (8 * (j & 3));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < SG; ++k) {
        const int q = t + k * D1_THREADS;
        if (q < ng) {
            // bytes R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3 -> one word per texel
            reinterpret_cast<uint4*>(foot)[q] =
                make_uint4(__byte_perm(w[k][0], 0u, 0x0210), __byte_perm(w[k][0], w[k][1], 0x0543),
                           __byte_perm(w[k][1], w[k][2], 0x0432), __byte_perm(w[k][2], 0u, 0x0321));
        }
    }
}

// 2^23 + byte j of w, as a float (exact)
__device__ __forceinline__ float d1_bf(uint32_t w, uint32_t j) { return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | j)); }

// Bilinear RGB of four texel words with fractions (fx, fy), times `scale`.  The arithmetic is that
// of sample_rgb (top = p00 + fx (p01 - p00), bot likewise, value = top + fy (bot - top), then the
// scale), on exact 2^23-offset values whose differences are the byte differences, so the result
// is bit-identical.  R and G go as one pair.
__device__ __forceinline__ void d1_bilerp(uint32_t w00, uint32_t w01, uint32_t w10, uint32_t w11, float fx, float fy,
                                          float scale, V4& s) {
    constexpr float K23 = 8388608.0f;
    const float2 a00 = make_float2(d1_bf(w00, 0), d1_bf(w00, 1)), a01 = make_float2(d1_bf(w01, 0), d1_bf(w01, 1));
    const float2 a10 = make_float2(d1_bf(w10, 0), d1_bf(w10, 1)), a11 = make_float2(d1_bf(w11, 0), d1_bf(w11, 1));
    const float2 fxx = f2(fx), fyy = f2(fy);
    const float2 top = f2fma(fxx, f2sub(a01, a00), f2sub(a00, f2(K23)));
    const float2 bot = f2fma(fxx, f2sub(a11, a10), f2sub(a10, f2(K23)));
    s.a = f2mul(f2fma(fyy, f2sub(bot, top), top), f2(scale));
    const float b00 = d1_bf(w00, 2), b01 = d1_bf(w01, 2), b10 = d1_bf(w10, 2), b11 = d1_bf(w11, 2);
    const float btop = fmaf(fx, b01 - b00, b00 - K23), bbot = fmaf(fx, b11 - b10, b10 - K23);
    s.b.x = fmaf(fy, bbot - btop, btop) * scale;
}

// Per-tile constants of the sweep.
struct D1Ctx {
    TileMap tm;
    const uint32_t* foot;  // staged footprint
    const float2* rowdy;   // (dy, dy) of every virtual row: canvas row minus the anchor row
    const float* wt;       // normalised weights of the tile's samples (67 x 19; all 1 on INTERIOR tiles)
    const uint8_t* px;     // frame (taps read from it)
    long long pitch;
    int S;                 // footprint row stride (words)
    int fw, fh, fx0, fy0;  // footprint
    unsigned ibase;        // index of the top-left tap from the floor constants, see d1_sample
    int maxidx;            // largest top-left index whose four taps lie in the footprint
    int W, H;
    float scale;
};

// Sample modes: the staged footprint without clamping (every input at least 0.01 px inside the
// image), the staged footprint with the image clamp of S1 (tiles at the image border), taps read
// from the frame (footprints too large to stage or reaching behind the camera).
enum D1Mode { D1M_STAGED = 0, D1M_CLAMP = 1, D1M_FRAME = 2 };

constexpr float D1_FLOOR_M = 12582912.0f;       // 1.5 * 2^23
constexpr unsigned D1_FLOOR_BITS = 0x4B400000u;  // its bit pattern

// Level-0 sample of virtual row r at the column whose anchored numerators and denominator at the
// anchor row are (nuv, dqc): (r, g, b, normalised weight a), weight 0 outside Omega^0 (a < 0).
// The colour there is whatever the taps give: Omega^0 holds the 5 x 5 support of every stored G^1
// sample, and a level-0 output of weight 0 adds nothing to a blend, so it is never read.
// Position and taps are those of map_pos + sample_rgb, so the three modes give bit-identical
// samples.  The floor of the offsets ru, rv (|ru|, |rv| < 2^22 on staged tiles, whose footprint
// the planner bounds) comes from one addition rounded toward -infinity:
// RD(ru + 1.5 2^23) = 1.5 2^23 + floor(ru), whose low bits hold the integer.
template <int MODE>
__device__ __forceinline__ V4 d1_sample(const D1Ctx& x, float2 nuv, float dqc, int r, float a) {
    const float2 dy = x.rowdy[r];
    const float den = fmaf(x.tm.q2, dy.x, dqc);
    const float2 n = f2fma(make_float2(x.tm.pu2, x.tm.pv2), dy, nuv);
    const float rden = __fdividef(1.0f, den);
    V4 s;
    s.b.y = fmaxf(a, 0.0f);
    if (MODE == D1M_FRAME) {
        float ru = n.x * rden, rv = n.y * rden;
        ru = fminf(fmaxf(ru, -1.0e7f), 1.0e7f);
        rv = fminf(fmaxf(rv, -1.0e7f), 1.0e7f);
        const float flu = floorf(ru), flv = floorf(rv);
        Pos p;
        p.iu = x.tm.U0 + (int)flu;
        p.iv = x.tm.V0 + (int)flv;
        p.fu = ru - flu;
        p.fv = rv - flv;
        const float3 v = sample_rgb(x.px, x.pitch, p, x.W, x.H, x.scale);
        s.a = make_float2(v.x, v.y);
        s.b.x = v.z;
    } else {
        const float2 ruv = f2mul(n, f2(rden));
        const float2 tt = f2add_rm(ruv, f2(D1_FLOOR_M));
        const float2 f = f2sub(ruv, f2add(tt, f2(-D1_FLOOR_M)));  // fractions in [0, 1)
        const unsigned tu = __float_as_uint(tt.x), tv = __float_as_uint(tt.y);
        uint32_t w00, w01, w10, w11;
        float fx = f.x, fy = f.y;
        if (MODE == D1M_STAGED) {
            // top-left tap (V0 + floor(rv) - fy0) S + (U0 + floor(ru) - fx0), clamped into the footprint
            // (the planner's footprint holds every tap; the debug build records one that it misses)
            const int raw = (int)(tv * (unsigned)x.S + tu + x.ibase);
            (void)STITCH_DCHECK(raw >= 0 && raw <= x.maxidx, 1, raw);
            const int idx = min(max(raw, 0), x.maxidx);
            const uint32_t* p = x.foot + idx;
            w00 = p[0];
            w01 = p[1];
            w10 = p[x.S];
            w11 = p[x.S + 1];
        } else {
            // image clamp of S1: outside [0, W-1) x [0, H-1) the border texel, fraction 0
            const int lu = (int)(tu - D1_FLOOR_BITS) + (x.tm.U0 - x.fx0), lv = (int)(tv - D1_FLOOR_BITS) + (x.tm.V0 - x.fy0);
            if ((unsigned)(lu + x.fx0) >= (unsigned)(x.W - 1)) fx = 0.0f;
            if ((unsigned)(lv + x.fy0) >= (unsigned)(x.H - 1)) fy = 0.0f;
            const int lx = min(max(lu, 0), x.fw - 1), ly = min(max(lv, 0), x.fh - 1);
            const int ox = lx < x.fw - 1 ? 1 : 0, oy = ly < x.fh - 1 ? x.S : 0;
            const uint32_t* p = x.foot + ly * x.S + lx;
            w00 = p[0];
            w01 = p[ox];
            w10 = p[oy];
            w11 = p[oy + ox];
        }
        d1_bilerp(w00, w01, w10, w11, fx, fy, x.scale, s);
    }
    return s;
}

// The slot element of a sample whose colours are 8-bit levels times `scale`; enc = SLOT_RGB / scale
// (0 for scale 0).  Each code is the low half of 2^23 + code, the result of one rounded addition.
__device__ __forceinline__ Slot slot_encode(V4 s, float enc) {
    const float2 rg = f2fma(s.a, f2(enc), f2(8388608.0f));
    const float2 ba = f2fma(s.b, make_float2(enc, SLOT_A), f2(8388608.0f));
    return make_uint2(__byte_perm(__float_as_uint(rg.x), __float_as_uint(rg.y), 0x5410),
                      __byte_perm(__float_as_uint(ba.x), __float_as_uint(ba.y), 0x5410));
}

// (R, G, B) of a slot element in scaled units (dsc = scale / SLOT_RGB) and its weight code.
__device__ __forceinline__ float4 slot_decode(Slot w, float dsc) {
    constexpr float K23 = 8388608.0f;
    const float2 c = make_float2(__uint_as_float(__byte_perm(w.x, 0x4B000000u, 0x7610)),
                                 __uint_as_float(__byte_perm(w.x, 0x4B000000u, 0x7632)));
    const float2 rg = f2mul(f2sub(c, f2(K23)), f2(dsc));
    const float b = (__uint_as_float(__byte_perm(w.y, 0x4B000000u, 0x7610)) - K23) * dsc;
    const float a = __uint_as_float(__byte_perm(w.y, 0x4B000000u, 0x7632)) - K23;
    return make_float4(rg.x, rg.y, b, a);
}

// Where a tile's level-0 samples go besides the pyramid: nowhere, the FULL canvas tile's level-0
// slot, or the SOLO canvas tile's pixels (8-bit or float).  The sweep thread of virtual column c
// writes the sample of virtual row r at canvas (X0 + c - 2, Y0 + r - 2) for 2 <= r < 18.
enum D1OutKind { D1O_NONE = 0, D1O_SLOT = 1, D1O_U8 = 2, D1O_F32 = 3, D1O_ANY = 4 };

template <typename T>
struct D1Out {
    char* p;         // the thread's element at r = 2 (slot element, or canvas pixel)
    long long step;  // bytes from one row to the next
    int rows;        // rows r - 2 < rows exist (canvas bottom; 0 right of the canvas)
    int kind;
    float enc;       // slot codes per scaled unit (slot_encode)
};

// OUTK: the output kind fixed at compile time, or D1O_ANY to take o.kind.  Slot rows always exist.
template <typename T, int OUTK>
__device__ __forceinline__ void d1_put(const D1Out<T>& o, int dy, V4 s) {
    const int kind = OUTK == D1O_ANY ? o.kind : OUTK;
    if (kind == D1O_NONE) return;
    if (kind != D1O_SLOT && dy >= o.rows) return;
    char* q = o.p + dy * o.step;
    if (kind == D1O_SLOT) {
        *reinterpret_cast<Slot*>(q) = slot_encode(s, o.enc);
    } else if (kind == D1O_U8) {
        unsigned char* b = reinterpret_cast<unsigned char*>(q);
        b[0] = quantize_u8(__saturatef(s.a.x));
        b[1] = quantize_u8(__saturatef(s.a.y));
        b[2] = quantize_u8(__saturatef(s.b.x));
    } else {
        float* f = reinterpret_cast<float*>(q);
        f[0] = __saturatef(s.a.x);
        f[1] = __saturatef(s.a.y);
        f[2] = __saturatef(s.b.x);
    }
}

// The sweep of one thread over the 19 rows of its virtual column c: the vertical REDUCE in
// registers (output row jj takes rows 2 jj .. 2 jj + 4 in order), level-0 outputs on the fly.  Rows
// go in pairs (2m, 2m + 1), m = 0 .. 8, with two running sums: on entry to pair m, C holds output
// row m - 2 (taps 0..3 applied) and B row m - 1 (taps 0, 1); row 2m completes C (stored from m = 2
// on), moves B on by tap 2 into C and starts row m in B; row 2m + 1 adds tap 3 to C and tap 1 to B.
// Row 18 completes output row 7.
template <typename T, int MODE, int OUTK, bool ONES>
__device__ __forceinline__ void d1_sweep(const D1Ctx& x, float4* __restrict__ vcol, const float* __restrict__ wcol,
                                         float2 nuv, float dqc, const D1Out<T>& o) {
    V4 B = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, C = B;
    // weights of INTERIOR tiles are all 1; the others are loaded one row pair ahead
    float we = ONES ? 1.0f : __ldg(wcol), wo = ONES ? 1.0f : __ldg(wcol + D1_SX);
    const float* wp = wcol + 2 * D1_SX;        // weights of row 2m + 2
    float4* vp = vcol - 2 * D1_VROW;           // vres row of output m - 2
    D1Out<T> oq = o;
    oq.p -= 2 * o.step;                        // output row 2m - 2
    oq.rows += 2;
#pragma unroll 1
    for (int m = 0; m <= D1_TY; ++m) {
        const float ae = we, ao = wo;
        if (!ONES) {
            we = __ldg(wp);
            wo = __ldg(m < D1_TY ? wp + D1_SX : wp);
        }
        const V4 se = d1_sample<MODE>(x, nuv, dqc, 2 * m, ae);
        const V4 so = d1_sample<MODE>(x, nuv, dqc, 2 * m + 1, ao);
        if (m >= 1) d1_put<T, OUTK>(oq, 0, se);
        if (m >= 2) *vp = f4_of(v4_fma(d1_w(4), se, C));
        C = v4_fma(d1_w(2), se, B);
        B = v4_mul(d1_w(0), se);
        if (m >= 1) d1_put<T, OUTK>(oq, 1, so);
        C = v4_fma(d1_w(3), so, C);
        B = v4_fma(d1_w(1), so, B);
        wp += 2 * D1_SX;
        vp += D1_VROW;
        oq.p += 2 * o.step;
        oq.rows -= 2;
    }

    const V4 se = d1_sample<MODE>(x, nuv, dqc, 2 * D1_TY + 2, we);
    vcol[(D1_TY - 1) * D1_VROW] = f4_of(v4_fma(d1_w(4), se, C));
}

// Barrier of the threads working on one down1 tile: the whole block (id 0), or a named barrier of
// the 64 threads of one group when a larger block works on several tiles at once.
__device__ __forceinline__ void d1_bar(int id) {
    if (id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(D1_THREADS) : "memory");
}

// One down1 tile, worked on by the D1_THREADS threads t = 0 .. 63 that share barrier `bar`.
template <typename T, int CAP = D1_FOOT>
__device__ __forceinline__ void down1_tile(const CamDev* __restrict__ cams, const RigGeom& g, const FramePtrs& fp,
                                           const OutDesc& od, const D1Tile& tl, const CamRef* __restrict__ refs,
                                           const float* __restrict__ d1w, const float4* __restrict__ d1cols,
                                           Slot* __restrict__ g0buf, float4* smem, int t = threadIdx.x, int bar = 0) {
    uint32_t* foot = reinterpret_cast<uint32_t*>(smem);
    constexpr int SM_FOOT = D1Cap<CAP>::SM_FOOT;
    float4* vres = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem) + SM_FOOT);
    float4* ext = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem) + SM_FOOT + D1_SM_V);  // [19][3]
    float2* rowdy = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem) + SM_FOOT + D1_SM_V + D1_SM_X);

    const int i = tl.cam;
    const CamDev& ci = cams[i];
    const Rect o1 = ci.Om[1];
    const int k0 = tl.k0, j0 = tl.j0;              // level-1 tile origin
    const int vx0 = 2 * k0 - 2, vy0 = 2 * j0 - 2;  // level-0 virtual origin
    const bool act = t < D1_THREADS;
    const CamRef ref = refs[tl.ref];
    const uint8_t* px_i = fp.p[i];
    const long long pitch_i = fp.pitch[i];

    if (tl.pf_fwh != 0 && act) {
        // L2 prefetch of the staging inputs of the tile one resident wave later: its footprint rows
        // (one 128-byte line per thread and row segment) and its weight block
        const int pc = tl.pf_cw & 0xff, pw = (tl.pf_cw >> 8) - 1;
        const int pfx = tl.pf_fxy & 0xffff, pfy = (int)((unsigned)tl.pf_fxy >> 16);
        const int pfw = tl.pf_fwh & 0xffff, pfh = tl.pf_fwh >> 16;
        const uint8_t* pp = fp.p[pc];
        const long long ppitch = fp.pitch[pc];
        const int len = 3 * pfw, segs = (len + 127) >> 7;
        for (int q = t; q < segs * pfh; q += D1_THREADS) {
            const int rr = q / segs, k = q - rr * segs;
            prefetch_l2(pp + (long long)(pfy + rr) * ppitch + 3 * pfx + min(128 * k, len - 1));
        }
        if (pw >= 0)
            for (int q = t; q < (4 * D1_NSAMP + 127) / 128; q += D1_THREADS)
                prefetch_l2(d1w + (long long)pw * D1_NSAMP + min(32 * q, D1_NSAMP - 1));
    }

    D1Ctx x;
    x.tm = ref.tm;
    x.rowdy = rowdy;
    x.wt = d1w + (long long)tl.wsel * D1_NSAMP;
    x.px = px_i;
    x.pitch = pitch_i;
    x.W = ci.W;
    x.H = ci.H;
    x.scale = ci.gain * (1.0f / 255.0f);
    x.foot = foot;
    const bool staged = tl.fwh != 0;
    x.fx0 = tl.fxy & 0xffff;
    x.fy0 = (int)((unsigned)tl.fxy >> 16);
    x.fw = tl.fwh & 0xffff;
    x.fh = tl.fwh >> 16;
    x.S = (x.fw + 3) & ~3;
    // footprint index of the top-left tap from the bit patterns tu, tv of the floor constants:
    // (tv - B + V0 - fy0) S + (tu - B + U0 - fx0), in arithmetic modulo 2^32
    x.ibase = (unsigned)(ref.tm.V0 - x.fy0) * (unsigned)x.S + (unsigned)(ref.tm.U0 - x.fx0) -
              D1_FLOOR_BITS * ((unsigned)x.S + 1u);
    x.maxidx = x.S * (x.fh - 1) - 2;
    if (staged && act) stage_footprint<CAP>(foot, px_i, pitch_i, x.W, x.fx0, x.fy0, x.fw, x.fh, t);
    if (t < D1_SY) {
        const float dy = (float)(fold101(vy0 + t, g.ny[0]) - ref.ay);
        rowdy[t] = make_float2(dy, dy);
    }
    // column terms: the anchored homography on the planar canvas, the column table on the
    // cylindrical one
    const float4* __restrict__ cols = g.cyl ? d1cols + (long long)tl.coltab * D1_SX : nullptr;
    auto colterms = [&](int c, float2& nuv, float& dqc) {
        if (cols) {
            const float4 cc = cols[c];
            nuv = make_float2(cc.x, cc.y);
            dqc = cc.z;
        } else {
            const float dx = (float)(fold101(vx0 + c, g.nx[0]) - ref.ax);
            nuv = make_float2(fmaf(x.tm.pu1, dx, x.tm.pu0), fmaf(x.tm.pv1, dx, x.tm.pv0));
            dqc = fmaf(x.tm.q1, dx, x.tm.q0);
        }
    };
    const int mode = staged ? (tl.flags & D1_NOCLAMP ? D1M_STAGED : D1M_CLAMP) : D1M_FRAME;
    const int flags = tl.flags;
    const int X0 = 2 * k0, Y0 = 2 * j0;
    d1_bar(bar);
    if (act) {
        // sweep thread t takes virtual column t + 2 (the 64 columns of the canvas tile's pixels);
        // the remaining columns 0, 1 and 66 are one sample per thread
        const int c = t + 2;
        float2 nuv;
        float dqc;
        colterms(c, nuv, dqc);
        D1Out<T> o{nullptr, 0, 0, D1O_NONE, 0.f};
        if (flags & D1_G0_OUT) {
            o.kind = D1O_SLOT;
            o.p = reinterpret_cast<char*>(g0buf + (long long)tl.g0 * D1_SLOT + ((j0 / D1_TY) & 1) * (2 * D1_TY) * (2 * D1_TX) + t);
            o.step = (long long)sizeof(Slot) * (2 * D1_TX);
            o.rows = 2 * D1_TY;
            o.enc = x.scale != 0.f ? SLOT_RGB / x.scale : 0.f;
        } else if (flags & D1_SOLO_OUT) {
            o.kind = od.is_float ? D1O_F32 : D1O_U8;
            const int xo = X0 + t;
            o.p = (char*)od.ptr + (long long)Y0 * od.pitch + (long long)xo * (od.is_float ? 12 : 3);
            o.step = od.pitch;
            o.rows = xo < g.nx[0] ? max(0, min(2 * D1_TY, g.ny[0] - Y0)) : 0;
        }
        float4* vcol = vres + d1_vslot(c);
        const float* wcol = x.wt + c;
        // the staged mode (nearly every tile) has a sweep per output kind; the rare clamping and
        // frame-reading modes take the kind at run time
        if (mode == D1M_STAGED && (flags & D1_INTERIOR)) {
            switch (o.kind) {
                case D1O_SLOT: d1_sweep<T, D1M_STAGED, D1O_SLOT, true>(x, vcol, wcol, nuv, dqc, o); break;
                case D1O_U8: d1_sweep<T, D1M_STAGED, D1O_U8, true>(x, vcol, wcol, nuv, dqc, o); break;
                case D1O_F32: d1_sweep<T, D1M_STAGED, D1O_F32, true>(x, vcol, wcol, nuv, dqc, o); break;
                default: d1_sweep<T, D1M_STAGED, D1O_NONE, true>(x, vcol, wcol, nuv, dqc, o); break;
            }
        } else if (mode == D1M_STAGED) {
            switch (o.kind) {
                case D1O_SLOT: d1_sweep<T, D1M_STAGED, D1O_SLOT, false>(x, vcol, wcol, nuv, dqc, o); break;
                case D1O_U8: d1_sweep<T, D1M_STAGED, D1O_U8, false>(x, vcol, wcol, nuv, dqc, o); break;
                case D1O_F32: d1_sweep<T, D1M_STAGED, D1O_F32, false>(x, vcol, wcol, nuv, dqc, o); break;
                default: d1_sweep<T, D1M_STAGED, D1O_NONE, false>(x, vcol, wcol, nuv, dqc, o); break;
            }
        } else if (mode == D1M_CLAMP) {
            d1_sweep<T, D1M_CLAMP, D1O_ANY, false>(x, vcol, wcol, nuv, dqc, o);
        } else {
            d1_sweep<T, D1M_FRAME, D1O_ANY, false>(x, vcol, wcol, nuv, dqc, o);
        }
        if (t < D1_XC * D1_SY && (flags & D1_G1_OUT)) {
            const int r = t / D1_XC, k = t - r * D1_XC, ce = k < 2 ? k : D1_SX - 1;
            colterms(ce, nuv, dqc);
            const float a = __ldg(x.wt + r * D1_SX + ce);
            V4 s;
            switch (mode) {
                case D1M_STAGED: s = d1_sample<D1M_STAGED>(x, nuv, dqc, r, a); break;
                case D1M_CLAMP: s = d1_sample<D1M_CLAMP>(x, nuv, dqc, r, a); break;
                default: s = d1_sample<D1M_FRAME>(x, nuv, dqc, r, a); break;
            }
            ext[t] = f4_of(s);
        }
    }
    if (!(flags & D1_G1_OUT)) return;  // no level-1 output of this tile is read
    d1_bar(bar);
    // vertical REDUCE of columns 0, 1 and 66
    if (t < D1_XC * D1_TY) {
        const int jj = t / D1_XC, k = t - jj * D1_XC, ce = k < 2 ? k : D1_SX - 1;
        V4 acc = v4_mul(d1_w(0), v4_of(ext[(2 * jj) * D1_XC + k]));
#pragma unroll
        for (int n = 1; n < 5; ++n) acc = v4_fma(d1_w(n), v4_of(ext[(2 * jj + n) * D1_XC + k]), acc);
        vres[jj * D1_VROW + d1_vslot(ce)] = f4_of(acc);
    }
    d1_bar(bar);
    // S3 horizontal pass and store of G^1: output (p, jj) takes columns 2p .. 2p+4
    if (act) {
        T* dst = reinterpret_cast<T*>(ci.FG[1]);
        const int p = t & 31, kk = k0 + p;
#pragma unroll
        for (int q = 0; q < D1_TY / 2; ++q) {
            const int jj = (t >> 5) + 2 * q, j = j0 + jj;
            const float4* ev = vres + jj * D1_VROW + p;  // columns 2p, 2p+2, 2p+4
            const float4* odp = ev + D1_VODD;           // columns 2p+1, 2p+3
            V4 acc = v4_mul(d1_w(0), v4_of(ev[0]));
            acc = v4_fma(d1_w(1), v4_of(odp[0]), acc);
            acc = v4_fma(d1_w(2), v4_of(ev[1]), acc);
            acc = v4_fma(d1_w(3), v4_of(odp[1]), acc);
            acc = v4_fma(d1_w(4), v4_of(ev[2]), acc);
            // tiles lie on the global grid, so they may start before and end after Omega^1
            if (o1.contains(kk, j)) st(dst + (long long)(j - o1.y0) * o1.w() + (kk - o1.x0), f4_of(acc));
        }
    }
}

template <typename T, int CAP>
__global__ void __launch_bounds__(D1_THREADS, D1Cap<CAP>::BLOCKS) k_down1(const CamDev* __restrict__ cams, RigGeom g,
                                                                        FramePtrs fp, OutDesc od,
                                                                        const D1Tile* __restrict__ tiles,
                                                                        const CamRef* __restrict__ refs,
                                                                        const float* __restrict__ d1w,
                                                                        const float4* __restrict__ d1cols,
                                                                        Slot* __restrict__ g0buf) {
    extern __shared__ float4 smem[];
    down1_tile<T, CAP>(cams, g, fp, od, tiles[blockIdx.x], refs, d1w, d1cols, g0buf, smem);
}

// ------------------------------------------------------------------------------------------------
// reduce (levels >= 1 -> next)

// Tiled separable REDUCE: 32 x 16 outputs of level l+1 from a 67 x 35 input region of level l
// staged in shared memory with coalesced loads.
// The tile shape is a template parameter (the batched schedule's tuner picks one per batch); the
// single-rig path uses 32 x 16.
template <int X, int Y>
struct RShape {
    static constexpr int TX = X, TY = Y;                  // outputs
    static constexpr int SX = 2 * X + 3, SY = 2 * Y + 3;  // staged inputs
    static constexpr int SXH = (SX + 1) / 2;              // inputs stored as even and odd column planes
    static constexpr size_t SMEM = sizeof(float4) * (2 * SXH * SY + 2 * SXH * Y);
};
using RS32x16 = RShape<32, 16>;
using RS64x8 = RShape<64, 8>;
using RSRig = RS32x16;  // the shape of a rig's own REDUCE tiles (the single-rig path, the persistent batch)
using RSAlt = RShape<RSRig::TY * 4, RSRig::TY / 2>;  // the batch tuner's other shape (64 x 8, column sweep)
constexpr int RT_X = RSRig::TX, RT_Y = RSRig::TY;
constexpr size_t RT_SMEM = RSRig::SMEM;

// L2 prefetch of a reduce tile's input rows (the part inside Omega^l; rows that fold at the canvas
// border are left to the loads), 16 threads per row, one 128-byte line each.
template <typename T, typename RS = RS32x16>
__device__ __forceinline__ void reduce_prefetch(const CamDev* __restrict__ cams, int l, const Tile& tn, int nthreads = 256) {
    const CamDev& c = cams[tn.cam];
    const Rect of = c.Om[l];
    const int vx0 = 2 * tn.x0 - 2, vy0 = 2 * tn.y0 - 2;
    const int x0 = max(vx0, of.x0), x1 = min(vx0 + RS::SX, of.x1);
    if (x1 <= x0) return;
    const char* base = reinterpret_cast<const char*>(c.FG[l]);
    const int len = (x1 - x0) * (int)sizeof(T);
    constexpr int LPR = (RS::SX * (int)sizeof(T) + 127) / 128 + 1;  // 128-byte lines a row may touch
    for (int q = threadIdx.x; q < LPR * RS::SY; q += nthreads) {
        const int rr = q / LPR, k = q - rr * LPR, y = vy0 + rr;
        if (y < of.y0 || y >= of.y1 || 128 * k >= len + 127) continue;
        prefetch_l2(base + ((long long)(y - of.y0) * of.w() + (x0 - of.x0)) * (long long)sizeof(T) + min(128 * k, len - 1));
    }
}

template <typename T, typename RS = RS32x16>
__device__ __forceinline__ void reduce_tile(const CamDev* __restrict__ cams, const RigGeom& g, int l, const Tile& tl,
                                            float4* smem, const Tile* pf = nullptr) {
    float4* s0 = smem;  // [SY][2][SXH]: even columns, then odd columns, of each row
    float4* sh = smem + 2 * RS::SXH * RS::SY;
    const CamDev& c = cams[tl.cam];
    const Rect oc = c.Om[l + 1], of = c.Om[l];
    const int vx0 = 2 * tl.x0 - 2, vy0 = 2 * tl.y0 - 2;
    const T* src = reinterpret_cast<const T*>(c.FG[l]);
    const int nxl = g.nx[l], nyl = g.ny[l];
    {
        // all loads of a thread in flight before the shared-memory stores; a tile whose inputs lie
        // inside Omega^l (so inside the level: nothing folds) reads them straight
        constexpr int NL = (RS::SX * RS::SY + 255) / 256;
        float4 v[NL];
        const bool inside = vx0 >= of.x0 && vx0 + RS::SX <= of.x1 && vy0 >= of.y0 && vy0 + RS::SY <= of.y1;
        const T* base = src + (long long)(vy0 - of.y0) * of.w() + (vx0 - of.x0);
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = threadIdx.x + 256 * k;
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < RS::SX * RS::SY) {
                const int r = q / RS::SX, cc = q - r * RS::SX;
                if (inside) {
                    v[k] = ld(base + (long long)r * of.w() + cc);
                } else {
                    const int x = fold101(vx0 + cc, nxl), y = fold101(vy0 + r, nyl);
                    if (of.contains(x, y)) v[k] = ld(src + (long long)(y - of.y0) * of.w() + (x - of.x0));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = threadIdx.x + 256 * k;
            if (q < RS::SX * RS::SY) {
                const int r = q / RS::SX, cc = q - r * RS::SX;
                s0[r * (2 * RS::SXH) + (cc & 1) * RS::SXH + (cc >> 1)] = v[k];
            }
        }
    }
    if (pf) reduce_prefetch<T, RS>(cams, l, *pf);  // the tile one resident wave later
    __syncthreads();
    // vertical pass (rows 2 jj .. 2 jj + 4 of every column, into even and odd column planes), then
    // horizontal: each output's operations in the order of reduce_col_tile, so both give the same bits
    for (int q = threadIdx.x; q < RS::SX * RS::TY; q += 256) {
        const int jj = q / RS::SX, cc = q - jj * RS::SX;
        const int slot = (cc & 1) * RS::SXH + (cc >> 1);
        const float4* col = s0 + (2 * jj) * (2 * RS::SXH) + slot;
        float4 acc = f4fma(c_w5[0], col[0], make_float4(0.f, 0.f, 0.f, 0.f));
#pragma unroll
        for (int n = 1; n < 5; ++n) acc = f4fma(c_w5[n], col[n * (2 * RS::SXH)], acc);
        sh[jj * (2 * RS::SXH) + slot] = acc;
    }
    __syncthreads();
    T* dst = reinterpret_cast<T*>(c.FG[l + 1]);
    for (int q = threadIdx.x; q < RS::TX * RS::TY; q += 256) {
        const int jj = q / RS::TX, p = q - jj * RS::TX;
        const int k = tl.x0 + p, j = tl.y0 + jj;
        if (k >= oc.x1 || j >= oc.y1) continue;
        if (!STITCH_DCHECK(k >= oc.x0 && j >= oc.y0, 3, (long long)k << 24 | j)) continue;
        const float4* ev = sh + jj * (2 * RS::SXH) + p;  // columns 2p, 2p+2, 2p+4
        const float4* od = ev + RS::SXH;                 // columns 2p+1, 2p+3
        float4 acc = f4fma(c_w5[0], ev[0], make_float4(0.f, 0.f, 0.f, 0.f));
        acc = f4fma(c_w5[1], od[0], acc);
        acc = f4fma(c_w5[2], ev[1], acc);
        acc = f4fma(c_w5[3], od[1], acc);
        acc = f4fma(c_w5[4], ev[2], acc);
        st(dst + (long long)(j - oc.y0) * oc.w() + (k - oc.x0), acc);
    }
}

// Blocks start in index order as resident ones finish, so block b prefetches into L2 the input of
// tile b + wave (wave = resident blocks on the device), which starts about when b ends.
// Column-sweep REDUCE of the single-rig path: 64 x 8 outputs of level l+1 from the 131 x 19 region
// of level l.  Thread t takes virtual column t + 2 and runs the vertical pass down its 19 rows in
// registers, with its loads straight from G^l a few rows ahead; the columns 0, 1 and 130 are one
// element per thread.  The vertically reduced rows go to shared memory (even and odd column
// planes, 16 banks apart) for the horizontal pass.  Shared memory carries 8 rows instead of the
// whole input region, and every operation is that of reduce_tile, in the same order.
using RSCol = RShape<64, 8>;
constexpr int RC_THREADS = 128;
constexpr int RC_VODD = 68, RC_VROW = 136;
constexpr size_t RC_SMEM = sizeof(float4) * (RC_VROW * RSCol::TY + 3 * RSCol::SY);
static_assert(RSCol::SX == RC_THREADS + 3 && RSCol::SY == 19 && RC_VODD >= RSCol::SXH && RC_VROW >= 2 * RC_VODD,
              "column per thread over a 131 x 19 region");
static_assert(RSAlt::TX == RSCol::TX && RSAlt::TY == RSCol::TY, "the staged schedule's 64 x 8 tiles run the column sweep");

template <typename T>
__device__ __forceinline__ void reduce_col_tile(const CamDev* __restrict__ cams, const RigGeom& g, int l, const Tile& tl,
                                                float4* smem, const Tile* pf) {
    constexpr int SX = RSCol::SX, SY = RSCol::SY, TX = RSCol::TX, TY = RSCol::TY;
    float4* vres = smem;                 // [TY][RC_VROW]
    float4* ext = smem + RC_VROW * TY;   // [SY][3]: columns 0, 1 and SX - 1
    const CamDev& c = cams[tl.cam];
    const Rect oc = c.Om[l + 1], of = c.Om[l];
    const int vx0 = 2 * tl.x0 - 2, vy0 = 2 * tl.y0 - 2;
    const T* src = reinterpret_cast<const T*>(c.FG[l]);
    const int nxl = g.nx[l], nyl = g.ny[l];
    const long long w = of.w();
    const int t = threadIdx.x;
    // a tile whose inputs lie inside Omega^l (so inside the level: nothing folds) reads them straight
    const bool inside = vx0 >= of.x0 && vx0 + SX <= of.x1 && vy0 >= of.y0 && vy0 + SY <= of.y1;
    auto elem = [&](int r, int x, bool xin) -> float4 {
        if (inside) return ld(src + (long long)(vy0 + r - of.y0) * w + (x - of.x0));
        const int y = fold101(vy0 + r, nyl);
        return xin && y >= of.y0 && y < of.y1 ? ld(src + (long long)(y - of.y0) * w + (x - of.x0))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto colx = [&](int cc, bool& xin) {
        const int x = inside ? vx0 + cc : fold101(vx0 + cc, nxl);
        xin = x >= of.x0 && x < of.x1;
        return x;
    };
    if (t < 3 * SY) {
        const int r = t / 3, k = t - 3 * r;
        bool xin;
        const int x = colx(k < 2 ? k : SX - 1, xin);
        ext[t] = elem(r, x, xin);
    }
    {
        const int cc = t + 2;
        bool xin;
        const int x = colx(cc, xin);
        float4* vcol = vres + (cc & 1) * RC_VODD + (cc >> 1);
        constexpr int D = 10;  // rows in flight ahead of the one being reduced
        float4 row[SY];
#pragma unroll
        for (int r = 0; r < D; ++r) row[r] = elem(r, x, xin);
        V4 B = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, C = B;
        // rows 2m complete output row m - 2 (stored from m = 2 on) and start row m; rows 2m + 1 add
        // their taps to rows m - 1 and m
#pragma unroll
        for (int r = 0; r < SY; ++r) {
            if (r + D < SY) row[r + D] = elem(r + D, x, xin);
            const V4 v = v4_of(row[r]);
            if ((r & 1) == 0) {
                if (r >= 4) vcol[(r / 2 - 2) * RC_VROW] = f4_of(v4_fma(d1_w(4), v, C));
                C = v4_fma(d1_w(2), v, B);
                B = v4_mul(d1_w(0), v);
            } else {
                C = v4_fma(d1_w(3), v, C);
                B = v4_fma(d1_w(1), v, B);
            }
        }
    }
    if (pf) reduce_prefetch<T, RSCol>(cams, l, *pf, RC_THREADS);  // the tile one resident wave later
    __syncthreads();
    if (t < 3 * TY) {
        const int jj = t / 3, k = t - 3 * jj, cc = k < 2 ? k : SX - 1;
        V4 acc = v4_mul(d1_w(0), v4_of(ext[(2 * jj) * 3 + k]));
#pragma unroll
        for (int n = 1; n < 5; ++n) acc = v4_fma(d1_w(n), v4_of(ext[(2 * jj + n) * 3 + k]), acc);
        vres[jj * RC_VROW + (cc & 1) * RC_VODD + (cc >> 1)] = f4_of(acc);
    }
    __syncthreads();
    T* dst = reinterpret_cast<T*>(c.FG[l + 1]);
    const int p = t % TX, k = tl.x0 + p;
#pragma unroll
    for (int q = 0; q < TY * TX / RC_THREADS; ++q) {
        const int jj = t / TX + q * (RC_THREADS / TX), j = tl.y0 + jj;
        const float4* ev = vres + jj * RC_VROW + p;  // columns 2p, 2p+2, 2p+4
        const float4* od = ev + RC_VODD;             // columns 2p+1, 2p+3
        V4 acc = v4_mul(d1_w(0), v4_of(ev[0]));
        acc = v4_fma(d1_w(1), v4_of(od[0]), acc);
        acc = v4_fma(d1_w(2), v4_of(ev[1]), acc);
        acc = v4_fma(d1_w(3), v4_of(od[1]), acc);
        acc = v4_fma(d1_w(4), v4_of(ev[2]), acc);
        if (k >= oc.x1 || j >= oc.y1) continue;
        if (!STITCH_DCHECK(k >= oc.x0 && j >= oc.y0, 3, (long long)k << 24 | j)) continue;
        st(dst + (long long)(j - oc.y0) * oc.w() + (k - oc.x0), f4_of(acc));
    }
}

template <typename T>
__global__ void __launch_bounds__(RC_THREADS, 8) k_reduce_t(const CamDev* __restrict__ cams, const __grid_constant__ RigGeom g,
                                                           int l, const Tile* __restrict__ tiles, int n, int wave) {
    extern __shared__ float4 smem[];
    const int nb = blockIdx.x + wave;
    reduce_col_tile<T>(cams, g, l, tiles[blockIdx.x], smem, nb < n ? tiles + nb : nullptr);
}

// ------------------------------------------------------------------------------------------------
// coarse levels

// Polyphase EXPAND of a 2x2 block of fine samples whose coarse 3x3 neighbourhood starts at
// a[oy][ox] (row stride ld): even-even, odd-even (x odd), even-odd (y odd), odd-odd.  R and G go
// as one pair, B alone; the fourth channel is not expanded.
struct V3 {
    float2 rg;
    float b;
};
__device__ __forceinline__ V3 v3_of(float4 v) { return {make_float2(v.x, v.y), v.z}; }
__device__ __forceinline__ V3 v3_zero() { return {make_float2(0.f, 0.f), 0.f}; }

__device__ __forceinline__ void expand_quad(const float4* __restrict__ a, int ld, int ox, int oy, V3 e[4]) {
    const float2 k75 = f2(0.75f), k125 = f2(0.125f), k5 = f2(0.5f);
    auto even = [&](V3 c0, V3 c1, V3 c2) -> V3 {  // (1, 6, 1) / 8
        return {f2fma(k75, c1.rg, f2mul(k125, f2add(c0.rg, c2.rg))), fmaf(0.75f, c1.b, 0.125f * (c0.b + c2.b))};
    };
    auto odd = [&](V3 c1, V3 c2) -> V3 {  // (4, 4) / 8
        return {f2mul(k5, f2add(c1.rg, c2.rg)), 0.5f * (c1.b + c2.b)};
    };
    V3 he[3], ho[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const V3 c0 = v3_of(a[(oy + r) * ld + ox]), c1 = v3_of(a[(oy + r) * ld + ox + 1]), c2 = v3_of(a[(oy + r) * ld + ox + 2]);
        he[r] = even(c0, c1, c2);
        ho[r] = odd(c1, c2);
    }
    e[0] = even(he[0], he[1], he[2]);
    e[1] = even(ho[0], ho[1], ho[2]);
    e[2] = odd(he[1], he[2]);
    e[3] = odd(ho[1], ho[2]);
}

// Tiled coarse level: R^l on a tile of level l (l >= 2), one 2 x 2 quad per thread, cameras in
// chunks of 2.  Virtual level-(l+1) region: origin (X0/2 - 2, Y0/2 - 2), TX/2 + 4 by TY/2 + 4.
// The tile shape is a template parameter (the batched schedule's tuner picks one per batch); the
// single-rig path uses 32 x 32.
constexpr int CT_NC = 2;
template <int X, int Y>
struct CShape {
    static constexpr int TX = X, TY = Y;                   // level-l outputs
    static constexpr int CX = X / 2 + 4, CY = Y / 2 + 4;   // level-(l+1) virtual region
    static constexpr int CN = CX * CY, TN = X * Y;
    static constexpr int QUADS = (X / 2) * (Y / 2);
    static constexpr int SMEM_F4 = CN + CT_NC * CN;  // shared memory in float4 units
    static_assert(QUADS == 256, "one 2 x 2 quad per thread of a 256-thread block");
};
using CS32x32 = CShape<32, 32>;
using CS64x16 = CShape<64, 16>;
using CSRig = CS32x32;  // the shape of a rig's own coarse tiles (the single-rig path, the persistent batch)
using CSAlt = CShape<CSRig::TX * 2, CSRig::TY / 2>;  // the batch tuner's other shape (64 x 16)
constexpr int CT_X = CSRig::TX, CT_Y = CSRig::TY;
constexpr int CT_SMEM_F4 = CSRig::SMEM_F4;

struct LevelTile {
    int x0, y0, first, count;  // level origin, range of camera indices in the list
};

template <typename T, typename CS = CS32x32>
__device__ __forceinline__ void coarse_tile(const CamDev* __restrict__ cams, const RigGeom& g, int l,
                                            T* __restrict__ Rl, const T* __restrict__ Rc, const LevelTile& tl,
                                            const int* __restrict__ camlist, float4* smem) {
    float4* rc = smem;                                                   // [CS::CN] R^{l+1}
    float4 (*gc)[CS::CN] = reinterpret_cast<float4 (*)[CS::CN]>(rc + CS::CN);  // [CT_NC][CS::CN] G^{l+1}, then R - G
    const bool top = l == g.levels - 1;
    const int X0 = tl.x0, Y0 = tl.y0;
    const int ax = X0 / 2 - 2, ay = Y0 / 2 - 2;
    const int nxl = g.nx[l], nyl = g.ny[l];
    const int t = threadIdx.x;
    if (!top) {
        for (int q = t; q < CS::CN; q += 256) {
            const int r = q / CS::CX, c = q - r * CS::CX;
            const int x = fold101(ax + c, g.nx[l + 1]), y = fold101(ay + r, g.ny[l + 1]);
            rc[q] = ld(Rc + (long long)y * g.nx[l + 1] + x);
        }
    }
    const int qx = t % (CS::TX / 2), qy = t / (CS::TX / 2);
    const bool has_quad = t < CS::QUADS;
    float2 nrg[4];
    float nb[4], den[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nrg[k] = make_float2(0.f, 0.f);
        nb[k] = den[k] = 0.f;
    }
    for (int c0 = 0; c0 < tl.count; c0 += CT_NC) {
        const int nc = min(CT_NC, tl.count - c0);
        __syncthreads();
        // the chunk's G^{l+1} regions into shared memory, all loads in flight before the stores
        {
            constexpr int NC2 = (CT_NC * CS::CN + 255) / 256;
            float4 w[NC2];
#pragma unroll
            for (int k = 0; k < NC2; ++k) {
                const int q = t + 256 * k;
                w[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!top && q < nc * CS::CN) {
                    const int ci = q / CS::CN, qq = q - ci * CS::CN;
                    const CamDev& c = cams[camlist[tl.first + c0 + ci]];
                    const int r = qq / CS::CX, cc = qq - r * CS::CX;
                    const int x = fold101(ax + cc, g.nx[l + 1]), y = fold101(ay + r, g.ny[l + 1]);
                    const Rect o = c.Om[l + 1];
                    if (o.contains(x, y))
                        w[k] = ld(reinterpret_cast<const T*>(c.FG[l + 1]) + (long long)(y - o.y0) * o.w() + (x - o.x0));
                }
            }
#pragma unroll
            for (int k = 0; k < NC2; ++k) {
                const int q = t + 256 * k;
                if (!top && q < nc * CS::CN) gc[q / CS::CN][q % CS::CN] = w[k];
            }
        }
        __syncthreads();
        if (!top) {
            for (int q = t; q < nc * CS::CN; q += 256) {
                const int ci = q / CS::CN, qq = q - ci * CS::CN;
                const float4 a = rc[qq], b = gc[ci][qq];
                gc[ci][qq] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f);
            }
            __syncthreads();
        }
        if (has_quad) {
            for (int ci = 0; ci < nc; ++ci) {
                // the quad's G^l of the camera: each value is read by this thread only, so it goes
                // straight into registers (only inside Z^l, where it enters the blend)
                const CamDev& c = cams[camlist[tl.first + c0 + ci]];
                const Rect z = c.Z[l], o = c.Om[l];
                const T* fg = reinterpret_cast<const T*>(c.FG[l]);
                float4 gq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int x = X0 + 2 * qx + (k & 1), y = Y0 + 2 * qy + (k >> 1);
                    gq[k] = z.contains(x, y) ? ld(fg + (long long)(y - o.y0) * o.w() + (x - o.x0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                V3 e[4] = {v3_zero(), v3_zero(), v3_zero(), v3_zero()};
                if (!top) expand_quad(gc[ci], CS::CX, qx + 1, qy + 1, e);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int x = X0 + 2 * qx + (k & 1), y = Y0 + 2 * qy + (k >> 1);
                    if (!z.contains(x, y)) continue;
                    const float4 gv = gq[k];
                    nrg[k] = f2fma(f2(gv.w), f2add(make_float2(gv.x, gv.y), e[k].rg), nrg[k]);
                    nb[k] = fmaf(gv.w, gv.z + e[k].b, nb[k]);
                    den[k] += gv.w;
                }
            }
        }
    }
    if (!has_quad) return;
    V3 e[4] = {v3_zero(), v3_zero(), v3_zero(), v3_zero()};
    bool need = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) need |= !(den[k] > 1e-12f);
    if (need && !top) expand_quad(rc, CS::CX, qx + 1, qy + 1, e);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = X0 + 2 * qx + (k & 1), y = Y0 + 2 * qy + (k >> 1);
        if (x >= nxl || y >= nyl) continue;
        if (!STITCH_DCHECK(x >= 0 && y >= 0, 4, (long long)x << 24 | y)) continue;
        float4 r = make_float4(e[k].rg.x, e[k].rg.y, e[k].b, 0.f);
        if (den[k] > 1e-12f) {
            const float rd = __frcp_rn(den[k]);  // one reciprocal, three products (within 1 ulp of division)
            const float2 q = f2mul(nrg[k], f2(rd));
            r = make_float4(q.x, q.y, nb[k] * rd, 0.f);
        }
        st(Rl + (long long)y * nxl + x, r);
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_coarse_t(const CamDev* __restrict__ cams, const __grid_constant__ RigGeom g, int l,
                                                   T* __restrict__ Rl, const T* __restrict__ Rc,
                                                   const LevelTile* __restrict__ tiles,
                                                   const int* __restrict__ camlist) {
    extern __shared__ float4 smem[];
    coarse_tile<T, CSRig>(cams, g, l, Rl, Rc, tiles[blockIdx.x], camlist, smem);
}

// ------------------------------------------------------------------------------------------------
// up: levels 1 and 0 of one canvas tile

constexpr int U_TX = 64, U_TY = 32;                     // level-0 pixels per tile
static_assert(D1_SLOT == U_TX * U_TY && 2 * D1_TX == U_TX && 4 * D1_TY == U_TY,
              "two down1 tiles over one canvas tile of up");
constexpr int U_THREADS = 256;
// virtual regions, origins (X0/2 - 2, Y0/2 - 2) at level 1 and (X0/4 - 2, Y0/4 - 2) at level 2
constexpr int U1_X = U_TX / 2 + 4, U1_Y = U_TY / 2 + 4;  // 36 x 20
constexpr int U2_X = U_TX / 4 + 4, U2_Y = U_TY / 4 + 4;  // 20 x 12
constexpr int U1_N = U1_X * U1_Y, U2_N = U2_X * U2_Y;
constexpr int U_QUADS0 = (U_TX / 2) * (U_TY / 2);        // 512 level-0 quads
constexpr int U_QUADS1 = (U1_X / 2) * (U1_Y / 2);        // 180 level-1 quads

// Write a tile's uint8 output staged in shared memory (rows of 3*U_TX bytes): 32-bit stores when
// the destination rows are 4-byte aligned and the tile is full width, bytes otherwise.
__device__ __forceinline__ void store_u8_tile(const unsigned char* __restrict__ stage, const OutDesc& od, int X0,
                                              int Y0, int X1, int Y1) {
    const int bytes = 3 * (X1 - X0), rows = Y1 - Y0;
    unsigned char* base = (unsigned char*)od.ptr + (long long)Y0 * od.pitch + 3LL * X0;
    const bool words = (bytes == 3 * U_TX) && ((((uintptr_t)base) | (uintptr_t)od.pitch) % 4 == 0);
    if (words) {
        constexpr int WPR = 3 * U_TX / 4;  // 48 words per row
        for (int q = threadIdx.x; q < rows * WPR; q += blockDim.x) {
            const int r = q / WPR, c = q - r * WPR;
            reinterpret_cast<uint32_t*>(base + (long long)r * od.pitch)[c] =
                reinterpret_cast<const uint32_t*>(stage + r * 3 * U_TX)[c];
        }
    } else {
        for (int q = threadIdx.x; q < rows * bytes; q += blockDim.x) {
            const int r = q / bytes, c = q - r * bytes;
            base[(long long)r * od.pitch + c] = stage[r * 3 * U_TX + c];
        }
    }
}

__device__ __forceinline__ void put_pixel(unsigned char* stage, const OutDesc& od, int dx, int dy, int x, int y,
                                          float r, float g, float b) {
    if (od.is_float) {
        float* o = (float*)((char*)od.ptr + (long long)y * od.pitch) + 3 * x;
        o[0] = r;
        o[1] = g;
        o[2] = b;
    } else {
        unsigned char* o = stage + dy * 3 * U_TX + 3 * dx;
        o[0] = quantize_u8(r);
        o[1] = quantize_u8(g);
        o[2] = quantize_u8(b);
    }
}

// ZERO and SOLO tiles: output 0, or the clamped warp of the one exclusive camera.
__device__ __forceinline__ void up_simple_tile(const CamDev* __restrict__ cams, const RigGeom& g, const FramePtrs& fp,
                                               const OutDesc& od, const UpTile& tl, const CamRef* __restrict__ refs,
                                               unsigned char* stage) {
    const int X0 = tl.x0, Y0 = tl.y0;
    const int X1 = min(X0 + U_TX, g.nx[0]), Y1 = min(Y0 + U_TY, g.ny[0]);
    if (tl.count == 0) {
        for (int p = threadIdx.x; p < U_TX * U_TY; p += U_THREADS) {
            const int dx = p % U_TX, dy = p / U_TX;
            if (X0 + dx < X1 && Y0 + dy < Y1) put_pixel(stage, od, dx, dy, X0 + dx, Y0 + dy, 0.f, 0.f, 0.f);
        }
    } else {
        const CamRef cr = refs[tl.first];
        const CamDev& c = cams[cr.cam];
        const int W = c.W, H = c.H;
        const float scale = c.gain * (1.0f / 255.0f);
        const float fU0 = (float)cr.tm.U0, fV0 = (float)cr.tm.V0;
        const uint8_t* px = fp.p[cr.cam];
        const long long pitch = fp.pitch[cr.cam];
        for (int p = threadIdx.x; p < U_TX * U_TY; p += U_THREADS) {
            const int dx = p % U_TX, dy = p / U_TX;
            const int x = X0 + dx, y = Y0 + dy;
            if (x >= X1 || y >= Y1) continue;
            const Pos ps = g.cyl ? map_pos64(c, g, x, y) : map_pos(cr.tm, fU0, fV0, (float)(x - cr.ax), (float)(y - cr.ay));
            const float3 v = sample_rgb(px, pitch, ps, W, H, scale);
            put_pixel(stage, od, dx, dy, x, y, __saturatef(v.x), __saturatef(v.y), __saturatef(v.z));
        }
    }
    if (!od.is_float) {
        __syncthreads();
        store_u8_tile(stage, od, X0, Y0, X1, Y1);
    }
}

__global__ void __launch_bounds__(U_THREADS) k_up_simple(const CamDev* __restrict__ cams, RigGeom g, FramePtrs fp,
                                                          OutDesc od, const UpTile* __restrict__ tiles,
                                                          const CamRef* __restrict__ refs) {
    __shared__ __align__(16) unsigned char stage[3 * U_TX * U_TY];
    up_simple_tile(cams, g, fp, od, tiles[blockIdx.x], refs, stage);
}

// FULL tiles with at most NC contributing cameras.
// Per-camera constants of a FULL tile, kept in shared memory.
template <int NC>
struct UpCams {
    CamRef cr[NC];
    Rect om1[NC], om2[NC];       // the cameras' Omega^1, Omega^2
    const void* fg1[NC];         // and their G^1, G^2
    const void* fg2[NC];
    float dsc[NC];               // scale / SLOT_RGB: slot codes to scaled units
};

// L2 prefetch of an up_full tile's largest inputs: the level-0 slots of its blended cameras
// (one 128-byte line per thread and pass) and their G^1 rows inside Omega^1.
template <typename T, int NC>
__device__ __forceinline__ void up_prefetch(const CamDev* __restrict__ cams, const UpTile& tn,
                                            const CamRef* __restrict__ refs, const Slot* __restrict__ g0buf) {
    const int nc = min(tn.count, NC);
    const int a1x = tn.x0 / 2 - 2, a1y = tn.y0 / 2 - 2;
    for (int c = 0; c < nc; ++c) {
        const CamRef& cr = refs[tn.first + c];
        if (cr.g0 >= 0) {
            const char* p = reinterpret_cast<const char*>(g0buf + (long long)cr.g0 * (U_TX * U_TY));
            for (int q = threadIdx.x; q < (int)(U_TX * U_TY * sizeof(Slot)) / 128; q += U_THREADS) prefetch_l2(p + 128 * q);
        }
        const CamDev& cd = cams[cr.cam];
        const Rect o1 = cd.Om[1];
        const int x0 = max(a1x, o1.x0), x1 = min(a1x + U1_X, o1.x1);
        if (x1 <= x0) continue;
        const char* base = reinterpret_cast<const char*>(cd.FG[1]);
        const int len = (x1 - x0) * (int)sizeof(T);
        for (int q = threadIdx.x; q < 8 * U1_Y; q += U_THREADS) {
            const int rr = q >> 3, k = q & 7, y = a1y + rr;
            if (y < o1.y0 || y >= o1.y1 || 128 * k >= len + 127) continue;
            prefetch_l2(base + ((long long)(y - o1.y0) * o1.w() + (x0 - o1.x0)) * (long long)sizeof(T) + min(128 * k, len - 1));
        }
    }
}

// NB: blended cameras whose level-0 slot loads are in flight at once (1 or 2)
template <typename T, int NC, int NB = (NC < 2 ? NC : 2)>
__device__ __forceinline__ void up_full_tile(const CamDev* __restrict__ cams, const RigGeom& g, const FramePtrs& fp,
                                             const OutDesc& od, const T* __restrict__ R2, const UpTile& tl,
                                             const CamRef* __restrict__ refs, const Slot* __restrict__ g0buf,
                                             float4* usm, const UpTile* pf = nullptr) {
    float4* d1 = usm;                // [NC][U1_N]: G^1 of each camera, then R^1 - G^1
    float4* d2 = d1 + NC * U1_N;     // [NC][U2_N]: G^2 of each camera, then R^2 - G^2
    float4* r2s = d2 + NC * U2_N;    // [U2_N]: R^2
    unsigned char* stage = reinterpret_cast<unsigned char*>(r2s + U2_N);
    UpCams<NC>& ucs = *reinterpret_cast<UpCams<NC>*>(stage + 3 * U_TX * U_TY);
    CamRef* cr = ucs.cr;

    const int L = g.levels;
    const int nc = min(tl.count, NC);
    const int X0 = tl.x0, Y0 = tl.y0;
    const int X1 = min(X0 + U_TX, g.nx[0]), Y1 = min(Y0 + U_TY, g.ny[0]);
    const int a1x = X0 / 2 - 2, a1y = Y0 / 2 - 2;
    const int a2x = X0 / 4 - 2, a2y = Y0 / 4 - 2;
    const int t = threadIdx.x;
    if (t < nc) {
        cr[t] = refs[tl.first + t];
        const CamDev& c = cams[cr[t].cam];
        ucs.om1[t] = c.Om[1];
        ucs.om2[t] = c.Om[2];
        ucs.fg1[t] = c.FG[1];
        ucs.fg2[t] = c.FG[2];
        ucs.dsc[t] = c.gain * (1.0f / 255.0f) * (1.0f / SLOT_RGB);
    }
    __syncthreads();
    // loads of level 1 and 2 data, all of a thread's loads in flight before the stores
    if (L >= 2) {
        constexpr int NL = (NC * U1_N + U_THREADS - 1) / U_THREADS;
        float4 v[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = t + k * U_THREADS;
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < nc * U1_N) {
                const int ci = q / U1_N, qq = q - ci * U1_N;
                const int r = qq / U1_X, cc = qq - r * U1_X;
                const int x = fold101(a1x + cc, g.nx[1]), y = fold101(a1y + r, g.ny[1]);
                const Rect o1 = ucs.om1[ci];
                if (o1.contains(x, y))
                    v[k] = ld(reinterpret_cast<const T*>(ucs.fg1[ci]) + (long long)(y - o1.y0) * o1.w() + (x - o1.x0));
            }
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = t + k * U_THREADS;
            if (q < nc * U1_N) d1[q] = v[k];
        }
    }
    if (L >= 3) {
        constexpr int NL = ((NC + 1) * U2_N + U_THREADS - 1) / U_THREADS;
        float4 v[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = t + k * U_THREADS;
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < (nc + 1) * U2_N) {
                const int ci = q / U2_N, qq = q - ci * U2_N;
                const int r = qq / U2_X, cc = qq - r * U2_X;
                const int x = fold101(a2x + cc, g.nx[2]), y = fold101(a2y + r, g.ny[2]);
                if (ci == nc) {
                    v[k] = ld(R2 + (long long)y * g.nx[2] + x);
                } else {
                    const Rect o2 = ucs.om2[ci];
                    if (o2.contains(x, y))
                        v[k] = ld(reinterpret_cast<const T*>(ucs.fg2[ci]) + (long long)(y - o2.y0) * o2.w() + (x - o2.x0));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int q = t + k * U_THREADS;
            if (q < (nc + 1) * U2_N) {
                const int ci = q / U2_N, qq = q - ci * U2_N;
                if (ci == nc) r2s[qq] = v[k];
                else d2[q] = v[k];
            }
        }
    }
    if (pf) up_prefetch<T, NC>(cams, *pf, refs, g0buf);  // the tile one resident wave later
    __syncthreads();
    if (L >= 3) {
        // Delta^2_i = R^2 - G^2_i
        for (int q = t; q < nc * U2_N; q += U_THREADS) {
            const float4 rv = r2s[q % U2_N], gv = d2[q];
            d2[q] = make_float4(rv.x - gv.x, rv.y - gv.y, rv.z - gv.z, 0.f);
        }
        __syncthreads();
    }
    if (L >= 2 && t < U_QUADS1) {
        // level 1: R^1 = sum_i a_i (G^1_i + EXPAND(Delta^2_i)), then Delta^1_i = R^1 - G^1_i in place
        const int qx = t % (U1_X / 2), qy = t / (U1_X / 2);
        float3 num[4];
        float den[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            num[k] = make_float3(0.f, 0.f, 0.f);
            den[k] = 0.f;
        }
        for (int c = 0; c < nc; ++c) {
            float3 e[4] = {make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 0.f),
                           make_float3(0.f, 0.f, 0.f)};
            if (L >= 3) {
                V3 e2[4];
                expand_quad(d2 + c * U2_N, U2_X, qx, qy, e2);
#pragma unroll
                for (int k = 0; k < 4; ++k) e[k] = make_float3(e2[k].rg.x, e2[k].rg.y, e2[k].b);
            }

            // outside the camera's Z^1 its weight pyramid is exactly 0, so those terms add nothing
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 gv = d1[c * U1_N + (2 * qy + (k >> 1)) * U1_X + 2 * qx + (k & 1)];
                num[k].x = fmaf(gv.w, gv.x + e[k].x, num[k].x);
                num[k].y = fmaf(gv.w, gv.y + e[k].y, num[k].y);
                num[k].z = fmaf(gv.w, gv.z + e[k].z, num[k].z);
                den[k] += gv.w;
            }
        }
        float3 r1[4];
        bool need_plain = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (den[k] > 1e-12f) {
                const float rd = __frcp_rn(den[k]);
                r1[k] = make_float3(num[k].x * rd, num[k].y * rd, num[k].z * rd);
            } else {
                r1[k] = make_float3(0.f, 0.f, 0.f);
                need_plain = true;
            }
        }
        if (need_plain && L >= 3) {
            V3 e[4];
            expand_quad(r2s, U2_X, qx, qy, e);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (!(den[k] > 1e-12f)) r1[k] = make_float3(e[k].rg.x, e[k].rg.y, e[k].b);
        }
        for (int c = 0; c < nc; ++c) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4& dv = d1[c * U1_N + (2 * qy + (k >> 1)) * U1_X + 2 * qx + (k & 1)];
                dv = make_float4(r1[k].x - dv.x, r1[k].y - dv.y, r1[k].z - dv.z, 0.f);
            }
        }
    }
    __syncthreads();
    if (L >= 2 && (a1x + U1_X > g.nx[1] || a1y + U1_Y > g.ny[1])) {
        // Past the right or bottom border the level-1 region's values are those of the folded
        // positions.  Delta^1 was evaluated there with EXPAND on the virtual level-2 grid, which
        // agrees with the folded position's value only where the level's size is odd (the fine and
        // coarse reflection points then correspond), so copy them from the folded positions.
        for (int q = t; q < nc * U1_N; q += U_THREADS) {
            const int ci = q / U1_N, qq = q - ci * U1_N;
            const int r = qq / U1_X, cc = qq - r * U1_X;
            if (a1x + cc < g.nx[1] && a1y + r < g.ny[1]) continue;
            const int sx = fold101(a1x + cc, g.nx[1]) - a1x, sy = fold101(a1y + r, g.ny[1]) - a1y;
            if (sx >= 0 && sx < U1_X && sy >= 0 && sy < U1_Y) d1[ci * U1_N + qq] = d1[ci * U1_N + sy * U1_X + sx];
        }
        __syncthreads();
    }
    // level 0: R^0 = sum_i a_i (G^0_i + EXPAND(Delta^1_i)) / sum_i a_i on covered pixels, with the
    // level-0 sample G^0_i and normalised weight a_i of every blended camera written by its down1
    // tile (slot g0)
    for (int qd = t; qd < U_QUADS0; qd += U_THREADS) {
        const int qx = qd % (U_TX / 2), qy = qd / (U_TX / 2);
        float3 num[4];
        float den[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            num[k] = make_float3(0.f, 0.f, 0.f);
            den[k] = 0.f;
        }
        // the level-0 samples of every blended camera, NB cameras at a time (all their loads in
        // flight at once); the weights enter as their slot codes

        for (int c0 = 0; c0 < nc; c0 += NB) {
            Slot gw[NB][4];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int slot = c0 + b < nc ? cr[c0 + b].g0 : -1;
                const Slot* gq = g0buf + (long long)max(slot, 0) * (U_TX * U_TY) + (2 * qy) * U_TX + 2 * qx;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    gw[b][k] = slot >= 0 ? __ldcg(gq + (k >> 1) * U_TX + (k & 1)) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int c = c0 + b;
                if (c >= nc || cr[c].g0 < 0) continue;
                V3 e[4];
                expand_quad(d1 + c * U1_N, U1_X, qx + 1, qy + 1, e);
                // a camera's weight is 0 (and its sample 0) where it does not cover the pixel: the
                // terms add nothing there, so no test is needed
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 gv = slot_decode(gw[b][k], ucs.dsc[c]);
                    num[k].x = fmaf(gv.w, gv.x + e[k].rg.x, num[k].x);
                    num[k].y = fmaf(gv.w, gv.y + e[k].rg.y, num[k].y);
                    num[k].z = fmaf(gv.w, gv.z + e[k].b, num[k].z);
                    den[k] += gv.w;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int dx = 2 * qx + (k & 1), dy = 2 * qy + (k >> 1);
            const int x = X0 + dx, y = Y0 + dy;
            if (x >= X1 || y >= Y1) continue;
            float rr = 0.f, gg = 0.f, bb = 0.f;
            if (den[k] > 0.f) {
                const float rd = __frcp_rn(den[k]);
                rr = __saturatef(num[k].x * rd);
                gg = __saturatef(num[k].y * rd);
                bb = __saturatef(num[k].z * rd);
            }
            put_pixel(stage, od, dx, dy, x, y, rr, gg, bb);
        }
    }
    if (!od.is_float) {
        __syncthreads();
        store_u8_tile(stage, od, X0, Y0, X1, Y1);
    }
}

// Blocks n .. n + n_simple - 1 take the ZERO (and fallback SOLO) canvas tiles `simple`, so that they
// need no launch of their own.
template <typename T, int NC, int NB>
__device__ __forceinline__ void up_full_block(const CamDev* __restrict__ cams, const RigGeom& g, const FramePtrs& fp,
                                              const OutDesc& od, const T* __restrict__ R2, const UpTile* __restrict__ tiles,
                                              const CamRef* __restrict__ refs, const Slot* __restrict__ g0buf, int n,
                                              int wave, const UpTile* __restrict__ simple, float4* usm) {
    if ((int)blockIdx.x >= n) {
        up_simple_tile(cams, g, fp, od, simple[blockIdx.x - n], refs, reinterpret_cast<unsigned char*>(usm));
        return;
    }
    const int nb = blockIdx.x + wave;  // prefetched: the tile one resident wave later (see k_reduce_t)
    up_full_tile<T, NC, NB>(cams, g, fp, od, R2, tiles[blockIdx.x], refs, g0buf, usm, nb < n ? tiles + nb : nullptr);
}
// Two occupancies: k_up_full_b4 holds four resident blocks per SM (64 registers, a few spilled in
// the level-1 phase, one camera's slot loads at a time), for rigs with many waves of canvas tiles;
// k_up_full three, with two cameras' slot loads in flight, which wins when the launch is a few waves.
template <typename T, int NC>
__global__ void __launch_bounds__(U_THREADS) k_up_full(const CamDev* __restrict__ cams, RigGeom g, FramePtrs fp,
                                                        OutDesc od, const T* __restrict__ R2,
                                                        const UpTile* __restrict__ tiles,
                                                        const CamRef* __restrict__ refs, const Slot* __restrict__ g0buf,
                                                        int n, int wave, const UpTile* __restrict__ simple) {
    extern __shared__ float4 usm[];
    up_full_block<T, NC, (NC < 2 ? NC : 2)>(cams, g, fp, od, R2, tiles, refs, g0buf, n, wave, simple, usm);
}
template <typename T, int NC>
__global__ void __launch_bounds__(U_THREADS, 4) k_up_full_b4(const CamDev* __restrict__ cams, RigGeom g, FramePtrs fp,
                                                              OutDesc od, const T* __restrict__ R2,
                                                              const UpTile* __restrict__ tiles,
                                                              const CamRef* __restrict__ refs,
                                                              const Slot* __restrict__ g0buf, int n, int wave,
                                                              const UpTile* __restrict__ simple) {
    extern __shared__ float4 usm[];
    up_full_block<T, NC, 1>(cams, g, fp, od, R2, tiles, refs, g0buf, n, wave, simple, usm);
}

template <int NC>
constexpr size_t up_full_smem() {
    return sizeof(float4) * (NC * U1_N + NC * U2_N + U2_N) + 3 * U_TX * U_TY + sizeof(UpCams<NC>);
}

// ------------------------------------------------------------------------------------------------
// GENERAL tiles (more than 4 contributing cameras): one camera at a time through shared memory.

constexpr int UG_PPT = U_TX * U_TY / U_THREADS;                  // level-0 pixels per thread (8)
constexpr int UG1_X = U_TX / 2 + 2, UG1_Y = U_TY / 2 + 2;       // level-1 virtual region (34 x 18)
constexpr int UG2_X = U_TX / 4 + 3, UG2_Y = U_TY / 4 + 3;       // level-2 virtual region (19 x 11)
constexpr int UG1_N = UG1_X * UG1_Y;
constexpr int UG1_PT = (UG1_N + U_THREADS - 1) / U_THREADS;

// EXPAND at fine offset (dx, dy) from a virtual coarse array whose index 0 sits one coarse
// sample before the fine origin's coarse position.
__device__ __forceinline__ float3 expand_smem(const float4* __restrict__ a, int ldx, int dx, int dy) {
    const int ky0 = (dy & 1) ? (dy + 1) / 2 : dy / 2, nky = (dy & 1) ? 2 : 3;
    const int kx0 = (dx & 1) ? (dx + 1) / 2 : dx / 2, nkx = (dx & 1) ? 2 : 3;
    float3 acc = make_float3(0.f, 0.f, 0.f);
    for (int p = 0; p < nky; ++p) {
        const float wy = (dy & 1) ? 0.5f : (p == 1 ? 0.75f : 0.125f);
        float3 row = make_float3(0.f, 0.f, 0.f);
        const float4* rp = a + (ky0 + p) * ldx + kx0;
        for (int q = 0; q < nkx; ++q) {
            const float wx = (dx & 1) ? 0.5f : (q == 1 ? 0.75f : 0.125f);
            const float4 v = rp[q];
            row.x = fmaf(wx, v.x, row.x);
            row.y = fmaf(wx, v.y, row.y);
            row.z = fmaf(wx, v.z, row.z);
        }
        acc.x = fmaf(wy, row.x, acc.x);
        acc.y = fmaf(wy, row.y, acc.y);
        acc.z = fmaf(wy, row.z, acc.z);
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void up_general_tile(const CamDev* __restrict__ cams, const RigGeom& g, const FramePtrs& fp,
                                                const OutDesc& od, const T* __restrict__ R2, const UpTile& tl,
                                                const CamRef* __restrict__ refs, float4* smem) {
    float4* g1 = smem;                   // [UG1_N]
    float4* g2 = g1 + UG1_N;             // [UG2_X * UG2_Y]
    float4* r2 = g2 + UG2_X * UG2_Y;     // [UG2_X * UG2_Y]
    float4* r1 = r2 + UG2_X * UG2_Y;     // [UG1_N]

    const int L = g.levels;
    const int X0 = tl.x0, Y0 = tl.y0;
    const int X1 = min(X0 + U_TX, g.nx[0]), Y1 = min(Y0 + U_TY, g.ny[0]);
    const int a1x = X0 / 2 - 1, a1y = Y0 / 2 - 1;          // level-1 virtual origin
    const int a2x = (a1x - 1) / 2, a2y = (a1y - 1) / 2;    // level-2 virtual origin (a1 odd)
    const int t = threadIdx.x;
    const int na = tl.count;
    if (L >= 3) {
        for (int q = t; q < UG2_X * UG2_Y; q += U_THREADS) {
            const int r = q / UG2_X, c = q - r * UG2_X;
            const int x = fold101(a2x + c, g.nx[2]), y = fold101(a2y + r, g.ny[2]);
            r2[q] = ld(R2 + (long long)y * g.nx[2] + x);
        }
    }
    __syncthreads();

    float ws[UG_PPT];
    int own[UG_PPT];  // seam weights: list position of the pixel's owner
    float4 n0[UG_PPT];
#pragma unroll
    for (int k = 0; k < UG_PPT; ++k) {
        const int p = t + k * U_THREADS;
        const int x = X0 + (p & (U_TX - 1)), y = Y0 + p / U_TX;
        float s = 0.f;
        own[k] = -1;
        if (g.seam) {
            if (x < X1 && y < Y1)
                own[k] = seam_owner(g, na, [&](int m) -> const CamDev& { return cams[refs[tl.first + m].cam]; }, x, y);
            s = own[k] >= 0 ? 1.f : 0.f;
        } else if (x < X1 && y < Y1) {
            for (int a = 0; a < na; ++a) {
                const CamRef cr = refs[tl.first + a];
                const CamDev& c = cams[cr.cam];
                if (!c.V.contains(x, y)) continue;
                const SrcPos sp = g.cyl ? map_point64(c, g, x, y) : map_point(cr.tm, (float)(x - cr.ax), (float)(y - cr.ay));
                s += feather_weight(sp, c.W, c.H);
            }
        }
        ws[k] = s;
        n0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 n1[UG1_PT];
#pragma unroll
    for (int k = 0; k < UG1_PT; ++k) n1[k] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (int a = 0; a < na; ++a) {
        const CamRef cr = refs[tl.first + a];
        const int i = cr.cam;
        const CamDev& c = cams[i];
        if (L >= 2) {
            const Rect o1 = c.Om[1];
            const T* G1 = reinterpret_cast<const T*>(c.FG[1]);
            for (int q = t; q < UG1_N; q += U_THREADS) {
                const int r = q / UG1_X, cc = q - r * UG1_X;
                const int x = fold101(a1x + cc, g.nx[1]), y = fold101(a1y + r, g.ny[1]);
                g1[q] = o1.contains(x, y) ? ld(G1 + (long long)(y - o1.y0) * o1.w() + (x - o1.x0))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (L >= 3) {
                const Rect o2 = c.Om[2];
                const T* G2 = reinterpret_cast<const T*>(c.FG[2]);
                for (int q = t; q < UG2_X * UG2_Y; q += U_THREADS) {
                    const int r = q / UG2_X, cc = q - r * UG2_X;
                    const int x = fold101(a2x + cc, g.nx[2]), y = fold101(a2y + r, g.ny[2]);
                    g2[q] = o2.contains(x, y) ? ld(G2 + (long long)(y - o2.y0) * o2.w() + (x - o2.x0))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
            const Rect z1 = c.Z[1];
#pragma unroll
            for (int k = 0; k < UG1_PT; ++k) {
                const int q = t + k * U_THREADS;
                if (q >= UG1_N) break;
                const int r = q / UG1_X, cc = q - r * UG1_X;
                const int x = fold101(a1x + cc, g.nx[1]), y = fold101(a1y + r, g.ny[1]);
                if (!z1.contains(x, y)) continue;
                const float4 gv = g1[q];
                float lr = gv.x, lg = gv.y, lb = gv.z;
                if (L >= 3) {
                    const float3 e = expand_smem(g2, UG2_X, cc - 1, r - 1);
                    lr -= e.x;
                    lg -= e.y;
                    lb -= e.z;
                }
                n1[k].x = fmaf(gv.w, lr, n1[k].x);
                n1[k].y = fmaf(gv.w, lg, n1[k].y);
                n1[k].z = fmaf(gv.w, lb, n1[k].z);
                n1[k].w += gv.w;
            }
        }
        const float scale = c.gain * (1.0f / 255.0f);
#pragma unroll
        for (int k = 0; k < UG_PPT; ++k) {
            const int p = t + k * U_THREADS;
            const int dx = p & (U_TX - 1), dy = p / U_TX;
            const int x = X0 + dx, y = Y0 + dy;
            if (x >= X1 || y >= Y1 || !(ws[k] > 0.f) || !c.V.contains(x, y)) continue;
            const SrcPos sp = g.cyl ? map_point64(c, g, x, y) : map_point(cr.tm, (float)(x - cr.ax), (float)(y - cr.ay));
            const float w = g.seam ? (own[k] == a ? 1.f : 0.f) : feather_weight(sp, c.W, c.H);
            if (!(w > 0.f)) continue;
            const float what = w / ws[k];
            float3 v = bilinear_rgb(fp.p[i], fp.pitch[i], clamp_tap(sp, c.W, c.H), scale);
            if (L >= 2) {
                const float3 e = expand_smem(g1, UG1_X, dx, dy);
                v.x -= e.x;
                v.y -= e.y;
                v.z -= e.z;
            }
            n0[k].x = fmaf(what, v.x, n0[k].x);
            n0[k].y = fmaf(what, v.y, n0[k].y);
            n0[k].z = fmaf(what, v.z, n0[k].z);
            n0[k].w += what;
        }
        __syncthreads();
    }
    if (L >= 2) {
#pragma unroll
        for (int k = 0; k < UG1_PT; ++k) {
            const int q = t + k * U_THREADS;
            if (q >= UG1_N) break;
            const int r = q / UG1_X, cc = q - r * UG1_X;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const float s = n1[k].w;
            if (s > 1e-12f) {
                v.x = n1[k].x / s;
                v.y = n1[k].y / s;
                v.z = n1[k].z / s;
            }
            if (L >= 3) {
                const float3 e = expand_smem(r2, UG2_X, cc - 1, r - 1);
                v.x += e.x;
                v.y += e.y;
                v.z += e.z;
            }
            r1[q] = v;
        }
        __syncthreads();
        if (a1x + UG1_X > g.nx[1] || a1y + UG1_Y > g.ny[1]) {
            // past the right or bottom border, R^1 is that of the folded positions (see up_full_tile)
            for (int q = t; q < UG1_N; q += U_THREADS) {
                const int r = q / UG1_X, cc = q - r * UG1_X;
                if (a1x + cc < g.nx[1] && a1y + r < g.ny[1]) continue;
                const int sx = fold101(a1x + cc, g.nx[1]) - a1x, sy = fold101(a1y + r, g.ny[1]) - a1y;
                if (sx >= 0 && sx < UG1_X && sy >= 0 && sy < UG1_Y) r1[q] = r1[sy * UG1_X + sx];
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int k = 0; k < UG_PPT; ++k) {
        const int p = t + k * U_THREADS;
        const int dx = p & (U_TX - 1), dy = p / U_TX;
        const int x = X0 + dx, y = Y0 + dy;
        if (x >= X1 || y >= Y1) continue;
        float3 v = make_float3(0.f, 0.f, 0.f);
        const float s = n0[k].w;
        if (s > 1e-12f) {
            v.x = n0[k].x / s;
            v.y = n0[k].y / s;
            v.z = n0[k].z / s;
        }
        if (L >= 2) {
            const float3 e = expand_smem(r1, UG1_X, dx, dy);
            v.x += e.x;
            v.y += e.y;
            v.z += e.z;
        }
        const bool cov = ws[k] > 0.f;
        const float rr = cov ? __saturatef(v.x) : 0.f, gg = cov ? __saturatef(v.y) : 0.f,
                    bb = cov ? __saturatef(v.z) : 0.f;
        if (od.is_float) {
            float* o = (float*)((char*)od.ptr + (long long)y * od.pitch) + 3 * x;
            o[0] = rr;
            o[1] = gg;
            o[2] = bb;
        } else {
            unsigned char* o = (unsigned char*)od.ptr + (long long)y * od.pitch + 3 * x;
            o[0] = quantize_u8(rr);
            o[1] = quantize_u8(gg);
            o[2] = quantize_u8(bb);
        }
    }
}

constexpr int UG_SMEM_F4 = 2 * UG1_N + 2 * UG2_X * UG2_Y;

template <typename T>
__global__ void __launch_bounds__(U_THREADS) k_up_general(const CamDev* __restrict__ cams, RigGeom g, FramePtrs fp,
                                                           OutDesc od, const T* __restrict__ R2,
                                                           const UpTile* __restrict__ tiles,
                                                           const CamRef* __restrict__ refs) {
    __shared__ float4 smem[UG_SMEM_F4];
    up_general_tile<T>(cams, g, fp, od, R2, tiles[blockIdx.x], refs, smem);
}

// ------------------------------------------------------------------------------------------------
// host side

enum UpKind { UP_SIMPLE = 0, UP_FULL2 = 1, UP_FULL4 = 2, UP_GENERAL = 3, UP_KINDS = 4 };

struct FusedState {
    D1Tile* d1_tiles = nullptr;
    int n_d1 = 0;
    Tile* red_tiles[MAXL] = {};  // tiles producing level l (l >= 2), RSRig shape (the batched schedules)
    int n_red[MAXL] = {};
    Tile* rc_tiles[MAXL] = {};   // the same levels in the column-sweep kernel's 64 x 8 tiles (stitch_frames)
    int n_rc[MAXL] = {};
    LevelTile* co_tiles[MAXL] = {};  // coarse tiles of level l (l >= 2)
    int n_co[MAXL] = {};
    int* camlist = nullptr;
    float* d1w = nullptr;        // normalised level-0 weights of the non-INTERIOR down1 tiles
    int n_wtab = 0;
    D1Cams* d1_cams = nullptr;   // weight normalisation cameras of every down1 tile
    float4* d1cols = nullptr;    // cylindrical canvas: column terms of every down1 tile
    void* g0buf = nullptr;       // level-0 samples of the FULL canvas tiles, one slot per camera
    int n_g0 = 0;
    int n_staged = 0;            // down1 tiles with a staged source footprint
    bool d1_small = false;       // down1 with the smaller footprint capacity (13 blocks per SM)
    bool up_four = false;        // up_full with four resident blocks per SM
    int wave_red = 0, wave_up2 = 0, wave_up4 = 0;  // resident blocks on the device (L2 prefetch distance)
    void* R[MAXL] = {};          // R^l on the canvas grid, l >= 2
    CamRef* refs = nullptr;
    UpTile* up_tiles[UP_KINDS] = {};
    int n_up[UP_KINDS] = {};
    int n_zero = 0, n_solo = 0;  // classification counts (UP_SIMPLE = zero + solo)
    bool fp16 = false;
    // host copies of the tile tables (the batched schedule embeds them in its tasks)
    std::vector<D1Tile> h_d1;
    std::vector<Tile> h_red[MAXL];
    std::vector<LevelTile> h_co[MAXL];
    std::vector<UpTile> h_up[UP_KINDS];
};

template <typename V>
stitch_status upload(stitch_rig* r, const std::vector<V>& v, V** out) {
    *out = nullptr;
    if (v.empty()) return STITCH_OK;
    *out = (V*)rig_alloc(r, sizeof(V) * v.size());
    if (!*out) return STITCH_ENOMEM;
    STITCH_CUDA_TRY(cudaMemcpy(*out, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
    return STITCH_OK;
}

// Canvas positions [lo, hi) that the virtual positions v0 .. v0 + n - 1 fold to on a grid of size m.
Span folded_span(int v0, int n, int m) {
    Span s{m, -1};
    for (int v = v0; v < v0 + n; ++v) {
        const int f = fold101(v, m);
        s.lo = std::min(s.lo, f);
        s.hi = std::max(s.hi, f + 1);
    }
    return s;
}

bool rects_meet(const Rect& a, int x0, int x1, int y0, int y1) {
    return !a.empty() && a.x0 < x1 && a.x1 > x0 && a.y0 < y1 && a.y1 > y0;
}

// A camera's reference for a tile.  Planar canvas: the homography anchored at the tile.
// Cylindrical canvas: U0, V0 at the anchor and the per-row slopes of the anchored numerators and
// denominator (they are affine in the canvas row on every column); the column terms come from the
// tile's column table (cyl_columns), or from the FP64 map on the paths that are not hot.
CamRef make_ref(const CamDev& c, const RigGeom& g, int cam, int X, int Y) {
    CamRef r;
    int ax, ay;
    tile_anchor(c.V, X, Y, &ax, &ay);
    if (g.cyl) {
        double u, v;
        source_point64(c, g, (double)ax, (double)ay, &u, &v);
        u = std::fmin(std::fmax(u, -1.0e8), 1.0e8);
        v = std::fmin(std::fmax(v, -1.0e8), 1.0e8);
        const double U = std::rint(u), V = std::rint(v);
        TileMap t{};
        t.U0 = (int)U;
        t.V0 = (int)V;
        t.pu2 = (float)((c.A[1] - U * c.A[7]) / g.cf);
        t.pv2 = (float)((c.A[4] - V * c.A[7]) / g.cf);
        t.q2 = (float)(c.A[7] / g.cf);
        r.tm = t;
    } else {
        r.tm = make_tile_map(c.A, ax, ay);
    }
    r.cam = cam;
    r.ax = ax;
    r.ay = ay;
    r.g0 = -1;
    return r;
}

// Column terms of a down1 tile on the cylindrical canvas: for virtual column k (canvas column
// x = fold(vx0 + k)) the anchored numerators and denominator at the anchor row, in FP64, so that
// a sample at row dy = y - ay is (col.x + pu2 dy, col.y + pv2 dy) / (col.z + q2 dy).
void cyl_columns(const CamDev& c, const RigGeom& g, const CamRef& r, int vx0, float4* out) {
    const double py = ((double)r.ay - g.ccy) / g.cf;
    for (int k = 0; k < D1_SX; ++k) {
        const double x = (double)fold101(vx0 + k, g.nx[0]);
        const double t = (x - g.ccx) / g.cf, sx = std::sin(t), cx = std::cos(t);
        const double nu = c.A[0] * sx + c.A[1] * py + c.A[2] * cx;
        const double nv = c.A[3] * sx + c.A[4] * py + c.A[5] * cx;
        const double w = c.A[6] * sx + c.A[7] * py + c.A[8] * cx;
        out[k] = make_float4((float)(nu - r.tm.U0 * w), (float)(nv - r.tm.V0 * w), (float)w, 0.f);
    }
}

// Level-0 rectangle on which the outputs of tile [x0,x1) x [y0,y1) depend (pyramid cone).
Rect cone_level0(const RigGeom& g, int x0, int x1, int y0, int y1) {
    const int L = g.levels;
    Span xs[MAXL], ys[MAXL];
    xs[0] = {x0, x1};
    ys[0] = {y0, y1};
    for (int l = 0; l + 1 < L; ++l) {
        xs[l + 1] = expand_reads(xs[l], g.nx[l + 1]);
        ys[l + 1] = expand_reads(ys[l], g.ny[l + 1]);
    }
    Span yx = xs[L - 1], yy = ys[L - 1];
    for (int l = L - 2; l >= 0; --l) {
        yx = span_union(xs[l], reduce_reads(yx, g.nx[l]));
        yy = span_union(ys[l], reduce_reads(yy, g.ny[l]));
    }
    return make_rect(yx, yy);
}

// Range of source coordinates of camera c over the pixels of rect q; false when some pixel is not
// in front of the camera or maps beyond |u|, |v| < 1e6.  Planar canvas: the image of a rectangle
// under a homography in front of the camera is convex, so its corners decide.  Cylindrical
// canvas: on every column u, v are Moebius functions of the row (monotonic where w > 0) and w is
// affine in it, so the top and bottom rows of every column decide.
bool source_range(const CamDev& c, const RigGeom& g, const Rect& q, double* umin, double* umax, double* vmin,
                  double* vmax) {
    *umin = *vmin = 1e300;
    *umax = *vmax = -1e300;
    const double ys[2] = {(double)q.y0, (double)(q.y1 - 1)};
    const int step = g.cyl ? 1 : std::max(1, q.x1 - 1 - q.x0);
    for (int xi = q.x0; xi < q.x1; xi += step)
        for (int pass = 0; pass < 2; ++pass) {
            const double x = pass == 0 ? (double)xi : (double)(q.x1 - 1);
            for (double y : ys) {
                double u, v;
                if (!(source_point64(c, g, x, y, &u, &v) > 0.0)) return false;
                if (!(std::fabs(u) < 1e6 && std::fabs(v) < 1e6)) return false;
                *umin = std::min(*umin, u);
                *umax = std::max(*umax, u);
                *vmin = std::min(*vmin, v);
                *vmax = std::max(*vmax, v);
            }
        }
    return true;
}

// Camera c maps every pixel of rect q into [m, W-1-m] x [m, H-1-m] of its image.  With m = 0 the
// feather weight is >= 0.5 everywhere; with m > 0 no sample needs coordinate clamping.
bool solidly_inside(const CamDev& c, const RigGeom& g, const Rect& q, double m = 0.0) {
    double umin, umax, vmin, vmax;
    if (!source_range(c, g, q, &umin, &umax, &vmin, &vmax)) return false;
    return umin >= m && umax <= c.W - 1.0 - m && vmin >= m && vmax <= c.H - 1.0 - m;
}

// Source-pixel footprint of camera c over the level-0 rectangle q: every tap of a bilinear sample
// of a point of q (after the image clamp of S1) lies in [fx0, fx0 + fw) x [fy0, fy0 + fh).  The
// kernels' FP32 positions err by ~1e-5 px; the footprint allows 1e-3 px.  fx0 is a multiple of 4
// and the footprint is at least 2 x 2 texels (grown inside the image where the rectangle maps
// beyond an image border).  False when q is not entirely in front of the camera, maps beyond
// |u|, |v| < 1e6, or the footprint (rows padded to 4 texels) exceeds the shared-memory capacity.
bool d1_footprint(const CamDev& c, const RigGeom& g, const Rect& q, int& fx0, int& fy0, int& fw, int& fh) {
    if (c.W < 2 || c.H < 2) return false;
    double umin, umax, vmin, vmax;
    if (!source_range(c, g, q, &umin, &umax, &vmin, &vmax)) return false;
    constexpr double eps = 1e-3;
    int x0 = std::min(std::max((int)std::floor(umin - eps), 0), c.W - 1);
    int x1 = std::min(std::max((int)std::floor(umax + eps) + 2, 1), c.W);
    int y0 = std::min(std::max((int)std::floor(vmin - eps), 0), c.H - 1);
    int y1 = std::min(std::max((int)std::floor(vmax + eps) + 2, 1), c.H);
    if (x1 - x0 < 2) {
        x0 = std::min(x0, c.W - 2);
        x1 = x0 + 2;
    }
    if (y1 - y0 < 2) {
        y0 = std::min(y0, c.H - 2);
        y1 = y0 + 2;
    }
    x0 &= ~3;
    if (x1 - x0 < 2 || y1 - y0 < 2 || (long long)((x1 - x0 + 3) & ~3) * (y1 - y0) > D1_FOOT || y0 > 0xffff ||
        x0 > 0xffff)
        return false;
    fx0 = x0;
    fy0 = y0;
    fw = x1 - x0;
    fh = y1 - y0;
    return true;
}

// Reduce tiles producing level l >= 2 of every visible camera: tx x ty outputs on its Omega^l.
void plan_reduce_tiles(const stitch_rig* r, int tx, int ty, std::vector<Tile> red[MAXL]) {
    const RigGeom& g = r->geom;
    for (int i = 0; i < g.ncam; ++i) {
        const CamDev& c = r->hcam[i];
        if (!c.visible) continue;
        for (int l = 2; l < g.levels; ++l) {
            const Rect o = c.Om[l];
            for (int y = o.y0; y < o.y1; y += ty)
                for (int x = o.x0; x < o.x1; x += tx) red[l].push_back({i, x, y, 0});
        }
    }
}

// Coarse tiles of tx x ty on levels l >= 2 and their cameras (those whose Z^l meets the tile).
// R^l is read only by the FULL and GENERAL canvas tiles (R^2, in a halo around the tile) and by the
// coarse tiles of level l - 1 (R^l, in a halo), so a coarse tile is emitted only where one of those
// readers needs it (the halos taken with a margin of 2).
void plan_coarse_tiles(const stitch_rig* r, const std::vector<UpTile>* up, int tx, int ty, std::vector<LevelTile> co[MAXL],
                       std::vector<int>& camlist) {
    const RigGeom& g = r->geom;
    const int L = g.levels;
    std::vector<char> need[MAXL];
    auto mark = [&](int l, int x0, int x1, int y0, int y1) {
        x0 = std::max(x0, 0);
        y0 = std::max(y0, 0);
        x1 = std::min(x1, g.nx[l]);
        y1 = std::min(y1, g.ny[l]);
        const int ntx = (g.nx[l] + tx - 1) / tx;
        for (int yy = y0 / ty; yy * ty < y1; ++yy)
            for (int xx = x0 / tx; xx * tx < x1; ++xx) need[l][(size_t)yy * ntx + xx] = 1;
    };
    for (int l = 2; l < L; ++l) need[l].assign((size_t)((g.nx[l] + tx - 1) / tx) * ((g.ny[l] + ty - 1) / ty), 0);
    if (L >= 3) {
        for (int kind : {UP_FULL2, UP_FULL4, UP_GENERAL})
            for (const UpTile& t : up[kind])
                mark(2, t.x0 / 4 - 4, t.x0 / 4 + U_TX / 4 + 4, t.y0 / 4 - 4, t.y0 / 4 + U_TY / 4 + 4);
        for (int l = 2; l + 1 < L; ++l) {
            const int ntx = (g.nx[l] + tx - 1) / tx;
            for (size_t k = 0; k < need[l].size(); ++k)
                if (need[l][k]) {
                    const int x = (int)(k % ntx) * tx, y = (int)(k / ntx) * ty;
                    mark(l + 1, x / 2 - 4, x / 2 + tx / 2 + 4, y / 2 - 4, y / 2 + ty / 2 + 4);
                }
        }
    }
    for (int l = 2; l < L; ++l) {
        const int ntx = (g.nx[l] + tx - 1) / tx;
        for (int y = 0; y < g.ny[l]; y += ty)
            for (int x = 0; x < g.nx[l]; x += tx) {
                if (!need[l][(size_t)(y / ty) * ntx + x / tx]) continue;
                LevelTile t{x, y, (int)camlist.size(), 0};
                for (int j = 0; j < g.ncam; ++j) {
                    const CamDev& cj = r->hcam[j];
                    if (!cj.visible || !rects_meet(cj.Z[l], x, std::min(x + tx, g.nx[l]), y, std::min(y + ty, g.ny[l])))
                        continue;
                    camlist.push_back(j);
                    ++t.count;
                }
                co[l].push_back(t);
            }
    }
}

template <typename T>
stitch_status launch_all(stitch_rig* r, FusedState* fs, const FramePtrs& fp, const OutDesc& od, cudaStream_t s) {
    const RigGeom& g = r->geom;
    const int L = g.levels;
    if (L >= 2 && fs->n_d1 > 0) {
        prof_mark(r, "fused_down1", s);
        if (fs->d1_small)
            k_down1<T, D1_FOOT_SMALL><<<fs->n_d1, D1_THREADS, D1Cap<D1_FOOT_SMALL>::SMEM, s>>>(
                r->dcam, g, fp, od, fs->d1_tiles, fs->refs, fs->d1w, fs->d1cols, (Slot*)fs->g0buf);
        else
            k_down1<T, D1_FOOT><<<fs->n_d1, D1_THREADS, D1_SMEM, s>>>(r->dcam, g, fp, od, fs->d1_tiles, fs->refs, fs->d1w,
                                                                     fs->d1cols, (Slot*)fs->g0buf);
    }
    for (int l = 1; l + 1 < L; ++l) {
        if (fs->n_rc[l + 1] == 0) continue;
        prof_mark(r, "fused_reduce", s);
        k_reduce_t<T><<<fs->n_rc[l + 1], RC_THREADS, RC_SMEM, s>>>(r->dcam, g, l, fs->rc_tiles[l + 1], fs->n_rc[l + 1],
                                                                   fs->wave_red);
    }
    for (int l = L - 1; l >= 2; --l) {
        if (fs->n_co[l] == 0) continue;
        prof_mark(r, "fused_coarse", s);
        k_coarse_t<T><<<fs->n_co[l], 256, sizeof(float4) * CT_SMEM_F4, s>>>(r->dcam, g, l, (T*)fs->R[l],
                                                   l + 1 < L ? (const T*)fs->R[l + 1] : nullptr, fs->co_tiles[l],
                                                   fs->camlist);
    }
    const T* R2 = L >= 3 ? (const T*)fs->R[2] : nullptr;
    // the ZERO canvas tiles ride along with the first up_full launch (or get their own)
    const int ns = fs->n_up[UP_SIMPLE];
    if (ns && !fs->n_up[UP_FULL2] && !fs->n_up[UP_FULL4]) {
        prof_mark(r, "fused_up_simple", s);
        k_up_simple<<<ns, U_THREADS, 0, s>>>(r->dcam, g, fp, od, fs->up_tiles[UP_SIMPLE], fs->refs);
    }
    if (fs->n_up[UP_FULL2]) {
        prof_mark(r, "fused_up_full", s);
        auto k = fs->up_four ? k_up_full_b4<T, 2> : k_up_full<T, 2>;
        k<<<fs->n_up[UP_FULL2] + ns, U_THREADS, up_full_smem<2>(), s>>>(
            r->dcam, g, fp, od, R2, fs->up_tiles[UP_FULL2], fs->refs, (const Slot*)fs->g0buf, fs->n_up[UP_FULL2],
            fs->wave_up2, fs->up_tiles[UP_SIMPLE]);
    }
    if (fs->n_up[UP_FULL4]) {
        const int extra = fs->n_up[UP_FULL2] ? 0 : ns;
        prof_mark(r, "fused_up_full4", s);
        auto k = fs->up_four ? k_up_full_b4<T, 4> : k_up_full<T, 4>;
        k<<<fs->n_up[UP_FULL4] + extra, U_THREADS, up_full_smem<4>(), s>>>(
            r->dcam, g, fp, od, R2, fs->up_tiles[UP_FULL4], fs->refs, (const Slot*)fs->g0buf, fs->n_up[UP_FULL4],
            fs->wave_up4, fs->up_tiles[UP_SIMPLE]);
    }
    if (fs->n_up[UP_GENERAL]) {
        prof_mark(r, "fused_up_general", s);
        k_up_general<T><<<fs->n_up[UP_GENERAL], U_THREADS, 0, s>>>(r->dcam, g, fp, od, R2,
                                                                    fs->up_tiles[UP_GENERAL], fs->refs);
    }
    return launch_status();
}

template <typename T>
stitch_status set_smem_attrs() {
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_down1<T, D1_FOOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D1_SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_down1<T, D1_FOOT_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)D1Cap<D1_FOOT_SMALL>::SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_reduce_t<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC_SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_up_full<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<2>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_up_full<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<4>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_up_full_b4<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<2>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_up_full_b4<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<4>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_coarse_t<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float4) * CT_SMEM_F4)));
    return STITCH_OK;
}

// Resident blocks of the reduce and up_full kernels on the rig's device: the distance of their L2
// prefetch chains.
template <typename T>
stitch_status set_waves(stitch_rig* r, FusedState* fs) {
    int sms = 0, pr = 0, p2 = 0, p4 = 0;
    STITCH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device));
    STITCH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pr, k_reduce_t<T>, RC_THREADS, RC_SMEM));
    // four resident up_full blocks per SM when the blended canvas tiles make many waves of them
    fs->up_four = fs->n_up[UP_FULL2] + fs->n_up[UP_FULL4] >= 8 * 4 * std::max(sms, 1);
    if (fs->up_four) {
        STITCH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_up_full_b4<T, 2>, U_THREADS, up_full_smem<2>()));
        STITCH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_up_full_b4<T, 4>, U_THREADS, up_full_smem<4>()));
    } else {
        STITCH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_up_full<T, 2>, U_THREADS, up_full_smem<2>()));
        STITCH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_up_full<T, 4>, U_THREADS, up_full_smem<4>()));
    }
    fs->wave_red = std::max(pr, 1) * sms;
    fs->wave_up2 = std::max(p2, 1) * sms;
    fs->wave_up4 = std::max(p4, 1) * sms;
    return STITCH_OK;
}

}  // namespace

stitch_status fused_plan(stitch_rig* r) {
    const RigGeom& g = r->geom;
    const int L = g.levels;
    FusedState* fs = new (std::nothrow) FusedState();
    if (!fs) return STITCH_ENOMEM;
    r->fused = fs;
    fs->fp16 = r->desc.band_fp16 != 0;
    const size_t elem = fs->fp16 ? sizeof(half4) : sizeof(float4);
    std::vector<CamRef> refs;
    std::vector<D1Tile> d1;
    std::vector<D1Cams> d1c;
    std::vector<float4> cols;  // cylindrical canvas: D1_SX column terms per down1 tile
    std::vector<Tile> red[MAXL];
    for (int i = 0; i < g.ncam; ++i) {
        CamDev& c = r->hcam[i];
        if (!c.visible) continue;
        for (int l = 1; l < L; ++l) {
            c.FG[l] = rig_alloc(r, elem * (size_t)c.Om[l].area());
            if (!c.FG[l]) return STITCH_ENOMEM;
        }
        if (L >= 2) {
            // tiles on the global grid of 32 x 8 level-1 samples, so that two vertically adjacent
            // tiles' level-0 interiors are exactly one 64 x 32 canvas tile of `up`; both tiles of
            // every such pair that meets Omega^1 exist
            const Rect o = c.Om[1];
            const int band = 2 * D1_TY;
            for (int y = (o.y0 / band) * band; y < o.y1 || y % band != 0; y += D1_TY)
                for (int x = (o.x0 / D1_TX) * D1_TX; x < o.x1; x += D1_TX) {
                    // level-0 bounding box of the tile's inputs: the canvas positions its virtual
                    // samples fold to (past the right or bottom border they fold back by as much
                    // as they reach beyond it)
                    const Span fx = folded_span(2 * x - 2, D1_SX, g.nx[0]), fy = folded_span(2 * y - 2, D1_SY, g.ny[0]);
                    const int bx0 = fx.lo, bx1 = fx.hi, by0 = fy.lo, by1 = fy.hi;
                    D1Tile t{i, x, y, -1, -1, 0, 0, 0, -1, -1, 0, 0, 0, -1};
                    D1Cams tc{(int)refs.size(), 0, -1, 0};
                    for (int j = 0; j < g.ncam; ++j) {
                        const CamDev& cj = r->hcam[j];
                        if (!cj.visible || (j != i && !rects_meet(cj.V, bx0, bx1, by0, by1))) continue;
                        if (j == i) tc.self = tc.count;
                        refs.push_back(make_ref(cj, g, j, bx0, by0));
                        ++tc.count;
                    }
                    t.ref = tc.first + tc.self;
                    if (g.cyl) {
                        t.coltab = (int)d1.size();
                        cols.resize(cols.size() + D1_SX);
                        cyl_columns(c, g, refs[t.ref], 2 * x - 2, cols.data() + (size_t)t.coltab * D1_SX);
                    }
                    // no clamping: every input at least 0.01 px inside the image (FP32 positions err
                    // by ~1e-5 px); interior: in addition no other camera, so the weight is 1
                    if (solidly_inside(c, g, Rect{bx0, bx1, by0, by1}, 0.01)) {
                        t.flags |= D1_NOCLAMP;
                        if (tc.count == 1) t.flags |= D1_INTERIOR;
                    }
                    t.wtab = (t.flags & D1_INTERIOR) ? -1 : fs->n_wtab++;
                    t.wsel = t.wtab;
                    int fx0, fy0, fw, fh;
                    if (d1_footprint(c, g, Rect{bx0, bx1, by0, by1}, fx0, fy0, fw, fh)) {
                        t.fxy = fx0 | (fy0 << 16);
                        t.fwh = fw | (fh << 16);
                        ++fs->n_staged;
                    }
                    d1.push_back(t);
                    d1c.push_back(tc);
                }
        }
    }
    plan_reduce_tiles(r, RT_X, RT_Y, red);
    std::vector<Tile> redc[MAXL];
    plan_reduce_tiles(r, RSCol::TX, RSCol::TY, redc);
    // classify the canvas tiles of `up`
    std::vector<UpTile> up[UP_KINDS];
    std::unordered_map<long long, size_t> d1_index;  // (camera, level-1 origin) -> down1 tile
    for (size_t k = 0; k < d1.size(); ++k)
        d1_index[((long long)d1[k].cam << 42) | ((long long)d1[k].k0 << 21) | d1[k].j0] = k;
    for (int Y0 = 0; Y0 < g.ny[0]; Y0 += U_TY)
        for (int X0 = 0; X0 < g.nx[0]; X0 += U_TX) {
            const int X1 = std::min(X0 + U_TX, g.nx[0]), Y1 = std::min(Y0 + U_TY, g.ny[0]);
            UpTile t{X0, Y0, (int)refs.size(), 0};
            // level-1 region read by the tile (actual coordinates; folding stays inside it)
            int bx0 = 0, bx1 = 0, by0 = 0, by1 = 0;
            if (L >= 2) {
                bx0 = std::max(X0 / 2 - 2, 0);
                bx1 = std::min(X0 / 2 - 2 + U1_X, g.nx[1]);
                by0 = std::max(Y0 / 2 - 2, 0);
                by1 = std::min(Y0 / 2 - 2 + U1_Y, g.ny[1]);
            }
            int nv = 0, last_v = -1;
            for (int j = 0; j < g.ncam; ++j) {
                const CamDev& cj = r->hcam[j];
                if (!cj.visible) continue;
                const bool at0 = rects_meet(cj.V, X0, X1, Y0, Y1);
                const bool at1 = L >= 2 && rects_meet(cj.Z[1], bx0, bx1, by0, by1);
                if (at0) {
                    ++nv;
                    last_v = j;
                }
                if (!(at0 || at1)) continue;
                refs.push_back(make_ref(cj, g, j, X0, Y0));
                ++t.count;
            }
            int kind;
            if (t.count == 0) {
                kind = UP_SIMPLE;
                ++fs->n_zero;
            } else {
                bool solo = false;
                if (nv == 1) {
                    const Rect cone = cone_level0(g, X0, X1, Y0, Y1);
                    solo = solidly_inside(r->hcam[last_v], g, cone);
                    for (int j = 0; j < g.ncam && solo; ++j)
                        if (j != last_v && r->hcam[j].visible && rects_meet(r->hcam[j].V, cone.x0, cone.x1, cone.y0, cone.y1))
                            solo = false;
                }
                if (solo) {
                    // one reference: the exclusive camera
                    refs.resize(t.first);
                    refs.push_back(make_ref(r->hcam[last_v], g, last_v, X0, Y0));
                    t.count = 1;
                    kind = UP_SIMPLE;
                    ++fs->n_solo;
                    // with a level-1 pass, the camera's down1 tile over this canvas tile writes the
                    // output (its level-0 samples are the output here)
                    if (L >= 2) {
                        auto it = d1_index.find(((long long)last_v << 42) | ((long long)(X0 / 2) << 21) | (Y0 / 2));
                        auto it2 = d1_index.find(((long long)last_v << 42) | ((long long)(X0 / 2) << 21) | (Y0 / 2 + D1_TY));
                        if (it != d1_index.end() && it2 != d1_index.end()) {
                            d1[it->second].flags |= D1_SOLO_OUT;
                            d1[it2->second].flags |= D1_SOLO_OUT;
                            kind = -1;
                        }
                    }
                } else if (t.count <= 4 && L >= 2) {
                    // FULL: every camera blended at level 0 takes its level-0 samples (value and
                    // normalised weight) from its down1 tile over this canvas tile
                    kind = t.count <= 2 ? UP_FULL2 : UP_FULL4;
                    size_t d1k[4][2];
                    for (int k = 0; k < t.count && kind != UP_GENERAL; ++k) {
                        const CamRef& rk = refs[t.first + k];
                        d1k[k][0] = d1k[k][1] = SIZE_MAX;
                        if (!rects_meet(r->hcam[rk.cam].V, X0, X1, Y0, Y1)) continue;
                        for (int h = 0; h < 2; ++h) {
                            auto it = d1_index.find(((long long)rk.cam << 42) | ((long long)(X0 / 2) << 21) | (Y0 / 2 + h * D1_TY));
                            if (it == d1_index.end()) kind = UP_GENERAL;
                            else d1k[k][h] = it->second;
                        }
                    }
                    if (kind != UP_GENERAL)
                        for (int k = 0; k < t.count; ++k) {
                            if (d1k[k][0] == SIZE_MAX) continue;
                            const int slot = fs->n_g0++;
                            for (int h = 0; h < 2; ++h) {
                                D1Tile& dt = d1[d1k[k][h]];
                                dt.g0 = slot;
                                dt.flags |= D1_G0_OUT;
                            }
                            refs[t.first + k].g0 = slot;
                        }
                } else {
                    kind = UP_GENERAL;
                }
            }
            if (kind >= 0) up[kind].push_back(t);
        }
    std::vector<LevelTile> co[MAXL];
    std::vector<int> camlist;
    for (int l = 2; l < L; ++l) {
        fs->R[l] = rig_alloc(r, elem * (size_t)g.nx[l] * g.ny[l]);
        if (!fs->R[l]) return STITCH_ENOMEM;
    }
    plan_coarse_tiles(r, up, CT_X, CT_Y, co, camlist);
    // Only part of every camera's Gaussian levels >= 1 is ever read: by the coarse tiles (G^l on the
    // tile, G^{l+1} on its halo), the FULL and GENERAL canvas tiles (G^1 and G^2 on their halos) and,
    // through REDUCE, by the needed part of the next level (its 5 x 5 support).  The needed pixels
    // are marked top-down; REDUCE tiles with no needed output are dropped, down1 tiles store G^1
    // only where it is needed, and a down1 tile with neither a needed G^1 nor a level-0 output is
    // dropped.  The rest of the level buffers is never written and never read.
    if (L >= 2) {
        std::vector<std::vector<uint8_t>> need[MAXL];  // [level][camera]: a byte per pixel of Omega^l
        for (int l = 1; l < L; ++l) {
            need[l].resize(g.ncam);
            for (int i = 0; i < g.ncam; ++i)
                if (r->hcam[i].visible) need[l][i].assign((size_t)r->hcam[i].Om[l].area(), 0);
        }
        // mark [x0, x1) x [y0, y1) of level l of camera i: the range is taken on the level grid (a
        // range reaching past a border also covers the positions it folds to), then cut to Omega^l
        auto fold_range = [](int a0, int a1, int n, int& lo, int& hi) {
            lo = std::max(a0, 0);
            hi = std::min(a1, n);
            if (a0 < 0) hi = std::max(hi, std::min(-a0 + 1, n));
            if (a1 > n) lo = std::min(lo, std::max(2 * n - 1 - a1, 0));
        };
        auto mark = [&](int l, int i, int x0, int x1, int y0, int y1) {
            const CamDev& c = r->hcam[i];
            if (!c.visible) return;
            int ax, bx, ay, by;
            fold_range(x0, x1, g.nx[l], ax, bx);
            fold_range(y0, y1, g.ny[l], ay, by);
            const Rect o = c.Om[l];
            ax = std::max(ax, o.x0);
            bx = std::min(bx, o.x1);
            ay = std::max(ay, o.y0);
            by = std::min(by, o.y1);
            for (int y = ay; y < by; ++y)
                if (bx > ax) memset(need[l][i].data() + (size_t)(y - o.y0) * o.w() + (ax - o.x0), 1, bx - ax);
        };
        auto any = [&](int l, int i, int x0, int x1, int y0, int y1) {
            const Rect o = r->hcam[i].Om[l];
            x0 = std::max(x0, o.x0);
            x1 = std::min(x1, o.x1);
            y0 = std::max(y0, o.y0);
            y1 = std::min(y1, o.y1);
            for (int y = y0; y < y1; ++y)
                if (x1 > x0 && memchr(need[l][i].data() + (size_t)(y - o.y0) * o.w() + (x0 - o.x0), 1, x1 - x0)) return true;
            return false;
        };
        for (int kind : {UP_FULL2, UP_FULL4, UP_GENERAL})
            for (const UpTile& t : up[kind])
                for (int k = 0; k < t.count; ++k) {
                    const int i = refs[t.first + k].cam;
                    mark(1, i, t.x0 / 2 - 3, t.x0 / 2 + U_TX / 2 + 3, t.y0 / 2 - 3, t.y0 / 2 + U_TY / 2 + 3);
                    if (L >= 3) mark(2, i, t.x0 / 4 - 3, t.x0 / 4 + U_TX / 4 + 3, t.y0 / 4 - 3, t.y0 / 4 + U_TY / 4 + 3);
                }
        // R^l (l >= 2) is needed on the FULL and GENERAL canvas tiles' level-2 halos and, from
        // level to level, on the EXPAND support of the needed part of the finer level; a coarse
        // tile computes R^l at a pixel from G^l_i there and from G^{l+1}_i on the support, so G^l_i
        // is needed wherever R^l is
        std::vector<uint8_t> needR[MAXL];
        for (int l = 2; l < L; ++l) needR[l].assign((size_t)g.nx[l] * g.ny[l], 0);
        auto markR = [&](int l, int x0, int x1, int y0, int y1) {
            int ax, bx, ay, by;
            fold_range(x0, x1, g.nx[l], ax, bx);
            fold_range(y0, y1, g.ny[l], ay, by);
            for (int y = ay; y < by; ++y)
                if (bx > ax) memset(needR[l].data() + (size_t)y * g.nx[l] + ax, 1, bx - ax);
        };
        if (L >= 3) {
            for (int kind : {UP_FULL2, UP_FULL4, UP_GENERAL})
                for (const UpTile& t : up[kind])
                    markR(2, t.x0 / 4 - 3, t.x0 / 4 + U_TX / 4 + 3, t.y0 / 4 - 3, t.y0 / 4 + U_TY / 4 + 3);
            for (int l = 2; l + 1 < L; ++l)
                for (int y = 0; y < g.ny[l]; ++y) {
                    const uint8_t* row = needR[l].data() + (size_t)y * g.nx[l];
                    for (int x = 0; x < g.nx[l];) {
                        if (!row[x]) {
                            ++x;
                            continue;
                        }
                        int e = x;
                        while (e < g.nx[l] && row[e]) ++e;
                        markR(l + 1, x / 2 - 2, (e - 1) / 2 + 3, y / 2 - 2, y / 2 + 3);
                        x = e;
                    }
                }
            for (int l = 2; l < L; ++l)
                for (int i = 0; i < g.ncam; ++i) {
                    const CamDev& c = r->hcam[i];
                    if (!c.visible) continue;
                    const Rect o = c.Om[l];
                    for (int y = o.y0; y < o.y1; ++y) {
                        const uint8_t* src = needR[l].data() + (size_t)y * g.nx[l] + o.x0;
                        uint8_t* dst = need[l][i].data() + (size_t)(y - o.y0) * o.w();
                        for (int x = 0; x < o.w(); ++x) dst[x] |= src[x];
                    }
                }
        }
        // top-down: the 5 x 5 support of every needed pixel of level l is needed at level l - 1,
        // row by row over runs of needed pixels
        for (int l = L - 1; l >= 2; --l)
            for (int i = 0; i < g.ncam; ++i) {
                const CamDev& c = r->hcam[i];
                if (!c.visible) continue;
                const Rect o = c.Om[l];
                for (int y = o.y0; y < o.y1; ++y) {
                    const uint8_t* row = need[l][i].data() + (size_t)(y - o.y0) * o.w();
                    for (int x = 0; x < o.w();) {
                        if (!row[x]) {
                            ++x;
                            continue;
                        }
                        int e = x;
                        while (e < o.w() && row[e]) ++e;
                        mark(l - 1, i, 2 * (o.x0 + x) - 2, 2 * (o.x0 + e - 1) + 3, 2 * y - 2, 2 * y + 3);
                        x = e;
                    }
                }
            }
        for (int l = 2; l < L; ++l) {
            std::vector<Tile> keep, keepc;
            for (const Tile& t : red[l])
                if (any(l, t.cam, t.x0, t.x0 + RT_X, t.y0, t.y0 + RT_Y)) keep.push_back(t);
            for (const Tile& t : redc[l])
                if (any(l, t.cam, t.x0, t.x0 + RSCol::TX, t.y0, t.y0 + RSCol::TY)) keepc.push_back(t);
            red[l].swap(keep);
            redc[l].swap(keepc);
        }
        // down1: G^1 only where needed; drop tiles without any output (renumbering weight tables)
        std::vector<D1Tile> kd;
        std::vector<D1Cams> kc;
        fs->n_wtab = 0;
        for (size_t k = 0; k < d1.size(); ++k) {
            D1Tile t = d1[k];
            if (any(1, t.cam, t.k0, t.k0 + D1_TX, t.j0, t.j0 + D1_TY)) t.flags |= D1_G1_OUT;
            if (!(t.flags & (D1_G1_OUT | D1_SOLO_OUT | D1_G0_OUT))) continue;
            if (t.wtab >= 0) t.wtab = t.wsel = fs->n_wtab++;
            kd.push_back(t);
            kc.push_back(d1c[k]);
        }
        d1.swap(kd);
        d1c.swap(kc);
    }
    // footprint capacity: the smaller one when at most 2 % of the staged tiles need more
    {
        int staged = 0, over = 0;
        for (const D1Tile& t : d1)
            if (t.fwh != 0) {
                ++staged;
                over += ((((t.fwh & 0xffff) + 3) & ~3) * (t.fwh >> 16)) > D1_FOOT_SMALL;
            }
        fs->d1_small = (long long)over * 50 <= staged;
        if (fs->d1_small)
            for (D1Tile& t : d1)
                if (t.fwh != 0 && (((t.fwh & 0xffff) + 3) & ~3) * (t.fwh >> 16) > D1_FOOT_SMALL) t.fxy = t.fwh = 0;
    }
    // L2 prefetch chain: blocks start in index order as resident ones finish, so tile i + K
    // (K = resident blocks of k_down1 on the device) starts about when tile i ends
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device) != cudaSuccess || sms < 1)
            return STITCH_ECUDA;
        int bpsm = 0;
        const cudaError_t oe =
            fs->d1_small ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_down1<float4, D1_FOOT_SMALL>, D1_THREADS,
                                                                         D1Cap<D1_FOOT_SMALL>::SMEM)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_down1<float4, D1_FOOT>, D1_THREADS, D1_SMEM);
        if (oe != cudaSuccess) return STITCH_ECUDA;
        const size_t K = (size_t)std::max(bpsm, 1) * sms;
        for (size_t k = 0; k + K < d1.size(); ++k) {
            const D1Tile& nx = d1[k + K];
            if (nx.fwh == 0) continue;
            d1[k].pf_fxy = nx.fxy;
            d1[k].pf_fwh = nx.fwh;
            d1[k].pf_cw = nx.cam | ((nx.wtab + 1) << 8);
        }
    }
    // INTERIOR tiles sample with the table of ones, after the tiles' own tables
    fs->n_staged = 0;
    for (D1Tile& t : d1) {
        if (t.wsel < 0) t.wsel = fs->n_wtab;
        fs->n_staged += t.fwh != 0;
    }
    fs->h_d1 = d1;
    for (int l = 0; l < MAXL; ++l) {
        fs->h_red[l] = red[l];
        fs->h_co[l] = co[l];
    }
    for (int k = 0; k < UP_KINDS; ++k) fs->h_up[k] = up[k];
    stitch_status st = upload(r, refs, &fs->refs);
    if (st != STITCH_OK) return st;
    st = upload(r, d1, &fs->d1_tiles);
    if (st != STITCH_OK) return st;
    st = upload(r, d1c, &fs->d1_cams);
    if (st != STITCH_OK) return st;
    st = upload(r, cols, &fs->d1cols);
    if (st != STITCH_OK) return st;
    fs->n_d1 = (int)d1.size();
    if (fs->n_d1 > 0) {
        fs->d1w = (float*)rig_alloc(r, sizeof(float) * D1_NSAMP * (size_t)(fs->n_wtab + 1));
        if (!fs->d1w) return STITCH_ENOMEM;
    }
    if (fs->n_g0 > 0) {
        fs->g0buf = rig_alloc(r, sizeof(Slot) * (size_t)U_TX * U_TY * fs->n_g0);
        if (!fs->g0buf) return STITCH_ENOMEM;
    }
    for (int l = 2; l < L; ++l) {
        st = upload(r, red[l], &fs->red_tiles[l]);
        if (st != STITCH_OK) return st;
        fs->n_red[l] = (int)red[l].size();
        st = upload(r, redc[l], &fs->rc_tiles[l]);
        if (st != STITCH_OK) return st;
        fs->n_rc[l] = (int)redc[l].size();
    }
    st = upload(r, camlist, &fs->camlist);
    if (st != STITCH_OK) return st;
    for (int l = 2; l < L; ++l) {
        st = upload(r, co[l], &fs->co_tiles[l]);
        if (st != STITCH_OK) return st;
        fs->n_co[l] = (int)co[l].size();
    }
    for (int k = 0; k < UP_KINDS; ++k) {
        st = upload(r, up[k], &fs->up_tiles[k]);
        if (st != STITCH_OK) return st;
        fs->n_up[k] = (int)up[k].size();
    }
    int kernels = 0;
    if (L >= 2 && fs->n_d1 > 0) kernels += 1;
    for (int l = 2; l < L; ++l) kernels += (fs->n_rc[l] > 0) + (fs->n_co[l] > 0);
    for (int k = 0; k < UP_KINDS; ++k) kernels += fs->n_up[k] > 0;
    if (fs->n_up[UP_SIMPLE] && (fs->n_up[UP_FULL2] || fs->n_up[UP_FULL4])) kernels -= 1;  // rides along
    r->kernels_per_frame = kernels;
    st = fs->fp16 ? set_smem_attrs<half4>() : set_smem_attrs<float4>();
    if (st != STITCH_OK) return st;
    return fs->fp16 ? set_waves<half4>(r, fs) : set_waves<float4>(r, fs);
}

stitch_status fused_frames(stitch_rig* r, const FramePtrs& fp, const OutDesc& od, cudaStream_t s) {
    FusedState* fs = (FusedState*)r->fused;
    if (!fs) return STITCH_EINVAL;
    return fs->fp16 ? launch_all<half4>(r, fs, fp, od, s) : launch_all<float4>(r, fs, fp, od, s);
}

stitch_status fused_precompute(stitch_rig* r) {
    FusedState* fs = (FusedState*)r->fused;
    if (!fs || fs->n_d1 == 0) return STITCH_OK;
    if (fs->n_wtab > 0) {
        k_d1_weights<<<fs->n_d1, D1W_THREADS>>>(r->dcam, r->geom, fs->d1_tiles, fs->d1_cams, fs->refs, fs->d1w);
        STITCH_CUDA_TRY(cudaGetLastError());
    }
    const std::vector<float> ones(D1_NSAMP, 1.0f);
    STITCH_CUDA_TRY(cudaMemcpy(fs->d1w + (size_t)fs->n_wtab * D1_NSAMP, ones.data(), sizeof(float) * D1_NSAMP,
                               cudaMemcpyHostToDevice));
    STITCH_CUDA_TRY(cudaDeviceSynchronize());
    return STITCH_OK;
}

void fused_release(stitch_rig* r) {
    delete (FusedState*)r->fused;
    r->fused = nullptr;
}

void fused_tile_counts(const stitch_rig* r, int counts[8]) {
    const FusedState* fs = (const FusedState*)r->fused;
    for (int k = 0; k < 8; ++k) counts[k] = 0;
    if (!fs) return;
    counts[0] = fs->n_zero;
    counts[1] = fs->n_solo;
    counts[2] = fs->n_up[UP_FULL2];
    counts[3] = fs->n_up[UP_FULL4];
    counts[4] = fs->n_up[UP_GENERAL];
    counts[5] = fs->n_d1;
    counts[6] = fs->n_staged;
    counts[7] = fs->n_d1 - fs->n_wtab;
}

// ================================================================================================
// Batched persistent schedule: several rigs stitched by one launch.
//
// Every rig's per-frame work is a chain of stages (down1, the REDUCEs, the coarse levels, the
// canvas tiles); each stage's tiles become tasks of one device task list spanning all rigs, ordered
// so that every task's inputs come from tasks earlier in the list.  A persistent grid of resident
// blocks dequeues tasks in list order with an atomic counter; before a task of stage s of rig r it
// waits until all tasks of stage s-1 of rig r have completed (a counter per rig and stage).  Since
// those tasks were dequeued earlier by resident blocks that only wait on still earlier tasks, the
// waits always end; each wait nevertheless has an iteration limit, after which the block records a
// status, raises an abort flag that stops every block, and returns.
// ================================================================================================

namespace {

enum BatchType { BT_D1 = 0, BT_RED = 1, BT_CO = 2, BT_UPS = 3, BT_UPF2 = 4, BT_UPF4 = 5, BT_UPG = 6 };
constexpr int B_MAXSTAGE = 2 * MAXL + 2;
constexpr int B_THREADS = 256;

struct BatchRigDev {
    const CamDev* cams;
    RigGeom g;
    FramePtrs fp;
    OutDesc od;
    const D1Tile* d1;
    const Tile* red[MAXL];
    const LevelTile* co[MAXL];
    const int* camlist;    // camera lists of the coarse tiles (32 x 32) ...
    const int* camlist_w;  // ... and of the batch's 64 x 16 coarse tiles
    const CamRef* refs;
    const float* d1w;
    const float4* d1cols;
    void* g0buf;
    const UpTile* up[UP_KINDS];
    void* R[MAXL];
};

// A task carries a copy of its tile record, so a block needs one load to start.  A down1 task of
// the persistent schedule stands for pad0 (<= 4) consecutive tiles from idx on, read from the rig's
// tile table.
struct BTask {
    int rig, type, idx, level, stage, pad0, pad1, pad2;
    int tile[14];
};
template <typename TL>
__device__ __forceinline__ const TL& task_tile(const BTask& tk) {
    static_assert(sizeof(TL) <= sizeof(tk.tile), "tile record fits the task");
    return *reinterpret_cast<const TL*>(tk.tile);
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr int B_D1_GROUPS = B_THREADS / D1_THREADS;  // down1 tiles a persistent block works on at once
static_assert(B_D1_GROUPS == 4 && D1_SMEM % 16 == 0, "four 64-thread down1 groups per block");
constexpr size_t B_SMEM = cmax(cmax(cmax(B_D1_GROUPS * D1_SMEM, RT_SMEM), sizeof(float4) * CT_SMEM_F4),
                               cmax(up_full_smem<4>(), (size_t)3 * U_TX * U_TY));

constexpr int B_MAXRIGS = 64;
constexpr int B_MAXCHUNK = 16;

// Persistent executor.  ctl[0] next task, ctl[1] status (1: a wait gave up), ctl[2] abort,
// ctl[3] spin limit.  Blocks dequeue `chunk` consecutive tasks at a time; a block remembers the
// latest stage of each rig it has seen complete, so it polls a rig's counter once per stage rather
// than once per task, and it publishes its completed tasks once per chunk (always before it starts
// waiting, so a block never waits on its own unpublished work).
template <typename T, int MINB>
__global__ void __launch_bounds__(B_THREADS, MINB) k_batch(const BatchRigDev* __restrict__ rigs,
                                                            const BTask* __restrict__ tasks, int ntasks, int* ctl,
                                                            int* done, const int* __restrict__ need, int nrigs,
                                                            int chunk) {
    extern __shared__ float4 smem[];
    __shared__ int s_base, s_go;
    __shared__ int s_seen[B_MAXRIGS];
    __shared__ int p_ix[B_MAXCHUNK], p_cnt[B_MAXCHUNK];
    __shared__ int s_np;
    volatile int* vctl = ctl;
    volatile int* vdone = done;
    const int t = threadIdx.x;
    for (int r = t; r < nrigs; r += blockDim.x) s_seen[r] = -1;
    if (t == 0) s_np = 0;
    __syncthreads();
    // publish pending completions (thread 0 only)
    auto flush = [&]() {
        if (s_np > 0) {
            __threadfence();
            for (int k = 0; k < s_np; ++k) atomicAdd(&done[p_ix[k]], p_cnt[k]);
            s_np = 0;
        }
    };
    for (;;) {
        if (t == 0) {
            const int base = atomicAdd(&ctl[0], chunk);
            s_base = base;
            s_go = base < ntasks && !vctl[2];
        }
        __syncthreads();
        if (!s_go) break;
        const int base = s_base;
        bool stop = false;
        for (int k = 0; k < chunk && base + k < ntasks; ++k) {
            const BTask tk = tasks[base + k];
            if (t == 0) {
                int go = 1;
                if (tk.stage > 0 && s_seen[tk.rig] < tk.stage - 1) {
                    flush();
                    const int ix = tk.rig * B_MAXSTAGE + tk.stage - 1;
                    const int limit = vctl[3];
                    int it = 0;
                    while (vdone[ix] < need[ix]) {
                        if (vctl[2]) {
                            go = 0;
                            break;
                        }
                        if (++it > limit) {
                            atomicExch(&ctl[1], 1);
                            atomicExch(&ctl[2], 1);
                            go = 0;
                            break;
                        }
                        __nanosleep(200);
                    }
                    if (go) s_seen[tk.rig] = tk.stage - 1;
                    __threadfence();
                }
                s_go = go;
            }
            __syncthreads();
            if (!s_go) {
                stop = true;
                break;
            }
            const BatchRigDev& rg = rigs[tk.rig];
            const T* R2 = rg.g.levels >= 3 ? (const T*)rg.R[2] : nullptr;
            switch (tk.type) {
                case BT_D1: {
                    // up to four consecutive down1 tiles of the rig, one per group of 64 threads
                    const int grp = t / D1_THREADS;
                    if (grp < tk.pad0)
                        down1_tile<T>(rg.cams, rg.g, rg.fp, rg.od, rg.d1[tk.idx + grp], rg.refs, rg.d1w, rg.d1cols,
                                      (Slot*)rg.g0buf, reinterpret_cast<float4*>(reinterpret_cast<char*>(smem) + grp * D1_SMEM),
                                      t % D1_THREADS, 1 + grp);
                    break;
                }
                case BT_RED:
                    reduce_tile<T, RSRig>(rg.cams, rg.g, tk.level - 1, task_tile<Tile>(tk), smem);
                    break;
                case BT_CO:
                    coarse_tile<T, CSRig>(rg.cams, rg.g, tk.level, (T*)rg.R[tk.level],
                                   tk.level + 1 < rg.g.levels ? (const T*)rg.R[tk.level + 1] : nullptr,
                                   task_tile<LevelTile>(tk), rg.camlist, smem);
                    break;
                case BT_UPS:
                    up_simple_tile(rg.cams, rg.g, rg.fp, rg.od, task_tile<UpTile>(tk), rg.refs,
                                   reinterpret_cast<unsigned char*>(smem));
                    break;
                case BT_UPF2:
                    up_full_tile<T, 2>(rg.cams, rg.g, rg.fp, rg.od, R2, task_tile<UpTile>(tk), rg.refs, (const Slot*)rg.g0buf, smem);
                    break;
                case BT_UPF4:
                    up_full_tile<T, 4>(rg.cams, rg.g, rg.fp, rg.od, R2, task_tile<UpTile>(tk), rg.refs, (const Slot*)rg.g0buf, smem);
                    break;
                default:
                    break;
            }
            __syncthreads();
            if (t == 0) {
                const int ix = tk.rig * B_MAXSTAGE + tk.stage;
                if (s_np > 0 && p_ix[s_np - 1] == ix) {
                    ++p_cnt[s_np - 1];
                } else {
                    if (s_np == B_MAXCHUNK) flush();
                    p_ix[s_np] = ix;
                    p_cnt[s_np] = 1;
                    ++s_np;
                }
            }
        }
        if (t == 0) flush();
        if (stop) break;
    }
    if (t == 0) flush();
}

// Canvas tiles with more than 4 contributing cameras, after the persistent launch.
template <typename T>
__global__ void __launch_bounds__(U_THREADS) k_batch_general(const BatchRigDev* __restrict__ rigs,
                                                              const BTask* __restrict__ tasks, const int* ctl) {
    __shared__ float4 smem[UG_SMEM_F4];
    if (((volatile const int*)ctl)[2]) return;
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    const T* R2 = rg.g.levels >= 3 ? (const T*)rg.R[2] : nullptr;
    up_general_tile<T>(rg.cams, rg.g, rg.fp, rg.od, R2, task_tile<UpTile>(tk), rg.refs, smem);
}

// Multi-rig stage kernels (the alternative batched schedule): one block per task of one task type,
// tasks of every rig in one launch, each kernel with its own register and shared-memory budget.
template <typename T, int CAP>
__global__ void __launch_bounds__(D1_THREADS, D1Cap<CAP>::BLOCKS) k_mr_down1(const BatchRigDev* __restrict__ rigs,
                                                             const BTask* __restrict__ tasks) {
    extern __shared__ float4 smem[];
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    down1_tile<T, CAP>(rg.cams, rg.g, rg.fp, rg.od, task_tile<D1Tile>(tk), rg.refs, rg.d1w, rg.d1cols, (Slot*)rg.g0buf, smem);
}

template <typename T, typename RS>
__global__ void __launch_bounds__(256) k_mr_reduce(const BatchRigDev* __restrict__ rigs, const BTask* __restrict__ tasks) {
    extern __shared__ float4 smem[];
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    reduce_tile<T, RS>(rg.cams, rg.g, tk.level - 1, task_tile<Tile>(tk), smem);
}

// The 64 x 8 REDUCE tiles of the staged schedule run the single-rig path's column sweep.
template <typename T>
__global__ void __launch_bounds__(RC_THREADS, 8) k_mr_reduce_col(const BatchRigDev* __restrict__ rigs,
                                                                const BTask* __restrict__ tasks) {
    extern __shared__ float4 smem[];
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    reduce_col_tile<T>(rg.cams, rg.g, tk.level - 1, task_tile<Tile>(tk), smem, nullptr);
}

// camlist: the rig's camera list of the coarse tiles of this shape
template <typename T, typename CS>
__global__ void __launch_bounds__(256, 3) k_mr_coarse(const BatchRigDev* __restrict__ rigs, const BTask* __restrict__ tasks) {
    extern __shared__ float4 smem[];
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    coarse_tile<T, CS>(rg.cams, rg.g, tk.level, (T*)rg.R[tk.level],
                       tk.level + 1 < rg.g.levels ? (const T*)rg.R[tk.level + 1] : nullptr, task_tile<LevelTile>(tk),
                       std::is_same<CS, CSRig>::value ? rg.camlist : rg.camlist_w, smem);
}

__global__ void __launch_bounds__(U_THREADS) k_mr_up_simple(const BatchRigDev* __restrict__ rigs,
                                                             const BTask* __restrict__ tasks) {
    __shared__ __align__(16) unsigned char stage[3 * U_TX * U_TY];
    const BTask tk = tasks[blockIdx.x];
    const BatchRigDev& rg = rigs[tk.rig];
    up_simple_tile(rg.cams, rg.g, rg.fp, rg.od, task_tile<UpTile>(tk), rg.refs, stage);
}

template <typename T, int NC, int NB>
__device__ __forceinline__ void mr_up_full_block(const BatchRigDev* __restrict__ rigs, const BTask* __restrict__ tasks) {
    extern __shared__ float4 usm[];
    // the rig's geometry and output descriptor in shared memory: the tile reads them inside its
    // loops, which from the rig record in global memory costs a load each time (1.9 ms against
    // 1.4 ms for the canvas tiles of the 16-rig batch)
    __shared__ RigGeom g;
    __shared__ OutDesc od;
    const BTask* tp = tasks + blockIdx.x;
    const BatchRigDev& rg = rigs[tp->rig];
    if (threadIdx.x == 0) {
        g = rg.g;
        od = rg.od;
    }
    __syncthreads();
    const T* R2 = g.levels >= 3 ? (const T*)rg.R[2] : nullptr;
    up_full_tile<T, NC, NB>(rg.cams, g, rg.fp, od, R2, task_tile<UpTile>(*tp), rg.refs, (const Slot*)rg.g0buf, usm);
}
// (the two occupancies of k_up_full)
template <typename T, int NC>
__global__ void __launch_bounds__(U_THREADS) k_mr_up_full(const BatchRigDev* __restrict__ rigs,
                                                           const BTask* __restrict__ tasks) {
    mr_up_full_block<T, NC, (NC < 2 ? NC : 2)>(rigs, tasks);
}
template <typename T, int NC>
__global__ void __launch_bounds__(U_THREADS, 4) k_mr_up_full_b4(const BatchRigDev* __restrict__ rigs,
                                                                 const BTask* __restrict__ tasks) {
    mr_up_full_block<T, NC, 1>(rigs, tasks);
}

// A launch of the staged schedule: all tasks of one type and level, over every rig.
struct StageGroup {
    int type, level, count;
    BTask* d_tasks;
};

// Tile shapes the staged schedule can take for its REDUCE and coarse launches (the tuner times the
// four combinations): reduce 32 x 16 or 64 x 8 outputs, coarse 32 x 32 or 64 x 16.
constexpr int B_SHAPES = 4;
__host__ __device__ constexpr int b_rs(int shape) { return shape & 1; }
__host__ __device__ constexpr int b_cs(int shape) { return shape >> 1; }

struct BatchState {
    int device = 0, n = 0;
    bool fp16 = false;
    std::vector<stitch_rig*> rigs;
    std::vector<void*> allocs;
    BatchRigDev* d_rigs = nullptr;
    BatchRigDev* h_rigs = nullptr;  // pinned
    BTask* d_tasks[2] = {};         // two orderings
    int ntasks = 0;
    BTask* d_gtasks = nullptr;
    int ngtasks = 0;
    int* d_ctl = nullptr;
    int* d_done = nullptr;
    int* d_need = nullptr;
    int* h_status = nullptr;  // pinned
    std::vector<int> need;
    int max_bpsm[2] = {1, 1}, sms = 1;
    int order = 1, grid = 0, variant = 1, chunk = 4;
    float tuned_ms = 0.f;
    bool tuned = false;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<StageGroup> groups[B_SHAPES];  // staged schedule per tile-shape combination, in launch order
    int shape = 0;                             // the combination chosen
    bool staged = false;             // schedule chosen by the tuner: staged launches or persistent
    bool d1_small = false;           // staged down1 launches with the smaller footprint capacity (every rig's)
    bool up_four = false;            // staged up_full launches at four blocks per SM
    bool streams = false;            // ... or every rig's own launch sequence on its own stream
    cudaStream_t rs[B_MAXRIGS] = {};
    cudaEvent_t rdone[B_MAXRIGS] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t last = nullptr;  // recorded after each call's work
    bool launched = false;
    bool from_cache = false;  // the schedule came from the tuning cache
    long long tasks_by_type[8] = {};
};

template <typename V>
stitch_status b_upload(BatchState* b, const std::vector<V>& v, V** out) {
    *out = nullptr;
    if (v.empty()) return STITCH_OK;
    if (cudaMalloc((void**)out, sizeof(V) * v.size()) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return STITCH_ENOMEM;
    }
    b->allocs.push_back(*out);
    STITCH_CUDA_TRY(cudaMemcpy(*out, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
    return STITCH_OK;
}

void b_free(BatchState* b) {
    for (int k = 0; k < B_MAXRIGS; ++k) {
        if (b->rs[k]) cudaStreamDestroy(b->rs[k]);
        if (b->rdone[k]) cudaEventDestroy(b->rdone[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->last) cudaEventDestroy(b->last);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_rigs) cudaFreeHost(b->h_rigs);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
}

// The persistent kernel's blocks wait on one another, so it is launched cooperatively: the grid
// (at most the resident capacity) is guaranteed to run at once.
template <typename T>
void* batch_kernel(int variant) {
    return variant == 0 ? (void*)k_batch<T, 2> : (void*)k_batch<T, 3>;
}

template <typename T>
stitch_status b_launch(BatchState* b, int order, int variant, int grid, int chunk, cudaStream_t s) {
    int ntasks = b->ntasks, nrigs = b->n;
    void* args[] = {(void*)&b->d_rigs, (void*)&b->d_tasks[order], (void*)&ntasks, (void*)&b->d_ctl,
                    (void*)&b->d_done, (void*)&b->d_need, (void*)&nrigs, (void*)&chunk};
    STITCH_CUDA_TRY(cudaLaunchCooperativeKernel(batch_kernel<T>(variant), dim3(grid), dim3(B_THREADS), args, B_SMEM, s));
    if (b->ngtasks) k_batch_general<T><<<b->ngtasks, U_THREADS, 0, s>>>(b->d_rigs, b->d_gtasks, b->d_ctl);
    return launch_status();
}

stitch_status b_prepare(BatchState* b, cudaStream_t s);

// Report a wait that gave up: clear the device status and its host copy, return STITCH_ETIMEOUT.
stitch_status b_clear_status(BatchState* b) {
    *b->h_status = 0;
    STITCH_CUDA_TRY(cudaMemset(b->d_ctl + 1, 0, sizeof(int)));
    return STITCH_ETIMEOUT;
}


template <typename T>
stitch_status b_launch_staged(BatchState* b, int shape, cudaStream_t s) {
    for (const StageGroup& gr : b->groups[shape]) {
        if (!gr.count) continue;
        switch (gr.type) {
            case BT_D1:
                if (b->d1_small)
                    k_mr_down1<T, D1_FOOT_SMALL><<<gr.count, D1_THREADS, D1Cap<D1_FOOT_SMALL>::SMEM, s>>>(b->d_rigs, gr.d_tasks);
                else
                    k_mr_down1<T, D1_FOOT><<<gr.count, D1_THREADS, D1_SMEM, s>>>(b->d_rigs, gr.d_tasks);
                break;
            case BT_RED:
                if (b_rs(shape)) k_mr_reduce_col<T><<<gr.count, RC_THREADS, RC_SMEM, s>>>(b->d_rigs, gr.d_tasks);
                else k_mr_reduce<T, RSRig><<<gr.count, 256, RSRig::SMEM, s>>>(b->d_rigs, gr.d_tasks);
                break;
            case BT_CO:
                if (b_cs(shape))
                    k_mr_coarse<T, CSAlt><<<gr.count, 256, sizeof(float4) * CSAlt::SMEM_F4, s>>>(b->d_rigs, gr.d_tasks);
                else
                    k_mr_coarse<T, CSRig><<<gr.count, 256, sizeof(float4) * CSRig::SMEM_F4, s>>>(b->d_rigs, gr.d_tasks);
                break;
            case BT_UPS: k_mr_up_simple<<<gr.count, U_THREADS, 0, s>>>(b->d_rigs, gr.d_tasks); break;
            case BT_UPF2:
                if (b->up_four) k_mr_up_full_b4<T, 2><<<gr.count, U_THREADS, up_full_smem<2>(), s>>>(b->d_rigs, gr.d_tasks);
                else k_mr_up_full<T, 2><<<gr.count, U_THREADS, up_full_smem<2>(), s>>>(b->d_rigs, gr.d_tasks);
                break;
            case BT_UPF4:
                if (b->up_four) k_mr_up_full_b4<T, 4><<<gr.count, U_THREADS, up_full_smem<4>(), s>>>(b->d_rigs, gr.d_tasks);
                else k_mr_up_full<T, 4><<<gr.count, U_THREADS, up_full_smem<4>(), s>>>(b->d_rigs, gr.d_tasks);
                break;
            case BT_UPG: k_batch_general<T><<<gr.count, U_THREADS, 0, s>>>(b->d_rigs, gr.d_tasks, b->d_ctl); break;
            default: break;
        }
    }
    return launch_status();
}

template <typename T>
stitch_status b_staged_attrs() {
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_down1<T, D1_FOOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D1_SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_down1<T, D1_FOOT_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)D1Cap<D1_FOOT_SMALL>::SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_up_full_b4<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<2>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_up_full_b4<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<4>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_reduce<T, RSRig>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)RSRig::SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_reduce_col<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)RC_SMEM));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_coarse<T, CSRig>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float4) * CSRig::SMEM_F4)));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_coarse<T, CSAlt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float4) * CSAlt::SMEM_F4)));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_up_full<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<2>()));
    STITCH_CUDA_TRY(cudaFuncSetAttribute(k_mr_up_full<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)up_full_smem<4>()));
    return STITCH_OK;
}

// Graph of the staged schedule, captured from a private stream: descriptor copy, status reset,
// the stage launches in dependency order, status readback.
template <typename T>
stitch_status b_build_staged_graph(BatchState* b) {
    cudaStream_t cs;
    STITCH_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    stitch_status st = STITCH_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = STITCH_ECUDA;
    if (st == STITCH_OK) st = b_prepare(b, cs);
    if (st == STITCH_OK) st = b_launch_staged<T>(b, b->shape, cs);
    if (st == STITCH_OK && cudaMemcpyAsync(b->h_status, b->d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        st = STITCH_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess) st = STITCH_ECUDA;
    cudaStreamDestroy(cs);
    if (st != STITCH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    b->graph = g;
    STITCH_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    return STITCH_OK;
}

// Per call: the rig descriptors, the next-task counter ctl[0] and the abort flag ctl[2] reset, the
// completion counters cleared.  The status ctl[1] stays set once a wait has given up, until the host
// has reported it (fused_batch_status), so no call's timeout goes unreported.
stitch_status b_prepare(BatchState* b, cudaStream_t s) {
    STITCH_CUDA_TRY(cudaMemcpyAsync(b->d_rigs, b->h_rigs, sizeof(BatchRigDev) * b->n, cudaMemcpyHostToDevice, s));
    STITCH_CUDA_TRY(cudaMemsetAsync(b->d_ctl, 0, sizeof(int), s));
    STITCH_CUDA_TRY(cudaMemsetAsync(b->d_ctl + 2, 0, sizeof(int), s));
    STITCH_CUDA_TRY(cudaMemsetAsync(b->d_done, 0, sizeof(int) * b->need.size(), s));
    return STITCH_OK;
}

template <typename T>
stitch_status b_build_graph(BatchState* b) {
    cudaGraph_t g;
    STITCH_CUDA_TRY(cudaGraphCreate(&g, 0));
    b->graph = g;
    cudaGraphNode_t cp, m1, m1b, m2, kb, kg = nullptr, st;
    STITCH_CUDA_TRY(cudaGraphAddMemcpyNode1D(&cp, g, nullptr, 0, b->d_rigs, b->h_rigs, sizeof(BatchRigDev) * b->n,
                                             cudaMemcpyHostToDevice));
    cudaMemsetParams ms{};
    ms.dst = b->d_ctl;
    ms.value = 0;
    ms.elementSize = sizeof(int);
    ms.width = 1;
    ms.height = 1;
    ms.pitch = 0;
    STITCH_CUDA_TRY(cudaGraphAddMemsetNode(&m1, g, nullptr, 0, &ms));
    ms.dst = b->d_ctl + 2;
    STITCH_CUDA_TRY(cudaGraphAddMemsetNode(&m1b, g, nullptr, 0, &ms));
    ms.dst = b->d_done;
    ms.width = b->need.size();
    STITCH_CUDA_TRY(cudaGraphAddMemsetNode(&m2, g, nullptr, 0, &ms));
    int ntasks = b->ntasks, nrigs = b->n, chunk = b->chunk;
    void* args[] = {(void*)&b->d_rigs, (void*)&b->d_tasks[b->order], (void*)&ntasks, (void*)&b->d_ctl,
                    (void*)&b->d_done, (void*)&b->d_need, (void*)&nrigs, (void*)&chunk};
    cudaKernelNodeParams kp{};
    kp.func = batch_kernel<T>(b->variant);
    kp.gridDim = dim3(b->grid);
    kp.blockDim = dim3(B_THREADS);
    kp.sharedMemBytes = (unsigned)B_SMEM;
    kp.kernelParams = args;
    cudaGraphNode_t deps[4] = {cp, m1, m1b, m2};
    STITCH_CUDA_TRY(cudaGraphAddKernelNode(&kb, g, deps, 4, &kp));
    cudaLaunchAttributeValue coop{};
    coop.cooperative = 1;
    STITCH_CUDA_TRY(cudaGraphKernelNodeSetAttribute(kb, cudaLaunchAttributeCooperative, &coop));
    cudaGraphNode_t last = kb;
    if (b->ngtasks) {
        void* gargs[] = {(void*)&b->d_rigs, (void*)&b->d_gtasks, (void*)&b->d_ctl};
        cudaKernelNodeParams gp{};
        gp.func = (void*)k_batch_general<T>;
        gp.gridDim = dim3(b->ngtasks);
        gp.blockDim = dim3(U_THREADS);
        gp.sharedMemBytes = 0;
        gp.kernelParams = gargs;
        STITCH_CUDA_TRY(cudaGraphAddKernelNode(&kg, g, &kb, 1, &gp));
        last = kg;
    }
    STITCH_CUDA_TRY(cudaGraphAddMemcpyNode1D(&st, g, &last, 1, b->h_status, b->d_ctl + 1, sizeof(int),
                                             cudaMemcpyDeviceToHost));
    STITCH_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    return STITCH_OK;
}

// The per-rig schedule on streams: every rig's own launch sequence (the single-rig kernels) on a
// stream of its own, forked from and joined back to the caller's stream, so that one rig's small
// latency-bound levels overlap another's large launches.
template <typename T>
stitch_status b_launch_streams(BatchState* b, cudaStream_t s) {
    if (!b->fork) {
        STITCH_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (int k = 0; k < b->n; ++k) {
            STITCH_CUDA_TRY(cudaStreamCreateWithFlags(&b->rs[k], cudaStreamNonBlocking));
            STITCH_CUDA_TRY(cudaEventCreateWithFlags(&b->rdone[k], cudaEventDisableTiming));
        }
    }
    STITCH_CUDA_TRY(cudaEventRecord(b->fork, s));
    for (int k = 0; k < b->n; ++k) {
        stitch_rig* r = b->rigs[k];
        STITCH_CUDA_TRY(cudaStreamWaitEvent(b->rs[k], b->fork, 0));
        const stitch_status st = launch_all<T>(r, (FusedState*)r->fused, b->h_rigs[k].fp, b->h_rigs[k].od, b->rs[k]);
        if (st != STITCH_OK) return st;
        STITCH_CUDA_TRY(cudaEventRecord(b->rdone[k], b->rs[k]));
        STITCH_CUDA_TRY(cudaStreamWaitEvent(s, b->rdone[k], 0));
    }
    return STITCH_OK;
}

// Tuning cache: a file of JSON lines (STITCH_TUNE_CACHE), one object per tuned batch:
//   {"key": "<GPU name>|<SMs>|<hash of every rig's description>", "mode": "staged", "order": 1,
//    "variant": 1, "chunk": 4, "shape": 2, "ms": 5.43}
// A later batch with the same key on the same kind of GPU takes the schedule without timing it;
// the last line with a key wins.
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t k = 0; k < n; ++k) h = (h ^ c[k]) * 1099511628211ull;
    return h;
}

std::string b_cache_key(const BatchState* b) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) return std::string();
    uint64_t h = 1469598103934665603ull;
    const char tag[] = "libstitch batch schedule 2";
    h = fnv1a(h, tag, sizeof(tag));
    h = fnv1a(h, &b->n, sizeof(b->n));
    for (const stitch_rig* r : b->rigs) {
        const stitch_rig_desc& d = r->desc;
        const int32_t f[9] = {d.num_cameras, d.canvas_w, d.canvas_h, d.levels, d.band_fp16, d.out_float, d.path,
                              d.weights, d.canvas_model};
        h = fnv1a(h, f, sizeof(f));
        h = fnv1a(h, d.cylinder, sizeof(d.cylinder));
        for (const stitch_camera& c : r->cams) {
            h = fnv1a(h, &c.width, sizeof(c.width));
            h = fnv1a(h, &c.height, sizeof(c.height));
            h = fnv1a(h, c.H, sizeof(c.H));
            h = fnv1a(h, &c.gain, sizeof(c.gain));
        }
    }
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == '"' || ch == '\\' || ch == '|' || (unsigned char)ch < 32) ch = '_';
    char buf[96];
    snprintf(buf, sizeof(buf), "|%d|%016llx", prop.multiProcessorCount, (unsigned long long)h);
    return name + buf;
}

// Integer field `name` of a cache line, or `fallback`.
long cache_field(const std::string& line, const char* name, long fallback) {
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return fallback;
    const char* p = line.c_str() + at + pat.size();
    if (*p == '"') {
        ++p;
        if (!strncmp(p, "persistent", 10)) return 0;
        if (!strncmp(p, "staged", 6)) return 1;
        if (!strncmp(p, "streams", 7)) return 2;
        return fallback;
    }
    char* end = nullptr;
    const long v = strtol(p, &end, 10);
    return end == p ? fallback : v;
}

bool b_cache_load(BatchState* b, const char* path, const std::string& key) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    std::string line, found;
    char buf[1024];
    const std::string kpat = "\"key\": \"" + key + "\"";
    while (fgets(buf, sizeof(buf), f)) {
        line = buf;
        if (line.find(kpat) != std::string::npos) found = line;
    }
    fclose(f);
    if (found.empty()) return false;
    const long mode = cache_field(found, "mode", -1), order = cache_field(found, "order", -1),
               variant = cache_field(found, "variant", -1), chunk = cache_field(found, "chunk", -1),
               shape = cache_field(found, "shape", -1);
    if (mode < 0 || mode > 2 || order < 0 || order > 1 || variant < 0 || variant > 1 ||
        (chunk != 1 && chunk != 4 && chunk != 8) || shape < 0 || shape >= B_SHAPES)
        return false;
    b->staged = mode == 1;
    b->streams = mode == 2;
    b->order = (int)order;
    b->variant = (int)variant;
    b->grid = b->max_bpsm[variant] * b->sms;
    b->chunk = (int)chunk;
    b->shape = (int)shape;
    b->from_cache = true;
    return true;
}

void b_cache_store(const BatchState* b, const char* path, const std::string& key) {
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"mode\": \"%s\", \"order\": %d, \"variant\": %d, \"chunk\": %d, \"shape\": %d, \"ms\": %.4f}\n",
            key.c_str(), b->streams ? "streams" : b->staged ? "staged" : "persistent", b->order, b->variant, b->chunk,
            b->shape, b->tuned_ms);
    fclose(f);
}

// Time every candidate schedule (stage ordering, register variant with its resident blocks per
// SM, tasks per dequeue; the staged launches; the per-rig streams) on the real frames and keep the
// fastest.
template <typename T>
stitch_status b_tune(BatchState* b, cudaStream_t s) {
    const char* mode = getenv("STITCH_TUNE");
    b->variant = 1;
    b->grid = b->max_bpsm[1] * b->sms;
    b->order = 1;
    b->chunk = 4;
    b->staged = false;
    if (mode && strcmp(mode, "off") == 0) return STITCH_OK;
    // a cached schedule for this batch and GPU (unless STITCH_TUNE forces a mode or a new timing)
    const char* cache = getenv("STITCH_TUNE_CACHE");
    const bool use_cache = cache && *cache && (!mode || !*mode || strcmp(mode, "cache") == 0);
    const bool store_cache = cache && *cache && (use_cache || (mode && strcmp(mode, "full") == 0));
    const std::string key = cache && *cache ? b_cache_key(b) : std::string();
    if (use_cache && !key.empty() && b_cache_load(b, cache, key)) return STITCH_OK;
    cudaEvent_t e0, e1;
    STITCH_CUDA_TRY(cudaEventCreate(&e0));
    STITCH_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    const int chunks[3] = {1, 4, 8};
    for (int order = 0; order < 2; ++order)
        for (int variant = 0; variant < 2; ++variant)
            for (int ci = 0; ci < 3; ++ci)
                for (int rep = 0; rep < 2; ++rep) {
                    const int grid = b->max_bpsm[variant] * b->sms;
                    stitch_status st = b_prepare(b, s);
                    if (st != STITCH_OK) return st;
                    cudaEventRecord(e0, s);
                    st = b_launch<T>(b, order, variant, grid, chunks[ci], s);
                    if (st != STITCH_OK) return st;
                    cudaEventRecord(e1, s);
                    STITCH_CUDA_TRY(cudaEventSynchronize(e1));
                    int status = 0;
                    STITCH_CUDA_TRY(cudaMemcpy(&status, b->d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost));
                    if (status) return b_clear_status(b);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep == 1 && ms < best) {
                        best = ms;
                        b->order = order;
                        b->variant = variant;
                        b->grid = grid;
                        b->chunk = chunks[ci];
                    }
                }
    // the staged schedule, every tile-shape combination
    float best_staged = 1e30f;
    for (int shape = 0; shape < B_SHAPES; ++shape)
        for (int rep = 0; rep < 2; ++rep) {
            stitch_status st = b_prepare(b, s);
            if (st != STITCH_OK) return st;
            cudaEventRecord(e0, s);
            st = b_launch_staged<T>(b, shape, s);
            if (st != STITCH_OK) return st;
            cudaEventRecord(e1, s);
            STITCH_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 && ms < best_staged) {
                best_staged = ms;
                b->shape = shape;
            }
        }
    if (best_staged < best) {
        best = best_staged;
        b->staged = true;
    }
    // the per-rig streams
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        stitch_status st = b_launch_streams<T>(b, s);
        if (st != STITCH_OK) return st;
        cudaEventRecord(e1, s);
        STITCH_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 && ms < best) {
            best = ms;
            b->streams = true;
        }
    }
    if (mode && strcmp(mode, "persistent") == 0) b->staged = b->streams = false;
    if (mode && strcmp(mode, "staged") == 0) {
        b->staged = true;
        b->streams = false;
    }
    if (mode && strcmp(mode, "streams") == 0) b->streams = true;
    b->tuned_ms = best;
    if (store_cache && !key.empty()) b_cache_store(b, cache, key);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return STITCH_OK;
}

}  // namespace

stitch_status fused_batch_create(stitch_rig* const* rigs, int n, void** out) {
    *out = nullptr;
    if (!rigs || n < 1) return STITCH_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!rigs[k] || rigs[k]->desc.path != STITCH_PATH_FUSED || !rigs[k]->fused) return STITCH_EINVAL;
    const int dev = rigs[0]->device;
    const bool fp16 = rigs[0]->desc.band_fp16 != 0;
    for (int k = 1; k < n; ++k)
        if (rigs[k]->device != dev || (rigs[k]->desc.band_fp16 != 0) != fp16) return STITCH_EUNSUPPORTED;
    if (cudaSetDevice(dev) != cudaSuccess) return STITCH_ECUDA;
    BatchState* b = new (std::nothrow) BatchState();
    if (!b) return STITCH_ENOMEM;
    b->device = dev;
    b->n = n;
    b->fp16 = fp16;
    b->rigs.assign(rigs, rigs + n);
    b->need.assign((size_t)n * B_MAXSTAGE, 0);
    // per rig: descriptor and stage lists
    std::vector<std::vector<std::vector<BTask>>> stages(n);
    std::vector<BTask> gtasks;
    if (cudaMallocHost((void**)&b->h_rigs, sizeof(BatchRigDev) * n) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        b_free(b);
        return STITCH_ENOMEM;
    }
    *b->h_status = 0;
    for (int k = 0; k < n; ++k) {
        stitch_rig* r = rigs[k];
        FusedState* fs = (FusedState*)r->fused;
        BatchRigDev& d = b->h_rigs[k];
        memset(&d, 0, sizeof(d));
        d.cams = r->dcam;
        d.g = r->geom;
        d.d1 = fs->d1_tiles;
        for (int l = 0; l < MAXL; ++l) {
            d.red[l] = fs->red_tiles[l];
            d.co[l] = fs->co_tiles[l];
            d.R[l] = fs->R[l];
        }
        d.camlist = fs->camlist;
        d.refs = fs->refs;
        d.d1w = fs->d1w;
        d.d1cols = fs->d1cols;
        d.g0buf = fs->g0buf;
        for (int q = 0; q < UP_KINDS; ++q) d.up[q] = fs->up_tiles[q];
        const int L = r->geom.levels;
        auto mk = [&](int type, int idx, int level, int st) {
            BTask tk{k, type, idx, level, st, 0, 0, 0, {}};
            switch (type) {
                case BT_D1: memcpy(tk.tile, &fs->h_d1[idx], sizeof(D1Tile)); break;
                case BT_RED: memcpy(tk.tile, &fs->h_red[level][idx], sizeof(Tile)); break;
                case BT_CO: memcpy(tk.tile, &fs->h_co[level][idx], sizeof(LevelTile)); break;
                case BT_UPS: memcpy(tk.tile, &fs->h_up[UP_SIMPLE][idx], sizeof(UpTile)); break;
                case BT_UPF2: memcpy(tk.tile, &fs->h_up[UP_FULL2][idx], sizeof(UpTile)); break;
                case BT_UPF4: memcpy(tk.tile, &fs->h_up[UP_FULL4][idx], sizeof(UpTile)); break;
                case BT_UPG: memcpy(tk.tile, &fs->h_up[UP_GENERAL][idx], sizeof(UpTile)); break;
                default: break;
            }
            return tk;
        };
        auto add_stage = [&](int type, int level, int count) {
            const int st = (int)stages[k].size();
            stages[k].emplace_back();
            for (int i = 0; i < count; ++i) stages[k].back().push_back(mk(type, i, level, st));
            b->need[(size_t)k * B_MAXSTAGE + st] = count;
            b->tasks_by_type[type] += count;
        };
        if (L >= 2) add_stage(BT_D1, 1, fs->n_d1);
        for (int l = 2; l < L; ++l) add_stage(BT_RED, l, fs->n_red[l]);
        for (int l = L - 1; l >= 2; --l) add_stage(BT_CO, l, fs->n_co[l]);
        {
            const int st = (int)stages[k].size();
            stages[k].emplace_back();
            int cnt = 0;
            for (int i = 0; i < fs->n_up[UP_SIMPLE]; ++i) stages[k].back().push_back(mk(BT_UPS, i, 0, st));
            for (int i = 0; i < fs->n_up[UP_FULL2]; ++i) stages[k].back().push_back(mk(BT_UPF2, i, 0, st));
            for (int i = 0; i < fs->n_up[UP_FULL4]; ++i) stages[k].back().push_back(mk(BT_UPF4, i, 0, st));
            cnt = (int)stages[k].back().size();
            b->need[(size_t)k * B_MAXSTAGE + st] = cnt;
            b->tasks_by_type[BT_UPS] += fs->n_up[UP_SIMPLE];
            b->tasks_by_type[BT_UPF2] += fs->n_up[UP_FULL2];
            b->tasks_by_type[BT_UPF4] += fs->n_up[UP_FULL4];
            for (int i = 0; i < fs->n_up[UP_GENERAL]; ++i) gtasks.push_back(mk(BT_UPG, i, 0, st));
        }
    }
    // the persistent schedule takes the down1 tiles four at a time (one per 64-thread group)
    std::vector<std::vector<std::vector<BTask>>> pstages(n);
    for (int k = 0; k < n; ++k)
        for (size_t st = 0; st < stages[k].size(); ++st) {
            const std::vector<BTask>& v = stages[k][st];
            pstages[k].emplace_back();
            if (v.empty() || v[0].type != BT_D1) {
                pstages[k].back() = v;
                continue;
            }
            for (size_t i = 0; i < v.size(); i += B_D1_GROUPS) {
                BTask tk = v[i];
                tk.pad0 = (int)std::min<size_t>(B_D1_GROUPS, v.size() - i);
                pstages[k].back().push_back(tk);
            }
            b->need[(size_t)k * B_MAXSTAGE + st] = (int)pstages[k].back().size();
        }
    // two orderings: stages ranked from the start, or aligned so that every rig ends together
    int maxs = 0;
    for (int k = 0; k < n; ++k) maxs = std::max(maxs, (int)pstages[k].size());
    std::vector<BTask> ord[2];
    for (int o = 0; o < 2; ++o)
        for (int rank = 0; rank < maxs; ++rank)
            for (int k = 0; k < n; ++k) {
                const int s = o == 0 ? rank : rank - (maxs - (int)pstages[k].size());
                if (s < 0 || s >= (int)pstages[k].size()) continue;
                ord[o].insert(ord[o].end(), pstages[k][s].begin(), pstages[k][s].end());
            }
    b->ntasks = (int)ord[0].size();
    stitch_status st = STITCH_OK;
    if ((st = b_upload(b, ord[0], &b->d_tasks[0])) != STITCH_OK || (st = b_upload(b, ord[1], &b->d_tasks[1])) != STITCH_OK ||
        (st = b_upload(b, gtasks, &b->d_gtasks)) != STITCH_OK || (st = b_upload(b, b->need, &b->d_need)) != STITCH_OK) {
        b_free(b);
        return st;
    }
    b->ngtasks = (int)gtasks.size();
    // staged schedule: groups by (type, level) in dependency order, for every tile-shape combination;
    // the 32 x 16 reduce and 32 x 32 coarse tiles are the rigs' own, the 64 x 8 and 64 x 16 ones are
    // planned here (with their own camera lists)
    {
        int maxL = 0;
        for (int k = 0; k < n; ++k) maxL = std::max(maxL, rigs[k]->geom.levels);
        // the occupancy variants the rigs' own launches take (down1: the smaller footprint capacity
        // when every rig takes it; up_full: four blocks per SM for many waves of blended tiles)
        {
            long long nfull = 0;
            b->d1_small = true;
            for (int k = 0; k < n; ++k) {
                const FusedState* fs = (const FusedState*)rigs[k]->fused;
                b->d1_small = b->d1_small && fs->d1_small;
                nfull += fs->n_up[UP_FULL2] + fs->n_up[UP_FULL4];
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, rigs[0]->device) != cudaSuccess) {
                cudaGetLastError();
                sms = 1;
            }
            b->up_four = nfull >= 8LL * 4 * std::max(sms, 1);
        }
        std::vector<BTask> wred[MAXL], wco[MAXL];
        for (int k = 0; k < n; ++k) {
            stitch_rig* r = rigs[k];
            FusedState* fs = (FusedState*)r->fused;
            std::vector<Tile> red[MAXL];
            std::vector<LevelTile> co[MAXL];
            std::vector<int> camlist;
            plan_reduce_tiles(r, RSAlt::TX, RSAlt::TY, red);
            plan_coarse_tiles(r, fs->h_up, CSAlt::TX, CSAlt::TY, co, camlist);
            int* d_cl = nullptr;
            if ((st = b_upload(b, camlist, &d_cl)) != STITCH_OK) {
                b_free(b);
                return st;
            }
            b->h_rigs[k].camlist_w = d_cl;
            for (int l = 2; l < MAXL; ++l) {
                for (size_t i = 0; i < red[l].size(); ++i) {
                    BTask tk{k, BT_RED, (int)i, l, 0, 0, 0, 0, {}};
                    memcpy(tk.tile, &red[l][i], sizeof(Tile));
                    wred[l].push_back(tk);
                }
                for (size_t i = 0; i < co[l].size(); ++i) {
                    BTask tk{k, BT_CO, (int)i, l, 0, 0, 0, 0, {}};
                    memcpy(tk.tile, &co[l][i], sizeof(LevelTile));
                    wco[l].push_back(tk);
                }
            }
        }
        std::vector<std::pair<int, int>> order_tl;
        order_tl.push_back({BT_D1, 1});
        for (int l = 2; l < maxL; ++l) order_tl.push_back({BT_RED, l});
        for (int l = maxL - 1; l >= 2; --l) order_tl.push_back({BT_CO, l});
        order_tl.push_back({BT_UPS, 0});
        order_tl.push_back({BT_UPF2, 0});
        order_tl.push_back({BT_UPF4, 0});
        for (auto [type, level] : order_tl) {
            std::vector<BTask> v;
            for (int k = 0; k < n; ++k)
                for (const auto& stv : stages[k])
                    for (const BTask& tk : stv)
                        if (tk.type == type && tk.level == level) v.push_back(tk);
            StageGroup gr{type, level, (int)v.size(), nullptr};
            if (!v.empty() && (st = b_upload(b, v, &gr.d_tasks)) != STITCH_OK) {
                b_free(b);
                return st;
            }
            StageGroup gw = gr;  // the same group with the batch's wide tiles
            const std::vector<BTask>* w = type == BT_RED ? &wred[level] : type == BT_CO ? &wco[level] : nullptr;
            if (w) {
                gw.count = (int)w->size();
                gw.d_tasks = nullptr;
                if (!w->empty() && (st = b_upload(b, *w, &gw.d_tasks)) != STITCH_OK) {
                    b_free(b);
                    return st;
                }
            }
            for (int shape = 0; shape < B_SHAPES; ++shape) {
                const bool wide = (type == BT_RED && b_rs(shape)) || (type == BT_CO && b_cs(shape));
                const StageGroup& use = wide ? gw : gr;
                if (use.count) b->groups[shape].push_back(use);
            }
        }
        if (!gtasks.empty())
            for (int shape = 0; shape < B_SHAPES; ++shape) b->groups[shape].push_back({BT_UPG, 0, (int)gtasks.size(), b->d_gtasks});
        const stitch_status as = fp16 ? b_staged_attrs<half4>() : b_staged_attrs<float4>();
        if (as != STITCH_OK) {
            b_free(b);
            return as;
        }
    }
    std::vector<int> zeros(b->need.size(), 0), ctl = {0, 0, 0, 1 << 22};
    if ((st = b_upload(b, zeros, &b->d_done)) != STITCH_OK || (st = b_upload(b, ctl, &b->d_ctl)) != STITCH_OK) {
        b_free(b);
        return st;
    }
    if (cudaMalloc((void**)&b->d_rigs, sizeof(BatchRigDev) * n) != cudaSuccess) {
        cudaGetLastError();
        b_free(b);
        return STITCH_ENOMEM;
    }
    b->allocs.push_back(b->d_rigs);
    // resident blocks per SM of the persistent kernel: the grid never exceeds what fits at once
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        b_free(b);
        return STITCH_ECUDA;
    }
    b->sms = prop.multiProcessorCount;
    if (n > B_MAXRIGS) {
        b_free(b);
        return STITCH_EUNSUPPORTED;
    }
    for (int variant = 0; variant < 2; ++variant) {
        int bpsm = 0;
        void* fn = fp16 ? batch_kernel<half4>(variant) : batch_kernel<float4>(variant);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B_SMEM);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, fn, B_THREADS, B_SMEM);
        if (e != cudaSuccess || bpsm < 1) {
            cudaGetLastError();
            b_free(b);
            return STITCH_ECUDA;
        }
        b->max_bpsm[variant] = bpsm;
    }
    b->grid = b->max_bpsm[1] * b->sms;
    if (cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        b_free(b);
        return STITCH_ECUDA;
    }
    *out = b;
    return STITCH_OK;
}

stitch_status fused_batch_frames(void* bp, const uint8_t* const* const* frames, const int64_t* const* pitches,
                                 void* const* outs, const int64_t* out_pitches, cudaStream_t s) {
    BatchState* b = (BatchState*)bp;
    if (!b || !frames || !pitches || !outs || !out_pitches) return STITCH_EINVAL;
    for (int k = 0; k < b->n; ++k) {
        stitch_rig* r = b->rigs[k];
        if (!frames[k] || !pitches[k] || !outs[k]) return STITCH_EINVAL;
        const long long row = (long long)r->geom.nx[0] * (r->desc.out_float ? 12 : 3);
        if (out_pitches[k] < row) return STITCH_EINVAL;
        FramePtrs& fp = b->h_rigs[k].fp;
        memset(&fp, 0, sizeof(fp));
        for (int i = 0; i < r->geom.ncam; ++i) {
            if (!r->hcam[i].visible) continue;
            if (!frames[k][i] || pitches[k][i] < 3LL * r->cams[i].width) return STITCH_EINVAL;
            fp.p[i] = frames[k][i];
            fp.pitch[i] = pitches[k][i];
        }
        b->h_rigs[k].od = OutDesc{outs[k], out_pitches[k], r->desc.out_float};
    }
    if (!b->tuned) {
        const stitch_status st = b->fp16 ? b_tune<half4>(b, s) : b_tune<float4>(b, s);
        if (st != STITCH_OK) return st;
        b->tuned = true;
        if (!b->streams) {
            const stitch_status gs = b->staged
                                         ? (b->fp16 ? b_build_staged_graph<half4>(b) : b_build_staged_graph<float4>(b))
                                         : (b->fp16 ? b_build_graph<half4>(b) : b_build_graph<float4>(b));
            if (gs != STITCH_OK) return gs;
        }
    }
    // a wait that gave up in an earlier call whose work has completed is reported now, before any
    // further launch; one that has not completed yet is reported by a later call or by
    // fused_batch_status
    if (b->launched && cudaEventQuery(b->last) == cudaSuccess && *b->h_status) return b_clear_status(b);
    cudaGetLastError();  // a cudaErrorNotReady of the query is not an error
    if (b->streams) {
        // the frame and output pointers are kernel arguments here: launched directly, no graph
        const stitch_status st = b->fp16 ? b_launch_streams<half4>(b, s) : b_launch_streams<float4>(b, s);
        if (st != STITCH_OK) return st;
    } else {
        STITCH_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    }
    STITCH_CUDA_TRY(cudaEventRecord(b->last, s));
    b->launched = true;
    return STITCH_OK;
}

stitch_status fused_batch_status(void* bp) {
    BatchState* b = (BatchState*)bp;
    if (!b) return STITCH_EINVAL;
    if (!b->launched) return STITCH_OK;
    STITCH_CUDA_TRY(cudaEventSynchronize(b->last));
    return *b->h_status ? b_clear_status(b) : STITCH_OK;
}

void fused_batch_destroy(void* bp) {
    BatchState* b = (BatchState*)bp;
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    b_free(b);
}

stitch_status fused_batch_info(void* bp, int32_t* order, int32_t* grid, int64_t* ntasks) {
    BatchState* b = (BatchState*)bp;
    if (!b) return STITCH_EINVAL;
    if (order)
        *order = (b->streams ? 0xE : b->staged ? (0xF | (b->shape << 8)) : (b->order | (b->variant << 4) | (b->chunk << 8))) |
                 (b->from_cache ? 1 << 24 : 0);
    if (grid) *grid = b->grid;
    if (ntasks) *ntasks = b->ntasks + b->ngtasks;
    return STITCH_OK;
}

// Test hook: spin limit of the waits, and optionally make the second stage of rig `rig` wait for a
// count that is never reached (the first stage's `need` raised), so the bounded wait runs out.
stitch_status fused_batch_wait_test(void* bp, int spin_limit, int rig) {
    BatchState* b = (BatchState*)bp;
    if (!b || spin_limit < 1) return STITCH_EINVAL;
    STITCH_CUDA_TRY(cudaMemcpy(b->d_ctl + 3, &spin_limit, sizeof(int), cudaMemcpyHostToDevice));
    std::vector<int> need = b->need;
    if (rig >= 0 && rig < b->n) need[(size_t)rig * B_MAXSTAGE] += 1 << 30;
    STITCH_CUDA_TRY(cudaMemcpy(b->d_need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice));
    return STITCH_OK;
}
