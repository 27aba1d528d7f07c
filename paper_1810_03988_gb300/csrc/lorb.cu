// L-ORB feature extraction (Sec. 4.1, Algorithms 1 and 2) on the GPU, in exact integer
// arithmetic so that every decision (FAST, threshold, non-maximum suppression, top-N, BRIEF
// bits) is the one of the definition:
//   gray = (77 R + 150 G + 29 B + 128) >> 8; candidates inside the detection areas and at least
//   LORB_MARGIN px from the image border; FAST-9 on the radius-3 circle with threshold t;
//   Ix, Iy central differences; A, B, C their products weighted by the binomial [1,4,6,4,1]^2
//   (the sigma = 1 Gaussian, unnormalised); R' = 25 (AB - C^2) - (A + B)^2 = 25 R with
//   alpha = 0.04, kept when R' > t_h; non-maximum suppression over the 8-neighbourhood with ties
//   to the lower index y W + x; the N strongest (R' descending, index ascending); BRIEF bits
//   [S(x + p_k) > S(x + q_k)] of the binomial-smoothed image S for 256 given point pairs.
//
// Kernels: lorb_maps (gray and S over the areas' neighbourhood, S by separable passes),
// lorb_response (FAST + Harris on 32 x 16 tiles staged in shared memory; FAST by a compass
// pre-test and 16-bit run masks), lorb_nms (survivors appended with warp-aggregated atomics, their
// order is irrelevant since the selection below is exact, and counted in a histogram of coarse
// response bins), lorb_prune (the survivors in the bins that can hold the N strongest),
// lorb_select (one block: radix selection of the N-th key, then a bitonic sort of the N winners),
// lorb_brief (a warp per keypoint, bits packed by ballots).
#include "stitch_internal.cuh"

namespace {

constexpr int LORB_MARGIN = 18;
constexpr int LORB_MAX_AREAS = 64;
constexpr int LORB_MAX_POINTS = 2048;
constexpr int LT_X = 32, LT_Y = 16;           // response tile
constexpr int LG_X = LT_X + 6, LG_Y = LT_Y + 6;  // gray with the radius-3 halo
constexpr int LD_X = LT_X + 4, LD_Y = LT_Y + 4;  // gradients at the tensor window positions
constexpr int SEL_THREADS = 1024;

struct LorbAreas {
    int n;
    int r[LORB_MAX_AREAS][4];  // x0, y0, x1, y1 clipped to the margin, half-open
};

struct LorbPattern {
    int8_t p[256][4];
};

struct Cand {
    long long r;
    int idx, pad;
};

__device__ __forceinline__ bool in_areas(const LorbAreas& a, int x, int y) {
    for (int k = 0; k < a.n; ++k)
        if (x >= a.r[k][0] && x < a.r[k][2] && y >= a.r[k][1] && y < a.r[k][3]) return true;
    return false;
}

// gray (uint8) and binomial-smoothed gray S (unnormalised, at most 255 * 256: uint16) on
// [x0, x1) x [y0, y1) (x0 a multiple of 4); S by a horizontal then a vertical [1,4,6,4,1] pass (the
// same integers as the 5 x 5 product weights).  The tile's gray, with a halo of 4 columns and 2
// rows, is staged from groups of 4 pixels: three aligned 32-bit words where the group lies inside
// the image and the frame's base and pitch are multiples of 4 bytes, clamped byte loads otherwise.
__device__ __forceinline__ int gray_of(int r, int g, int b) { return (77 * r + 150 * g + 29 * b + 128) >> 8; }

__global__ void __launch_bounds__(256) lorb_maps(const uint8_t* __restrict__ frame, long long pitch, int W, int H,
                                                 int x0, int y0, int x1, int y1, uint8_t* __restrict__ gray,
                                                 uint16_t* __restrict__ smooth) {
    __shared__ int g[20][40];  // columns bx - 4 .. bx + 35, rows by - 2 .. by + 17
    __shared__ int hs[20][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const int bx = x0 + blockIdx.x * 32, by = y0 + blockIdx.y * 16;
    const bool words = ((reinterpret_cast<uintptr_t>(frame) | (uintptr_t)pitch) & 3) == 0;
    for (int q = threadIdx.x; q < 20 * 10; q += 256) {
        const int r = q / 10, j = q - r * 10;
        const int y = min(max(by - 2 + r, 0), H - 1), gx0 = bx - 4 + 4 * j;
        const uint8_t* row = frame + (long long)y * pitch;
        if (words && gx0 >= 0 && gx0 + 3 < W) {
            const uint32_t* w = reinterpret_cast<const uint32_t*>(row + 3LL * gx0);
            const uint32_t a = __ldg(w), b = __ldg(w + 1), c = __ldg(w + 2);
            // bytes R G B R | G B R G | B R G B
            g[r][4 * j] = gray_of(a & 255, (a >> 8) & 255, (a >> 16) & 255);
            g[r][4 * j + 1] = gray_of(a >> 24, b & 255, (b >> 8) & 255);
            g[r][4 * j + 2] = gray_of((b >> 16) & 255, b >> 24, c & 255);
            g[r][4 * j + 3] = gray_of((c >> 8) & 255, (c >> 16) & 255, c >> 24);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = min(max(gx0 + k, 0), W - 1);
                const uint8_t* p = row + 3LL * x;
                g[r][4 * j + k] = gray_of(p[0], p[1], p[2]);
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 20 * 32; q += 256) {
        const int r = q >> 5, c = q & 31;  // window columns c + 2 .. c + 6 (canvas x - 2 .. x + 2)
        hs[r][c] = g[r][c + 2] + 4 * g[r][c + 3] + 6 * g[r][c + 4] + 4 * g[r][c + 5] + g[r][c + 6];
    }
    __syncthreads();
    for (int rr = ty; rr < 16; rr += 8) {
        const int x = bx + tx, y = by + rr;
        if (x >= x1 || y >= y1) continue;
        gray[(long long)y * W + x] = (uint8_t)g[rr + 2][tx + 4];
        // S only where its 5 x 5 window is inside the image (BRIEF never reads it elsewhere)
        if (x < 2 || y < 2 || x >= W - 2 || y >= H - 2) continue;
        smooth[(long long)y * W + x] =
            (uint16_t)(hs[rr][tx] + 4 * hs[rr + 1][tx] + 6 * hs[rr + 2][tx] + 4 * hs[rr + 3][tx] + hs[rr + 4][tx]);
    }
}

// FAST-9 + Harris response R' (INT64_MIN where not a candidate) on [x0, x1) x [y0, y1)
__global__ void __launch_bounds__(256) lorb_response(const uint8_t* __restrict__ gray, int W, int x0, int y0,
                                                     int x1, int y1, const __grid_constant__ LorbAreas areas,
                                                     int fast_t, long long harris_t, long long* __restrict__ resp) {
    __shared__ int g[LG_Y][LG_X];
    __shared__ int dxs[LD_Y][LD_X], dys[LD_Y][LD_X];
    __shared__ int hxx[LD_Y][LT_X], hyy[LD_Y][LT_X], hxy[LD_Y][LT_X];
    const int bx = x0 + blockIdx.x * LT_X, by = y0 + blockIdx.y * LT_Y;
    const int t = threadIdx.x;
    // gray of the tile and its radius-3 halo (inside the image: candidates keep a wider margin)
    for (int q = t; q < LG_X * LG_Y; q += 256) {
        const int r = q / LG_X, c = q - r * LG_X;
        const int x = bx - 3 + c, y = by - 3 + r;
        g[r][c] = (x >= 0 && y >= 0 && x < x1 + 3 && y < y1 + 3) ? gray[(long long)y * W + x] : 0;
    }
    __syncthreads();
    for (int q = t; q < LD_X * LD_Y; q += 256) {
        const int r = q / LD_X, c = q - r * LD_X;  // position (bx - 2 + c, by - 2 + r)
        dxs[r][c] = g[r + 1][c + 2] - g[r + 1][c];
        dys[r][c] = g[r + 2][c + 1] - g[r][c + 1];
    }
    __syncthreads();
    const int b5[5] = {1, 4, 6, 4, 1};
    for (int q = t; q < LT_X * LD_Y; q += 256) {
        const int r = q / LT_X, c = q - r * LT_X;
        int sxx = 0, syy = 0, sxy = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int ix = dxs[r][c + k], iy = dys[r][c + k];
            sxx += b5[k] * ix * ix;
            syy += b5[k] * iy * iy;
            sxy += b5[k] * ix * iy;
        }
        hxx[r][c] = sxx;
        hyy[r][c] = syy;
        hxy[r][c] = sxy;
    }
    __syncthreads();
    constexpr int fdx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
    constexpr int fdy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};
    for (int q = t; q < LT_X * LT_Y; q += 256) {
        const int r = q / LT_X, c = q - r * LT_X;
        const int x = bx + c, y = by + r;
        if (x >= x1 || y >= y1) continue;
        long long out = LLONG_MIN;
        if (in_areas(areas, x, y)) {
            // FAST-9: a run of >= 9 contiguous circle pixels all brighter than p + t, or all darker
            // than p - t.  Such an arc holds at least 2 of the 4 compass pixels (0, 4, 8, 12), so a
            // pixel with fewer than 2 brighter and fewer than 2 darker compass pixels is no corner;
            // the others test the 16-bit masks, doubled so that a run may wrap around.
            const int p = g[r + 3][c + 3], hi = p + fast_t, lo = p - fast_t;
            int nb = 0, nd = 0;
#pragma unroll
            for (int k = 0; k < 16; k += 4) {
                const int v = g[r + 3 + fdy[k]][c + 3 + fdx[k]];
                nb += v > hi;
                nd += v < lo;
            }
            bool corner = false;
            if (nb >= 2 || nd >= 2) {
                unsigned mb = 0, md = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int v = g[r + 3 + fdy[k]][c + 3 + fdx[k]];
                    mb |= (unsigned)(v > hi) << k;
                    md |= (unsigned)(v < lo) << k;
                }
                mb |= mb << 16;
                md |= md << 16;
                unsigned rb = mb, rd = md;
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    rb &= mb >> k;
                    rd &= md >> k;
                }
                corner = (rb | rd) != 0;
            }
            if (corner) {
                long long A = 0, B = 0, C = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    A += (long long)b5[k] * hxx[r + k][c];
                    B += (long long)b5[k] * hyy[r + k][c];
                    C += (long long)b5[k] * hxy[r + k][c];
                }
                const long long rr = 25 * (A * B - C * C) - (A + B) * (A + B);
                if (rr > harris_t) out = rr;
            }
        }
        resp[(long long)y * W + x] = out;
    }
}

// Coarse, monotone (non-decreasing in R') bin of a response: the position of its leading bit and
// the 4 bits below it; R' <= 0 in bin 0.  The N strongest candidates all lie in the bins at or above
// the bin where the count from the top reaches N.
constexpr int LORB_BINS = 1024;
__device__ __forceinline__ int lorb_bin(long long r) {
    if (r <= 0) return 0;
    const int e = 64 - __clzll(r);  // 1 .. 63
    const int m = e > 5 ? (int)((r >> (e - 5)) & 15) : (int)(r & 15);
    return 16 * e + m;
}

// non-maximum suppression: survivors appended to cand (ties to the lower index), and counted in
// the bin histogram
__global__ void __launch_bounds__(256) lorb_nms(const long long* __restrict__ resp, int W, int x0, int y0, int x1,
                                                int y1, Cand* __restrict__ cand, int* __restrict__ ncand, int cap,
                                                int* __restrict__ hist) {
    const int x = x0 + blockIdx.x * 32 + (threadIdx.x & 31), y = y0 + blockIdx.y * 8 + (threadIdx.x >> 5);
    bool keep = false;
    long long r = LLONG_MIN;
    int idx = 0;
    if (x < x1 && y < y1) {
        idx = y * W + x;
        r = resp[idx];
        keep = r != LLONG_MIN;
        for (int dy = -1; dy <= 1 && keep; ++dy)
            for (int dx = -1; dx <= 1 && keep; ++dx) {
                if (!dx && !dy) continue;
                const int xx = x + dx, yy = y + dy;
                if (xx < x0 || yy < y0 || xx >= x1 || yy >= y1) continue;  // outside: never a candidate
                const int q = yy * W + xx;
                const long long o = resp[q];
                if (o == LLONG_MIN) continue;
                keep = r > o || (r == o && idx < q);
            }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    int base = 0;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(ncand, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
        const int pos = base + __popc(m & ((1u << lane) - 1));
        if (pos < cap) {
            cand[pos] = Cand{r, idx, 0};
            atomicAdd(&hist[lorb_bin(r)], 1);
        }
    }
}

// The candidates in the bins at or above the threshold bin (where the count from the top reaches
// N) appended to cand2: a superset of the N strongest, typically a small one.  Grid-stride; every
// block finds the threshold bin from the histogram (a suffix sum over the bins).
constexpr int PRUNE_THREADS = 1024, PRUNE_BLOCKS = 64;
__global__ void __launch_bounds__(PRUNE_THREADS) lorb_prune(const Cand* __restrict__ cand, const int* __restrict__ ncand,
                                                            int cap, int npts, const int* __restrict__ hist,
                                                            Cand* __restrict__ cand2, int* __restrict__ n2,
                                                            int* __restrict__ overflow) {
    static_assert(PRUNE_THREADS == LORB_BINS, "one bin per thread");
    __shared__ int wsum[32];
    __shared__ int s_b;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int total = *ncand, n = min(total, cap), want = min(n, npts);
    if (blockIdx.x == 0 && t == 0) *overflow = total > cap ? 1 : 0;
    if (t == 0) s_b = LORB_BINS;  // want == 0: nothing
    // suffix sums: thread t takes bin 1023 - t and an inclusive prefix sum over t
    const int b = LORB_BINS - 1 - t;
    int v = hist[b];
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += o;
        }
        wsum[lane] = x;
    }
    __syncthreads();
    const int S = v + (w > 0 ? wsum[w - 1] : 0);  // candidates in bins >= b
    const int S_above = S - hist[b];             // in bins > b
    if (want > 0 && S >= want && S_above < want) s_b = b;
    __syncthreads();
    const int bT = s_b;
    for (int i0 = blockIdx.x * PRUNE_THREADS; i0 < n; i0 += gridDim.x * PRUNE_THREADS) {
        const int i = i0 + t;
        Cand cv{0, 0, 0};
        bool keep = false;
        if (i < n) {
            cv = cand[i];
            keep = lorb_bin(cv.r) >= bT;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        int base = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(n2, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (keep) cand2[base + __popc(m & ((1u << lane) - 1))] = cv;
    }
}

// key order: R' descending, index ascending == (u, ~idx) descending with u = R' with the sign
// bit flipped
__device__ __forceinline__ unsigned long long ukey(long long r) { return (unsigned long long)r ^ (1ull << 63); }

// Threshold digit of one radix-selection pass over the 256-bin histogram (threads 0..255 take a
// bin each; every thread of the block calls this): from the top, the bin b where the count of the
// bins from the top down to b first reaches `need` (the largest keys); from the bottom, the same
// counting up (the smallest indices).  Returns b and leaves in `need` what is still wanted among
// the keys of bin b.  If the count never reaches `need`, the last bin and the remainder, as a
// sequential scan would leave them.
__device__ __forceinline__ int select_digit(const int* hist, int* wsum, int& need, bool from_top, int* s_out) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const bool act = t < 256;
    const int b = from_top ? 255 - t : t;
    const int own = act ? hist[b] : 0;
    int v = own;  // inclusive prefix over the bins in scan order
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (act && lane == 31) wsum[w] = v;
    const int nd = need;
    __syncthreads();
    int S = v;
    if (act)
        for (int k = 0; k < w; ++k) S += wsum[k];
    if (t == 255) {  // the last bin in scan order: the fallback
        s_out[0] = b;
        s_out[1] = nd - (S - own);
    }
    __syncthreads();
    if (act && t < 255 && S >= nd && S - own < nd) {
        s_out[0] = b;
        s_out[1] = nd - (S - own);
    }
    __syncthreads();
    need = s_out[1];
    const int r = s_out[0];
    __syncthreads();
    return r;
}

// One block: the N strongest survivors, sorted.  Radix selection (8-bit digits, most
// significant first) of the N-th largest u; survivors above it are taken, and among those equal
// to it the lowest indices (a second radix selection on the index); then a bitonic sort.
__global__ void __launch_bounds__(SEL_THREADS) lorb_select(const Cand* __restrict__ cand,
                                                           const int* __restrict__ ncand, int cap, int npts,
                                                           int W, int* __restrict__ out_xy,
                                                           long long* __restrict__ out_resp, int* __restrict__ count,
                                                           int* __restrict__ overflow) {
    __shared__ int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_need;
    __shared__ Cand win[LORB_MAX_POINTS];
    __shared__ int s_nwin;
    __shared__ int s_wsum[32], s_pick[2];
    const int t = threadIdx.x;
    const int total = *ncand;
    if (t == 0 && overflow) *overflow = total > cap ? 1 : 0;
    const int n = min(total, cap);
    const int want = min(n, npts);
    if (t == 0) {
        s_prefix = 0;
        s_need = want;
        s_nwin = 0;
    }
    __syncthreads();
    // radix selection of the want-th largest u (threshold value uT)
    unsigned long long mask = 0;
    for (int d = 7; d >= 0 && want > 0; --d) {
        for (int k = t; k < 256; k += SEL_THREADS) hist[k] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        for (int i = t; i < n; i += SEL_THREADS) {
            const unsigned long long u = ukey(cand[i].r);
            if ((u & mask) == prefix) atomicAdd(&hist[(u >> (8 * d)) & 255], 1);
        }
        __syncthreads();
        int need = s_need;
        const int b = select_digit(hist, s_wsum, need, true, s_pick);
        if (t == 0) {
            s_prefix = prefix | ((unsigned long long)b << (8 * d));
            s_need = need;  // how many of the keys equal to the final prefix are still wanted
        }
        __syncthreads();
        mask |= 255ull << (8 * d);
    }
    const unsigned long long uT = s_prefix;
    const int need_eq = s_need;
    // the index threshold among keys equal to uT: the need_eq-th smallest index
    int iT = INT_MAX;
    if (want > 0) {
        unsigned prefix = 0, imask = 0;
        if (t == 0) s_need = need_eq;
        __syncthreads();
        for (int d = 3; d >= 0; --d) {
            for (int k = t; k < 256; k += SEL_THREADS) hist[k] = 0;
            __syncthreads();
            for (int i = t; i < n; i += SEL_THREADS) {
                if (ukey(cand[i].r) != uT) continue;
                const unsigned ix = (unsigned)cand[i].idx;
                if ((ix & imask) == prefix) atomicAdd(&hist[(ix >> (8 * d)) & 255], 1);
            }
            __syncthreads();
            int need = s_need;
            const int b = select_digit(hist, s_wsum, need, false, s_pick);
            if (t == 0) {
                s_prefix = prefix | ((unsigned)b << (8 * d));
                s_need = need;
            }
            __syncthreads();
            prefix = (unsigned)s_prefix;
            imask |= 255u << (8 * d);
        }
        iT = (int)prefix;
    }
    // gather the winners: u > uT, or u == uT with index <= iT
    for (int i = t; i < n && want > 0; i += SEL_THREADS) {
        const Cand c = cand[i];
        const unsigned long long u = ukey(c.r);
        if (u > uT || (u == uT && c.idx <= iT)) {
            const int pos = atomicAdd(&s_nwin, 1);
            if (pos < LORB_MAX_POINTS) win[pos] = c;
        }
    }
    __syncthreads();
    // bitonic sort of the winners (padded with the weakest key)
    int m = 1;
    while (m < want) m <<= 1;
    for (int i = want + t; i < m; i += SEL_THREADS) win[i] = Cand{LLONG_MIN, INT_MAX, 0};
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < m; i += SEL_THREADS) {
                const int l = i ^ j;
                if (l <= i) continue;
                const Cand a = win[i], b = win[l];
                // a before b when a is stronger: R' descending, index ascending
                const bool a_first = a.r > b.r || (a.r == b.r && a.idx < b.idx);
                const bool up = (i & k) == 0;
                if (up != a_first) {
                    win[i] = b;
                    win[l] = a;
                }
            }
            __syncthreads();
        }
    for (int i = t; i < want; i += SEL_THREADS) {
        out_xy[2 * i] = win[i].idx % W;
        out_xy[2 * i + 1] = win[i].idx / W;
        out_resp[i] = win[i].r;
    }
    if (t == 0) *count = want;
}

// BRIEF: a warp per keypoint, lane l computes bits l, l + 32, ..., packed by ballots
__global__ void __launch_bounds__(256) lorb_brief(const uint16_t* __restrict__ smooth, int W,
                                                  const __grid_constant__ LorbPattern pat,
                                                  const int* __restrict__ xy, const int* __restrict__ count,
                                                  unsigned* __restrict__ desc) {
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= *count) return;
    const int x = xy[2 * k], y = xy[2 * k + 1];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int b = 32 * j + lane;
        const int sp = smooth[(long long)(y + pat.p[b][1]) * W + x + pat.p[b][0]];
        const int sq = smooth[(long long)(y + pat.p[b][3]) * W + x + pat.p[b][2]];  // uint16 -> int
        const unsigned bits = __ballot_sync(0xffffffffu, sp > sq);
        if (lane == 0) desc[8 * k + j] = bits;  // bit b of the descriptor: byte b/8, bit b%8 (little endian)
    }
}

}  // namespace

struct stitch_lorb {
    int device = 0;
    int max_w = 0, max_h = 0, max_points = 0, cap = 0;
    uint8_t* gray = nullptr;
    uint16_t* smooth = nullptr;
    long long* resp = nullptr;
    Cand* cand = nullptr;
    Cand* cand2 = nullptr;  // the pruned candidates
    int* ncand = nullptr;   // [0] survivors, [1] overflow flag, [2] pruned count, then the bin histogram
};

static void lorb_free(stitch_lorb* c) {
    if (!c) return;
    cudaFree(c->gray);
    cudaFree(c->smooth);
    cudaFree(c->resp);
    cudaFree(c->cand);
    cudaFree(c->cand2);
    cudaFree(c->ncand);
    delete c;
}

extern "C" stitch_status stitch_lorb_create(int32_t max_width, int32_t max_height, int32_t max_points, int32_t device,
                                            stitch_lorb** out) {
    if (!out) return STITCH_EINVAL;
    *out = nullptr;
    if (max_width < 2 * LORB_MARGIN + 1 || max_height < 2 * LORB_MARGIN + 1 || max_points < 1 ||
        max_points > LORB_MAX_POINTS || (long long)max_width * max_height > (1LL << 30))
        return STITCH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return STITCH_ECUDA;
    }
    if (device < 0 || device >= ndev) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return STITCH_ECUDA;
    stitch_lorb* c = new (std::nothrow) stitch_lorb();
    if (!c) return STITCH_ENOMEM;
    c->device = device;
    c->max_w = max_width;
    c->max_h = max_height;
    c->max_points = max_points;
    const size_t N = (size_t)max_width * max_height;
    c->cap = (int)(((size_t)max_width + 1) / 2 * (((size_t)max_height + 1) / 2));  // NMS survivors are never adjacent
    stitch_status st = STITCH_OK;
    if (cudaMalloc(&c->gray, N) != cudaSuccess || cudaMalloc(&c->smooth, N * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&c->resp, N * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&c->cand, (size_t)c->cap * sizeof(Cand)) != cudaSuccess ||
        cudaMalloc(&c->cand2, (size_t)c->cap * sizeof(Cand)) != cudaSuccess ||
        cudaMalloc(&c->ncand, (4 + LORB_BINS) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        st = STITCH_ENOMEM;
    }
    if (st == STITCH_OK && cudaMemset(c->ncand, 0, (4 + LORB_BINS) * sizeof(int)) != cudaSuccess) st = STITCH_ECUDA;
    if (prev >= 0) cudaSetDevice(prev);
    if (st != STITCH_OK) {
        lorb_free(c);
        return st;
    }
    *out = c;
    return STITCH_OK;
}

extern "C" void stitch_lorb_destroy(stitch_lorb* c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    lorb_free(c);
    if (prev >= 0) cudaSetDevice(prev);
}

extern "C" stitch_status stitch_lorb_detect(stitch_lorb* c, const uint8_t* frame, int32_t width, int32_t height,
                                            int64_t pitch, const int32_t* areas, int32_t n_areas,
                                            const stitch_lorb_params* params, const int8_t* pattern,
                                            int32_t* xy, int64_t* resp, uint8_t* desc, int32_t* count,
                                            void* stream) {
    if (!c || !frame || !params || !pattern || !xy || !resp || !desc || !count) return STITCH_EINVAL;
    if (width < 1 || height < 1 || width > c->max_w || height > c->max_h || pitch < 3LL * width || n_areas < 0 ||
        n_areas > LORB_MAX_AREAS || (n_areas > 0 && !areas) || params->fast_t < 0 || params->max_points < 0 ||
        params->max_points > c->max_points)
        return STITCH_EINVAL;
    LorbPattern pat;
    for (int k = 0; k < 256; ++k)
        for (int j = 0; j < 4; ++j) {
            if (pattern[4 * k + j] < -15 || pattern[4 * k + j] > 15) return STITCH_EINVAL;
            pat.p[k][j] = pattern[4 * k + j];
        }
    // areas clipped to the margin; bounding box of the candidates, and of what BRIEF reads
    LorbAreas ar{};
    int bx0 = width, by0 = height, bx1 = 0, by1 = 0;
    for (int k = 0; k < n_areas; ++k) {
        const int x0 = std::max(areas[4 * k], LORB_MARGIN), y0 = std::max(areas[4 * k + 1], LORB_MARGIN);
        const int x1 = std::min(areas[4 * k + 2], width - LORB_MARGIN), y1 = std::min(areas[4 * k + 3], height - LORB_MARGIN);
        if (x1 <= x0 || y1 <= y0) continue;
        ar.r[ar.n][0] = x0;
        ar.r[ar.n][1] = y0;
        ar.r[ar.n][2] = x1;
        ar.r[ar.n][3] = y1;
        ++ar.n;
        bx0 = std::min(bx0, x0);
        by0 = std::min(by0, y0);
        bx1 = std::max(bx1, x1);
        by1 = std::max(by1, y1);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return STITCH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    stitch_status st = STITCH_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == STITCH_OK) st = STITCH_ECUDA;
    };
    int* hist = c->ncand + 4;
    ok(cudaMemsetAsync(c->ncand, 0, (4 + LORB_BINS) * sizeof(int), s));
    if (ar.n > 0) {
        // gray and S on the candidates' box grown by the BRIEF reach (15 + 2) and the FAST / tensor
        // halo, inside the image
        const int mx0 = std::max(bx0 - 17, 0) & ~3, my0 = std::max(by0 - 17, 0);  // x0 on a 4-pixel group
        const int mx1 = std::min(bx1 + 17, (int)width), my1 = std::min(by1 + 17, (int)height);
        lorb_maps<<<dim3((mx1 - mx0 + 31) / 32, (my1 - my0 + 15) / 16), 256, 0, s>>>(
            frame, pitch, width, height, mx0, my0, mx1, my1, c->gray, c->smooth);
        lorb_response<<<dim3((bx1 - bx0 + LT_X - 1) / LT_X, (by1 - by0 + LT_Y - 1) / LT_Y), 256, 0, s>>>(
            c->gray, width, bx0, by0, bx1, by1, ar, params->fast_t, (long long)params->harris_t, c->resp);
        lorb_nms<<<dim3((bx1 - bx0 + 31) / 32, (by1 - by0 + 7) / 8), 256, 0, s>>>(c->resp, width, bx0, by0, bx1, by1,
                                                                               c->cand, c->ncand, c->cap, hist);
    }
    lorb_prune<<<PRUNE_BLOCKS, PRUNE_THREADS, 0, s>>>(c->cand, c->ncand, c->cap, params->max_points, hist, c->cand2,
                                                      c->ncand + 2, c->ncand + 1);
    lorb_select<<<1, SEL_THREADS, 0, s>>>(c->cand2, c->ncand + 2, c->cap, params->max_points, width, xy,
                                          reinterpret_cast<long long*>(resp), count, nullptr);
    lorb_brief<<<(params->max_points + 7) / 8 + 1, 256, 0, s>>>(c->smooth, width, pat, xy, count,
                                                                reinterpret_cast<unsigned*>(desc));
    ok(cudaGetLastError());
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return st;
}
