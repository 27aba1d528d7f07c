// S7 (an extension beyond the paper, which fixes its homographies by feature matching, Sec. 4.2,
// Algorithm 4 step 5): overlap photometric loss and its gradient with respect to each camera's
// canvas->camera homography entries a11..a32 (a33 = +-1 fixed by the rig) and gain.
//
//   loss = sum_x sum_{i<j} v_i(x) v_j(x) |I_i(x) - I_j(x)|^2,  I = gain * bilinear(frame, A x) / 255
//
// with validity masks held constant.  For camera i at pixel x with k valid cameras,
// dloss/dI_i = 2 r_i, r_i = k I_i - sum_j I_j, and by the chain rule through u = nu/w, v = nv/w:
//   d/da11 = gu x/w, d/da12 = gu y/w, d/da13 = gu/w, d/da2k likewise with gv,
//   d/da31 = -(gu u + gv v) x/w, d/da32 = -(gu u + gv v) y/w, d/dgain = 2 r . bilinear/255,
// where gu = 2 r . dI/du and gv = 2 r . dI/dv (bilinear derivative inside the cell, zero along a
// clamped axis).  Sample coordinates are recomputed per pixel, never stored.
//
// Sums run in local coordinates x' = x - c_i (c_i a fixed point of camera i's footprint) so the
// single-precision terms stay small: with S(f) = sum f, d/da11 = S(gu x'/w) + c_x S(gu/w) etc.,
// applied in double precision at the end.  Per pixel and camera the 10 terms are reduced by warp
// shuffles and a block tree to one partial per (tile, camera slot); a second kernel sums each
// camera's partials with compensated (TwoSum) single-precision arithmetic and applies the chain
// rule to canvas coordinates in double precision.
#include "stitch_internal.cuh"

namespace {

constexpr int BW_TX = 64, BW_TY = 8;  // canvas pixels per tile
constexpr int BW_THREADS = 256;
constexpr int BW_PPT = BW_TX * BW_TY / BW_THREADS;  // 2 pixels per thread
constexpr int BW_SLOTS = 4;                          // cameras accumulated per pass
constexpr int BW_NV = 10;                            // values per camera
constexpr int BW_MARGIN = 64;                        // px: how far params may move footprints

struct BwTile {
    int x0, y0, first, count;  // canvas origin, candidate cameras (range in the camera list)
};

// One camera's sample at a pixel: bilinear value and its derivatives (before gain, in [0,1]
// units), source position and w.
struct GSample {
    float b[3], bu[3], bv[3];
    float u, v, w;
    bool valid;
};

__device__ __forceinline__ void gsample(const uint8_t* __restrict__ px, long long pitch, int W, int H,
                                        const TileMap& t, float dx, float dy, GSample& s) {
    const Pos p = map_pos(t, (float)t.U0, (float)t.V0, dx, dy);
    s.u = p.u;
    s.v = p.v;
    s.w = p.den;
    s.valid = (p.den > 0.f) & (p.u >= -0.5f) & (p.u < (float)W - 0.5f) & (p.v >= -0.5f) & (p.v < (float)H - 0.5f);
    int i0, j0;
    float fx, fy;
    bool cu = false, cv = false;
    if (p.iu < 0) { i0 = 0; fx = 0.f; cu = true; }
    else if (p.iu >= W - 1) { i0 = W - 1; fx = 0.f; cu = true; }
    else { i0 = p.iu; fx = p.fu; }
    if (p.iv < 0) { j0 = 0; fy = 0.f; cv = true; }
    else if (p.iv >= H - 1) { j0 = H - 1; fy = 0.f; cv = true; }
    else { j0 = p.iv; fy = p.fv; }
    // an exact integer u = W-1 sits on the last texel: one-sided derivative there is 0 as well
    const int di = (i0 + 1 < W) ? 3 : 0;
    const long long dj = (j0 + 1 < H) ? pitch : 0;
    const uint8_t* a = px + (long long)j0 * pitch + 3 * i0;
    const uint8_t* b = a + dj;
    const float k255 = 1.0f / 255.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p00 = u8_to_f(__ldg(a + c)), p01 = u8_to_f(__ldg(a + di + c));
        const float p10 = u8_to_f(__ldg(b + c)), p11 = u8_to_f(__ldg(b + di + c));
        const float top = fmaf(fx, p01 - p00, p00), bot = fmaf(fx, p11 - p10, p10);
        s.b[c] = fmaf(fy, bot - top, top) * k255;
        s.bu[c] = cu ? 0.f : fmaf(fy, (p11 - p10) - (p01 - p00), p01 - p00) * k255;
        s.bv[c] = cv ? 0.f : (bot - top) * k255;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Canvas->camera parameters of one camera as doubles: a11..a32, gain (a33 comes from the rig).
struct BwCam {
    double a[9];  // a11 a12 a13 a21 a22 a23 a31 a32 a33
    float gain;
    int cx, cy;   // local origin
    int W, H;
};

__global__ void __launch_bounds__(BW_THREADS) k_backward(const CamDev* __restrict__ cams, FramePtrs fp,
                                                          const double* __restrict__ params,
                                                          const BwTile* __restrict__ tiles,
                                                          const int* __restrict__ camlist,
                                                          const int* __restrict__ centers, int canvas_w,
                                                          int canvas_h, float* __restrict__ partials,
                                                          float* __restrict__ loss_partials) {
    __shared__ TileMap tm[MAXC];
    __shared__ int cw[MAXC], chh[MAXC];
    __shared__ float cgain[MAXC];
    __shared__ int ccx[MAXC], ccy[MAXC], cid[MAXC];
    __shared__ float red[BW_THREADS / 32][BW_SLOTS * BW_NV + 1];

    const BwTile tl = tiles[blockIdx.x];
    const int n = tl.count;  // <= MAXC
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < n) {
        const int c = camlist[tl.first + t];
        const double* p = params + 9 * c;
        double A[9] = {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], cams[c].A[8]};
        // anchor at the tile origin clamped into the canvas; w > 0 there for every candidate is
        // not guaranteed, so anchor where w is largest among the tile corners
        int ax = tl.x0, ay = tl.y0;
        double best = -1e300;
        for (int k = 0; k < 4; ++k) {
            const int x = min(tl.x0 + (k & 1) * (BW_TX - 1), canvas_w - 1);
            const int y = min(tl.y0 + (k >> 1) * (BW_TY - 1), canvas_h - 1);
            const double w = A[6] * x + A[7] * y + A[8];
            if (w > best) {
                best = w;
                ax = x;
                ay = y;
            }
        }
        tm[t] = make_tile_map(A, ax, ay);
        // store the anchor in the tile map's frame: dx, dy are taken from (ax, ay)
        ccx[t] = ax;
        ccy[t] = ay;
        cid[t] = c;
        cw[t] = cams[c].W;
        chh[t] = cams[c].H;
        cgain[t] = (float)p[8];
    }
    __syncthreads();

    float loss = 0.f;
    for (int g0 = 0; g0 < max(n, 1); g0 += BW_SLOTS) {
        float acc[BW_SLOTS][BW_NV];
#pragma unroll
        for (int s = 0; s < BW_SLOTS; ++s)
#pragma unroll
            for (int v = 0; v < BW_NV; ++v) acc[s][v] = 0.f;
#pragma unroll
        for (int k = 0; k < BW_PPT; ++k) {
            const int q = t + k * BW_THREADS;
            const int x = tl.x0 + q % BW_TX, y = tl.y0 + q / BW_TX;
            if (x >= canvas_w || y >= canvas_h) continue;
            // pass 1: number of valid cameras and the sum of their intensities
            int kv = 0;
            float S[3] = {0.f, 0.f, 0.f};
            for (int a = 0; a < n; ++a) {
                GSample s;
                gsample(fp.p[cid[a]], fp.pitch[cid[a]], cw[a], chh[a], tm[a], (float)(x - ccx[a]),
                        (float)(y - ccy[a]), s);
                if (!s.valid) continue;
                ++kv;
#pragma unroll
                for (int c = 0; c < 3; ++c) S[c] = fmaf(cgain[a], s.b[c], S[c]);
            }
            if (kv < 2) continue;
            // pass 2: loss (first group only) and gradient terms of this group's cameras
            for (int a = 0; a < n; ++a) {
                GSample s;
                gsample(fp.p[cid[a]], fp.pitch[cid[a]], cw[a], chh[a], tm[a], (float)(x - ccx[a]),
                        (float)(y - ccy[a]), s);
                if (!s.valid) continue;
                const float g = cgain[a];
                float r[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) r[c] = (float)kv * (g * s.b[c]) - S[c];
                if (g0 == 0) {
                    // with the mean m = S/k, sum_{i<j} |I_i - I_j|^2 = k sum_i |I_i - m|^2
                    // = sum_i |r_i|^2 / k; r_i is small and accurate, so no cancellation
                    loss += (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) / (float)kv;
                }
                const int slot = a - g0;
                if (slot < 0 || slot >= BW_SLOTS) continue;
                const float gu = 2.f * g * (r[0] * s.bu[0] + r[1] * s.bu[1] + r[2] * s.bu[2]);
                const float gv = 2.f * g * (r[0] * s.bv[0] + r[1] * s.bv[1] + r[2] * s.bv[2]);
                const float gg = 2.f * (r[0] * s.b[0] + r[1] * s.b[1] + r[2] * s.b[2]);
                const float iw = 1.0f / s.w;
                const float xl = (float)(x - centers[2 * cid[a]]), yl = (float)(y - centers[2 * cid[a] + 1]);
                const float q = -(gu * s.u + gv * s.v) * iw;
                const float guw = gu * iw, gvw = gv * iw;
                // unrolled slot selection keeps the accumulators in registers
#pragma unroll
                for (int ss = 0; ss < BW_SLOTS; ++ss) {
                    if (ss != slot) continue;
                    acc[ss][0] = fmaf(guw, xl, acc[ss][0]);
                    acc[ss][1] = fmaf(guw, yl, acc[ss][1]);
                    acc[ss][2] += guw;
                    acc[ss][3] = fmaf(gvw, xl, acc[ss][3]);
                    acc[ss][4] = fmaf(gvw, yl, acc[ss][4]);
                    acc[ss][5] += gvw;
                    acc[ss][6] = fmaf(q, xl, acc[ss][6]);
                    acc[ss][7] = fmaf(q, yl, acc[ss][7]);
                    acc[ss][8] += q;
                    acc[ss][9] += gg;
                }
            }
        }
        // block reduction of this group's slots: warp shuffles, then a tree over warps
#pragma unroll
        for (int s = 0; s < BW_SLOTS; ++s)
#pragma unroll
            for (int v = 0; v < BW_NV; ++v) {
                const float w = warp_sum(acc[s][v]);
                if (lane == 0) red[warp][s * BW_NV + v] = w;
            }
        __syncthreads();
        if (t < BW_SLOTS * BW_NV) {
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < BW_THREADS / 32; ++w) sum += red[w][t];
            const int s = t / BW_NV, v = t - s * BW_NV;
            if (g0 + s < n) partials[(long long)(tl.first + g0 + s) * BW_NV + v] = sum;
        }
        __syncthreads();
    }
    const float lw = warp_sum(loss);
    if (lane == 0) red[warp][BW_SLOTS * BW_NV] = lw;
    __syncthreads();
    if (t == 0) {
        float sum = 0.f;
        for (int w = 0; w < BW_THREADS / 32; ++w) sum += red[w][BW_SLOTS * BW_NV];
        loss_partials[blockIdx.x] = sum;
    }
}

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated sum of (sum, compensation) pairs across a block.
__device__ __forceinline__ void block_csum(float& s, float& c, float* sh_s, float* sh_c) {
    sh_s[threadIdx.x] = s;
    sh_c[threadIdx.x] = c;
    __syncthreads();
    for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) {
            float ns, ne;
            two_sum(sh_s[threadIdx.x], sh_s[threadIdx.x + stride], ns, ne);
            sh_s[threadIdx.x] = ns;
            sh_c[threadIdx.x] += sh_c[threadIdx.x + stride] + ne;
        }
        __syncthreads();
    }
    s = sh_s[0];
    c = sh_c[0];
}

// One block per camera (blockIdx.x < ncam) and one for the loss (blockIdx.x == ncam).
__global__ void __launch_bounds__(256) k_backward_final(const CamDev* __restrict__ cams, int ncam,
                                                         const float* __restrict__ partials,
                                                         const float* __restrict__ loss_partials, int ntiles,
                                                         const int* __restrict__ cam_slots,
                                                         const int* __restrict__ cam_slot_start,
                                                         const int* __restrict__ centers, double* __restrict__ loss,
                                                         double* __restrict__ grad) {
    __shared__ float sh_s[256], sh_c[256];
    const int b = blockIdx.x;
    if (b == ncam) {
        float s = 0.f, c = 0.f;
        for (int k = threadIdx.x; k < ntiles; k += blockDim.x) {
            float ns, ne;
            two_sum(s, loss_partials[k], ns, ne);
            s = ns;
            c += ne;
        }
        block_csum(s, c, sh_s, sh_c);
        if (threadIdx.x == 0) *loss = (double)s + (double)c;
        return;
    }
    // the camera's BW_NV sums at once: each slot's values are read together (one index load, five
    // 8-byte loads); per value the order of the additions, and the tree, are those of block_csum
    __shared__ float ss[BW_NV][256], sc[BW_NV][256];
    double S[BW_NV];
    const int lo = cam_slot_start[b], hi = cam_slot_start[b + 1];
    float s[BW_NV], c[BW_NV];
#pragma unroll
    for (int v = 0; v < BW_NV; ++v) s[v] = c[v] = 0.f;
    static_assert(BW_NV % 2 == 0, "pairs of values per load");
#pragma unroll 2
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const float2* p = reinterpret_cast<const float2*>(partials + (long long)cam_slots[k] * BW_NV);
        float x[BW_NV];
#pragma unroll
        for (int v = 0; v < BW_NV / 2; ++v) {
            const float2 q = p[v];
            x[2 * v] = q.x;
            x[2 * v + 1] = q.y;
        }
#pragma unroll
        for (int v = 0; v < BW_NV; ++v) {
            float ns, ne;
            two_sum(s[v], x[v], ns, ne);
            s[v] = ns;
            c[v] += ne;
        }
    }
    const int t = threadIdx.x;
#pragma unroll
    for (int v = 0; v < BW_NV; ++v) {
        ss[v][t] = s[v];
        sc[v][t] = c[v];
    }
    __syncthreads();
    for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
        if (t < stride) {
#pragma unroll
            for (int v = 0; v < BW_NV; ++v) {
                float ns, ne;
                two_sum(ss[v][t], ss[v][t + stride], ns, ne);
                ss[v][t] = ns;
                sc[v][t] += sc[v][t + stride] + ne;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < BW_NV; ++v) S[v] = (double)ss[v][0] + (double)sc[v][0];
    if (threadIdx.x == 0 && grad) {
        const double cx = centers[2 * b], cy = centers[2 * b + 1];
        double* gr = grad + 9 * b;
        gr[0] = S[0] + cx * S[2];
        gr[1] = S[1] + cy * S[2];
        gr[2] = S[2];
        gr[3] = S[3] + cx * S[5];
        gr[4] = S[4] + cy * S[5];
        gr[5] = S[5];
        gr[6] = S[6] + cx * S[8];
        gr[7] = S[7] + cy * S[8];
        gr[8] = S[9];
    }
    (void)cams;
}

struct BwState {
    BwTile* tiles = nullptr;
    int ntiles = 0;
    int* camlist = nullptr;
    int* centers = nullptr;
    int* cam_slots = nullptr;
    int* cam_slot_start = nullptr;
    float* partials = nullptr;
    float* loss_partials = nullptr;
};

template <typename V>
stitch_status upload_bw(stitch_rig* r, const std::vector<V>& v, V** out) {
    *out = nullptr;
    if (v.empty()) return STITCH_OK;
    *out = (V*)rig_alloc(r, sizeof(V) * v.size());
    if (!*out) return STITCH_ENOMEM;
    STITCH_CUDA_TRY(cudaMemcpy(*out, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
    return STITCH_OK;
}

}  // namespace

// Candidate tiles: canvas tiles met by the footprint boxes (grown by BW_MARGIN px) of at least two
// cameras; parameters that move a footprint further than that leave pixels uncounted.
stitch_status backward_plan(stitch_rig* r) {
    const RigGeom& g = r->geom;
    BwState* bs = new (std::nothrow) BwState();
    if (!bs) return STITCH_ENOMEM;
    r->bw = bs;
    std::vector<BwTile> tiles;
    std::vector<int> camlist, centers(2 * g.ncam, 0);
    std::vector<std::vector<int>> slots(g.ncam);
    for (int i = 0; i < g.ncam; ++i) {
        const Rect v = r->hcam[i].V;
        centers[2 * i] = r->hcam[i].visible ? (v.x0 + v.x1) / 2 : 0;
        centers[2 * i + 1] = r->hcam[i].visible ? (v.y0 + v.y1) / 2 : 0;
    }
    const int Wc = g.nx[0], Hc = g.ny[0];
    for (int y0 = 0; y0 < Hc; y0 += BW_TY)
        for (int x0 = 0; x0 < Wc; x0 += BW_TX) {
            const int x1 = std::min(x0 + BW_TX, Wc), y1 = std::min(y0 + BW_TY, Hc);
            BwTile t{x0, y0, (int)camlist.size(), 0};
            for (int i = 0; i < g.ncam; ++i) {
                const CamDev& c = r->hcam[i];
                if (!c.visible) continue;
                const Rect v = c.V;
                if (v.x0 - BW_MARGIN < x1 && v.x1 + BW_MARGIN > x0 && v.y0 - BW_MARGIN < y1 && v.y1 + BW_MARGIN > y0) {
                    camlist.push_back(i);
                    ++t.count;
                }
            }
            if (t.count < 2) {
                camlist.resize(t.first);
                continue;
            }
            for (int k = 0; k < t.count; ++k) slots[camlist[t.first + k]].push_back(t.first + k);
            tiles.push_back(t);
        }
    std::vector<int> cam_slots, start(g.ncam + 1, 0);
    for (int i = 0; i < g.ncam; ++i) {
        start[i] = (int)cam_slots.size();
        cam_slots.insert(cam_slots.end(), slots[i].begin(), slots[i].end());
    }
    start[g.ncam] = (int)cam_slots.size();
    stitch_status st;
    if ((st = upload_bw(r, tiles, &bs->tiles)) != STITCH_OK) return st;
    if ((st = upload_bw(r, camlist, &bs->camlist)) != STITCH_OK) return st;
    if ((st = upload_bw(r, centers, &bs->centers)) != STITCH_OK) return st;
    if ((st = upload_bw(r, cam_slots, &bs->cam_slots)) != STITCH_OK) return st;
    if ((st = upload_bw(r, start, &bs->cam_slot_start)) != STITCH_OK) return st;
    bs->ntiles = (int)tiles.size();
    bs->partials = (float*)rig_alloc(r, sizeof(float) * BW_NV * std::max<size_t>(camlist.size(), 1));
    bs->loss_partials = (float*)rig_alloc(r, sizeof(float) * std::max(bs->ntiles, 1));
    if (!bs->partials || !bs->loss_partials) return STITCH_ENOMEM;
    return STITCH_OK;
}

stitch_status backward_run(stitch_rig* r, const FramePtrs& fp, const double* params, double* loss, double* grad,
                           cudaStream_t s) {
    BwState* bs = (BwState*)r->bw;
    if (!bs) return STITCH_EINVAL;
    const RigGeom& g = r->geom;
    if (bs->ntiles > 0) {
        prof_mark(r, "backward", s);
        k_backward<<<bs->ntiles, BW_THREADS, 0, s>>>(r->dcam, fp, params, bs->tiles, bs->camlist, bs->centers, g.nx[0],
                                                    g.ny[0], bs->partials, bs->loss_partials);
    }
    prof_mark(r, "backward_final", s);
    k_backward_final<<<g.ncam + 1, 256, 0, s>>>(r->dcam, g.ncam, bs->partials, bs->loss_partials, bs->ntiles,
                                                bs->cam_slots, bs->cam_slot_start, bs->centers, loss, grad);
    return launch_status();
}

void backward_release(stitch_rig* r) {
    delete (BwState*)r->bw;
    r->bw = nullptr;
}
