// Plain path: one kernel per step of the stitching definition (Algorithm 4, step 6, with the
// multi-band fusion of Sec. 1), FP32 intermediates in HBM.
// It is the comparison path for the fused implementation and follows the steps literally:
//   warp+weights (S1, S2) -> REDUCE per level (S3) -> Laplacian per level (S4)
//   -> per-level normalised blend on the canvas grid (S5) -> collapse + output (S6).
#include "stitch_internal.cuh"

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }

// S1 + S2: level 0 of camera i on Om[0]: (I_i rgb, What_i).
__global__ void __launch_bounds__(BX* BY) k_plain_warp(const CamDev* __restrict__ cams, int ncam, int i,
                                                        FramePtrs fp, const __grid_constant__ RigGeom g) {
    __shared__ TileMap tm[MAXC];
    __shared__ int act[MAXC];
    __shared__ int ax[MAXC], ay[MAXC];
    const CamDev& ci = cams[i];
    const Rect om = ci.Om[0];
    const int X = om.x0 + blockIdx.x * BX, Y = om.y0 + blockIdx.y * BY;
    const int t = threadIdx.y * BX + threadIdx.x;
    if (t < ncam) {
        const CamDev& cj = cams[t];
        const Rect v = cj.V;
        // camera t matters for this block if it is camera i or its validity box meets the block
        const int a = cj.visible && (t == i || (v.x0 < X + BX && v.x1 > X && v.y0 < Y + BY && v.y1 > Y));
        act[t] = a;
        if (a) {
            int px, py;
            tile_anchor(v, X, Y, &px, &py);
            ax[t] = px;
            ay[t] = py;
            tm[t] = make_tile_map(cj.A, px, py);
        }
    }
    __syncthreads();
    const int x = X + threadIdx.x, y = Y + threadIdx.y;
    if (x >= om.x1 || y >= om.y1) return;
    float3 rgb = make_float3(0.f, 0.f, 0.f);
    float wi = 0.f, ws = 0.f;
    // seam weights: the pixel's owner among all cameras (FP64 decision)
    const int own = g.seam ? seam_owner(g, ncam, [&](int k) -> const CamDev& { return cams[k]; }, x, y) : -1;
    for (int j = 0; j < ncam; ++j) {
        if (!act[j]) continue;
        const CamDev& cj = cams[j];
        const SrcPos s = g.cyl ? map_point64(cj, g, x, y) : map_point(tm[j], (float)(x - ax[j]), (float)(y - ay[j]));
        const float w = g.seam ? (own == j ? 1.f : 0.f) : (cj.V.contains(x, y) ? feather_weight(s, cj.W, cj.H) : 0.f);
        ws += w;
        if (j == i) {
            wi = w;
            rgb = bilinear_rgb(fp.p[i], fp.pitch[i], clamp_tap(s, cj.W, cj.H), cj.gain * (1.0f / 255.0f));
        }
    }
    const float what = ws > 0.f ? wi / ws : 0.f;
    ci.G[0][(long long)(y - om.y0) * om.w() + (x - om.x0)] = make_float4(rgb.x, rgb.y, rgb.z, what);
}

// S3: G^{l+1} = REDUCE(G^l) on Om[l+1] (all four channels), 25 taps read straight from HBM/L2.
__global__ void __launch_bounds__(BX* BY) k_plain_reduce(const CamDev* __restrict__ cams, int i, int l, RigGeom g) {
    const CamDev& c = cams[i];
    const Rect oc = c.Om[l + 1], of = c.Om[l];
    const int k = oc.x0 + blockIdx.x * BX + threadIdx.x, j = oc.y0 + blockIdx.y * BY + threadIdx.y;
    if (k >= oc.x1 || j >= oc.y1) return;
    const float w5[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
    const float4* src = c.G[l];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int n = -2; n <= 2; ++n) {
        const int yy = fold101(2 * j + n, g.ny[l]) - of.y0;
        float4 row = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m = -2; m <= 2; ++m) {
            const int xx = fold101(2 * k + m, g.nx[l]) - of.x0;
            const float4 v = ld4(src + (long long)yy * of.w() + xx);
            const float wm = w5[m + 2];
            row.x = fmaf(wm, v.x, row.x);
            row.y = fmaf(wm, v.y, row.y);
            row.z = fmaf(wm, v.z, row.z);
            row.w = fmaf(wm, v.w, row.w);
        }
        const float wn = w5[n + 2];
        acc.x = fmaf(wn, row.x, acc.x);
        acc.y = fmaf(wn, row.y, acc.y);
        acc.z = fmaf(wn, row.z, acc.z);
        acc.w = fmaf(wn, row.w, acc.w);
    }
    c.G[l + 1][(long long)(j - oc.y0) * oc.w() + (k - oc.x0)] = acc;
}

// EXPAND of a coarse buffer (rect r of a level of size nxc x nyc) at fine (x, y), rgb only.
__device__ __forceinline__ float3 expand_rgb(const float4* __restrict__ buf, const Rect& r, int nxc, int nyc, int x,
                                             int y) {
    int jy[3], kx[3];
    float wy[3], wx[3];
    int ny_, nx_;
    if ((y & 1) == 0) {
        jy[0] = y / 2 - 1; jy[1] = y / 2; jy[2] = y / 2 + 1;
        wy[0] = 0.125f; wy[1] = 0.75f; wy[2] = 0.125f;
        ny_ = 3;
    } else {
        jy[0] = (y - 1) / 2; jy[1] = (y + 1) / 2;
        wy[0] = 0.5f; wy[1] = 0.5f;
        ny_ = 2;
    }
    if ((x & 1) == 0) {
        kx[0] = x / 2 - 1; kx[1] = x / 2; kx[2] = x / 2 + 1;
        wx[0] = 0.125f; wx[1] = 0.75f; wx[2] = 0.125f;
        nx_ = 3;
    } else {
        kx[0] = (x - 1) / 2; kx[1] = (x + 1) / 2;
        wx[0] = 0.5f; wx[1] = 0.5f;
        nx_ = 2;
    }
    float3 acc = make_float3(0.f, 0.f, 0.f);
    for (int a = 0; a < ny_; ++a) {
        const int yy = fold101(jy[a], nyc) - r.y0;
        float3 row = make_float3(0.f, 0.f, 0.f);
        for (int b = 0; b < nx_; ++b) {
            const int xx = fold101(kx[b], nxc) - r.x0;
            const float4 v = ld4(buf + (long long)yy * r.w() + xx);
            row.x = fmaf(wx[b], v.x, row.x);
            row.y = fmaf(wx[b], v.y, row.y);
            row.z = fmaf(wx[b], v.z, row.z);
        }
        acc.x = fmaf(wy[a], row.x, acc.x);
        acc.y = fmaf(wy[a], row.y, acc.y);
        acc.z = fmaf(wy[a], row.z, acc.z);
    }
    return acc;
}

// S4: (L^l rgb, G^l weight) on Z[l], l < L-1.
__global__ void __launch_bounds__(BX* BY) k_plain_laplacian(const CamDev* __restrict__ cams, int i, int l, RigGeom g) {
    const CamDev& c = cams[i];
    const Rect z = c.Z[l], o = c.Om[l], oc = c.Om[l + 1];
    const int x = z.x0 + blockIdx.x * BX + threadIdx.x, y = z.y0 + blockIdx.y * BY + threadIdx.y;
    if (x >= z.x1 || y >= z.y1) return;
    const float4 gv = ld4(c.G[l] + (long long)(y - o.y0) * o.w() + (x - o.x0));
    const float3 e = expand_rgb(c.G[l + 1], oc, g.nx[l + 1], g.ny[l + 1], x, y);
    c.Lp[l][(long long)(y - z.y0) * z.w() + (x - z.x0)] = make_float4(gv.x - e.x, gv.y - e.y, gv.z - e.z, gv.w);
}

// S5: B^l = sum_i G^l(What_i) L^l_i / S^l on the whole level grid; .w keeps S^l > 0 (coverage).
__global__ void __launch_bounds__(BX* BY) k_plain_blend(const CamDev* __restrict__ cams, int l, RigGeom g,
                                                         float4* __restrict__ B) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= g.nx[l] || y >= g.ny[l]) return;
    const bool top = l == g.levels - 1;
    float nr = 0.f, ng = 0.f, nb = 0.f, s = 0.f;
    for (int i = 0; i < g.ncam; ++i) {
        const CamDev& c = cams[i];
        if (!c.visible) continue;
        const Rect z = c.Z[l];
        if (!z.contains(x, y)) continue;
        float4 v;
        if (top) {
            const Rect o = c.Om[l];
            v = ld4(c.G[l] + (long long)(y - o.y0) * o.w() + (x - o.x0));
        } else {
            v = ld4(c.Lp[l] + (long long)(y - z.y0) * z.w() + (x - z.x0));
        }
        nr = fmaf(v.w, v.x, nr);
        ng = fmaf(v.w, v.y, ng);
        nb = fmaf(v.w, v.z, nb);
        s += v.w;
    }
    float4 out = make_float4(0.f, 0.f, 0.f, s > 0.f ? 1.f : 0.f);
    if (s > 1e-12f) {
        out.x = nr / s;
        out.y = ng / s;
        out.z = nb / s;
    }
    B[(long long)y * g.nx[l] + x] = out;
}

// S6: R^l = B^l + EXPAND(R^{l+1}) in place for l >= 1; at level 0 mask, clamp and write out.
__global__ void __launch_bounds__(BX* BY) k_plain_collapse(int l, RigGeom g, float4* __restrict__ Bl,
                                                            const float4* __restrict__ Rc, OutDesc od) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= g.nx[l] || y >= g.ny[l]) return;
    float4 b = Bl[(long long)y * g.nx[l] + x];
    if (Rc) {
        const Rect rc{0, g.nx[l + 1], 0, g.ny[l + 1]};
        const float3 e = expand_rgb(Rc, rc, g.nx[l + 1], g.ny[l + 1], x, y);
        b.x += e.x;
        b.y += e.y;
        b.z += e.z;
    }
    if (l > 0) {
        Bl[(long long)y * g.nx[l] + x] = b;
        return;
    }
    const bool cov = b.w > 0.f;
    const float r = cov ? __saturatef(b.x) : 0.f, gg = cov ? __saturatef(b.y) : 0.f, bb = cov ? __saturatef(b.z) : 0.f;
    if (od.is_float) {
        float* o = (float*)((char*)od.ptr + (long long)y * od.pitch) + 3 * x;
        o[0] = r;
        o[1] = gg;
        o[2] = bb;
    } else {
        unsigned char* o = (unsigned char*)od.ptr + (long long)y * od.pitch + 3 * x;
        o[0] = quantize_u8(r);
        o[1] = quantize_u8(gg);
        o[2] = quantize_u8(bb);
    }
}

dim3 grid_for(const Rect& r) { return dim3((r.w() + BX - 1) / BX, (r.h() + BY - 1) / BY); }

bool launchable(const Rect& r) { return !r.empty(); }

}  // namespace

stitch_status plain_plan(stitch_rig* r) {
    const RigGeom& g = r->geom;
    int kernels = 0;
    for (int i = 0; i < g.ncam; ++i) {
        CamDev& c = r->hcam[i];
        if (!c.visible) continue;
        for (int l = 0; l < g.levels; ++l) {
            c.G[l] = (float4*)rig_alloc(r, sizeof(float4) * (size_t)c.Om[l].area());
            if (!c.G[l]) return STITCH_ENOMEM;
            if (l + 1 < g.levels) {
                c.Lp[l] = (float4*)rig_alloc(r, sizeof(float4) * (size_t)c.Z[l].area());
                if (!c.Lp[l]) return STITCH_ENOMEM;
            }
        }
        kernels += 1 + 2 * (g.levels - 1);
    }
    for (int l = 0; l < g.levels; ++l) {
        r->Bl[l] = (float4*)rig_alloc(r, sizeof(float4) * (size_t)g.nx[l] * g.ny[l]);
        if (!r->Bl[l]) return STITCH_ENOMEM;
    }
    kernels += g.levels + (g.levels > 1 ? g.levels - 1 : 1);
    r->kernels_per_frame = kernels;
    return STITCH_OK;
}

stitch_status plain_frames(stitch_rig* r, const FramePtrs& fp, const OutDesc& od, cudaStream_t s) {
    const RigGeom& g = r->geom;
    const dim3 blk(BX, BY);
    for (int i = 0; i < g.ncam; ++i) {
        if (!r->hcam[i].visible || !launchable(r->hcam[i].Om[0])) continue;
        prof_mark(r, "plain_warp", s);
        k_plain_warp<<<grid_for(r->hcam[i].Om[0]), blk, 0, s>>>(r->dcam, g.ncam, i, fp, g);
    }
    for (int i = 0; i < g.ncam; ++i) {
        if (!r->hcam[i].visible) continue;
        for (int l = 0; l + 1 < g.levels; ++l) {
            if (!launchable(r->hcam[i].Om[l + 1])) continue;
            prof_mark(r, "plain_reduce", s);
            k_plain_reduce<<<grid_for(r->hcam[i].Om[l + 1]), blk, 0, s>>>(r->dcam, i, l, g);
        }
    }
    for (int i = 0; i < g.ncam; ++i) {
        if (!r->hcam[i].visible) continue;
        for (int l = 0; l + 1 < g.levels; ++l) {
            if (!launchable(r->hcam[i].Z[l])) continue;
            prof_mark(r, "plain_laplacian", s);
            k_plain_laplacian<<<grid_for(r->hcam[i].Z[l]), blk, 0, s>>>(r->dcam, i, l, g);
        }
    }
    for (int l = 0; l < g.levels; ++l) {
        prof_mark(r, "plain_blend", s);
        k_plain_blend<<<grid_for(Rect{0, g.nx[l], 0, g.ny[l]}), blk, 0, s>>>(r->dcam, l, g, r->Bl[l]);
    }
    if (g.levels == 1) {
        prof_mark(r, "plain_collapse", s);
        k_plain_collapse<<<grid_for(Rect{0, g.nx[0], 0, g.ny[0]}), blk, 0, s>>>(0, g, r->Bl[0], nullptr, od);
    }
    for (int l = g.levels - 2; l >= 0; --l) {
        prof_mark(r, "plain_collapse", s);
        k_plain_collapse<<<grid_for(Rect{0, g.nx[l], 0, g.ny[l]}), blk, 0, s>>>(l, g, r->Bl[l], r->Bl[l + 1], od);
    }
    return launch_status();
}
