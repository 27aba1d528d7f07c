// libstitch host side: rig validation and planning, buffer ownership, C-ABI entry points,
// host staging and per-kernel profiling.  Every buffer the per-frame path needs is allocated when
// the rig is created, the counterpart of the paper's start-up preallocation (Sec. 4.3.2).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "stitch_internal.cuh"

namespace {

bool invert_normalised(const double* M, double* A) {
    const double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], k = M[8];
    const double c00 = e * k - f * h, c01 = f * g - d * k, c02 = d * h - e * g;
    const double det = a * c00 + b * c01 + c * c02;
    if (!(fabs(det) > 0.0) || !std::isfinite(det)) return false;
    double inv[9] = {c00, c * h - b * k, b * f - c * e, c01, a * k - c * g, c * d - a * f, c02, b * g - a * h,
                     a * e - b * d};
    for (double& v : inv) v /= det;
    // scale by the positive factor 1/|a33|: the third component of A x stays 1/w_c(p) up to that
    // factor, positive exactly for canvas points whose camera point p is in front (a33 = -1 when
    // the canvas origin lies behind the camera)
    const double s = fabs(inv[8]);
    if (!(s > 0.0)) return false;
    for (int i = 0; i < 9; ++i) A[i] = inv[i] / s;
    A[8] = inv[8] > 0.0 ? 1.0 : -1.0;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(A[i])) return false;
    return true;
}

}  // namespace

// Validate one camera and plan its regions (validity box V, weight support Z^l, pyramid region
// Omega^l).  Adds the camera's level-0 region area to *roi.
// Footprint on the cylindrical canvas of camera P's pixel-edge rectangle: its border, sampled
// every 0.25 px, mapped through the rays P^-1 (u, v, 1).  False when a border ray points along
// the axis or the border crosses the back of the cylinder (the footprint would wrap around).
static bool cylinder_footprint(const stitch_camera& c, const RigGeom& g, double* xmin, double* xmax, double* ymin,
                               double* ymax) {
    // P^-1 (adjugate over the determinant)
    const double* M = c.H;
    const double a = M[0], b = M[1], cc = M[2], d = M[3], e = M[4], f = M[5], gg = M[6], h = M[7], k = M[8];
    const double det = a * (e * k - f * h) + b * (f * gg - d * k) + cc * (d * h - e * gg);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    const double Pi[9] = {(e * k - f * h) / det,  (cc * h - b * k) / det, (b * f - cc * e) / det,
                          (f * gg - d * k) / det, (a * k - cc * gg) / det, (cc * d - a * f) / det,
                          (d * h - e * gg) / det, (b * gg - a * h) / det, (a * e - b * d) / det};
    const double W = c.width, H = c.height;
    const long long nu = (long long)std::ceil(W * 4.0), nv = (long long)std::ceil(H * 4.0);
    double tprev = 0.0;
    bool first = true;
    *xmin = *ymin = 1e300;
    *xmax = *ymax = -1e300;
    for (int side = 0; side < 4; ++side) {
        const long long n = (side % 2 == 0) ? nu : nv;
        for (long long k = 0; k <= n; ++k) {
            const double s = (double)k / (double)n;
            double u, v;
            if (side == 0) { u = -0.5 + s * W; v = -0.5; }
            else if (side == 1) { u = W - 0.5; v = -0.5 + s * H; }
            else if (side == 2) { u = W - 0.5 - s * W; v = H - 0.5; }
            else { u = -0.5; v = H - 0.5 - s * H; }
            double r[3];
            // P r = (u, v, 1): in front of the camera
            for (int i = 0; i < 3; ++i) r[i] = Pi[3 * i] * u + Pi[3 * i + 1] * v + Pi[3 * i + 2];
            const double rxz = std::hypot(r[0], r[2]);
            if (!(rxz > 0.0)) return false;
            const double t = std::atan2(r[0], r[2]);
            if (!first && std::fabs(t - tprev) > 1.0) return false;
            first = false;
            tprev = t;
            const double x = g.ccx + g.cf * t, y = g.ccy + g.cf * r[1] / rxz;
            *xmin = std::min(*xmin, x);
            *xmax = std::max(*xmax, x);
            *ymin = std::min(*ymin, y);
            *ymax = std::max(*ymax, y);
        }
    }
    return true;
}

stitch_status plan_camera_geometry(const stitch_camera& c, const RigGeom& g, CamDev& d, long long* roi) {
    memset(&d, 0, sizeof(d));
    const int L = g.levels, Wc = g.nx[0], Hc = g.ny[0];
    if (c.width < 1 || c.height < 1 || !std::isfinite(c.gain)) return STITCH_EINVAL;
    for (double v : c.H)
        if (!std::isfinite(v)) return STITCH_EINVAL;
    if (g.cyl) {
        for (int i = 0; i < 9; ++i) d.A[i] = c.H[i];  // P acts on the canvas ray as given
    } else if (!invert_normalised(c.H, d.A)) {
        return STITCH_EINVAL;
    }
    d.W = c.width;
    d.H = c.height;
    d.gain = c.gain;

    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, margin = 1.0;
    if (g.cyl) {
        if (!cylinder_footprint(c, g, &xmin, &xmax, &ymin, &ymax)) return STITCH_EINVAL;
        margin = 2.0;  // the border is sampled, not mapped exactly
    } else {
        // footprint of the validity rectangle: image of its corners under H (must stay in front)
        const double cu[4] = {-0.5, c.width - 0.5, -0.5, c.width - 0.5};
        const double cv[4] = {-0.5, -0.5, c.height - 0.5, c.height - 0.5};
        for (int k = 0; k < 4; ++k) {
            const double X = c.H[0] * cu[k] + c.H[1] * cv[k] + c.H[2];
            const double Y = c.H[3] * cu[k] + c.H[4] * cv[k] + c.H[5];
            const double Wh = c.H[6] * cu[k] + c.H[7] * cv[k] + c.H[8];
            // the corner must be in front of the camera for the footprint to be a bounded quad
            if (!(Wh > 0.0)) return STITCH_EINVAL;
            xmin = std::min(xmin, X / Wh);
            xmax = std::max(xmax, X / Wh);
            ymin = std::min(ymin, Y / Wh);
            ymax = std::max(ymax, Y / Wh);
        }
    }
    // a margin beyond the footprint so single-precision evaluation near its edge is still inside
    // the box (outside the box the camera's weight is exactly zero)
    const double bx0 = std::max(0.0, floor(xmin) - margin), bx1 = std::min((double)Wc, ceil(xmax) + margin + 1.0);
    const double by0 = std::max(0.0, floor(ymin) - margin), by1 = std::min((double)Hc, ceil(ymax) + margin + 1.0);
    if (bx1 <= bx0 || by1 <= by0) {
        d.visible = 0;
        return STITCH_OK;
    }
    d.visible = 1;
    Span zx[MAXL], zy[MAXL];
    zx[0] = {(int)bx0, (int)bx1};
    zy[0] = {(int)by0, (int)by1};
    d.V = make_rect(zx[0], zy[0]);
    for (int l = 0; l + 1 < L; ++l) {
        zx[l + 1] = reduce_touch(zx[l], g.nx[l], g.nx[l + 1]);
        zy[l + 1] = reduce_touch(zy[l], g.ny[l], g.ny[l + 1]);
    }
    // Omega: everything the bands on Z depend on
    Span ox[MAXL], oy[MAXL];
    for (int l = L - 1; l >= 0; --l) {
        ox[l] = zx[l];
        oy[l] = zy[l];
        if (l >= 1) {
            ox[l] = span_union(ox[l], expand_reads(zx[l - 1], g.nx[l]));
            oy[l] = span_union(oy[l], expand_reads(zy[l - 1], g.ny[l]));
        }
        if (l + 1 < L) {
            ox[l] = span_union(ox[l], reduce_reads(ox[l + 1], g.nx[l]));
            oy[l] = span_union(oy[l], reduce_reads(oy[l + 1], g.ny[l]));
        }
    }
    for (int l = 0; l < L; ++l) {
        d.Z[l] = make_rect(zx[l], zy[l]);
        d.Om[l] = make_rect(ox[l], oy[l]);
    }
    // the camera must be in front (w > 0) everywhere its level-0 values are evaluated: w is affine
    // in (x, y) on the planar canvas (corners decide) and affine in y on every column of the
    // cylindrical one (the top and bottom rows of every column decide)
    const Rect& o = d.Om[0];
    const double qy[2] = {(double)o.y0, (double)(o.y1 - 1)};
    const int step = g.cyl ? 1 : std::max(1, o.x1 - 1 - o.x0);
    for (int xi = o.x0; xi < o.x1; xi += step) {
        for (int pass = 0; pass < 2; ++pass) {
            const double x = pass == 0 ? (double)xi : (double)(o.x1 - 1);
            for (double y : qy) {
                double u, v;
                if (!(source_point64(d, g, x, y, &u, &v) > 0.0)) return STITCH_EINVAL;
            }
        }
    }
    *roi += o.area();
    return STITCH_OK;
}

namespace {

stitch_status plan_camera(stitch_rig* r, int i) {
    return plan_camera_geometry(r->cams[i], r->geom, r->hcam[i], &r->roi_pixels);
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void free_all(stitch_rig* r) {
    for (void* p : r->allocs) cudaFree(p);
    r->allocs.clear();
    for (int i = 0; i < MAXC; ++i)
        if (r->stage_frames[i]) cudaFree(r->stage_frames[i]);
    if (r->stage_out) cudaFree(r->stage_out);
    for (cudaEvent_t e : r->ev_pool) cudaEventDestroy(e);
    r->ev_pool.clear();
}

bool frames_ok(const stitch_rig* r, const uint8_t* const* frames, const int64_t* pitches, FramePtrs* fp) {
    if (!frames || !pitches) return false;
    memset(fp, 0, sizeof(*fp));
    for (int i = 0; i < r->geom.ncam; ++i) {
        if (!r->hcam[i].visible) continue;
        if (!frames[i] || pitches[i] < 3LL * r->cams[i].width) return false;
        fp->p[i] = frames[i];
        fp->pitch[i] = pitches[i];
    }
    return true;
}

}  // namespace

// ------------------------------------------------------------------------------------------------

#ifdef STITCH_DEBUG
namespace {
__global__ void k_guard_fill(uint32_t* p, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        p[k] = kGuardWord;
}
__global__ void k_guard_check(const uint32_t* p, size_t n, unsigned long long* damaged) {
    unsigned long long bad = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        bad += p[k] != kGuardWord;
    if (bad) atomicAdd(damaged, bad);
}
}  // namespace
#endif

// Device allocation owned by the rig.  The debug build puts a guard band of kGuardBytes before and
// after it (the allocation rounded up to 16 bytes), filled with a NaN word and checked by
// stitch_rig_debug_check.
void* rig_alloc(stitch_rig* r, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
#ifdef STITCH_DEBUG
    const size_t body = (bytes + 15) & ~(size_t)15;
    if (cudaMalloc(&p, body + 2 * kGuardBytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    r->allocs.push_back(p);
    uint32_t* lo = (uint32_t*)p;
    uint32_t* hi = (uint32_t*)((char*)p + kGuardBytes + body);
    for (uint32_t* gp : {lo, hi}) {
        k_guard_fill<<<1, 64>>>(gp, kGuardBytes / 4);
        r->guards.push_back({gp, kGuardBytes / 4});
    }
    r->scratch_bytes += (long long)bytes;
    return (char*)p + kGuardBytes;
#else
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    r->allocs.push_back(p);
    r->scratch_bytes += (long long)bytes;
    return p;
#endif
}

void prof_mark(stitch_rig* r, const char* name, cudaStream_t s) {
    if (!r->prof) return;
    if (r->ev_used == r->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            r->prof = false;
            return;
        }
        r->ev_pool.push_back(e);
    }
    cudaEvent_t e = r->ev_pool[r->ev_used++];
    cudaEventRecord(e, s);
    r->marks.push_back({name, e});
}

extern "C" {

const char* stitch_status_string(stitch_status s) {
    switch (s) {
        case STITCH_OK: return "STITCH_OK";
        case STITCH_EINVAL: return "STITCH_EINVAL: invalid argument or geometry";
        case STITCH_ENOMEM: return "STITCH_ENOMEM: allocation failed";
        case STITCH_ECUDA: return "STITCH_ECUDA: CUDA error";
        case STITCH_ETIMEOUT: return "STITCH_ETIMEOUT: bounded device wait gave up";
        case STITCH_EUNSUPPORTED: return "STITCH_EUNSUPPORTED: not supported by this build";
        case STITCH_ETOOLARGE: return "STITCH_ETOOLARGE: request exceeds the static scratch array";
    }
    return "unknown stitch_status";
}

stitch_status stitch_rig_create(const stitch_rig_desc* desc, int device, stitch_rig** out) {
    if (!out) return STITCH_EINVAL;
    *out = nullptr;
    if (!desc || !desc->cameras || desc->num_cameras < 1 || desc->num_cameras > MAXC || desc->canvas_w < 1 ||
        desc->canvas_h < 1 || desc->levels < 1 || desc->levels > MAXL || desc->canvas_w > (1 << 28) ||
        desc->canvas_h > (1 << 28) || (desc->band_fp16 != 0 && desc->band_fp16 != 1) ||
        (desc->out_float != 0 && desc->out_float != 1) ||
        (desc->path != STITCH_PATH_FUSED && desc->path != STITCH_PATH_PLAIN) ||
        (desc->weights != STITCH_WEIGHTS_FEATHER && desc->weights != STITCH_WEIGHTS_SEAM) ||
        (desc->canvas_model != STITCH_CANVAS_PLANAR && desc->canvas_model != STITCH_CANVAS_CYLINDRICAL) ||
        (desc->canvas_model == STITCH_CANVAS_CYLINDRICAL &&
         !(std::isfinite(desc->cylinder[0]) && desc->cylinder[0] > 0.0 && std::isfinite(desc->cylinder[1]) &&
           std::isfinite(desc->cylinder[2]))))
        return STITCH_EINVAL;
    if ((long long)desc->canvas_w * desc->canvas_h > (1LL << 31)) return STITCH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return STITCH_ECUDA;
    }
    if (device < 0 || device >= ndev) return STITCH_EINVAL;
    DeviceGuard dg(device);  // the caller's current device is restored on return
    if (!dg.ok) return STITCH_ECUDA;

    stitch_rig* r = new (std::nothrow) stitch_rig();
    if (!r) return STITCH_ENOMEM;
    r->device = device;
    r->desc = *desc;
    r->cams.assign(desc->cameras, desc->cameras + desc->num_cameras);
    r->desc.cameras = nullptr;
    RigGeom& g = r->geom;
    g.ncam = desc->num_cameras;
    g.levels = desc->levels;
    g.seam = desc->weights == STITCH_WEIGHTS_SEAM;
    g.cyl = desc->canvas_model == STITCH_CANVAS_CYLINDRICAL;
    g.cf = g.cyl ? desc->cylinder[0] : 0.0;
    g.ccx = g.cyl ? desc->cylinder[1] : 0.0;
    g.ccy = g.cyl ? desc->cylinder[2] : 0.0;
    g.nx[0] = desc->canvas_w;
    g.ny[0] = desc->canvas_h;
    for (int l = 1; l < g.levels; ++l) {
        g.nx[l] = (g.nx[l - 1] + 1) / 2;
        g.ny[l] = (g.ny[l - 1] + 1) / 2;
    }
    stitch_status st = STITCH_OK;
    for (int i = 0; i < g.ncam && st == STITCH_OK; ++i) st = plan_camera(r, i);
    if (st == STITCH_OK && desc->path == STITCH_PATH_PLAIN && desc->band_fp16) st = STITCH_EUNSUPPORTED;
    if (st == STITCH_OK) st = desc->path == STITCH_PATH_PLAIN ? plain_plan(r) : fused_plan(r);
    if (st == STITCH_OK) st = backward_plan(r);
    if (st == STITCH_OK) {
        r->dcam = (CamDev*)rig_alloc(r, sizeof(CamDev) * g.ncam);
        if (!r->dcam) st = STITCH_ENOMEM;
    }
    if (st == STITCH_OK && cudaMemcpy(r->dcam, r->hcam, sizeof(CamDev) * g.ncam, cudaMemcpyHostToDevice) != cudaSuccess)
        st = STITCH_ECUDA;
    if (st == STITCH_OK && desc->path != STITCH_PATH_PLAIN) st = fused_precompute(r);
    if (st != STITCH_OK) {
        fused_release(r);
        backward_release(r);
        free_all(r);
        delete r;
        return st;
    }
    *out = r;
    return STITCH_OK;
}

void stitch_rig_destroy(stitch_rig* r) {
    if (!r) return;
    DeviceGuard dg(r->device);
    cudaDeviceSynchronize();
    pipeline_release(r);
    fused_release(r);
    backward_release(r);
    free_all(r);
    delete r;
}

stitch_status stitch_rig_debug_check(stitch_rig* r, int64_t* damaged_words, int64_t* failed_check) {
    if (!r || !damaged_words || !failed_check) return STITCH_EINVAL;
    *damaged_words = 0;
    *failed_check = 0;
#ifdef STITCH_DEBUG
    DeviceGuard dg(r->device);
    if (!dg.ok) return STITCH_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return STITCH_ECUDA;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return STITCH_ECUDA;
    unsigned long long h = 0;
    stitch_status st = cudaMemset(d, 0, sizeof(*d)) == cudaSuccess ? STITCH_OK : STITCH_ECUDA;
    for (const auto& gd : r->guards)
        if (st == STITCH_OK) k_guard_check<<<1, 64>>>(gd.first, gd.second, d);
    if (st == STITCH_OK && cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) st = STITCH_ECUDA;
    cudaFree(d);
    *damaged_words = (int64_t)h;
    *failed_check = fused_debug_take(r->device);
    return st;
#else
    return STITCH_EUNSUPPORTED;
#endif
}

stitch_status stitch_rig_get_info(const stitch_rig* r, stitch_rig_info* info) {
    if (!r || !info) return STITCH_EINVAL;
    info->scratch_bytes = r->scratch_bytes;
    info->num_kernels = r->kernels_per_frame;
    info->path = r->desc.path;
    info->roi_pixels = r->roi_pixels;
    int tc[8];
    fused_tile_counts(r, tc);
    info->tiles_zero = tc[0];
    info->tiles_solo = tc[1];
    info->tiles_full2 = tc[2];
    info->tiles_full4 = tc[3];
    info->tiles_general = tc[4];
    info->tiles_down1 = tc[5];
    info->tiles_down1_staged = tc[6];
    info->tiles_down1_interior = tc[7];
    return STITCH_OK;
}

stitch_status stitch_rig_get_camera(const stitch_rig* r, int32_t index, double* a, int32_t* visible) {
    if (!r || !a || index < 0 || index >= r->geom.ncam) return STITCH_EINVAL;
    for (int k = 0; k < 9; ++k) a[k] = r->hcam[index].A[k];
    if (visible) *visible = r->hcam[index].visible;
    return STITCH_OK;
}

stitch_status stitch_frames(stitch_rig* r, const uint8_t* const* frames, const int64_t* pitches, void* out,
                            int64_t out_pitch, void* stream) {
    if (!r || !out) return STITCH_EINVAL;
    const long long row = (long long)r->geom.nx[0] * (r->desc.out_float ? 12 : 3);
    if (out_pitch < row) return STITCH_EINVAL;
    FramePtrs fp;
    if (!frames_ok(r, frames, pitches, &fp)) return STITCH_EINVAL;
    DeviceGuard dg(r->device);
    if (!dg.ok) return STITCH_ECUDA;
    OutDesc od{out, out_pitch, r->desc.out_float};
    cudaStream_t s = (cudaStream_t)stream;
    stitch_status st = r->desc.path == STITCH_PATH_PLAIN ? plain_frames(r, fp, od, s) : fused_frames(r, fp, od, s);
    prof_mark(r, nullptr, s);
    return st;
}

stitch_status stitch_frames_host(stitch_rig* r, const uint8_t* const* host_frames, const int64_t* pitches,
                                 void* host_out, int64_t out_pitch, void* stream) {
    if (!r || !host_frames || !pitches || !host_out) return STITCH_EINVAL;
    const int bpp = r->desc.out_float ? 12 : 3;
    const long long row = (long long)r->geom.nx[0] * bpp;
    if (out_pitch < row) return STITCH_EINVAL;
    DeviceGuard dg(r->device);
    if (!dg.ok) return STITCH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t* dframes[MAXC] = {};
    int64_t dpitch[MAXC] = {};
    for (int i = 0; i < r->geom.ncam; ++i) {
        const stitch_camera& c = r->cams[i];
        if (!r->hcam[i].visible) continue;
        if (!host_frames[i] || pitches[i] < 3LL * c.width) return STITCH_EINVAL;
        if (!r->stage_frames[i] &&
            cudaMalloc((void**)&r->stage_frames[i], (size_t)c.width * c.height * 3) != cudaSuccess) {
            cudaGetLastError();
            r->stage_frames[i] = nullptr;
            return STITCH_ENOMEM;
        }
        STITCH_CUDA_TRY(cudaMemcpy2DAsync(r->stage_frames[i], (size_t)c.width * 3, host_frames[i], (size_t)pitches[i],
                                          (size_t)c.width * 3, c.height, cudaMemcpyHostToDevice, s));
        dframes[i] = r->stage_frames[i];
        dpitch[i] = (int64_t)c.width * 3;
    }
    if (!r->stage_out && cudaMalloc(&r->stage_out, (size_t)row * r->geom.ny[0]) != cudaSuccess) {
        cudaGetLastError();
        r->stage_out = nullptr;
        return STITCH_ENOMEM;
    }
    stitch_status st = stitch_frames(r, dframes, dpitch, r->stage_out, row, stream);
    if (st != STITCH_OK) return st;
    STITCH_CUDA_TRY(cudaMemcpy2DAsync(host_out, (size_t)out_pitch, r->stage_out, (size_t)row, (size_t)row,
                                      r->geom.ny[0], cudaMemcpyDeviceToHost, s));
    STITCH_CUDA_TRY(cudaStreamSynchronize(s));
    return STITCH_OK;
}

stitch_status stitch_backward(stitch_rig* r, const uint8_t* const* frames, const int64_t* pitches,
                              const double* params, double* loss, double* grad, void* stream) {
    if (!r || !params || !loss) return STITCH_EINVAL;
    if (!frames || !pitches) return STITCH_EINVAL;
    if (r->geom.cyl) return STITCH_EUNSUPPORTED;  // the loss is parametrised by planar homographies
    FramePtrs fp;
    memset(&fp, 0, sizeof(fp));
    for (int i = 0; i < r->geom.ncam; ++i) {
        if (!frames[i] || pitches[i] < 3LL * r->cams[i].width) return STITCH_EINVAL;
        fp.p[i] = frames[i];
        fp.pitch[i] = pitches[i];
    }
    DeviceGuard dg(r->device);
    if (!dg.ok) return STITCH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    stitch_status st = backward_run(r, fp, params, loss, grad, s);
    prof_mark(r, nullptr, s);
    return st;
}

stitch_status stitch_rig_set_profiling(stitch_rig* r, int enable) {
    if (!r) return STITCH_EINVAL;
    r->prof = enable != 0;
    r->marks.clear();
    r->ev_used = 0;
    r->stats.clear();
    return STITCH_OK;
}

stitch_status stitch_rig_kernel_times(stitch_rig* r, const char** names, double* ms, int64_t* launches, int32_t cap,
                                      int32_t* count) {
    if (!r || !count) return STITCH_EINVAL;
    DeviceGuard dg(r->device);
    if (!r->marks.empty()) STITCH_CUDA_TRY(cudaEventSynchronize(r->marks.back().ev));
    for (size_t k = 0; k + 1 < r->marks.size(); ++k) {
        const ProfMark& a = r->marks[k];
        if (!a.name) continue;
        float t = 0.0f;
        STITCH_CUDA_TRY(cudaEventElapsedTime(&t, a.ev, r->marks[k + 1].ev));
        auto it = std::find_if(r->stats.begin(), r->stats.end(),
                               [&](const KernelStat& s) { return strcmp(s.name, a.name) == 0; });
        if (it == r->stats.end()) {
            r->stats.push_back({a.name, 0.0, 0});
            it = r->stats.end() - 1;
        }
        it->ms += t;
        it->launches += 1;
    }
    r->marks.clear();
    r->ev_used = 0;
    const int n = (int)r->stats.size();
    for (int k = 0; k < n && k < cap; ++k) {
        if (names) names[k] = r->stats[k].name;
        if (ms) ms[k] = r->stats[k].ms;
        if (launches) launches[k] = r->stats[k].launches;
    }
    *count = n;
    return STITCH_OK;
}

}  // extern "C"
