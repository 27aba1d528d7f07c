// stitch_frames_static: the plain stitching path for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: real-time loops whose latency budget forbids the
// allocator's implicit device synchronisation, embedded hosts that hand the library a fixed memory
// budget at start-up, or plugins whose host application owns every allocation and forbids its
// plugins to allocate device memory of their own.  For them this entry point runs the same
// plain-path kernels as a STITCH_PATH_PLAIN rig, but every scratch buffer (the per-camera
// pyramid and band buffers, the per-level blend buffers and the camera descriptors) is carved out
// of one file-scope device array of fixed size.  The caller passes the frames and the output
// exactly as for stitch_frames.
//
// The array is a `static __device__` symbol: every GPU that loads this module holds it until the
// process exits.  Host code cannot use the symbol's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that device current) and
// caches it; that first call should therefore come before any stream capture.  The cached address
// belongs to the device's current context: after cudaDeviceReset the module is loaded again and
// further calls on that device are not supported.  Calls share the array and keep the last call's
// contents; nothing in it needs to start at zero, because every kernel writes each scratch
// element before any kernel reads it.  Calls whose kernels overlap on the GPU (different streams,
// or different host threads on one device) race on the array.
#include <cmath>
#include <mutex>

#include "stitch_internal.cuh"

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = (size_t)STITCH_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the static array on the current device (looked up once per device).
stitch_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return STITCH_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return STITCH_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return STITCH_OK;
}

// Camera descriptors travel as a kernel parameter (copied at launch, so the host copy may go out
// of scope as soon as the launch returns) and are written into the array by one small kernel.
struct CamPack {
    CamDev c[MAXC];
};
static_assert(sizeof(CamDev) % 8 == 0, "CamDev is copied in 8-byte words");
static_assert(sizeof(CamPack) + sizeof(void*) + sizeof(int) <= 32764, "kernel parameter limit");

__global__ void k_put_cams(const __grid_constant__ CamPack pk, int n, CamDev* __restrict__ dst) {
    const uint2* src = reinterpret_cast<const uint2*>(pk.c);
    uint2* d = reinterpret_cast<uint2*>(dst);
    const int words = n * (int)(sizeof(CamDev) / 8);
    for (int k = threadIdx.x; k < words; k += blockDim.x) d[k] = src[k];
}

// Bump allocator over the static array (256-byte aligned pieces); returns false when full.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    bool take(size_t bytes, void** out) {
        const size_t off = (used + 255) & ~(size_t)255;
        if (off > STATIC_SCRATCH_BYTES || bytes > STATIC_SCRATCH_BYTES - off) return false;
        *out = base ? (void*)(base + off) : nullptr;  // sizing pass: no addresses yet
        used = off + bytes;
        return true;
    }
};

}  // namespace

extern "C" stitch_status stitch_frames_static(const stitch_rig_desc* desc, const uint8_t* const* frames,
                                              const int64_t* pitches, void* out, int64_t out_pitch, void* stream) {
    if (!desc || !desc->cameras || !frames || !pitches || !out) return STITCH_EINVAL;
    if (desc->num_cameras < 1 || desc->num_cameras > MAXC || desc->canvas_w < 1 || desc->canvas_h < 1 ||
        desc->levels < 1 || desc->levels > MAXL || desc->canvas_w > (1 << 28) || desc->canvas_h > (1 << 28) ||
        desc->band_fp16 != 0 || (desc->out_float != 0 && desc->out_float != 1) ||
        (desc->weights != STITCH_WEIGHTS_FEATHER && desc->weights != STITCH_WEIGHTS_SEAM) ||
        (desc->canvas_model != STITCH_CANVAS_PLANAR && desc->canvas_model != STITCH_CANVAS_CYLINDRICAL) ||
        (desc->canvas_model == STITCH_CANVAS_CYLINDRICAL &&
         !(std::isfinite(desc->cylinder[0]) && desc->cylinder[0] > 0.0 && std::isfinite(desc->cylinder[1]) &&
           std::isfinite(desc->cylinder[2]))))
        return STITCH_EINVAL;
    if ((long long)desc->canvas_w * desc->canvas_h > (1LL << 31)) return STITCH_EINVAL;
    const long long row = (long long)desc->canvas_w * (desc->out_float ? 12 : 3);
    if (out_pitch < row) return STITCH_EINVAL;

    // plan on the host, in this stack frame only
    stitch_rig r;
    r.desc = *desc;
    r.desc.cameras = nullptr;
    r.desc.path = STITCH_PATH_PLAIN;
    RigGeom& g = r.geom;
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
    for (int i = 0; i < g.ncam; ++i) {
        const stitch_status st = plan_camera_geometry(desc->cameras[i], g, r.hcam[i], &r.roi_pixels);
        if (st != STITCH_OK) return st;
    }
    FramePtrs fp;
    memset(&fp, 0, sizeof(fp));
    for (int i = 0; i < g.ncam; ++i) {
        if (!r.hcam[i].visible) continue;
        if (!frames[i] || pitches[i] < 3LL * desc->cameras[i].width) return STITCH_EINVAL;
        fp.p[i] = frames[i];
        fp.pitch[i] = pitches[i];
    }

    // carve the plain path's buffers out of the static array: a sizing pass first (no device
    // interaction), then the real pass at the array's device address
    for (int pass = 0; pass < 2; ++pass) {
        void* base = nullptr;
        if (pass == 1) {
            const stitch_status st = scratch_address(&base);
            if (st != STITCH_OK) return st;
        }
        Carver cv{pass == 1 ? (unsigned char*)base : nullptr};
        void* p = nullptr;
        if (!cv.take(sizeof(CamDev) * g.ncam, &p)) return STITCH_ETOOLARGE;
        r.dcam = (CamDev*)p;
        for (int i = 0; i < g.ncam; ++i) {
            CamDev& c = r.hcam[i];
            if (!c.visible) continue;
            for (int l = 0; l < g.levels; ++l) {
                if (!cv.take(sizeof(float4) * (size_t)c.Om[l].area(), &p)) return STITCH_ETOOLARGE;
                c.G[l] = (float4*)p;
                if (l + 1 < g.levels) {
                    if (!cv.take(sizeof(float4) * (size_t)c.Z[l].area(), &p)) return STITCH_ETOOLARGE;
                    c.Lp[l] = (float4*)p;
                }
            }
        }
        for (int l = 0; l < g.levels; ++l) {
            if (!cv.take(sizeof(float4) * (size_t)g.nx[l] * g.ny[l], &p)) return STITCH_ETOOLARGE;
            r.Bl[l] = (float4*)p;
        }
    }

    // camera descriptors into the array, ordered on the stream before the path's kernels
    cudaStream_t s = (cudaStream_t)stream;
    static_assert(sizeof(r.hcam) == sizeof(CamPack), "descriptor pack layout");
    k_put_cams<<<1, 256, 0, s>>>(*reinterpret_cast<const CamPack*>(r.hcam), g.ncam, r.dcam);
    if (cudaGetLastError() != cudaSuccess) return STITCH_ECUDA;
    OutDesc od{out, out_pitch, desc->out_float};
    return plain_frames(&r, fp, od, s);
}
