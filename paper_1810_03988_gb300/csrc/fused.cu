// Fused forward path (work in progress).
#include "stitch_internal.cuh"

stitch_status fused_plan(stitch_rig* r) { (void)r; return STITCH_EUNSUPPORTED; }
stitch_status fused_frames(stitch_rig* r, const FramePtrs& fp, const OutDesc& od, cudaStream_t s) {
    (void)r; (void)fp; (void)od; (void)s;
    return STITCH_EUNSUPPORTED;
}
void fused_release(stitch_rig* r) { (void)r; }
