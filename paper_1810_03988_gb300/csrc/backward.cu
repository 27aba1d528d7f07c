// S7 backward (work in progress).
#include "stitch_internal.cuh"

stitch_status backward_plan(stitch_rig* r) { (void)r; return STITCH_OK; }
stitch_status backward_run(stitch_rig* r, const FramePtrs& fp, const double* params, double* loss, double* grad,
                           cudaStream_t s) {
    (void)r; (void)fp; (void)params; (void)loss; (void)grad; (void)s;
    return STITCH_EUNSUPPORTED;
}
