// C-ABI entry points of the batched schedule (the machinery lives with the fused kernels).  It
// takes the place of the paper's per-image CUDA streams (Sec. 4.3.2) for device-resident frames.
#include "stitch_internal.cuh"

struct stitch_batch {
    void* impl;
    int device;
};

extern "C" {

stitch_status stitch_batch_create(stitch_rig* const* rigs, int32_t n, stitch_batch** out) {
    if (!out) return STITCH_EINVAL;
    *out = nullptr;
    void* impl = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    const stitch_status st = fused_batch_create(rigs, n, &impl);
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    if (st != STITCH_OK) return st;
    stitch_batch* b = new (std::nothrow) stitch_batch{impl, rigs[0]->device};
    if (!b) {
        fused_batch_destroy(impl);
        return STITCH_ENOMEM;
    }
    *out = b;
    return STITCH_OK;
}

stitch_status stitch_batch_frames(stitch_batch* batch, const uint8_t* const* const* frames,
                                  const int64_t* const* pitches, void* const* outs, const int64_t* out_pitches,
                                  void* stream) {
    if (!batch) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device && cudaSetDevice(batch->device) != cudaSuccess) return STITCH_ECUDA;
    const stitch_status st = fused_batch_frames(batch->impl, frames, pitches, outs, out_pitches, (cudaStream_t)stream);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    return st;
}

stitch_status stitch_batch_sync(stitch_batch* batch) {
    if (!batch) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device && cudaSetDevice(batch->device) != cudaSuccess) return STITCH_ECUDA;
    const stitch_status st = fused_batch_status(batch->impl);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    return st;
}

void stitch_batch_destroy(stitch_batch* batch) {
    if (!batch) return;
    int prev = -1;
    cudaGetDevice(&prev);
    fused_batch_destroy(batch->impl);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    delete batch;
}

stitch_status stitch_batch_get_schedule(const stitch_batch* batch, int32_t* order, int32_t* grid, int64_t* tasks) {
    if (!batch) return STITCH_EINVAL;
    return fused_batch_info(batch->impl, order, grid, tasks);
}

stitch_status stitch_batch_wait_test(stitch_batch* batch, int32_t spin_limit, int32_t rig) {
    if (!batch) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device && cudaSetDevice(batch->device) != cudaSuccess) return STITCH_ECUDA;
    const stitch_status st = fused_batch_wait_test(batch->impl, spin_limit, rig);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
