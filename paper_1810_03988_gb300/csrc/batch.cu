// Batched persistent schedule (work in progress).
#include "stitch_internal.cuh"

extern "C" {
stitch_status stitch_batch_create(stitch_rig* const* rigs, int32_t n, stitch_batch** out) {
    (void)rigs; (void)n;
    if (out) *out = nullptr;
    return STITCH_EUNSUPPORTED;
}
stitch_status stitch_batch_frames(stitch_batch* batch, const uint8_t* const* const* frames,
                                  const int64_t* const* pitches, void* const* outs, const int64_t* out_pitches,
                                  void* stream) {
    (void)batch; (void)frames; (void)pitches; (void)outs; (void)out_pitches; (void)stream;
    return STITCH_EUNSUPPORTED;
}
void stitch_batch_destroy(stitch_batch* batch) { (void)batch; }
}
