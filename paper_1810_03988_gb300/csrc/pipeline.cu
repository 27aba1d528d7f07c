// stitch_frames_host_async: host buffers in and out, with upload, stitching and download of
// consecutive calls overlapped (the stream strategy of the paper, Sec. 4.3.2 and Fig. 3b: the next
// frame is uploaded while the current one is processed).
//
// Three rig-owned streams (copy-in, compute, copy-out) and two staging slots (device frames and
// canvas) alternate between calls.  Call k uses slot k % 2; its upload waits until the stitch of
// call k-2 has read the slot's frames, its stitch waits for its upload and for the download of
// call k-2 (which read the slot's canvas), its download waits for its stitch.  The caller's stream
// waits for the download, so synchronising that stream makes the output valid; the upload does
// not wait for earlier work on the caller's stream.  Stitches run in
// order on one stream, so the rig's pyramid scratch is never used by two calls at once.
#include "stitch_internal.cuh"

namespace {

struct PipeSlot {
    uint8_t* frames[MAXC];
    void* out;
    cudaEvent_t in_done, comp_done, out_done;
};

struct Pipe {
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    PipeSlot slot[2] = {};
    long long calls = 0;
    std::vector<void*> allocs;
};

void pipe_free(Pipe* p) {
    if (!p) return;
    for (auto& sl : p->slot) {
        if (sl.in_done) cudaEventDestroy(sl.in_done);
        if (sl.comp_done) cudaEventDestroy(sl.comp_done);
        if (sl.out_done) cudaEventDestroy(sl.out_done);
    }
    for (cudaStream_t s : {p->s_in, p->s_comp, p->s_out})
        if (s) cudaStreamDestroy(s);
    for (void* a : p->allocs) cudaFree(a);
    delete p;
}

stitch_status pipe_create(stitch_rig* r, Pipe** out) {
    *out = nullptr;
    Pipe* p = new (std::nothrow) Pipe();
    if (!p) return STITCH_ENOMEM;
    auto fail = [&](stitch_status st) {
        cudaGetLastError();
        pipe_free(p);
        return st;
    };
    if (cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) != cudaSuccess)
        return fail(STITCH_ECUDA);
    const size_t row = (size_t)r->geom.nx[0] * (r->desc.out_float ? 12 : 3);
    for (auto& sl : p->slot) {
        if (cudaEventCreateWithFlags(&sl.in_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.comp_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.out_done, cudaEventDisableTiming) != cudaSuccess)
            return fail(STITCH_ECUDA);
        for (int i = 0; i < r->geom.ncam; ++i) {
            if (!r->hcam[i].visible) continue;
            const stitch_camera& c = r->cams[i];
            if (cudaMalloc((void**)&sl.frames[i], (size_t)c.width * c.height * 3) != cudaSuccess) return fail(STITCH_ENOMEM);
            p->allocs.push_back(sl.frames[i]);
        }
        if (cudaMalloc(&sl.out, row * r->geom.ny[0]) != cudaSuccess) return fail(STITCH_ENOMEM);
        p->allocs.push_back(sl.out);
    }
    *out = p;
    return STITCH_OK;
}

}  // namespace

void pipeline_release(stitch_rig* r) {
    pipe_free((Pipe*)r->pipe);
    r->pipe = nullptr;
}

extern "C" stitch_status stitch_frames_host_async(stitch_rig* r, const uint8_t* const* host_frames,
                                                  const int64_t* pitches, void* host_out, int64_t out_pitch,
                                                  void* stream) {
    if (!r || !host_frames || !pitches || !host_out) return STITCH_EINVAL;
    const size_t row = (size_t)r->geom.nx[0] * (r->desc.out_float ? 12 : 3);
    if (out_pitch < (int64_t)row) return STITCH_EINVAL;
    for (int i = 0; i < r->geom.ncam; ++i)
        if (r->hcam[i].visible && (!host_frames[i] || pitches[i] < 3LL * r->cams[i].width)) return STITCH_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != r->device && cudaSetDevice(r->device) != cudaSuccess) return STITCH_ECUDA;
    stitch_status st = STITCH_OK;
    if (!r->pipe) {
        Pipe* p = nullptr;
        st = pipe_create(r, &p);
        r->pipe = p;
    }
    Pipe* p = (Pipe*)r->pipe;
    cudaStream_t cs = (cudaStream_t)stream;
    if (st == STITCH_OK) {
        PipeSlot& sl = p->slot[p->calls & 1];
        const uint8_t* dframes[MAXC] = {};
        int64_t dpitch[MAXC] = {};
        auto ok = [&](cudaError_t e) {
            if (e != cudaSuccess && st == STITCH_OK) st = STITCH_ECUDA;
        };
        // upload: after call k-2's stitch has read this slot.  It does not wait for work queued
        // earlier on the caller's stream: that stream waits for every earlier call's download, so
        // waiting for it would serialise consecutive calls.
        ok(cudaStreamWaitEvent(p->s_in, sl.comp_done, 0));
        for (int i = 0; i < r->geom.ncam && st == STITCH_OK; ++i) {
            if (!r->hcam[i].visible) continue;
            const stitch_camera& c = r->cams[i];
            ok(cudaMemcpy2DAsync(sl.frames[i], (size_t)c.width * 3, host_frames[i], (size_t)pitches[i],
                                 (size_t)c.width * 3, c.height, cudaMemcpyHostToDevice, p->s_in));
            dframes[i] = sl.frames[i];
            dpitch[i] = (int64_t)c.width * 3;
        }
        ok(cudaEventRecord(sl.in_done, p->s_in));
        // stitch: after the upload and after call k-2's download read this slot's canvas
        ok(cudaStreamWaitEvent(p->s_comp, sl.in_done, 0));
        ok(cudaStreamWaitEvent(p->s_comp, sl.out_done, 0));
        if (st == STITCH_OK) st = stitch_frames(r, dframes, dpitch, sl.out, (int64_t)row, p->s_comp);
        ok(cudaEventRecord(sl.comp_done, p->s_comp));
        // download, and the caller's stream waits for it
        ok(cudaStreamWaitEvent(p->s_out, sl.comp_done, 0));
        ok(cudaMemcpy2DAsync(host_out, (size_t)out_pitch, sl.out, row, row, r->geom.ny[0], cudaMemcpyDeviceToHost,
                             p->s_out));
        ok(cudaEventRecord(sl.out_done, p->s_out));
        ok(cudaStreamWaitEvent(cs, sl.out_done, 0));
        ++p->calls;
    }
    if (prev >= 0 && prev != r->device) cudaSetDevice(prev);
    return st;
}
