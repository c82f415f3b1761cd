// The closed-loop single-frame mode (Section 1: motion correction for
// real-time, closed-loop experiments): one frame in from host memory, its
// shift out, as fast as possible. The whole step (host-to-device copy, the
// plan's alignment of one frame, device-to-host copy of the shift) is
// captured once into a CUDA graph; each moco_stream_align replays it and
// waits for the shift.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "moco.h"
#include "plan.h"

namespace moco {
moco_status fail(moco_status s, const std::string& msg);
moco_status cuda_fail(cudaError_t e, const char* what);
moco_status align_frames(ShapePlan& sp, const uint16_t* frames, int64_t T, int32_t* shifts, double* best_cost,
                         float* margin, double* final_cost, cudaStream_t st);
}  // namespace moco

using namespace moco;

struct moco_stream_s {
    moco_plan_t plan = nullptr;
    int device = 0;
    uint16_t* dframe = nullptr;  // one frame
    int32_t* dshift = nullptr;   // (s, t)
    cudaStream_t cap = nullptr;  // the stream the graph was captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
struct DevGuard {
    int prev = 0;
    explicit DevGuard(int dev) {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~DevGuard() { cudaSetDevice(prev); }
};

void release(moco_stream_s* s) {
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->dframe) cudaFree(s->dframe);
    if (s->dshift) cudaFree(s->dshift);
    delete s;
}
}  // namespace

extern "C" moco_status moco_stream_create(moco_plan_t plan, int32_t shape_idx, const uint16_t* frame_host,
                                          int32_t* shift_host, moco_stream_t* out) {
    if (!out) return fail(MOCO_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!plan || !frame_host || !shift_host) return fail(MOCO_ERR_INVALID_ARG, "null plan or host buffer");
    if (shape_idx < 0 || shape_idx >= (int)plan->shapes.size()) return fail(MOCO_ERR_INVALID_ARG, "bad shape_idx");
    ShapePlan& sp = plan->shapes[shape_idx];
    if (sp.f32 && sp.levels) return fail(MOCO_ERR_UNSUPPORTED, "float template with levels");
    DevGuard guard(plan->device);
    moco_stream_s* s = new moco_stream_s;
    s->plan = plan;
    s->device = plan->device;
    const size_t bytes = (size_t)sp.desc.m * sp.desc.n * 2;
    cudaError_t e = cudaMalloc(&s->dframe, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->dshift, 8);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release(s);
        return e == cudaErrorMemoryAllocation ? fail(MOCO_ERR_OOM, "stream buffers") : cuda_fail(e, "stream set-up");
    }
    // One eager pass first: kernel attributes are set outside the capture.
    e = cudaMemcpyAsync(s->dframe, frame_host, bytes, cudaMemcpyHostToDevice, s->cap);
    if (e != cudaSuccess) {
        release(s);
        return cuda_fail(e, "stream warm-up copy");
    }
    const bool prof = plan->prof.on;
    plan->prof.on = false;  // no event records inside the graph
    moco_status r = align_frames(sp, s->dframe, 1, s->dshift, nullptr, nullptr, nullptr, s->cap);
    if (r == MOCO_OK) {
        e = cudaStreamSynchronize(s->cap);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(s->dframe, frame_host, bytes, cudaMemcpyHostToDevice, s->cap);
            r = align_frames(sp, s->dframe, 1, s->dshift, nullptr, nullptr, nullptr, s->cap);
            cudaMemcpyAsync(shift_host, s->dshift, 8, cudaMemcpyDeviceToHost, s->cap);
            const cudaError_t e2 = cudaStreamEndCapture(s->cap, &s->graph);
            if (e2 != cudaSuccess && r == MOCO_OK) r = cuda_fail(e2, "stream capture");
        } else {
            r = cuda_fail(e, "stream warm-up");
        }
        if (r == MOCO_OK) {
            e = cudaGraphInstantiate(&s->exec, s->graph, 0);
            if (e != cudaSuccess) r = cuda_fail(e, "stream graph instantiation");
        }
    }
    plan->prof.on = prof;
    if (r != MOCO_OK) {
        release(s);
        return r;
    }
    *out = s;
    return MOCO_OK;
}

extern "C" moco_status moco_stream_align(moco_stream_t s, void* stream) {
    if (!s) return fail(MOCO_ERR_INVALID_ARG, "null stream handle");
    DevGuard guard(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGraphLaunch(s->exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MOCO_OK : cuda_fail(e, "moco_stream_align");
}

extern "C" moco_status moco_stream_destroy(moco_stream_t s) {
    if (!s) return fail(MOCO_ERR_INVALID_ARG, "null stream handle");
    DevGuard guard(s->device);
    cudaStreamSynchronize(s->cap);
    release(s);
    return MOCO_OK;
}
