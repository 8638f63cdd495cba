// autotune.cu -- the timing driver of the tiling autotuner (pattern 2 of
// the batched pyramid window: the tile shape, and with it the staging batch
// and the threads per tile, is chosen by measurement on the caller's own
// workload; the rendered image does not depend on it).
//
// The caller owns the candidates' state; a callback sets a candidate up,
// enqueues one of its steps on the stream, or releases it.  The driver times
// every candidate's steps with CUDA events on that stream (after warm-up,
// each step bracketed by its own pair of events) and returns the medians and
// the fastest candidate.
#include <algorithm>
#include <vector>

#include "gsr_internal.cuh"

using namespace gsr;

extern "C" int32_t gsr_autotune(int32_t ncand, gsr_autotune_fn fn, void *ctx, int32_t warmup, int32_t steps,
                                gsr_stream_t stream, float *ms, int32_t *best) {
    if (ncand <= 0 || !fn || warmup < 0 || steps <= 0 || !ms || !best) {
        set_error("gsr_autotune: need candidates, a callback, warmup >= 0, steps > 0 and output pointers");
        return GSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = as_cuda(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return check_launch("gsr_autotune: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return check_launch("gsr_autotune: event");
    }
    int32_t rc = GSR_OK;
    std::vector<float> t((size_t)steps);
    *best = -1;
    for (int32_t c = 0; c < ncand && rc == GSR_OK; ++c) {
        if ((rc = fn(c, GSR_AUTOTUNE_SETUP, ctx)) != GSR_OK) break;
        for (int32_t k = 0; k < warmup && rc == GSR_OK; ++k) rc = fn(c, GSR_AUTOTUNE_STEP, ctx);
        if (rc == GSR_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = check_launch("gsr_autotune: warm-up");
        for (int32_t k = 0; k < steps && rc == GSR_OK; ++k) {
            cudaEventRecord(e0, st);
            if ((rc = fn(c, GSR_AUTOTUNE_STEP, ctx)) != GSR_OK) break;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[(size_t)k], e0, e1) != cudaSuccess)
                rc = check_launch("gsr_autotune: timing");
        }
        const int32_t rel = fn(c, GSR_AUTOTUNE_RELEASE, ctx);
        if (rc != GSR_OK) break;
        if ((rc = rel) != GSR_OK) break;
        std::vector<float> s(t);
        std::nth_element(s.begin(), s.begin() + (ptrdiff_t)(steps / 2), s.end());
        ms[c] = s[(size_t)(steps / 2)];
        if (*best < 0 || ms[c] < ms[*best]) *best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GSR_OK) *best = -1;
    return rc;
}
