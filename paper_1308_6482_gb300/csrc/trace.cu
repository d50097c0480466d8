// Kernel trace and pipe probes (no counterpart in the paper): measurement
// support for the roofline of each hot kernel.
//
// Trace: with lub_trace_enable(ctx, 1), the launchers record one CUDA event
// right before and one right after each traced kernel (the cell sweep, the
// closest-point solve, the resistance, the atomic apply), in eager calls only
// (not while the stream is captured into a graph).  lub_trace_read waits for
// a kernel's events and returns the sum of their intervals.  The events
// separate the traced kernel from its neighbours in the programmatic
// dependent-launch chain, so traced calls run a little slower than untraced
// ones; the intervals themselves are the kernels' own.
//
// Probe: long chains of fused multiply-adds, eight independent chains per
// thread and eight 256-thread blocks per SM, timed with events: the sustained
// FMA throughput of the FP32 or the FP64 pipe at the current clocks
// (2 FLOP per FMA).
#include <string.h>

#include "lub_internal.cuh"

void lub_trace_mark(lub_ctx *ctx, int id, cudaStream_t st)
{
    if (!ctx || !ctx->trace || id < 0 || id >= LUB_TRACE_COUNT) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return;
    }
    cudaEvent_t e;
    if (!ctx->trace_pool.empty()) {
        e = ctx->trace_pool.back();
        ctx->trace_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (cudaEventRecord(e, st) != cudaSuccess) {
        (void)cudaGetLastError();
        ctx->trace_pool.push_back(e);
        return;
    }
    ctx->trace_ev[id].push_back(e);
}

void lub_trace_free(lub_ctx *ctx)
{
    for (auto &v : ctx->trace_ev) {
        for (cudaEvent_t e : v) cudaEventDestroy(e);
        v.clear();
    }
    for (cudaEvent_t e : ctx->trace_pool) cudaEventDestroy(e);
    ctx->trace_pool.clear();
}

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T *sink, int write)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (write) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never taken: keeps the chains live
}

template <typename T>
int probe(lub_ctx *ctx, int iters, double *tflops, cudaStream_t st)
{
    const int grid = 8 * ctx->num_sms, block = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return lub_check_cuda(ctx, cudaGetLastError(), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return lub_check_cuda(ctx, cudaGetLastError(), "event");
    }
    double best = 0.0;
    int rc = LUB_OK;
    for (int r = 0; r < 4 && !rc; ++r) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<grid, block, 0, st>>>(iters, (T)0.999999, (T)1e-6, (T *)nullptr, 0);
        cudaEventRecord(e1, st);
        rc = lub_check_cuda(ctx, cudaEventSynchronize(e1), "probe");
        float ms = 0.f;
        if (!rc) rc = lub_check_cuda(ctx, cudaEventElapsedTime(&ms, e0, e1), "probe timing");
        const double flop = 2.0 * 8.0 * (double)iters * grid * block;
        if (!rc && r > 0 && ms > 0.f) best = fmax(best, flop / (ms * 1e-3) / 1e12);  // the first run warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) *tflops = best;
    return rc;
}

}  // namespace

extern "C" {

int lub_trace_enable(lub_ctx *ctx, int32_t on)
{
    if (!ctx) return LUB_ERR_ARG;
    if (!on) lub_trace_free(ctx);
    ctx->trace = on != 0;
    return LUB_OK;
}

int lub_trace_read(lub_ctx *ctx, int32_t kernel, double *ms_total, int64_t *launches)
{
    if (!ctx || !ms_total || !launches) return LUB_ERR_ARG;
    if (kernel < 0 || kernel >= LUB_TRACE_COUNT) return lub_set_error(ctx, LUB_ERR_ARG, "trace kernel %d", kernel);
    auto &v = ctx->trace_ev[kernel];
    double sum = 0.0;
    int64_t n = 0;
    int rc = LUB_OK;
    if (!v.empty()) rc = lub_check_cuda(ctx, cudaEventSynchronize(v.back()), "trace wait");
    for (size_t k = 0; !rc && k + 1 < v.size(); k += 2) {
        float ms = 0.f;
        rc = lub_check_cuda(ctx, cudaEventElapsedTime(&ms, v[k], v[k + 1]), "trace timing");
        sum += ms;
        ++n;
    }
    for (cudaEvent_t e : v) ctx->trace_pool.push_back(e);
    v.clear();
    *ms_total = sum;
    *launches = n;
    return rc;
}

int lub_probe_peak(lub_ctx *ctx, int32_t pipe, double *tflops, void *stream)
{
    if (!ctx || !tflops) return LUB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (pipe == LUB_PROBE_FP32) return probe<float>(ctx, 1 << 17, tflops, st);
    if (pipe == LUB_PROBE_FP64) return probe<double>(ctx, 1 << 12, tflops, st);
    return lub_set_error(ctx, LUB_ERR_ARG, "probe pipe %d", pipe);
}

}  // extern "C"
