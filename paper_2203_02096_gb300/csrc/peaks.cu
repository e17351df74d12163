// peaks.cu -- microbenchmarks of the device rates the evaluator's rooflines
// are stated against: FP32 fused multiply-add throughput, special-function
// (MUFU ex2) throughput and L2->SM load bandwidth.  Measurement
// infrastructure, not part of the docking method.
#include <algorithm>

#include "internal.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// kChains independent FMA chains per thread, iters steps each: 2 FLOP per
// FMA.  The result is written only when it equals an impossible value, so the
// work cannot be removed and nothing is stored.
__global__ void __launch_bounds__(256) ffma_kernel(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.2345e30f) out[blockIdx.x] = s;
}

// kChains independent chains x <- 2^(-x) per thread (values stay in (0, 1]).
__global__ void __launch_bounds__(256) ex2_kernel(float *out, int iters) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0.25f + 0.01f * k + threadIdx.x * 1e-5f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
            x[k] = y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.2345e30f) out[blockIdx.x] = s;
}

// Every thread reads float4 words of buf (n4 of them) in a grid-stride loop,
// `passes` times, through L2 only (ld.global.cg).
__global__ void __launch_bounds__(256) l2_read_kernel(const float4 *buf, size_t n4, int passes, float *out) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    if (acc.x + acc.y + acc.z + acc.w == -1.2345e30f) out[blockIdx.x] = acc.x;
}

}  // namespace

extern "C" int dock_microbench(dock_ctx *ctx, int what, double *value) {
    if (!ctx || !value) return ctx ? set_err(ctx, DOCK_ERR_INVALID, "null argument") : DOCK_ERR_INVALID;
    if (what != DOCK_PEAK_FFMA && what != DOCK_PEAK_EX2 && what != DOCK_PEAK_L2_READ)
        return set_err(ctx, DOCK_ERR_INVALID, "unknown microbenchmark");
    cudaStream_t s = nullptr;
    const int blocks = ctx->num_sms * 8, threads = 256;
    const size_t l2_bytes = (size_t)48 << 20;  // well inside the 129 MB L2
    float *out = (float *)dev_alloc(ctx, (size_t)blocks * 4, s);
    float4 *buf = what == DOCK_PEAK_L2_READ ? (float4 *)dev_alloc(ctx, l2_bytes, s) : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DOCK_OK;
    if (!out || (what == DOCK_PEAK_L2_READ && !buf)) rc = set_err(ctx, DOCK_ERR_OOM, "microbenchmark allocation");
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaEventCreate(&e0);
    if (!rc && !e) e = cudaEventCreate(&e1);
    if (!rc && !e && buf) e = cudaMemsetAsync(buf, 0, l2_bytes, s);
    double best = 0.0;
    const int iters = 1 << 14, passes = 200;
    for (int rep = 0; rep < 4 && !rc && !e; ++rep) {  // rep 0 warms up (clocks, L2)
        e = cudaEventRecord(e0, s);
        if (what == DOCK_PEAK_FFMA) ffma_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.9999f, 1e-6f);
        else if (what == DOCK_PEAK_EX2) ex2_kernel<<<blocks, threads, 0, s>>>(out, iters);
        else l2_read_kernel<<<blocks, threads, 0, s>>>(buf, l2_bytes / 16, passes, out);
        ++ctx->launches;
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e1, s);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e || rep == 0 || ms <= 0.f) continue;
        const double n = (double)blocks * threads;
        double v = 0.0;
        if (what == DOCK_PEAK_FFMA) v = n * iters * kChains * 2.0 / (ms * 1e-3) / 1e12;      // TFLOP/s
        else if (what == DOCK_PEAK_EX2) v = n * iters * kChains / (ms * 1e-3) / 1e9;        // Gop/s
        else v = (double)l2_bytes * passes / (ms * 1e-3) / 1e9;                             // GB/s
        best = std::max(best, v);
    }
    if (!rc && e) rc = cuda_err(ctx, e, "microbenchmark");
    if (!rc) *value = best;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, out, s);
    dev_free(ctx, buf, s);
    return rc;
}
