// gfc_measure_pipe_peaks: throughput of the scalar pipes that bound the
// evaluation kernels (binary64 FMA, binary32 FMA, the binary32 reciprocal of
// the special-function unit), measured on the current device. Each probe
// kernel runs ILP independent dependency chains per thread on a grid of SMs x
// 8 blocks of 256 threads, long enough (about `seconds`) for the clocks to
// settle; the rate is the number of thread operations over the CUDA-event
// time. These are the denominators of the kernels' executed-work fractions.
#include <cuda_runtime.h>

#include <algorithm>

#include "gfc.h"
#include "gfc_internal.h"

namespace gfc {
namespace {

constexpr int kIlp = 8;
constexpr int kUnroll = 4;   // chain steps per loop iteration
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) probe_dfma(int iters, double b, double c, double *sink)
{
    double a[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) a[j] = 1e-3 * threadIdx.x + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kIlp; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) s += a[j];
    if (s == -1.0) sink[0] = s;   // never true for these inputs; keeps the chains live
}

__global__ void __launch_bounds__(kThreads) probe_ffma(int iters, float b, float c, float *sink)
{
    float a[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) a[j] = 1e-3f * threadIdx.x + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kIlp; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) s += a[j];
    if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) probe_rcp32(int iters, float *sink)
{
    float a[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) a[j] = 1.0f + 1e-3f * threadIdx.x + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kIlp; ++j) asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a[j]) : "f"(a[j]));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) s += a[j];
    if (s == -1.0f) sink[0] = s;
}

// thread operations per launch of `iters` iterations
double ops_of(int blocks, int iters) { return (double)blocks * kThreads * iters * kUnroll * kIlp; }

// seconds of one launch of probe `which` with `iters` iterations, or < 0
double time_probe(int which, int blocks, int iters, double *dsink, cudaStream_t st,
                  cudaEvent_t e0, cudaEvent_t e1)
{
    if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0;
    if (which == 0) probe_dfma<<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-6, dsink);
    else if (which == 1) probe_ffma<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, (float *)dsink);
    else probe_rcp32<<<blocks, kThreads, 0, st>>>(iters, (float *)dsink);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    if (cudaEventRecord(e1, st) != cudaSuccess) return -1.0;
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
    return 1e-3 * ms;
}

}  // namespace
}  // namespace gfc

using namespace gfc;

extern "C" int gfc_measure_pipe_peaks(gfc_pipe_peaks *out, double seconds, void *stream)
{
    if (!out) return fail(GFC_EINVAL, "out is NULL");
    if (!(seconds > 0.0 && seconds <= 10.0)) return fail(GFC_EINVAL, "seconds must be in (0, 10]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    cudaStream_t st = (cudaStream_t)stream;
    double *sink = nullptr;
    if ((e = dev_malloc((void **)&sink, 64)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(probe)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    const int blocks = sms * kBlocksPerSm;
    double rate[3] = {0.0, 0.0, 0.0};
    int rc = GFC_OK;
    for (int which = 0; which < 3 && rc == GFC_OK; ++which) {
        // calibrate the iteration count to about `seconds` per launch, then
        // keep the best of two timed launches
        int iters = 64;
        double t = time_probe(which, blocks, iters, sink, st, e0, e1);
        for (int k = 0; k < 20 && t >= 0.0 && t < 0.05 * seconds && iters < (1 << 24); ++k) {
            iters *= 4;
            t = time_probe(which, blocks, iters, sink, st, e0, e1);
        }
        if (t < 0.0) {
            rc = fail(GFC_ECUDA, "probe launch failed");
            break;
        }
        const double scale = std::min(seconds / std::max(t, 1e-6), 2e9 / iters);
        iters = (int)std::max(1.0, iters * scale);
        for (int k = 0; k < 2; ++k) {
            t = time_probe(which, blocks, iters, sink, st, e0, e1);
            if (t <= 0.0) {
                rc = fail(GFC_ECUDA, "probe launch failed");
                break;
            }
            rate[which] = std::max(rate[which], ops_of(blocks, iters) / t);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != GFC_OK) return rc;
    out->dfma_per_s = rate[0];
    out->ffma_per_s = rate[1];
    out->rcp32_per_s = rate[2];
    out->sm_count = sms;
    return GFC_OK;
}
