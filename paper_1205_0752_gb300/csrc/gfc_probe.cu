// gfc_measure_pipe_peaks: throughput of the scalar pipes that bound the
// evaluation kernels (binary64 FMA, multiply and add, binary32 FMA, the
// binary32 reciprocal of the special-function unit), measured on the current
// device. Each probe kernel runs 8 or 16 independent dependency chains per
// thread on SMs x 4 or 8 blocks of 256 threads; the rate is the number of
// thread operations over the CUDA-event time of the best configuration.
// These are the denominators of the kernels' executed-work fractions.
#include <cuda_runtime.h>

#include <algorithm>

#include "gfc.h"
#include "gfc_internal.h"

namespace gfc {
namespace {

constexpr int kUnroll = 4;   // chain steps per loop iteration
constexpr int kThreads = 256;

// OP: 0 binary64 FMA, 1 binary64 multiply, 2 binary64 add, 3 binary32 FMA,
// 4 binary32 approximate reciprocal (each followed by a binary32 add of a
// tiny constant, which the FMA pipes absorb), 5 binary64 FMA interleaved
// with an independent binary32 FMA chain, 6 binary64 FMA, multiply and add in
// the proportions 5 : 2 : 1 (those of the binary64 evaluation kernel, whose
// FP64 pipe issues mixed streams faster than any one operation alone); ILP
// independent chains per thread.
// Thread 0 of block 0 records the SM clock and the global timer around its
// loop, so that the SM frequency of the launch is known.
template <int OP, int ILP>
__global__ void __launch_bounds__(kThreads) probe_kernel(int iters, double b, double c, double *sink,
                                                         long long *clk)
{
    long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    if constexpr (OP <= 2 || OP >= 5) {
        double a[ILP];
        float f[OP == 5 ? ILP : 1];
        const float bf = (float)b, cf = (float)c;
#pragma unroll
        for (int j = 0; j < ILP; ++j) a[j] = 1.0 + 1e-3 * threadIdx.x + j;
#pragma unroll
        for (int j = 0; j < (OP == 5 ? ILP : 1); ++j) f[j] = 1.0f + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < ILP; ++j) {
                    if constexpr (OP == 0 || OP == 5) {
                        a[j] = fma(a[j], b, c);
                    } else if constexpr (OP == 1) {
                        a[j] = a[j] * b;
                    } else if constexpr (OP == 2) {
                        a[j] = a[j] + c;
                    } else {
                        const int q = (j + u) & 7;   // the op of chain j at step u
                        if (q < 5) a[j] = fma(a[j], b, c);
                        else if (q < 7) a[j] = a[j] * b;
                        else a[j] = a[j] + c;
                    }
                    if constexpr (OP == 5) f[j] = fmaf(f[j], bf, cf);
                }
        }
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < ILP; ++j) s += a[j];
#pragma unroll
        for (int j = 0; j < (OP == 5 ? ILP : 1); ++j) s += f[j];
        if (s == -1.0) sink[0] = s;   // never true for these inputs; keeps the chains live
    } else {
        const float bf = (float)b, cf = (float)c;
        float a[ILP];
#pragma unroll
        for (int j = 0; j < ILP; ++j) a[j] = 1.0f + 1e-3f * threadIdx.x + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < ILP; ++j) {
                    if constexpr (OP == 3) {
                        a[j] = fmaf(a[j], bf, cf);
                    } else {
                        float r;
                        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[j]));
                        a[j] = r + 1e-30f;
                    }
                }
        }
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < ILP; ++j) s += a[j];
        if (s == -1.0f) sink[0] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = clock64() - c0;
        clk[1] = t1 - t0;
    }
}

template <int OP>
cudaError_t launch_probe(int ilp, int blocks, int iters, double *sink, cudaStream_t st)
{
    // multiply and FMA chains converge (b < 1); add chains grow slowly
    const double b = OP == 3 ? 0.999 : 0.9999999, c = OP == 3 ? 1e-3 : 1e-9;
    long long *clk = reinterpret_cast<long long *>(sink + 4);
    if (ilp == 8) probe_kernel<OP, 8><<<blocks, kThreads, 0, st>>>(iters, b, c, sink, clk);
    else probe_kernel<OP, 16><<<blocks, kThreads, 0, st>>>(iters, b, c, sink, clk);
    return cudaGetLastError();
}

// seconds of one launch of probe `op` with `iters` iterations, or < 0
double time_probe(int op, int ilp, int blocks, int iters, double *sink, cudaStream_t st,
                  cudaEvent_t e0, cudaEvent_t e1)
{
    if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0;
    cudaError_t e;
    switch (op) {
    case 0: e = launch_probe<0>(ilp, blocks, iters, sink, st); break;
    case 1: e = launch_probe<1>(ilp, blocks, iters, sink, st); break;
    case 2: e = launch_probe<2>(ilp, blocks, iters, sink, st); break;
    case 3: e = launch_probe<3>(ilp, blocks, iters, sink, st); break;
    case 4: e = launch_probe<4>(ilp, blocks, iters, sink, st); break;
    case 5: e = launch_probe<5>(ilp, blocks, iters, sink, st); break;
    default: e = launch_probe<6>(ilp, blocks, iters, sink, st); break;
    }
    if (e != cudaSuccess) return -1.0;
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
    if ((e = dev_malloc((void **)&sink, 128)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(probe)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    // every probe at 8 and 16 chains per thread and 4 and 8 blocks per SM;
    // the best configuration gives the pipe's rate
    double rate[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, mhz[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int rc = GFC_OK;
    for (int op = 0; op < 7 && rc == GFC_OK; ++op) {
        for (int cfg = 0; cfg < 4 && rc == GFC_OK; ++cfg) {
            const int ilp = cfg & 1 ? 16 : 8, blocks = sms * (cfg & 2 ? 8 : 4);
            const double per = seconds / 4.0;
            // calibrate the iteration count to about `per` per launch, then
            // keep the best of two timed launches
            int iters = 16;
            double t = time_probe(op, ilp, blocks, iters, sink, st, e0, e1);
            for (int k = 0; k < 20 && t >= 0.0 && t < 0.05 * per && iters < (1 << 24); ++k) {
                iters *= 4;
                t = time_probe(op, ilp, blocks, iters, sink, st, e0, e1);
            }
            if (t < 0.0) {
                rc = fail(GFC_ECUDA, "probe launch failed");
                break;
            }
            const double scale = std::min(per / std::max(t, 1e-6), 2e9 / iters);
            iters = (int)std::max(1.0, iters * scale);
            for (int k = 0; k < 2; ++k) {
                t = time_probe(op, ilp, blocks, iters, sink, st, e0, e1);
                if (t <= 0.0) {
                    rc = fail(GFC_ECUDA, "probe launch failed");
                    break;
                }
                const double ops = (double)blocks * kThreads * iters * kUnroll * ilp;
                if (ops / t > rate[op]) {
                    rate[op] = ops / t;
                    long long ck[2] = {0, 0};
                    if (cudaMemcpy(ck, sink + 4, sizeof ck, cudaMemcpyDeviceToHost) == cudaSuccess &&
                        ck[1] > 0)
                        mhz[op] = 1e3 * (double)ck[0] / (double)ck[1];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != GFC_OK) return rc;
    // binary64 FMA: the better of the plain chains and the chains interleaved
    // with binary32 work
    if (rate[5] > rate[0]) {
        rate[0] = rate[5];
        mhz[0] = mhz[5];
    }
    out->dfma_per_s = rate[0];
    out->fp64_mix_per_s = rate[6];
    out->dfma_mhz = mhz[0];
    out->ffma_mhz = mhz[3];
    out->dmul_per_s = rate[1];
    out->dadd_per_s = rate[2];
    out->ffma_per_s = rate[3];
    out->rcp32_per_s = rate[4];
    out->sm_count = sms;
    return GFC_OK;
}
