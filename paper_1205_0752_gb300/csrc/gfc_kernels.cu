// Kernels of libgfc for sm_103a that are not instantiated per arithmetic:
// G0(mu2) (the subtraction point of Sect. 2, in binary64) and the grid of
// Step 4 when a caller asks for it alone, plus the host-side dispatch of the
// evaluation kernels to their (arithmetic, pair count) instantiations.
#include <type_traits>

#include "gfc_kernels.cuh"

namespace gfc {

// G0(mu2) in binary64: the radial nodes of the real-axis ray are split over
// warps (one node per lane); the last warp to finish sums the partials in a
// fixed order. The first thread also resets the work counters of the
// evaluation launches that follow on the stream.
template <int NP, int NT>
__global__ void __launch_bounds__(256)
g0mu_kernel(const __grid_constant__ KParams kp,
            const __grid_constant__ AngTab<double, tab_size<NP>()> tab,
            const double *__restrict__ gtab, double mu2, double *partials, unsigned *ticket,
            double *g0mu_out, unsigned long long *counters)
{
    const double *stab;
    const void *srules;
    stage_tables<double, NP>(kp, gtab, kp.npair, stab, srules);
    if (blockIdx.x == 0 && threadIdx.x < kCounters) counters[threadIdx.x] = 0ULL;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    Plan<double> P = make_plan<double, 1>(kp, mu2, 0.0);
    C<double> x = {mu2, 0.0};
    C<double> e2 = P.eth * P.eth;
    C<double> eD = kp.dim == 4 ? e2 * e2 : e2 * P.eth;
    double sr = 0.0, si = 0.0;
    // the real-axis point has one ray pass
    const int nn = kp.n_r;
    const PassPre<double, 2> pp2 = pass_pre<double, 2>(kp, P, 0, x);
    const PassPre<double, 1> pp1 = pass_pre<double, 1>(kp, P, 0, x);
    for (int k = warp * 32 + lane; k < nn; k += nwarps * 32) {
        Node<double> nd = P.clus ? ray_node_cl<double>(kp, k, e2, eD, P.cl_c, P.cl_d, P.cl_eta)
                                 : ray_node<double>(kp, k, e2, eD);
        ErrAcc<double> ea = {0.0, 0.0};
        double qm;
        int np;
        C<double> v = P.nterm[0] == 2
                          ? node_value<double, NP, 2, 1>(kp, tab, stab, srules, pp2, x, nd, ea, qm, np, false)
                          : node_value<double, NP, 1, 1>(kp, tab, stab, srules, pp1, x, nd, ea, qm, np, false);
        sr += v.r;
        si += v.i;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    __shared__ bool last;
    if (lane == 0) {
        partials[2 * warp] = sr;
        partials[2 * warp + 1] = si;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double ar = 0.0, ai = 0.0;
        for (int w = 0; w < nwarps; ++w) {
            ar += ((volatile double *)partials)[2 * w];
            ai += ((volatile double *)partials)[2 * w + 1];
        }
        g0mu_out[0] = mu2 == 0.0 ? 0.0 : kp.K_D * ar;
        g0mu_out[1] = mu2 == 0.0 ? 0.0 : kp.K_D * ai;
        *ticket = 0u;
    }
}

__global__ void grid_points_kernel(double re0, double dre, double im0, double dim_im, int m,
                                   int n, double *x)
{
    int64_t total = (int64_t)m * n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        x[2 * p] = __dadd_rn(re0, __dmul_rn(i + 0.5, dre));
        x[2 * p + 1] = __dadd_rn(im0, __dmul_rn(j + 0.5, dim_im));
    }
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
// double-float runs the generic angular loop only: fully unrolled
// double-float bodies cost minutes of compile time for no speed gain
template <typename T>
static cudaError_t eval_np(const KParams &kp, const DevTables &tb, cudaStream_t st)
{
    // the closed-form angle and the clustered radial rule: generic variant kernels
    if (kp.radial_rule == 1 || kp.ang_exact) return eval_inst<T, 0>(kp, tb, st);
    if constexpr (std::is_same<T, df>::value) {
        return eval_inst<T, 0>(kp, tb, st);
    } else {
        switch (kp.npair) {
        case 32: return eval_inst<T, 32>(kp, tb, st);
        case 64: return eval_inst<T, 64>(kp, tb, st);
        case 128: return eval_inst<T, 128>(kp, tb, st);
        default: return eval_inst<T, 0>(kp, tb, st);
        }
    }
}

template <typename T>
static cudaError_t batch_np(const BatchLaunch &bl, const DevTables &tb, bool two_terms,
                            cudaStream_t st)
{
    if (bl.radial_rule == 1 || bl.ang_exact) return batch_inst<T, 0>(bl, tb, two_terms, st);
    if constexpr (std::is_same<T, df>::value) {
        return batch_inst<T, 0>(bl, tb, two_terms, st);
    } else {
        switch (bl.npair) {
        case 32: return batch_inst<T, 32>(bl, tb, two_terms, st);
        case 64: return batch_inst<T, 64>(bl, tb, two_terms, st);
        case 128: return batch_inst<T, 128>(bl, tb, two_terms, st);
        default: return batch_inst<T, 0>(bl, tb, two_terms, st);
        }
    }
}

cudaError_t launch_batch(const BatchLaunch &bl, const DevTables &tb, int arith, bool two_terms,
                         cudaStream_t st)
{
    if (take_injected_launch_failure()) return cudaErrorLaunchOutOfResources;
    if (arith == ARITH_F32) return batch_np<float>(bl, tb, two_terms, st);
    if (arith == ARITH_DF) return batch_np<df>(bl, tb, two_terms, st);
    return batch_np<double>(bl, tb, two_terms, st);
}

cudaError_t launch_eval(const KParams &kp, const DevTables &tb, int arith, cudaStream_t st)
{
    if (take_injected_launch_failure()) return cudaErrorLaunchOutOfResources;
    if (arith == ARITH_F32) return eval_np<float>(kp, tb, st);
    if (arith == ARITH_DF) return eval_np<df>(kp, tb, st);
    return eval_np<double>(kp, tb, st);
}

template <int NP, int NT>
static cudaError_t run_g0mu(const KParams &kp, const DevTables &tb, double mu2, double *partials,
                            int nwarps, unsigned *ticket, double *g0mu_out,
                            unsigned long long *counters, cudaStream_t st)
{
    AngTab<double, tab_size<NP>()> tab;
    fill_tab(tab, tb, NP > 0 ? kp.npair : 0);
    size_t smem = smem_bytes<double, NP>(kp.npair, kp.rules_total);
    int blocks = (nwarps + 7) / 8;
    g0mu_kernel<NP, NT><<<blocks, 256, smem, st>>>(kp, tab, tb.ang64, mu2, partials, ticket,
                                                   g0mu_out, counters);
    return cudaGetLastError();
}

cudaError_t launch_g0mu(const KParams &kp, const DevTables &tb, double mu2, double *partials,
                        int nwarps, unsigned *ticket, double *g0mu_out,
                        unsigned long long *counters, cudaStream_t st)
{
    const bool two = kp.pc.kind == 2;
#define GFC_G0(NP)                                                                               \
    return two ? run_g0mu<NP, 2>(kp, tb, mu2, partials, nwarps, ticket, g0mu_out, counters, st) \
               : run_g0mu<NP, 1>(kp, tb, mu2, partials, nwarps, ticket, g0mu_out, counters, st)
    switch (kp.npair) {
    case 32: GFC_G0(32);
    case 64: GFC_G0(64);
    case 128: GFC_G0(128);
    default: GFC_G0(0);
    }
#undef GFC_G0
}

cudaError_t launch_grid_points(double re0, double dre, double im0, double dim_im, int m, int n,
                               double *x, cudaStream_t st)
{
    int64_t total = (int64_t)m * n;
    int64_t blocks = (total + 255) / 256;
    int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    grid_points_kernel<<<(unsigned)blocks, 256, 0, st>>>(re0, dre, im0, dim_im, m, n, x);
    return cudaGetLastError();
}

}  // namespace gfc
