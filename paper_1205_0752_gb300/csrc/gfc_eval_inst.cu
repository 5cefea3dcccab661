// Instantiations of the evaluation kernels for one binary arithmetic and one
// unrolled angular pair count, selected at compile time by GFC_INST_T (double,
// float or df) and GFC_INST_NP (32, 64, 128 or 0 for the generic loop). The
// build compiles this file once per pair (T, NP); without the two macros it
// compiles to an empty object.
#include "gfc_kernels.cuh"

#if defined(GFC_INST_T) && defined(GFC_INST_NP)

namespace gfc {

// The closed-form angle and the clustered radial rule have variant kernels of
// their own, with the generic pair loop only (NP = 0): the dispatch sends
// them here.
// The kernel kind of a launch (see eval_loop): 1 the node groups of the
// mixed precision's partial routing (binary64 and double-float), 2 the
// binary32 bulk that records them, else 0.
template <typename T>
static int launch_kind(const KParams &kp)
{
    if constexpr (std::is_same<T, float>::value)
        return kp.mode == MODE_BULK32 && kp.node_list && kp.mixed_rtol > 0.0 ? 2 : 0;
    else
        return kp.mode == MODE_NODES ? 1 : 0;
}

template <typename T, int NP, int CL>
static cudaError_t eval_kind(const KParams &kp, const DevTables &tb, cudaStream_t st)
{
    const bool two = kp.pc.kind == 2;
    const int k = launch_kind<T>(kp);
    if constexpr (std::is_same<T, float>::value) {
        if (k == 2) return two ? run_eval<T, NP, 2, CL, 2>(kp, tb, st) : run_eval<T, NP, 1, CL, 2>(kp, tb, st);
    } else {
        if (k == 1) return two ? run_eval<T, NP, 2, CL, 1>(kp, tb, st) : run_eval<T, NP, 1, CL, 1>(kp, tb, st);
    }
    return two ? run_eval<T, NP, 2, CL>(kp, tb, st) : run_eval<T, NP, 1, CL>(kp, tb, st);
}

template <typename T, int NP>
cudaError_t eval_inst(const KParams &kp, const DevTables &tb, cudaStream_t st)
{
    if constexpr (NP == 0) {
        if (kp.radial_rule == 1 || kp.ang_exact) return eval_kind<T, 0, 1>(kp, tb, st);
    }
    return eval_kind<T, NP, 0>(kp, tb, st);
}

template <typename T, int NP>
cudaError_t batch_inst(const BatchLaunch &bl, const DevTables &tb, bool two_terms, cudaStream_t st)
{
    if constexpr (NP == 0) {
        if (bl.radial_rule == 1 || bl.ang_exact)
            return two_terms ? run_batch<T, 0, 2, 1>(bl, tb, st) : run_batch<T, 0, 1, 1>(bl, tb, st);
    }
    return two_terms ? run_batch<T, NP, 2, 0>(bl, tb, st) : run_batch<T, NP, 1, 0>(bl, tb, st);
}

template cudaError_t eval_inst<GFC_INST_T, GFC_INST_NP>(const KParams &, const DevTables &,
                                                        cudaStream_t);
template cudaError_t batch_inst<GFC_INST_T, GFC_INST_NP>(const BatchLaunch &, const DevTables &,
                                                         bool, cudaStream_t);

}  // namespace gfc

#endif
