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
template <typename T, int NP>
cudaError_t eval_inst(const KParams &kp, const DevTables &tb, cudaStream_t st)
{
    if constexpr (NP == 0) {
        if (kp.radial_rule == 1 || kp.ang_exact)
            return kp.pc.kind == 2 ? run_eval<T, 0, 2, 1>(kp, tb, st) : run_eval<T, 0, 1, 1>(kp, tb, st);
    }
    return kp.pc.kind == 2 ? run_eval<T, NP, 2, 0>(kp, tb, st) : run_eval<T, NP, 1, 0>(kp, tb, st);
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
