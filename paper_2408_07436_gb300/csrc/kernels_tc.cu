// Tensor-core (tcgen05) contraction for the split precisions TF32x3 and BF16x3.
#include "internal.h"
#include "kernels.cuh"

namespace m2l {

int split_tc_operators(m2l_plan_t *pl, int precision) {
    (void)pl;
    (void)precision;
    set_error("split tensor-core precisions are not built yet");
    return M2L_EUNSUPPORTED;
}

int launch_split_rows(const float *, long long, int, void *, void *, int, cudaStream_t) {
    set_error("split tensor-core precisions are not built yet");
    return M2L_EUNSUPPORTED;
}

template <class T>
int launch_contract_tc(m2l_plan_t *, const LevelsArg &, const ContractTile *, long long, int, const void *,
                       const void *, long long, T *, int, cudaStream_t) {
    set_error("split tensor-core precisions are not built yet");
    return M2L_EUNSUPPORTED;
}
template int launch_contract_tc<float>(m2l_plan_t *, const LevelsArg &, const ContractTile *, long long, int,
                                       const void *, const void *, long long, float *, int, cudaStream_t);
template int launch_contract_tc<double>(m2l_plan_t *, const LevelsArg &, const ContractTile *, long long, int,
                                        const void *, const void *, long long, double *, int, cudaStream_t);

}  // namespace m2l
