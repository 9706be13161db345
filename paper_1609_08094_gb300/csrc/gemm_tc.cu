// tcgen05 W contractions (TF32x3 / BF16x3): placeholder until the tensor-core
// kernel lands; the mixed precisions report TCORR_EUNSUPPORTED meanwhile.
#include "tcorr_internal.cuh"

namespace tcorr {

bool tc_supported(int, int) { return false; }

cudaError_t tc_build_tensor_maps(Handle *, std::string &err) {
    err = "tensor-core path not built";
    return cudaErrorNotSupported;
}

cudaError_t launch_ugemm_tc(Handle *, const GemmArgs &, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace tcorr
