// BF16 tensor-core (tcgen05) MLP decode and backward.
#include "npg_internal.cuh"

namespace npg {

bool decode_bf16_supported(int H, int D) { return false; }
cudaError_t launch_decode_bf16(npg_ctx* c) { return cudaErrorNotSupported; }
cudaError_t launch_mlp_backward_bf16(npg_ctx* c) { return cudaErrorNotSupported; }

}  // namespace npg
