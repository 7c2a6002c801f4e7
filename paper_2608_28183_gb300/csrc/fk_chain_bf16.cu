// Fused f-k lateral transforms, bf16 storage.
#include "fk_chain.cuh"
namespace nlos {
cudaError_t launch_fk_chain_bf16(const FkChainLaunch& l, cudaStream_t s) { return launch_fk_chain_typed<__nv_bfloat162>(l, s); }
}  // namespace nlos
