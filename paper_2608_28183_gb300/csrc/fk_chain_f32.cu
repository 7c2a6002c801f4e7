// Fused f-k lateral transforms, f32 storage.
#include "fk_chain.cuh"
namespace nlos {
cudaError_t launch_fk_chain_f32(const FkChainLaunch& l, cudaStream_t s) { return launch_fk_chain_typed<float2>(l, s); }
}  // namespace nlos
