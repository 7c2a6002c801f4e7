// Fused f-k lateral transforms, f16 storage.
#include "fk_chain.cuh"
namespace nlos {
cudaError_t launch_fk_chain_f16(const FkChainLaunch& l, cudaStream_t s) { return launch_fk_chain_typed<__half2>(l, s); }
}  // namespace nlos
