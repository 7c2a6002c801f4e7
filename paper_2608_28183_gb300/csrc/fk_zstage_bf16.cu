// f-k temporal-frequency stage instantiations for __nv_bfloat162 storage.
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_bf16(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__nv_bfloat162>(p, tile, s); }
}  // namespace nlos
