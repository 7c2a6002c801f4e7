// f-k temporal-frequency stage instantiations: bfloat16 storage, length range 0.
#define FK_RANGE 0
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_bf16_r0(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__nv_bfloat162, 0>(p, tile, s); }
}  // namespace nlos
