// f-k temporal-frequency stage instantiations: bfloat16 storage, length range 2.
#define FK_RANGE 2
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_bf16_r2(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__nv_bfloat162, 2>(p, tile, s); }
}  // namespace nlos
