// f-k temporal-frequency stage instantiations: float2 storage, length range 2.
#define FK_RANGE 2
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_f32_r2(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<float2, 2>(p, tile, s); }
}  // namespace nlos
