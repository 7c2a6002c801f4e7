// f-k temporal-frequency stage instantiations for float2 storage.
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_f32(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<float2>(p, tile, s); }
}  // namespace nlos
