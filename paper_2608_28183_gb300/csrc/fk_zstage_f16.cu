// f-k temporal-frequency stage instantiations for __half2 storage.
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_f16(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__half2>(p, tile, s); }
}  // namespace nlos
