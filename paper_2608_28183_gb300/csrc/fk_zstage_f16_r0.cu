// f-k temporal-frequency stage instantiations: IEEE half storage, length range 0.
#define FK_RANGE 0
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_f16_r0(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__half2, 0>(p, tile, s); }
}  // namespace nlos
