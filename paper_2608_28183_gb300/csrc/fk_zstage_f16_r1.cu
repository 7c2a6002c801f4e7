// f-k temporal-frequency stage instantiations: IEEE half storage, length range 1.
#define FK_RANGE 1
#include "fk_zstage.cuh"
namespace nlos {
cudaError_t launch_fk_zstage_f16_r1(const FkZParams& p, int tile, cudaStream_t s) { return launch_fk_typed<__half2, 1>(p, tile, s); }
}  // namespace nlos
