// f-k with the inverse temporal transform last: __half2 storage, lengths 2048-8192.
#include "fk_zsplit.cuh"
namespace nlos {
cudaError_t launch_fk_stolt_f16_r1(const FkZParams& p, int tile, cudaStream_t s) {
  switch (p.L) {
    case 2048: return launch_fk_stolt_len<2048, __half2>(p, tile, s);
    case 4096: return launch_fk_stolt_len<4096, __half2>(p, tile, s);
    case 8192: return launch_fk_stolt_len<8192, __half2>(p, tile, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_fk_zinv_f16_r1(const FkZInvParams& p, int tile, cudaStream_t s) {
  switch (p.L) {
    case 2048: return launch_fk_zinv_len<2048, __half2>(p, tile, s);
    case 4096: return launch_fk_zinv_len<4096, __half2>(p, tile, s);
    case 8192: return launch_fk_zinv_len<8192, __half2>(p, tile, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nlos
