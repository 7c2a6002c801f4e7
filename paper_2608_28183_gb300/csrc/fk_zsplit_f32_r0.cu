// f-k with the inverse temporal transform last: float2 storage, lengths 32-1024.
#include "fk_zsplit.cuh"
namespace nlos {
cudaError_t launch_fk_stolt_f32_r0(const FkZParams& p, int tile, cudaStream_t s) {
  switch (p.L) {
    case 32: return launch_fk_stolt_len<32, float2>(p, tile, s);
    case 64: return launch_fk_stolt_len<64, float2>(p, tile, s);
    case 128: return launch_fk_stolt_len<128, float2>(p, tile, s);
    case 256: return launch_fk_stolt_len<256, float2>(p, tile, s);
    case 512: return launch_fk_stolt_len<512, float2>(p, tile, s);
    case 1024: return launch_fk_stolt_len<1024, float2>(p, tile, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_fk_zinv_f32_r0(const FkZInvParams& p, int tile, cudaStream_t s) {
  switch (p.L) {
    case 32: return launch_fk_zinv_len<32, float2>(p, tile, s);
    case 64: return launch_fk_zinv_len<64, float2>(p, tile, s);
    case 128: return launch_fk_zinv_len<128, float2>(p, tile, s);
    case 256: return launch_fk_zinv_len<256, float2>(p, tile, s);
    case 512: return launch_fk_zinv_len<512, float2>(p, tile, s);
    case 1024: return launch_fk_zinv_len<1024, float2>(p, tile, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nlos
