// Strided-axis FFT instantiations: __nv_bfloat162 storage, lengths in the large range.
#define AXIS_LARGE
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_bf16_large(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__nv_bfloat162, kAxisLarge>(l, s); }
}  // namespace nlos
