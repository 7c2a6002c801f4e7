// Strided-axis FFT instantiations: __nv_bfloat162 storage, lengths in the small range.
#define AXIS_SMALL
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_bf16_small(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__nv_bfloat162, kAxisSmall>(l, s); }
}  // namespace nlos
