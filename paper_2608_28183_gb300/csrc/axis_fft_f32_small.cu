// Strided-axis FFT instantiations: float2 storage, lengths in the small range.
#define AXIS_SMALL
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f32_small(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<float2, kAxisSmall>(l, s); }
}  // namespace nlos
