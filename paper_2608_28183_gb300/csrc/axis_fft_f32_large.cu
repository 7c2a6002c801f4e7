// Strided-axis FFT instantiations: float2 storage, lengths in the large range.
#define AXIS_LARGE
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f32_large(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<float2, kAxisLarge>(l, s); }
}  // namespace nlos
