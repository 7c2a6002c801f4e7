// Strided-axis FFT instantiations for float2 storage.
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f32(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<float2>(l, s); }
}  // namespace nlos
