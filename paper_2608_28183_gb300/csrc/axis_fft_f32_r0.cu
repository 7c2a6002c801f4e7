// Strided-axis FFT instantiations: float2 storage, length range 0.
#define AXIS_RANGE 0
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f32_r0(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<float2, 0>(l, s); }
}  // namespace nlos
