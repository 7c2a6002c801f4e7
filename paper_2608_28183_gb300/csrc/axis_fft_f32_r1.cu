// Strided-axis FFT instantiations: float2 storage, length range 1.
#define AXIS_RANGE 1
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f32_r1(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<float2, 1>(l, s); }
}  // namespace nlos
