// Strided-axis FFT instantiations: IEEE half storage, length range 1.
#define AXIS_RANGE 1
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16_r1(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2, 1>(l, s); }
}  // namespace nlos
