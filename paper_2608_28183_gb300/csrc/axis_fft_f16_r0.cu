// Strided-axis FFT instantiations: IEEE half storage, length range 0.
#define AXIS_RANGE 0
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16_r0(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2, 0>(l, s); }
}  // namespace nlos
