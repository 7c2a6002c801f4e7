// Strided-axis FFT instantiations: IEEE half storage, length range 2.
#define AXIS_RANGE 2
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16_r2(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2, 2>(l, s); }
}  // namespace nlos
