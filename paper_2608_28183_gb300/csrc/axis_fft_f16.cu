// Strided-axis FFT instantiations for __half2 storage.
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2>(l, s); }
}  // namespace nlos
