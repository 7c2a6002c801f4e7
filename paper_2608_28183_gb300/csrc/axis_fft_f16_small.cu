// Strided-axis FFT instantiations: __half2 storage, lengths in the small range.
#define AXIS_SMALL
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16_small(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2, kAxisSmall>(l, s); }
}  // namespace nlos
