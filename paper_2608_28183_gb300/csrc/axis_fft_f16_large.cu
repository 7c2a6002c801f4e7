// Strided-axis FFT instantiations: __half2 storage, lengths in the large range.
#define AXIS_LARGE
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_f16_large(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__half2, kAxisLarge>(l, s); }
}  // namespace nlos
