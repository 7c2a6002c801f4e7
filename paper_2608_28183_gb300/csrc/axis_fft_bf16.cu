// Strided-axis FFT instantiations for __nv_bfloat162 storage.
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_bf16(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__nv_bfloat162>(l, s); }
}  // namespace nlos
