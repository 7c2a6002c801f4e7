// Strided-axis FFT instantiations: bfloat16 storage, length range 2.
#define AXIS_RANGE 2
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_bf16_r2(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__nv_bfloat162, 2>(l, s); }
}  // namespace nlos
