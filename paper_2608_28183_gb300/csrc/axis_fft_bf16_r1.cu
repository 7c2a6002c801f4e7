// Strided-axis FFT instantiations: bfloat16 storage, length range 1.
#define AXIS_RANGE 1
#include "axis_fft.cuh"
namespace nlos {
cudaError_t launch_axis_fft_bf16_r1(const AxisLaunch& l, cudaStream_t s) { return launch_axis_typed<__nv_bfloat162, 1>(l, s); }
}  // namespace nlos
