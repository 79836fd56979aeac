// Inverse FFTs, f32 arithmetic, float output: one instantiation unit of
// fft_core.cuh (the units compile in parallel).
#include "fft_launch.cuh"

namespace fftmv {
cudaError_t launch_irfft_inv_f32_float(const InvDesc& d, cudaStream_t s) { return inv_launch<float, float>(d, s); }
}  // namespace fftmv
