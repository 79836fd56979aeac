// Forward FFTs, double input, f32 arithmetic: one instantiation unit of
// fft_core.cuh (the units compile in parallel).
#include "fft_launch.cuh"

namespace fftmv {
cudaError_t launch_rfft_fwd_double_f32(const FwdDesc& d, cudaStream_t s) { return fwd_launch<double, float>(d, s); }
}  // namespace fftmv
