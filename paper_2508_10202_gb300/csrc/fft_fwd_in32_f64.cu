// Forward FFTs, float input, f64 arithmetic: one instantiation unit of
// fft_core.cuh (the units compile in parallel).
#include "fft_launch.cuh"

namespace fftmv {
cudaError_t launch_rfft_fwd_float_f64(const FwdDesc& d, cudaStream_t s) { return fwd_launch<float, double>(d, s); }
}  // namespace fftmv
