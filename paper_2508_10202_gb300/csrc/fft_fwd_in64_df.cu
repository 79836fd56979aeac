// Forward FFTs, double input, df arithmetic: one instantiation unit of
// fft_core.cuh (the units compile in parallel).
#include "fft_launch.cuh"

namespace fftmv {
cudaError_t launch_rfft_fwd_double_df(const FwdDesc& d, cudaStream_t s) { return fwd_launch<double, DFA>(d, s); }
}  // namespace fftmv
