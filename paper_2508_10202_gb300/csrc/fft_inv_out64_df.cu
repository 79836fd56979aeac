// Inverse FFTs, df arithmetic, double output: one instantiation unit of
// fft_core.cuh (the units compile in parallel).
#include "fft_launch.cuh"

namespace fftmv {
cudaError_t launch_irfft_inv_df_double(const InvDesc& d, cudaStream_t s) { return inv_launch<DFA, double>(d, s); }
}  // namespace fftmv
