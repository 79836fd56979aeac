// Entry points of the batched real FFTs.  fft_core.cuh holds the kernels;
// the fft_fwd_* / fft_inv_* units instantiate them per I/O dtype and
// arithmetic.
#include "fftmv_internal.h"

namespace fftmv {

cudaError_t launch_rfft_fwd_double_f64(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_rfft_fwd_double_f32(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_rfft_fwd_double_df(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_rfft_fwd_float_f64(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_rfft_fwd_float_f32(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_rfft_fwd_float_df(const FwdDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_f64_double(const InvDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_f32_double(const InvDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_df_double(const InvDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_f64_float(const InvDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_f32_float(const InvDesc& d, cudaStream_t s);
cudaError_t launch_irfft_inv_df_float(const InvDesc& d, cudaStream_t s);

// one signal per CTA: at most 1024 threads x the per-thread element count
// (16 FP32 complexes, 8 FP64 or double-float ones)
int fft_max_length(int prec) { return prec == FFT_F32 ? 16384 : 8192; }

cudaError_t launch_rfft_fwd(const FwdDesc& d, bool in_f32, int prec, cudaStream_t s) {
  if (d.rows == 0 || d.out_cols == 0 || d.K == 0) return cudaSuccess;
  if (in_f32) {
    if (prec == FFT_F64) return launch_rfft_fwd_float_f64(d, s);
    if (prec == FFT_DF) return launch_rfft_fwd_float_df(d, s);
    return launch_rfft_fwd_float_f32(d, s);
  }
  if (prec == FFT_F64) return launch_rfft_fwd_double_f64(d, s);
  if (prec == FFT_DF) return launch_rfft_fwd_double_df(d, s);
  return launch_rfft_fwd_double_f32(d, s);
}

cudaError_t launch_irfft_inv(const InvDesc& d, int prec, bool out_f32, cudaStream_t s) {
  if (d.cols == 0 || d.K == 0) return cudaSuccess;
  if (out_f32) {
    if (prec == FFT_F64) return launch_irfft_inv_f64_float(d, s);
    if (prec == FFT_DF) return launch_irfft_inv_df_float(d, s);
    return launch_irfft_inv_f32_float(d, s);
  }
  if (prec == FFT_F64) return launch_irfft_inv_f64_double(d, s);
  if (prec == FFT_DF) return launch_irfft_inv_df_double(d, s);
  return launch_irfft_inv_f32_double(d, s);
}

}  // namespace fftmv
