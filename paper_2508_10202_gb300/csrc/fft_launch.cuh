// Dispatch of the batched real FFTs: the compile-time-length kernels
// (in-place decimation in frequency for FP32, fft_dif.cuh, and for
// double-float, fft_dif_df.cuh; Stockham for FP64 and the other lengths,
// fft_core.cuh) and the runtime-length Stockham kernels.
#pragma once

#include "fft_dif.cuh"
#include "fft_dif_df.cuh"

namespace fftmv {
namespace {

#ifndef FFTMV_DIF
#define FFTMV_DIF 1
#endif
// the lengths with in-place decimation-in-frequency FP32 kernels (dif_plan)
#define FFTMV_DIF_LENGTHS(X) X(128) X(256) X(512) X(1000) X(2000)
// ... and double-float ones (dfd_plan, fft_dif_df.cuh)
#ifndef FFTMV_DFD
#define FFTMV_DFD 1
#endif

template <typename Tin, typename P>
cudaError_t fwd_launch(const FwdDesc& d, cudaStream_t s) {
  // the tensor-core B planes are written 8 channels (4 pairs) at a time
  const int np = d.fmt == FMT_TC ? fft_pairs<P>(d.plan.L)
                                 : fft_pairs_for_grid<P>(d.plan.L, [&](int n) {
                                     return (int64_t)d.rows * ((d.out_cols + 2 * n - 1) / (2 * n)) * d.K;
                                   });
#if FFTMV_DIF
  if constexpr (std::is_same<P, float>::value) {
    if (d.twd != nullptr && np == fft_pairs<P>(d.plan.L)) {
      switch (d.plan.L) {
#define FFTMV_CASE(LL) \
  case LL: return fwd_dif_launch<Tin, fft_pairs<float>(LL), LL>(d, s);
        FFTMV_DIF_LENGTHS(FFTMV_CASE)
#undef FFTMV_CASE
        default: break;
      }
    }
  }
#endif
#if FFTMV_DFD
  if constexpr (std::is_same<P, DFA>::value) {
    cudaError_t e;
    if (fwd_dfd_try<Tin>(d, np, s, e)) return e;
  }
#endif
  if (np == fft_pairs<P>(d.plan.L)) {
    switch (d.plan.L) {
#define FFTMV_CASE(LL) \
  case LL: return fwd_launch_np<Tin, P, fft_pairs<P>(LL), LL>(d, s);
      FFTMV_FIXED_LENGTHS(FFTMV_CASE)
#undef FFTMV_CASE
      default: break;
    }
  }
  switch (np) {
    case 8: return fwd_launch_np<Tin, P, 8, 0>(d, s);
    case 4: return fwd_launch_np<Tin, P, 4, 0>(d, s);
    case 2: return fwd_launch_np<Tin, P, 2, 0>(d, s);
    default: return fwd_launch_np<Tin, P, 1, 0>(d, s);
  }
}

template <typename P, typename Tout>
cudaError_t inv_launch(const InvDesc& d, cudaStream_t s) {
  const int np = fft_pairs_for_grid<P>(d.plan.L, [&](int n) { return (int64_t)((d.cols + 2 * n - 1) / (2 * n)) * d.K; });
#if FFTMV_DIF
  if constexpr (std::is_same<P, float>::value) {
    if (d.twd != nullptr && np == fft_pairs<P>(d.plan.L)) {
      switch (d.plan.L) {
#define FFTMV_CASE(LL) \
  case LL: return inv_dif_launch<Tout, fft_pairs<float>(LL), LL>(d, s);
        FFTMV_DIF_LENGTHS(FFTMV_CASE)
#undef FFTMV_CASE
        default: break;
      }
    }
  }
#endif
#if FFTMV_DFD
  if constexpr (std::is_same<P, DFA>::value) {
    cudaError_t e;
    if (inv_dfd_try<Tout>(d, np, s, e)) return e;
  }
#endif
  if (np == fft_pairs<P>(d.plan.L)) {
    switch (d.plan.L) {
#define FFTMV_CASE(LL) \
  case LL: return inv_launch_np<P, Tout, fft_pairs<P>(LL), LL>(d, s);
      FFTMV_FIXED_LENGTHS(FFTMV_CASE)
#undef FFTMV_CASE
      default: break;
    }
  }
  switch (np) {
    case 8: return inv_launch_np<P, Tout, 8, 0>(d, s);
    case 4: return inv_launch_np<P, Tout, 4, 0>(d, s);
    case 2: return inv_launch_np<P, Tout, 2, 0>(d, s);
    default: return inv_launch_np<P, Tout, 1, 0>(d, s);
  }
}

}  // namespace
}  // namespace fftmv
