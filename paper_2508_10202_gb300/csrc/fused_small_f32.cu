// Fused single-launch matvec for small operators: the FP32 kernels (every
// phase in FP32, the all-single configuration of Section 3.2; the kernel is in
// fused_small.cuh).
//
// Cluster size: 16 CTAs where the device schedules them (cl16), else 8.  The
// FP32 arithmetic of a call is small, but 16 CTAs halve each one's channel
// pairs and frequencies, and so its dependent shared-memory and L2 round trips:
// 8.2 against 9.2 us per call (Nt=64, Nd=8, Nm=32, in a CUDA graph).
#include "fused_small.cuh"

#ifndef FFTMV_FUSED32_CL16
#define FFTMV_FUSED32_CL16 1
#endif

namespace fftmv {
namespace {

template <int CL>
cudaError_t launch_f32_cl(const FusedDesc& d, cudaStream_t s) {
  if (d.io_f32)
    return d.L == 128 ? fused_launch_np<float, float, 128, CL>(d, s) : fused_launch_np<float, float, 256, CL>(d, s);
  return d.L == 128 ? fused_launch_np<float, double, 128, CL>(d, s) : fused_launch_np<float, double, 256, CL>(d, s);
}

}  // namespace

cudaError_t launch_fused_small_f32(const FusedDesc& d, bool cl16, cudaStream_t s) {
#if FFTMV_FUSED32_CL16
  if (cl16) return launch_f32_cl<16>(d, s);
#else
  (void)cl16;
#endif
  return launch_f32_cl<8>(d, s);
}

}  // namespace fftmv
