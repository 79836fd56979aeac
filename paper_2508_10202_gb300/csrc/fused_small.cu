// Fused single-launch matvec for small operators: the FP64 kernels, the size
// check and the entry point (the kernel itself is in fused_small.cuh; the FP32
// kernels in fused_small_f32.cu).
//
// FP64 clusters have 16 CTAs (a non-portable size) where the device schedules
// them, else the portable 8: FP64 runs at about two FMAs per clock per SM on
// this GPU, so its work is spread over as many SMs as a cluster can hold.
#include <mutex>

#include "fused_small.cuh"

#ifndef FFTMV_FUSED_CL16
#define FFTMV_FUSED_CL16 1
#endif

namespace fftmv {
namespace {

// whether the current device schedules CL-CTA clusters of the largest fused
// kernel (checked once per device and cluster size)
template <int CL>
bool clusters_ok() {
  static int cache[64];
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::call_once(once[dev], [&] {
    auto kern = fused_small_kernel<double, double, 4, 256, CL>;
    constexpr size_t smem = fused_smem_bytes<double, 256, 4, CL>();
    int n = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const bool ok = prep(kern, smem) == cudaSuccess &&
                    (CL <= 8 || cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                                    cudaSuccess) &&
                    cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();
    cache[dev] = ok ? 1 : 0;
  });
  return cache[dev] == 1;
}

template <typename Tio, int L>
cudaError_t fused_launch_cl(const FusedDesc& d, cudaStream_t s) {
#if FFTMV_FUSED_CL16
  if (clusters_ok<16>()) return fused_launch_np<double, Tio, L, 16>(d, s);
#endif
  return fused_launch_np<double, Tio, L, 8>(d, s);
}

}  // namespace

bool fused_small_fits(int64_t L, int64_t Cin, int64_t Cout) {
  // the sizes one cluster takes, on a device that schedules 8-CTA clusters of
  // the largest FP64 kernel (the FP32 kernels need less shared memory; else
  // every call takes the three-kernel path)
  return (L == 128 || L == 256) && Cin >= 1 && Cout >= 1 && Cin <= kFusedMaxChannels && Cout <= kFusedMaxChannels &&
         clusters_ok<8>();
}

cudaError_t launch_fused_small(const FusedDesc& d, cudaStream_t s) {
  if (d.K == 0) return cudaSuccess;
  if (!fused_small_fits(d.L, d.Cin, d.Cout) || d.K > 65535) return cudaErrorInvalidValue;
  if (d.f32) return launch_fused_small_f32(d, FFTMV_FUSED_CL16 && clusters_ok<16>(), s);
  if (d.io_f32) return d.L == 128 ? fused_launch_cl<float, 128>(d, s) : fused_launch_cl<float, 256>(d, s);
  return d.L == 128 ? fused_launch_cl<double, 128>(d, s) : fused_launch_cl<double, 256>(d, s);
}

}  // namespace fftmv
