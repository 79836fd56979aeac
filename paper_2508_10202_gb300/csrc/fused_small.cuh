// Fused single-launch matvec for small operators (Section 2.4, all five
// phases in one kernel; the FFT <-> block-matvec fusion for operators whose
// spectra fit on chip), in FP64 (fused_small.cu) or FP32 (fused_small_f32.cu):
// every phase in the arithmetic P, as the three-kernel path computes the
// all-FP64 and all-FP32 configurations of Section 3.2.
//
// One thread-block cluster of CL CTAs per right-hand side:
//   1. every CTA pads and transforms NP channel pairs of the input (the
//      Stockham passes of fft_core.cuh) and keeps their half spectra in its
//      shared memory;
//   2. cluster barrier; CTA r then takes the frequencies w = r, r + CL, ...:
//      it gathers their whole input spectra from the other CTAs' shared
//      memory (distributed shared memory) in one sweep, applies F-hat_w (N for
//      F, conjugate transpose for F*) with F-hat read from global memory, all
//      its frequencies' outputs at once, and keeps them in its own shared
//      memory;
//   3. cluster barrier; every CTA gathers the output spectra of its NP output
//      channel pairs at every frequency, the last cluster barrier releases the
//      other CTAs, and it runs the inverse passes and writes t < Nt.
// The spectra never reach global memory and the whole matvec is one launch;
// the CPU-launched three-kernel path takes over where the signals no longer
// fit (fused_small_fits).
#pragma once

#include <cooperative_groups.h>

#include "fft_core.cuh"

namespace fftmv {
namespace {

namespace cg = cooperative_groups;

constexpr int kFusedThreads = 128;
constexpr int kFusedMaxChannels = 64;   // input and output channels one cluster takes

template <typename P, int L, int NP, int CL>
__host__ __device__ constexpr size_t fused_smem_bytes() {
  constexpr int Nf = L / 2 + 1;
  constexpr int NWL = (Nf + CL - 1) / CL;
  constexpr int MAXC = 2 * NP * CL;
  return (size_t)(L * NP + Nf * 2 * NP + 2 * NWL * MAXC) * sizeof(typename Ar<P>::C);
}

template <typename P>
__device__ __forceinline__ P fused_fma(P a, P b, P c) {
  if constexpr (std::is_same<P, float>::value) return fmaf(a, b, c);
  else return fma(a, b, c);
}

template <typename P, typename Tio, int NP, int L, int CL>
__global__ void __launch_bounds__(kFusedThreads) fused_small_kernel(FusedDesc d) {
  using A = Ar<P>;
  using C = typename A::C;
  constexpr int T = kFusedThreads;
  constexpr int E = kFftE<P>;
  constexpr int NPASS = cplan<P>(L).npass;
  constexpr int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;         // channels per CTA
  constexpr int MAXC = NCH * CL;      // channels per cluster
  constexpr int NWL = (Nf + CL - 1) / CL;
  // the Stockham passes give each thread ceil(E / R) butterflies of radix R <= E
  static_assert(T * E >= L * NP, "too few threads for one pass over the CTA's signals");
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int b = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [L NP] signals (swizzled)
  C* Xh = buf + L * NP;                      // [Nf][NCH] half spectra of this CTA's input channels
  C* Yh = Xh + Nf * NCH;                     // [NWL][MAXC] output spectra of this CTA's frequencies
  C* G = Yh + NWL * MAXC;                    // [NWL][MAXC] input spectra of this CTA's frequencies
  const P h = (P)0.5;
  const C zero = A::mk(A::zero(), A::zero());
  const C* tw = static_cast<const C*>(d.tw);
  const C* Fh = static_cast<const C*>(d.F);
  auto sdst = [&](int, int, int e, C v) { buf[swz<C>(e)] = v; };
  auto ssrc = [&](int, int, int e) -> C { return buf[swz<C>(e)]; };

  // 1. pad (the cast to P) + forward FFT of input channels c0 .. c0 + NCH - 1
  // (zero past Cin)
  const int c0 = rank * NCH;
  const Tio* x = static_cast<const Tio*>(d.x) + b * d.x_ld_b;
  auto gsrc = [&](int t, int p, int) -> C {
    const int c = c0 + 2 * p;
    if (t >= d.Nt || c >= d.Cin) return zero;
    const Tio* xp = x + (int64_t)t * d.Cin + c;
    return A::mk((P)xp[0], c + 1 < d.Cin ? (P)xp[1] : A::zero());
  };
  cpass<P, false, NP, E, L, 0, 0, false>(T, tw, gsrc, sdst);
  __syncthreads();
  cpasses<P, false, NP, E, L, 1, NPASS>(T, tw, ssrc, sdst);
  // X_a = (Z_w + conj Z_{L-w}) / 2, X_b = (Z_w - conj Z_{L-w}) / (2i)
  for (int i = threadIdx.x; i < Nf * NCH; i += T) {
    const int w = i / NCH, cc = i - w * NCH;
    const C z = buf[sidx<C, NP>(w, cc >> 1)];
    const C zc = buf[sidx<C, NP>(w == 0 ? 0 : L - w, cc >> 1)];
    Xh[i] = (cc & 1) ? A::mk(h * (z.y + zc.y), h * (zc.x - z.x)) : A::mk(h * (z.x + zc.x), h * (z.y - zc.y));
  }
  cl.sync();

  // 2. block matvec of frequencies w = rank + CL j: first every input value
  // those frequencies need, gathered from the other CTAs in one sweep (all
  // loads in flight together), then every output of them at once
  const int nw = (Nf - rank + CL - 1) / CL;   // frequencies this CTA owns
  for (int i = threadIdx.x; i < nw * d.Cin; i += T) {
    const int j = i / d.Cin, n = i - j * d.Cin;
    const int owner = n / NCH;
    const C* rx = cl.map_shared_rank(Xh, owner);
    G[j * MAXC + n] = rx[(rank + CL * j) * NCH + (n - owner * NCH)];
  }
  __syncthreads();
  if (!d.adjoint) {
    // d-hat_w[r] = sum_n F-hat_w[r][n] m-hat_w[n]: GR threads per (w, r), each
    // over every GR-th n, then a shuffle sum (the loop is warp-uniform)
    constexpr int GR = 4;
    const int ntask = nw * d.Nd;
    for (int base = 0; base < ntask; base += T / GR) {
      const int t = base + threadIdx.x / GR, g = threadIdx.x % GR;
      P sr = A::zero(), si = A::zero();
      if (t < ntask) {
        const int j = t / d.Nd, r = t - j * d.Nd;
        const C* Fr = Fh + ((int64_t)(rank + CL * j) * d.Nd + r) * d.ldn;
        const C* v = G + j * MAXC;
#pragma unroll 4
        for (int n = g; n < d.Cin; n += GR) {
          const C f = __ldg(Fr + n), u = v[n];
          sr = fused_fma<P>(f.x, u.x, fused_fma<P>(-f.y, u.y, sr));
          si = fused_fma<P>(f.x, u.y, fused_fma<P>(f.y, u.x, si));
        }
      }
#pragma unroll
      for (int o = GR / 2; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (t < ntask && g == 0) {
        const int j = t / d.Nd;
        Yh[j * MAXC + (t - j * d.Nd)] = A::mk(sr, si);
      }
    }
  } else {
    // m-hat_w[n] = sum_r conj(F-hat_w[r][n]) d-hat_w[r]: a thread per (w, n)
    const int ntask = nw * d.Cout;
    for (int t = threadIdx.x; t < ntask; t += T) {
      const int j = t / d.Cout, n = t - j * d.Cout;
      const C* Fn = Fh + (int64_t)(rank + CL * j) * d.Nd * d.ldn + n;
      const C* v = G + j * MAXC;
      P sr = A::zero(), si = A::zero();
#pragma unroll 4
      for (int r = 0; r < d.Cin; ++r) {
        const C f = __ldg(Fn + (int64_t)r * d.ldn), u = v[r];
        sr = fused_fma<P>(f.x, u.x, fused_fma<P>(f.y, u.y, sr));
        si = fused_fma<P>(f.x, u.y, fused_fma<P>(-f.y, u.x, si));
      }
      Yh[j * MAXC + n] = A::mk(sr, si);
    }
  }
  cl.sync();

  // 3. Hermitian assembly of output channels o0 .. o0 + NCH - 1 from the
  // owners of each frequency, then the inverse passes and the unpad
  const int o0 = rank * NCH;
  for (int i = threadIdx.x; i < Nf * NP; i += T) {
    const int w = i / NP, p = i - w * NP;
    const int ca = o0 + 2 * p, cb = ca + 1;
    const C* ry = cl.map_shared_rank(Yh, w % CL) + (w / CL) * MAXC;
    const C a = ca < d.Cout ? ry[ca] : zero;
    const C bb = cb < d.Cout ? ry[cb] : zero;
    if (w == 0 || w == Nf - 1) {
      buf[sidx<C, NP>(w, p)] = A::mk(a.x, bb.x);
    } else {
      buf[sidx<C, NP>(w, p)] = A::mk(a.x - bb.y, a.y + bb.x);
      buf[sidx<C, NP>(L - w, p)] = A::mk(a.x + bb.y, bb.x - a.y);
    }
  }
  cl.sync();   // no CTA reads another's shared memory after this point
  cpasses<P, true, NP, E, L, 0, NPASS - 1>(T, tw, ssrc, sdst);
  Tio* y = static_cast<Tio*>(d.y) + b * d.y_ld_b;
  const P invL = (P)d.inv_L;   // 1/L, a power of two
  auto gdst = [&](int t, int p, int, C v) {
    const int c = o0 + 2 * p;
    if (t >= d.Nt || c >= d.Cout) return;
    Tio* yp = y + (int64_t)t * d.Cout + c;
    yp[0] = (Tio)(v.x * invL);
    if (c + 1 < d.Cout) yp[1] = (Tio)(v.y * invL);
  };
  cpass<P, true, NP, E, L, NPASS - 1, 2, false>(T, tw, ssrc, gdst);
}

template <typename P, typename Tio, int NP, int L, int CL>
cudaError_t fused_launch(const FusedDesc& d, cudaStream_t s) {
  auto kern = fused_small_kernel<P, Tio, NP, L, CL>;
  constexpr size_t smem = fused_smem_bytes<P, L, NP, CL>();
  cudaError_t e = prep(kern, smem);
  if (e == cudaSuccess && CL > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, d.K, 1);
  cfg.blockDim = dim3(kFusedThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d);
}

// channel pairs per CTA: the fewest of 1, 2, 4 that cover the wider side
template <typename P, typename Tio, int L, int CL>
cudaError_t fused_launch_np(const FusedDesc& d, cudaStream_t s) {
  const int pairs = (((d.Cin > d.Cout ? d.Cin : d.Cout) + 1) / 2 + CL - 1) / CL;
  if (pairs <= 1) return fused_launch<P, Tio, 1, L, CL>(d, s);
  if (pairs <= 2) return fused_launch<P, Tio, 2, L, CL>(d, s);
  return fused_launch<P, Tio, 4, L, CL>(d, s);
}

}  // namespace
}  // namespace fftmv
