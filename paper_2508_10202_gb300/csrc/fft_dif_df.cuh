// In-place decimation-in-frequency FFTs in double-float arithmetic (the
// FP64-class FFT phases of Section 3.2 at the compile-time lengths 2000 and
// 1000: phases 1-2, zero pad + forward real FFT, and phases 4-5, inverse real
// FFT + unpad).
//
// The structure of the FP32 kernels of fft_dif.cuh (NP channel pairs per CTA,
// pair (c, c+1) packed as one complex signal, the NP signals interleaved in
// shared memory; every pass a Gentleman-Sande step of a dfd_plan whose
// butterflies read their rad[s] inputs, transform them, multiply by their
// twiddles and write them back in place, one barrier per pass, compile-time
// offsets), with the arithmetic, the loads and the stores of the Stockham
// double-float kernels of fft_core.cuh: pad cast and range scaling as the
// samples load, any spectrum format out of the forward and into the inverse,
// the 1/L scale, range scaling and output cast in the inverse's final pass.
//
// A double-float complex is 16 bytes and four registers, so the radices stay
// at 8 and below (five passes for 2000, one barrier each, against the
// Stockham kernels' five passes with two), with 256 threads and three CTAs per
// SM.  The arithmetic renormalises lazily (Ar<DFL>), the spectra only where
// they are stored.
#pragma once

#include "fft_core.cuh"

namespace fftmv {
namespace {

// the arithmetic: DFA, double-float with lazy renormalisation (fft_core.cuh)
using DfdP = DFA;
#ifndef FFTMV_DIF_HALF
#define FFTMV_DIF_HALF 1
#endif

template <int L, int NP>
__device__ __forceinline__ int dfd_e(int pos, int p) {
  return pos * NP + p;
}
template <int L, int NP>
__host__ __device__ constexpr int dfd_smem_elems() {
  return L * NP;
}
// threads (0: one per butterfly of the first pass) and resident CTAs per SM;
// 256 and 3 took 0.233 / 0.200 ms for the F forward / F* inverse at the paper
// shape, 500 and 2 0.239 / 0.222, 320 and 3 about the same as 256
#ifndef FFTMV_DFD_T
#define FFTMV_DFD_T 256
#endif
#ifndef FFTMV_DFD_MINB
#define FFTMV_DFD_MINB 3
#endif
template <int L, int NP>
__host__ __device__ constexpr int dfd_threads() {
  return FFTMV_DFD_T > 0 ? FFTMV_DFD_T : (NP * L / dfd_plan(L).rad[0] + 31) / 32 * 32;
}
// the position of index k once every pass has run (digit reversal)
template <int L>
__device__ __forceinline__ int dfd_pos(int k) {
  constexpr DifPlan pl = dfd_plan(L);
  int pos = 0;
#pragma unroll
  for (int s = 0; s < pl.n; ++s) {
    pos += (k % pl.rad[s]) * dfd_S(L, s);
    k /= pl.rad[s];
  }
  return pos;
}

// v[q] *= W^{j q} (INV: conj) for q = 1 .. R-1 from a table row
template <bool INV, int R>
__device__ __forceinline__ void dfd_twiddle(float4* v, const float4* __restrict__ row) {
  using A = Ar<DfdP>;
#pragma unroll
  for (int q = 1; q < R; ++q) {
    float4 w = __ldg(row + q - 1);
    if (INV) w = A::conj(w);
    v[q] = A::cmul(v[q], w);
  }
}

// pass s (of the plan) in shared memory
template <bool INV, int NP, int L, int s, int T>
__device__ __forceinline__ void dfd_pass(float4* __restrict__ buf, const float4* __restrict__ twd) {
  constexpr int R = dfd_plan(L).rad[s], M = dfd_M(L, s), S = M / R;
  constexpr int NBUT = (L / M) * S * NP;
  constexpr int ES = S * NP;
#pragma unroll 1
  for (int bt = threadIdx.x; bt < NBUT; bt += T) {
    const int p = bt % NP, r = bt / NP, j = r % S, blk = r / S;
    float4* base = buf + dfd_e<L, NP>(blk * M + j, p);
    float4 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = base[q * ES];
    Dft<DfdP, R, INV>::run(v);
    if constexpr (S > 1) dfd_twiddle<INV, R>(v, twd + dfd_tw_offset(L, s) + j * (R - 1));
#pragma unroll
    for (int q = 0; q < R; ++q) base[q * ES] = v[q];
  }
}

template <bool INV, int NP, int L, int s, int T>
__device__ __forceinline__ void dfd_passes(float4* __restrict__ buf, const float4* __restrict__ twd, int last) {
  if constexpr (s < dfd_plan(L).n) {
    if (s < last) {
      dfd_pass<INV, NP, L, s, T>(buf, twd);
      __syncthreads();
      dfd_passes<INV, NP, L, s + 1, T>(buf, twd, last);
    }
  }
}

// Forward: pad + real FFT; grid (row x channel group, K), as rfft_fwd_kernel,
// with any output format but the tensor-core planes.
template <typename Tin, int NP, int L>
__global__ void __launch_bounds__(dfd_threads<L, NP>(), FFTMV_DFD_MINB) rfft_dfd_kernel(FwdDesc d) {
  using P = DfdP;
  using A = Ar<P>;
  using C = float4;
  using R = dfr;
  constexpr int T = dfd_threads<L, NP>();
  constexpr DifPlan pl = dfd_plan(L);
  constexpr int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int groups = (d.out_cols + NCH - 1) / NCH;
  const int row = blockIdx.x / groups;
  const int c0 = (blockIdx.x - row * groups) * NCH;
  const int b = blockIdx.y;
  const int64_t xo = b * d.x_ld_b + row * d.x_ld_row;
  const C* twd = static_cast<const C*>(d.twdd);
  const C zero = A::mk(A::zero(), A::zero());
  // range scaling: right-hand side b is divided by 2^e_b as it loads
  const int in_exp = d.in_absmax != nullptr ? range_exp(d.in_absmax[b]) : 0;
  const bool scaled = in_exp != 0;
  const double insc = scaled ? ldexp(1.0, -in_exp) : 1.0;

  // pass 0 straight from HBM: butterfly j takes samples j + q S_0, q < R_0 / 2
  // (t >= L/2 >= Nt is padding, never read nor added); SC: range-scaled loads
  // (the pass is instantiated once per case)
  auto first = [&](auto sc_t) {
    constexpr bool SC = decltype(sc_t)::value;
    constexpr int R0 = dfd_plan(L).rad[0], S0 = dfd_S(L, 0), ES = S0 * NP;
    static_assert(R0 % 2 == 0, "the first radix skips the zero half");
    auto cvt = [&](Tin x) -> R {
      if constexpr (SC) return cvt_real_scaled<P, Tin>(x, d.pad_single, insc);
      else return cvt_real<P, Tin>(x, d.pad_single);
    };
#pragma unroll 1
    for (int bt = threadIdx.x; bt < S0 * NP; bt += T) {
      const int p = bt % NP, j = bt / NP;
      const int c = c0 + 2 * p;
      C v[R0];
#pragma unroll
      for (int q = 0; q < R0 / 2; ++q) {
        const int t = j + q * S0;
        v[q] = zero;
        if (t < d.Nt && c < d.cols) {
          const int64_t o = xo + t * d.x_ld_t + c;
          if (d.pair_ok && c + 1 < d.cols) {   // both channels in one 8- or 16-byte load
            using V = typename std::conditional<sizeof(Tin) == 4, float2, double2>::type;
            const V x = __ldg(reinterpret_cast<const V*>(static_cast<const Tin*>(d.x) + o));
            v[q] = A::mk(cvt(x.x), cvt(x.y));
          } else {
            const Tin* xp = static_cast<const Tin*>(d.x) + o;
            v[q] = A::mk(cvt(__ldg(xp)), cvt(c + 1 < d.cols ? __ldg(xp + 1) : Tin(0)));
          }
        }
      }
#pragma unroll
      for (int q = R0 / 2; q < R0; ++q) v[q] = zero;
      DftHalf<P, R0, false>::run(v);
      dfd_twiddle<false, R0>(v, twd + j * (R0 - 1));
      C* base = buf + dfd_e<L, NP>(j, p);
#pragma unroll
      for (int q = 0; q < R0; ++q) base[q * ES] = v[q];
    }
  };
  if (scaled) first(std::true_type{});
  else first(std::false_type{});
  __syncthreads();
  dfd_passes<false, NP, L, 1, T>(buf, twd, pl.n);

  // split: X_a = (Z_w + conj Z_{L-w}) / 2,  X_b = (Z_w - conj Z_{L-w}) / (2i);
  // frequency-major spectra X[b][w][row][col].  A thread takes one channel
  // pair at one frequency (the two positions found once), consecutive
  // threads on consecutive pairs.
  const int64_t Xo = b * d.X_ld_b + row * d.X_ld_row;
  for (int i = threadIdx.x; i < Nf * NP; i += T) {
    const int w = i / NP, p = i - w * NP;
    const int c = c0 + 2 * p;
    if (c >= d.out_cols) continue;
    R ar = A::zero(), ai = A::zero(), br = A::zero(), bi = A::zero();
    if (c < d.cols) {
      const C z = buf[dfd_e<L, NP>(dfd_pos<L>(w), p)];
      const C zc = buf[dfd_e<L, NP>(dfd_pos<L>(w == 0 ? 0 : L - w), p)];
      ar = A::half(A::add(A::re(z), A::re(zc)));
      ai = A::half(A::sub(A::im(z), A::im(zc)));
      if (c + 1 < d.cols) {
        br = A::half(A::add(A::im(z), A::im(zc)));
        bi = A::half(A::sub(A::re(zc), A::re(z)));
      }
    }
    const int64_t o = Xo + w * d.X_ld_w + c;
    store_cx<P>(d.X, o, d.fmt, ar, ai);
    if (c + 1 < d.out_cols) store_cx<P>(d.X, o + 1, d.fmt, br, bi);
  }
}

// Inverse: Hermitian assembly + inverse complex FFT + unpad; grid (channel
// group, K), as irfft_inv_kernel.  The last pass writes t < Nt straight to HBM
// (1/L scale, range scaling, unpad and output cast fused).
// HALF: Nt = L / 2, so which of the final pass's outputs fall in t < Nt is
// known at compile time
template <typename Tout, int NP, int L, bool HALF>
__global__ void __launch_bounds__(dfd_threads<L, NP>(), FFTMV_DFD_MINB) irfft_dfd_kernel(InvDesc d) {
  using P = DfdP;
  using A = Ar<P>;
  using C = float4;
  constexpr int T = dfd_threads<L, NP>();
  constexpr DifPlan pl = dfd_plan(L);
  constexpr int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int c0 = blockIdx.x * NCH;
  const int b = blockIdx.y;
  const int64_t Xo = b * d.X_ld_b;
  const C zero = A::mk(A::zero(), A::zero());
  // Z_w = X_a(w) + i X_b(w) over the full circle, X(L-w) = conj X(w); the DC
  // and Nyquist terms are taken as real.  Thread i reads channel pair i % NP
  // at frequency i / NP; U of them in flight.
  constexpr int U = 4;
  const bool midsc = d.rhs_absmax != nullptr && d.in_fmt == FMT_C128 && d.mid_exp != 0;
  const double midf = midsc ? ldexp(1.0, d.mid_exp) : 1.0;
  for (int i0 = threadIdx.x; i0 < Nf * NP; i0 += U * T) {
    C a[U], bb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * T;
      const int w = i / NP, p = i - w * NP;
      const int ca = c0 + 2 * p, cb = ca + 1;
      const bool in = i < Nf * NP;
      if (in && d.pair_ok && cb < d.cols) {   // FP32 spectra of both channels in one 16-byte load
        const float4 v = __ldg(reinterpret_cast<const float4*>(static_cast<const float2*>(d.X) + Xo + w * d.X_ld_w + ca));
        a[u] = A::mk(A::from_f(v.x), A::from_f(v.y));
        bb[u] = A::mk(A::from_f(v.z), A::from_f(v.w));
      } else if (midsc) {   // FP64 spectra brought into the double-float range
        a[u] = in && ca < d.cols ? load_cx_scaled<P>(d.X, Xo + w * d.X_ld_w + ca, midf) : zero;
        bb[u] = in && cb < d.cols ? load_cx_scaled<P>(d.X, Xo + w * d.X_ld_w + cb, midf) : zero;
      } else {
        a[u] = in && ca < d.cols ? load_cx<P>(d.X, Xo + w * d.X_ld_w + ca, d.in_fmt) : zero;
        bb[u] = in && cb < d.cols ? load_cx<P>(d.X, Xo + w * d.X_ld_w + cb, d.in_fmt) : zero;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * T;
      if (i >= Nf * NP) break;
      const int w = i / NP, p = i - w * NP;
      if (w == 0 || w == Nf - 1) {
        buf[dfd_e<L, NP>(w, p)] = A::mk(A::re(a[u]), A::re(bb[u]));
      } else {
        buf[dfd_e<L, NP>(w, p)] = A::mk(A::sub(A::re(a[u]), A::im(bb[u])), A::add(A::im(a[u]), A::re(bb[u])));
        buf[dfd_e<L, NP>(L - w, p)] = A::mk(A::add(A::re(a[u]), A::im(bb[u])), A::sub(A::re(bb[u]), A::im(a[u])));
      }
    }
  }
  __syncthreads();
  const C* twd = static_cast<const C*>(d.twdd);
  dfd_passes<true, NP, L, 0, T>(buf, twd, pl.n - 1);

  const Kc inv_L{d.inv_L, d.inv_L_hi, d.inv_L_lo};
  // range scaling: outputs of right-hand side b times 2^(e_b + out_exp), in two
  // exact steps (each factor a normal double; the product may not be)
  const int oexp = d.rhs_absmax != nullptr ? range_exp(d.rhs_absmax[b]) + d.out_exp : 0;
  const bool scaled = oexp != 0;
  double s1 = 1.0, s2 = 1.0;
  if (scaled) {
    s1 = ldexp(1.0, oexp / 2);
    s2 = ldexp(1.0, oexp - oexp / 2);
  }
  // last pass: blocks of R contiguous positions; output q of block blk is time
  // t = tb(blk) + (L / R) q, tb from the digits of blk's position.  SC:
  // range-scaled outputs (the pass is instantiated once per case)
  auto last = [&](auto sc_t) {
    constexpr bool SC = decltype(sc_t)::value;
    constexpr int s = dfd_plan(L).n - 1;
    constexpr int R = dfd_plan(L).rad[s];
    constexpr int NBUT = (L / R) * NP;
#pragma unroll 1
    for (int bt = threadIdx.x; bt < NBUT; bt += T) {
      const int p = bt % NP, blk = bt / NP;
      const int c = c0 + 2 * p;
      C* base = buf + dfd_e<L, NP>(blk * R, p);
      C v[R];
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = base[q * NP];
      Dft<P, R, true>::run(v);
      if (c >= d.cols) continue;
      int rest = blk * R, tb = 0, mul = 1;
#pragma unroll
      for (int k = 0; k < s; ++k) {
        tb += (rest / dfd_S(L, k)) * mul;
        rest %= dfd_S(L, k);
        mul *= dfd_plan(L).rad[k];
      }
      const bool two = c + 1 < d.cols;
      const int64_t o0 = b * d.y_ld_b + (int64_t)tb * d.y_ld_t + c;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if constexpr (HALF) {
          if ((q * (L / R)) >= L / 2) continue;
          if ((q + 1) * (L / R) > L / 2 && tb + (L / R) * q >= L / 2) continue;
        } else {
          if (tb + (L / R) * q >= d.Nt) continue;
        }
        const int64_t o = o0 + (int64_t)q * (L / R) * d.y_ld_t;
        if constexpr (SC) {
          store_real_scaled<Tout, P>(d.y, o, A::mulk(A::re(v[q]), inv_L), d.unpad_single, s1, s2);
          if (two) store_real_scaled<Tout, P>(d.y, o + 1, A::mulk(A::im(v[q]), inv_L), d.unpad_single, s1, s2);
        } else {
          store_real<Tout, P>(d.y, o, A::mulk(A::re(v[q]), inv_L), d.unpad_single);
          if (two) store_real<Tout, P>(d.y, o + 1, A::mulk(A::im(v[q]), inv_L), d.unpad_single);
        }
      }
    }
  };
  if (scaled) last(std::true_type{});
  else last(std::false_type{});
}

// the double-float in-place kernels apply (fft_launch.cuh falls back to the
// Stockham kernels otherwise): a length with a dfd_plan, its twiddle table,
// the full tile of channel pairs, and no tensor-core output
template <int L>
bool dfd_fwd_ok(const FwdDesc& d, int np) {
  return dfd_plan(L).n > 0 && d.twdd != nullptr && d.fmt != FMT_TC && np == fft_pairs<DfdP>(L) && 2 * d.Nt <= L;
}
template <int L>
bool dfd_inv_ok(const InvDesc& d, int np) {
  return dfd_plan(L).n > 0 && d.twdd != nullptr && np == fft_pairs<DfdP>(L) && d.Nt <= L;
}

template <typename Tin, int L>
cudaError_t fwd_dfd_launch(const FwdDesc& d, cudaStream_t s) {
  constexpr int NP = fft_pairs<DfdP>(L);
  const int groups = (d.out_cols + 2 * NP - 1) / (2 * NP);
  dim3 grid(d.rows * groups, d.K);
  constexpr size_t smem = (size_t)dfd_smem_elems<L, NP>() * sizeof(float4);
  cudaError_t e = prep(rfft_dfd_kernel<Tin, NP, L>, smem);
  if (e != cudaSuccess) return e;
  rfft_dfd_kernel<Tin, NP, L><<<grid, dfd_threads<L, NP>(), smem, s>>>(d);
  return cudaGetLastError();
}

template <typename Tout, int L, bool HALF>
cudaError_t inv_dfd_launch_h(const InvDesc& d, cudaStream_t s) {
  constexpr int NP = fft_pairs<DfdP>(L);
  dim3 grid((d.cols + 2 * NP - 1) / (2 * NP), d.K);
  constexpr size_t smem = (size_t)dfd_smem_elems<L, NP>() * sizeof(float4);
  cudaError_t e = prep(irfft_dfd_kernel<Tout, NP, L, HALF>, smem);
  if (e != cudaSuccess) return e;
  irfft_dfd_kernel<Tout, NP, L, HALF><<<grid, dfd_threads<L, NP>(), smem, s>>>(d);
  return cudaGetLastError();
}
template <typename Tout, int L>
cudaError_t inv_dfd_launch(const InvDesc& d, cudaStream_t s) {
#if FFTMV_DIF_HALF
  if (2 * d.Nt == L) return inv_dfd_launch_h<Tout, L, true>(d, s);
#endif
  return inv_dfd_launch_h<Tout, L, false>(d, s);
}

// launch the double-float in-place kernel when it applies; false: it does not
template <typename Tin>
bool fwd_dfd_try(const FwdDesc& d, int np, cudaStream_t s, cudaError_t& e) {
  switch (d.plan.L) {
    case 2000:
      if (!dfd_fwd_ok<2000>(d, np)) return false;
      e = fwd_dfd_launch<Tin, 2000>(d, s);
      return true;
    case 1000:
      if (!dfd_fwd_ok<1000>(d, np)) return false;
      e = fwd_dfd_launch<Tin, 1000>(d, s);
      return true;
    default: return false;
  }
}
template <typename Tout>
bool inv_dfd_try(const InvDesc& d, int np, cudaStream_t s, cudaError_t& e) {
  switch (d.plan.L) {
    case 2000:
      if (!dfd_inv_ok<2000>(d, np)) return false;
      e = inv_dfd_launch<Tout, 2000>(d, s);
      return true;
    case 1000:
      if (!dfd_inv_ok<1000>(d, np)) return false;
      e = inv_dfd_launch<Tout, 1000>(d, s);
      return true;
    default: return false;
  }
}

}  // namespace
}  // namespace fftmv
