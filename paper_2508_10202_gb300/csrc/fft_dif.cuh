// In-place decimation-in-frequency FFTs for the compile-time lengths in FP32
// (Section 2.4: phases 1-2, zero pad + forward real FFT, and phases 4-5,
// inverse real FFT + unpad; the multi-right-hand-side path runs them).
//
// The same CTA tiling as the Stockham kernels of fft_core.cuh (NP channel
// pairs per CTA, pair (c, c+1) packed as one complex signal, the NP signals
// interleaved in shared memory), but each pass is the Gentleman-Sande
// decimation-in-frequency step of a DifPlan (fftmv_internal.h): a butterfly
// reads its rad[s] inputs, transforms them, multiplies by its twiddles and
// writes them back to the same places.  Butterflies own disjoint positions, so
// a thread handles one butterfly at a time with no barrier between its reads
// and writes (one barrier per pass), and every position a butterfly touches is
// a compile-time offset from one base address: no per-element index or
// swizzle arithmetic.  Twiddles come from a per-plan table laid out row by
// row (one 16-byte-aligned row per butterfly, read with vector loads).  The
// transform ends in digit-reversed order, which the output stage (forward) or
// the final store (inverse) undoes by index.
//
// Shared memory: element (pos, p) at pos NP + p, plus kDifPad elements after
// each block of S_0 positions.  The forward output stage reads consecutive
// frequencies, which lie S_0 positions apart; the padding puts consecutive
// threads' 16-byte reads on different banks.  The butterflies of every pass
// read consecutive elements across consecutive threads.
#pragma once

#include "fft_core.cuh"

namespace fftmv {
namespace {

constexpr int kDifPad = 2;
#ifndef FFTMV_DIF_HALF
#define FFTMV_DIF_HALF 1
#endif
#ifndef FFTMV_DIF_UNROLL
#define FFTMV_DIF_UNROLL 1
#endif
constexpr int kDifUnroll = FFTMV_DIF_UNROLL;

template <int L, int NP>
__device__ __forceinline__ int dif_e(int pos, int p) {
  constexpr int S0 = dif_S(L, 0);
  return pos * NP + p + (pos / S0) * kDifPad;
}
template <int L, int NP>
__host__ __device__ constexpr int dif_smem_elems() {
  return L * NP + dif_plan(L).rad[0] * kDifPad;
}
// element stride between the inputs of a pass-s butterfly
template <int L, int NP, int s>
__host__ __device__ constexpr int dif_es() {
  return s == 0 ? dif_S(L, 0) * NP + kDifPad : dif_S(L, s) * NP;
}
// threads: enough for one butterfly of the largest radix each (at least 64)
template <int L, int NP>
__host__ __device__ constexpr int dif_threads() {
  int rmax = 1;
  for (int s = 0; s < dif_plan(L).n; ++s) rmax = dif_plan(L).rad[s] > rmax ? dif_plan(L).rad[s] : rmax;
  const int t = (NP * L / rmax + 31) / 32 * 32;
  return t < 64 ? 64 : t;
}
#ifndef FFTMV_DIF_MINB
#define FFTMV_DIF_MINB 2
#endif
template <int L, int NP>
__host__ __device__ constexpr int dif_min_blocks() {
  return dif_threads<L, NP>() <= 320 ? FFTMV_DIF_MINB : 1;
}

// the position of index k (frequency of the forward, time of the inverse)
// once every pass has run: digit reversal over the plan's radices
template <int L>
__device__ __forceinline__ int dif_pos(int k) {
  constexpr DifPlan pl = dif_plan(L);
  int pos = 0;
#pragma unroll
  for (int s = 0; s < pl.n; ++s) {
    pos += (k % pl.rad[s]) * dif_S(L, s);
    k /= pl.rad[s];
  }
  return pos;
}

// a twiddle-table row (W^{j q}, q = 1 .. R-1, two per 16-byte load), loaded
// ahead of the butterfly's data so that both latencies overlap
template <int R>
struct DifTw {
  float4 w[dif_tw_row(R) / 2];
  __device__ __forceinline__ void load(const float2* __restrict__ row) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int h = 0; h < dif_tw_row(R) / 2; ++h) w[h] = __ldg(r4 + h);
  }
  // v[q] *= W^{j q} (INV: conj), q = 1 .. R-1
  template <bool INV>
  __device__ __forceinline__ void apply(float2* v) const {
#pragma unroll
    for (int h = 0; h < dif_tw_row(R) / 2; ++h) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = 1 + 2 * h + u;
        if (q < R) {
          const float wr = u ? w[h].z : w[h].x, wi = u ? w[h].w : w[h].y;
          const float2 a = v[q];
          v[q] = INV ? make_float2(fmaf(a.x, wr, a.y * wi), fmaf(a.y, wr, -(a.x * wi)))
                     : make_float2(fmaf(a.x, wr, -(a.y * wi)), fmaf(a.x, wi, a.y * wr));
        }
      }
    }
  }
};

// pass s (of the plan) in shared memory
template <bool INV, int NP, int L, int s, int T>
__device__ __forceinline__ void dif_pass(float2* __restrict__ buf, const float2* __restrict__ twd) {
  constexpr int R = dif_plan(L).rad[s], M = dif_M(L, s), S = M / R;
  constexpr int NBUT = (L / M) * S * NP;
  constexpr int ES = dif_es<L, NP, s>();
#pragma unroll kDifUnroll
  for (int bt = threadIdx.x; bt < NBUT; bt += T) {
    const int p = bt % NP, r = bt / NP, j = r % S, blk = r / S;
    float2* base = buf + dif_e<L, NP>(blk * M + j, p);
    DifTw<R> tw;
    if constexpr (S > 1) tw.load(twd + dif_tw_offset(L, s) + j * dif_tw_row(R));
    float2 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = base[q * ES];
    Dft<float, R, INV>::run(v);
    if constexpr (S > 1) tw.template apply<INV>(v);
#pragma unroll
    for (int q = 0; q < R; ++q) base[q * ES] = v[q];
  }
}

template <bool INV, int NP, int L, int s, int T>
__device__ __forceinline__ void dif_passes(float2* __restrict__ buf, const float2* __restrict__ twd, int last) {
  if constexpr (s < dif_plan(L).n) {
    if (s < last) {
      dif_pass<INV, NP, L, s, T>(buf, twd);
      __syncthreads();
      dif_passes<INV, NP, L, s + 1, T>(buf, twd, last);
    }
  }
}

// Forward: pad + real FFT; grid (row x channel group, K), as rfft_fwd_kernel.
template <typename Tin, int NP, int L>
__global__ void __launch_bounds__(dif_threads<L, NP>(), dif_min_blocks<L, NP>()) rfft_dif_kernel(FwdDesc d) {
  using P = float;
  using A = Ar<P>;
  using C = float2;
  using R = float;
  constexpr int T = dif_threads<L, NP>();
  constexpr DifPlan pl = dif_plan(L);
  constexpr int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int groups = (d.out_cols + NCH - 1) / NCH;
  const int row = blockIdx.x / groups;
  const int c0 = (blockIdx.x - row * groups) * NCH;
  const int b = blockIdx.y;
  const int64_t xo = b * d.x_ld_b + row * d.x_ld_row;
  const C* twd = static_cast<const C*>(d.twd);
  const C zero = make_float2(0.f, 0.f);
  const int in_exp = d.in_absmax != nullptr ? range_exp(d.in_absmax[b]) : 0;
  const bool scaled = in_exp != 0;
  const double insc = scaled ? ldexp(1.0, -in_exp) : 1.0;

  // sample t of channels (c, c+1), with the pad cast and zero padding
  auto gload = [&](int t, int c) -> C {
    if (t >= d.Nt || c >= d.cols) return zero;
    const int64_t o = xo + t * d.x_ld_t + c;
    if (d.pair_ok && c + 1 < d.cols) {
      using V = typename std::conditional<sizeof(Tin) == 4, float2, double2>::type;
      const V v = __ldg(reinterpret_cast<const V*>(static_cast<const Tin*>(d.x) + o));
      if (scaled)
        return A::mk(cvt_real_scaled<P, Tin>(v.x, d.pad_single, insc), cvt_real_scaled<P, Tin>(v.y, d.pad_single, insc));
      return A::mk(cvt_real<P, Tin>(v.x, d.pad_single), cvt_real<P, Tin>(v.y, d.pad_single));
    }
    const Tin* xp = static_cast<const Tin*>(d.x) + o;
    const Tin xa = __ldg(xp), xb = c + 1 < d.cols ? __ldg(xp + 1) : Tin(0);
    if (scaled) return A::mk(cvt_real_scaled<P, Tin>(xa, d.pad_single, insc), cvt_real_scaled<P, Tin>(xb, d.pad_single, insc));
    return A::mk(cvt_real<P, Tin>(xa, d.pad_single), cvt_real<P, Tin>(xb, d.pad_single));
  };

  // pass 0 straight from HBM: butterfly j takes samples j + q S_0; for an even
  // radix the upper half (t >= L/2 >= Nt) is padding, never read nor added
  {
    constexpr int R0 = pl.rad[0], S0 = dif_S(L, 0), ES = dif_es<L, NP, 0>();
    constexpr bool half = R0 % 2 == 0;
    // every channel of the CTA present and no padding below L/2: plain vector
    // loads at a fixed stride
    const bool fast = half && d.pair_ok && !scaled && c0 + NCH <= d.cols && 2 * d.Nt == L;
    using V = typename std::conditional<sizeof(Tin) == 4, float2, double2>::type;
    const int64_t st = (int64_t)S0 * d.x_ld_t;
#pragma unroll 1
    for (int bt = threadIdx.x; bt < S0 * NP; bt += T) {
      const int p = bt % NP, j = bt / NP;
      const int c = c0 + 2 * p;
      DifTw<R0> tw;
      tw.load(twd + j * dif_tw_row(R0));
      C v[R0];
      if (fast) {
        const Tin* xp = static_cast<const Tin*>(d.x) + xo + (int64_t)j * d.x_ld_t + c;
#pragma unroll
        for (int q = 0; q < R0 / 2; ++q) {
          const V x = __ldg(reinterpret_cast<const V*>(xp + q * st));
          v[q] = A::mk(cvt_real<P, Tin>(x.x, d.pad_single), cvt_real<P, Tin>(x.y, d.pad_single));
        }
#pragma unroll
        for (int q = R0 / 2; q < R0; ++q) v[q] = zero;
      } else {
#pragma unroll
        for (int q = 0; q < R0; ++q) v[q] = (half && q >= R0 / 2) ? zero : gload(j + q * S0, c);
      }
      if constexpr (half) DftHalf<P, R0, false>::run(v);
      else Dft<P, R0, false>::run(v);
      tw.template apply<false>(v);
      C* base = buf + dif_e<L, NP>(j, p);
#pragma unroll
      for (int q = 0; q < R0; ++q) base[q * ES] = v[q];
    }
  }
  __syncthreads();
  dif_passes<false, NP, L, 1, T>(buf, twd, pl.n);

  // real/imaginary split of pair p at frequency w from Z at w and L - w:
  //   X_a = (Z_w + conj Z_{L-w}) / 2,  X_b = (Z_w - conj Z_{L-w}) / (2i)
  // Positions of the frequencies a thread visits: it steps w by DW, a multiple
  // of the product PI of all radices but the last, which moves the last digit
  // only, so the positions of w and of L - w move by +-DW / PI (their first
  // digit, and with it the padding, stays put).
  constexpr int PI = L / pl.rad[pl.n - 1];
  if (d.fmt == FMT_TC) {
    // bf16 (or FP16) hi/lo B planes [2][J][ldb/g][Nf][g] (g = 2^tc_group_log2):
    // a thread takes one frequency and G adjacent channels and writes them as
    // one 2G-byte run into each of the four rows (Re, Im) x (hi, lo);
    // consecutive threads take consecutive frequencies.  The planes hold 2 X:
    // the split's 1/2 is applied in the contraction's epilogue.
    constexpr int G = NCH < 8 ? NCH : 8;
    constexpr int NG = NCH / G;
    constexpr int DW = T / NG;
    static_assert(DW % PI == 0, "frequency step must keep the leading digits");
    using Vec = typename std::conditional<G == 8, uint4, typename std::conditional<G == 4, uint2, uint32_t>::type>::type;
    unsigned short* B = static_cast<unsigned short*>(d.X);
    const bool f16 = d.tc_inv_scale != nullptr;
    const float sc = f16 ? d.tc_inv_scale[b] : 1.f;
    const int ch = b / d.tc_KC, q = b - ch * d.tc_KC;
    const int64_t jr = (int64_t)ch * d.tc_N + q, ji = jr + d.tc_KC;
    const int64_t row_el = (int64_t)d.out_cols * Nf;
    const int64_t plane_el = (int64_t)d.tc_J * row_el;
    const int g = threadIdx.x % NG, w0 = threadIdx.x / NG;
    const int cg = g * G, c = c0 + cg;
    if (c >= d.out_cols) return;
    const bool full = c + G <= d.cols;
    const int sh = d.tc_group_log2;
    unsigned short* Bw = B + jr * row_el + ((((int64_t)(c >> sh) * Nf + w0) << sh) + (c & ((1 << sh) - 1)));
    const int64_t di = (ji - jr) * row_el;
    int ew = dif_e<L, NP>(dif_pos<L>(w0), cg / 2);
    int ec = w0 == 0 ? dif_e<L, NP>(dif_pos<L>(L - DW), cg / 2) + (DW / PI) * NP : dif_e<L, NP>(dif_pos<L>(L - w0), cg / 2);
    // the loop once per (all channels present, FP16) case: no per-channel
    // checks or format branches inside
    auto run = [&](auto full_t, auto f16_t) {
      constexpr bool FULL = decltype(full_t)::value, F16 = decltype(f16_t)::value;
      int ew_ = ew, ec_ = ec;
      unsigned short* Bw_ = Bw;
      for (int w = w0; w < Nf; w += DW, ew_ += (DW / PI) * NP, ec_ -= (DW / PI) * NP, Bw_ += (int64_t)DW << sh) {
        const int ecw = w == 0 ? ew_ : ec_;
        C zw[G / 2], zc[G / 2];
        if constexpr (G >= 4) {
#pragma unroll
          for (int u = 0; u < G / 2; u += 2) {
            const float4 a = *reinterpret_cast<const float4*>(buf + ew_ + u);
            const float4 bq = *reinterpret_cast<const float4*>(buf + ecw + u);
            zw[u] = make_float2(a.x, a.y);
            zw[u + 1] = make_float2(a.z, a.w);
            zc[u] = make_float2(bq.x, bq.y);
            zc[u + 1] = make_float2(bq.z, bq.w);
          }
        } else {
#pragma unroll
          for (int u = 0; u < G / 2; ++u) {
            zw[u] = buf[ew_ + u];
            zc[u] = buf[ecw + u];
          }
        }
        // pair u of the G channels: X_a = Z_w + conj Z_{L-w}, X_b = (Z_w - conj Z_{L-w}) / i
        uint32_t hr[G / 2], lr[G / 2], hm[G / 2], lm[G / 2];   // Re hi, Re lo, Im hi, Im lo
#pragma unroll
        for (int u = 0; u < G / 2; ++u) {
          const C z = zw[u], y = zc[u];
          float ar = z.x + y.x, ai = z.y - y.y, br = z.y + y.y, bi = y.x - z.x;
          if constexpr (!FULL) {
            if (c + 2 * u >= d.cols) ar = ai = 0.f;
            if (c + 2 * u + 1 >= d.cols) br = bi = 0.f;
          }
          if constexpr (F16) {
            ar *= sc;
            ai *= sc;
            br *= sc;
            bi *= sc;
            const __half2 rh = __floats2half2_rn(ar, br), ih = __floats2half2_rn(ai, bi);
            const float2 rf = __half22float2(rh), mf = __half22float2(ih);
            const __half2 rl = __floats2half2_rn(ar - rf.x, br - rf.y), il = __floats2half2_rn(ai - mf.x, bi - mf.y);
            hr[u] = *reinterpret_cast<const uint32_t*>(&rh);
            lr[u] = *reinterpret_cast<const uint32_t*>(&rl);
            hm[u] = *reinterpret_cast<const uint32_t*>(&ih);
            lm[u] = *reinterpret_cast<const uint32_t*>(&il);
          } else {
            // bf16: hi = round(x); float(hi) of the low half is the word
            // shifted up, of the high half the word with its low half cleared
            const __nv_bfloat162 rh = __floats2bfloat162_rn(ar, br), ih = __floats2bfloat162_rn(ai, bi);
            const uint32_t rw = *reinterpret_cast<const uint32_t*>(&rh), iw = *reinterpret_cast<const uint32_t*>(&ih);
            const __nv_bfloat162 rl =
                __floats2bfloat162_rn(ar - __uint_as_float(rw << 16), br - __uint_as_float(rw & 0xFFFF0000u));
            const __nv_bfloat162 il =
                __floats2bfloat162_rn(ai - __uint_as_float(iw << 16), bi - __uint_as_float(iw & 0xFFFF0000u));
            hr[u] = rw;
            lr[u] = *reinterpret_cast<const uint32_t*>(&rl);
            hm[u] = iw;
            lm[u] = *reinterpret_cast<const uint32_t*>(&il);
          }
        }
        Vec vhr, vlr, vhm, vlm;
        if constexpr (G == 8) {
          vhr = make_uint4(hr[0], hr[1], hr[2], hr[3]);
          vlr = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          vhm = make_uint4(hm[0], hm[1], hm[2], hm[3]);
          vlm = make_uint4(lm[0], lm[1], lm[2], lm[3]);
        } else if constexpr (G == 4) {
          vhr = make_uint2(hr[0], hr[1]);
          vlr = make_uint2(lr[0], lr[1]);
          vhm = make_uint2(hm[0], hm[1]);
          vlm = make_uint2(lm[0], lm[1]);
        } else {
          vhr = hr[0];
          vlr = lr[0];
          vhm = hm[0];
          vlm = lm[0];
        }
        *reinterpret_cast<Vec*>(Bw_) = vhr;
        *reinterpret_cast<Vec*>(Bw_ + plane_el) = vlr;
        *reinterpret_cast<Vec*>(Bw_ + di) = vhm;
        *reinterpret_cast<Vec*>(Bw_ + di + plane_el) = vlm;
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (full) {
      if (f16) run(T_{}, T_{});
      else run(T_{}, F_{});
    } else {
      if (f16) run(F_{}, T_{});
      else run(F_{}, F_{});
    }
    return;
  }
  // frequency-major spectra X[b][w][row][col]: a thread takes one channel
  // pair at every DW-th frequency (consecutive threads on consecutive pairs),
  // and FP32 spectra go out as one 16-byte store
  const int64_t Xo = b * d.X_ld_b + row * d.X_ld_row;
  const bool vec = d.fmt == FMT_C64 && ((d.X_ld_w | d.X_ld_b | d.X_ld_row) & 1) == 0;
  constexpr int DW = T / NP;
  constexpr bool incr = DW % PI == 0;
  const int p = threadIdx.x % NP, w0 = threadIdx.x / NP;
  const int c = c0 + 2 * p;
  if (c >= d.out_cols) return;
  int ew = dif_e<L, NP>(dif_pos<L>(w0), p);
  int ec = w0 == 0 ? dif_e<L, NP>(dif_pos<L>(L - DW), p) + (DW / PI) * NP : dif_e<L, NP>(dif_pos<L>(L - w0), p);
  for (int w = w0; w < Nf; w += DW) {
    if constexpr (!incr) {
      ew = dif_e<L, NP>(dif_pos<L>(w), p);
      ec = dif_e<L, NP>(dif_pos<L>(w == 0 ? 0 : L - w), p);
    }
    const C z = buf[ew];
    const C zc = buf[w == 0 ? ew : ec];
    if constexpr (incr) {
      ew += (DW / PI) * NP;
      ec -= (DW / PI) * NP;
    }
    R ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
    if (c < d.cols) {
      ar = 0.5f * (z.x + zc.x);
      ai = 0.5f * (z.y - zc.y);
    }
    if (c + 1 < d.cols) {
      br = 0.5f * (z.y + zc.y);
      bi = 0.5f * (zc.x - z.x);
    }
    const int64_t o = Xo + w * d.X_ld_w + c;
    if (vec && c + 1 < d.out_cols) {
      *reinterpret_cast<float4*>(static_cast<float2*>(d.X) + o) = make_float4(ar, ai, br, bi);
    } else {
      store_cx<P>(d.X, o, d.fmt, ar, ai);
      if (c + 1 < d.out_cols) store_cx<P>(d.X, o + 1, d.fmt, br, bi);
    }
  }
}

// Inverse: Hermitian assembly + inverse complex FFT + unpad; grid (channel
// group, K), as irfft_inv_kernel.  The last pass writes t < Nt straight to HBM.
// HALF: Nt = L / 2, so which of the final pass's outputs fall in t < Nt is
// known at compile time (all of the first R/2, none past it but one)
template <typename Tout, int NP, int L, bool HALF>
__global__ void __launch_bounds__(dif_threads<L, NP>(), dif_min_blocks<L, NP>()) irfft_dif_kernel(InvDesc d) {
  using P = float;
  using A = Ar<P>;
  using C = float2;
  constexpr int T = dif_threads<L, NP>();
  constexpr DifPlan pl = dif_plan(L);
  constexpr int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int c0 = blockIdx.x * NCH;
  const int b = blockIdx.y;
  const int64_t Xo = b * d.X_ld_b;
  const C zero = make_float2(0.f, 0.f);
  // Z_w = X_a(w) + i X_b(w) over the full circle, X(L-w) = conj X(w); the DC
  // and Nyquist terms are taken as real.  Loads in flight as in irfft_inv_kernel.
  constexpr int U = fft_inv_loads(sizeof(C), 25, Nf, NP, T);
  const bool midsc = d.rhs_absmax != nullptr && d.in_fmt == FMT_C128 && d.mid_exp != 0;
  const double midf = midsc ? ldexp(1.0, d.mid_exp) : 1.0;
  // every channel of the CTA present in FP32 pairs: one 16-byte load per
  // item and no per-item checks but the end of the spectrum
  // (variants that issue the pair loads without the per-item branches were
  // slower at K = 64: checks hoisted out or indices clamped, 2.70 against
  // 2.48 ms; every address and position a compile-time offset from the
  // thread's own, with the edge items found at compile time, 2.53 against
  // 2.44 ms)
  for (int i0 = threadIdx.x; i0 < Nf * NP; i0 += U * T) {
    C a[U], bb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * T;
      const int w = i / NP, p = i - w * NP;
      const int ca = c0 + 2 * p, cb = ca + 1;
      const bool in = i < Nf * NP;
      if (in && d.pair_ok && cb < d.cols) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(static_cast<const float2*>(d.X) + Xo + w * d.X_ld_w + ca));
        a[u] = make_float2(v.x, v.y);
        bb[u] = make_float2(v.z, v.w);
      } else if (midsc) {
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
        buf[dif_e<L, NP>(w, p)] = make_float2(a[u].x, bb[u].x);
      } else {
        buf[dif_e<L, NP>(w, p)] = make_float2(a[u].x - bb[u].y, a[u].y + bb[u].x);
        buf[dif_e<L, NP>(L - w, p)] = make_float2(a[u].x + bb[u].y, bb[u].x - a[u].y);
      }
    }
  }
  __syncthreads();
  const C* twd = static_cast<const C*>(d.twd);
  dif_passes<true, NP, L, 0, T>(buf, twd, pl.n - 1);

  // last pass: contiguous blocks of R points; output q of block blk is time
  // t = tb(blk) + (L / R) q, tb from the digits of blk's position
  constexpr int s = pl.n - 1;
  constexpr int R = pl.rad[s];
  constexpr int NBUT = (L / R) * NP;
  const int oexp = d.rhs_absmax != nullptr ? range_exp(d.rhs_absmax[b]) + d.out_exp : 0;
  const bool scaled = oexp != 0;
  double s1 = 1.0, s2 = 1.0;
  if (scaled) {
    s1 = ldexp(1.0, oexp / 2);
    s2 = ldexp(1.0, oexp - oexp / 2);
  }
  const float invL = (float)d.inv_L;
  const bool vec = d.out_pair_ok && !d.unpad_single && !scaled;
  const int Nt = d.Nt;
  const int64_t ystep = (int64_t)(L / R) * d.y_ld_t;
#pragma unroll 1
  for (int bt = threadIdx.x; bt < NBUT; bt += T) {
    const int p = bt % NP, blk = bt / NP;
    const int c = c0 + 2 * p;
    C* base = buf + dif_e<L, NP>(blk * R, p);
    C v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = base[q * NP];
    Dft<P, R, true>::run(v);
    if (c >= d.cols) continue;
    int rest = blk * R, tb = 0, mul = 1;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      tb += (rest / dif_S(L, k)) * mul;
      rest %= dif_S(L, k);
      mul *= pl.rad[k];
    }
    Tout* yb = static_cast<Tout*>(d.y) + b * d.y_ld_b + (int64_t)tb * d.y_ld_t + c;
    const bool two = c + 1 < d.cols;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if constexpr (HALF) {
        // t = tb + (L/R) q with 0 <= tb < L/R: always below L/2 for
        // (q + 1) (L/R) <= L/2, never for q (L/R) >= L/2
        if ((q * (L / R)) >= L / 2) continue;
        if ((q + 1) * (L / R) > L / 2 && tb + (L / R) * q >= L / 2) continue;
      } else {
        if (tb + (L / R) * q >= Nt) continue;
      }
      Tout* yq = yb + q * ystep;
      const float re = v[q].x * invL, im = v[q].y * invL;
      if (vec && two) {
        using V = typename std::conditional<sizeof(Tout) == 4, float2, double2>::type;
        V pv;
        pv.x = (Tout)re;
        pv.y = (Tout)im;
        *reinterpret_cast<V*>(yq) = pv;
      } else if (scaled) {
        store_real_scaled<Tout, P>(yq, 0, re, d.unpad_single, s1, s2);
        if (two) store_real_scaled<Tout, P>(yq, 1, im, d.unpad_single, s1, s2);
      } else {
        store_real<Tout, P>(yq, 0, re, d.unpad_single);
        if (two) store_real<Tout, P>(yq, 1, im, d.unpad_single);
      }
    }
  }
}

template <typename Tin, int NP, int L>
cudaError_t fwd_dif_launch(const FwdDesc& d, cudaStream_t s) {
  const int groups = (d.out_cols + 2 * NP - 1) / (2 * NP);
  dim3 grid(d.rows * groups, d.K);
  constexpr size_t smem = (size_t)dif_smem_elems<L, NP>() * sizeof(float2);
  cudaError_t e = prep(rfft_dif_kernel<Tin, NP, L>, smem);
  if (e != cudaSuccess) return e;
  rfft_dif_kernel<Tin, NP, L><<<grid, dif_threads<L, NP>(), smem, s>>>(d);
  return cudaGetLastError();
}

template <typename Tout, int NP, int L, bool HALF>
cudaError_t inv_dif_launch_h(const InvDesc& d, cudaStream_t s) {
  dim3 grid((d.cols + 2 * NP - 1) / (2 * NP), d.K);
  constexpr size_t smem = (size_t)dif_smem_elems<L, NP>() * sizeof(float2);
  cudaError_t e = prep(irfft_dif_kernel<Tout, NP, L, HALF>, smem);
  if (e != cudaSuccess) return e;
  irfft_dif_kernel<Tout, NP, L, HALF><<<grid, dif_threads<L, NP>(), smem, s>>>(d);
  return cudaGetLastError();
}
template <typename Tout, int NP, int L>
cudaError_t inv_dif_launch(const InvDesc& d, cudaStream_t s) {
#if FFTMV_DIF_HALF
  if (2 * d.Nt == L) return inv_dif_launch_h<Tout, NP, L, true>(d, s);
#endif
  return inv_dif_launch_h<Tout, NP, L, false>(d, s);
}

}  // namespace
}  // namespace fftmv
