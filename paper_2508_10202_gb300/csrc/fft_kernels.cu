// Batched real FFTs along time for the block-Toeplitz matvec (Section 2.4,
// phases 1-2 and 4-5 of the paper's algorithm), written for sm_103a.
//
// One CTA transforms one pair of real channels (c, c+1) as the complex signal
// z = x_c + i x_{c+1}: the real-to-complex split is done in the epilogue
// (forward) or the Hermitian assembly in the prologue (inverse).  The complex
// FFT of length L = 2^a 3^b 5^c is a Stockham auto-sort sequence of radix-2,
// 3, 4, 5, 8 passes ping-ponging between two shared-memory buffers, so the
// result lands in natural order with no bit reversal.  Twiddles come from a
// per-length table exp(-2 pi i j / L) built once on the host.
//
// Zero padding (phase 1) and unpadding (phase 5) are fused: samples t >= Nt
// are zero in shared memory and never read from HBM, and only t < Nt is
// written back.  Casts between the I/O dtype, the pad/unpad precision and the
// FFT precision are fused into the loads and stores (Section 3.2).
//
// Arithmetic.  The same transform is instantiated for three precisions:
//   double : FP64 FMA (GB300 runs it at ~1.2 TFLOP/s, so FP64 FFTs are
//            FP64-pipe bound);
//   float  : FP32;
//   DFP    : double-float, an FP64-class format on the FP32 pipe.  A real is
//            an unevaluated pair hi + lo of floats (|lo| <= ulp(hi)/2, about
//            48 significant bits); sums use TwoSum + Fast2Sum renormalisation,
//            products an FMA-exact TwoProd plus the hi*lo cross terms.  The
//            adds are the normwise-accurate ("sloppy") double-word sums, which
//            is the accuracy an FFT's normwise error analysis needs.

#include <cuda_bf16.h>

#include <type_traits>

#include "fftmv_internal.h"

namespace fftmv {
namespace {

struct DFP {};  // precision tag: double-float on the FP32 pipe

// a real constant in every precision: FP64 value and its FP32 hi/lo split
struct Kc {
  double d;
  float h, l;
};
// cos/sin of 2 pi / 5, 4 pi / 5, pi / 3 and 1 / sqrt(2)
__device__ constexpr Kc KC1{0.30901699437494742410, 0.30901700258255005f, -8.207602597565256e-09f};
__device__ constexpr Kc KC2{-0.80901699437494742410, -0.80901700258255f, 8.207602597565256e-09f};
__device__ constexpr Kc KS1{0.95105651629515357212, 0.9510565400123596f, -2.3717205976936384e-08f};
__device__ constexpr Kc KS2{0.58778525229247312917, 0.5877852439880371f, 8.304436249773062e-09f};
__device__ constexpr Kc KS3{0.86602540378443864676, 0.8660253882408142f, 1.5543625053737742e-08f};
__device__ constexpr Kc KR2{0.70710678118654752440, 0.7071067690849304f, 1.2101617485882343e-08f};

// ---------------------------------------------------------------------------
// double-float reals
// ---------------------------------------------------------------------------
struct dfr {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dfr fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfr{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfr df_add(dfr a, dfr b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ dfr df_neg(dfr a) { return dfr{-a.h, -a.l}; }
__device__ __forceinline__ dfr df_mul(dfr a, dfr b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// a.re*b.re - s*a.im*b.im (s = +1) in one renormalisation
__device__ __forceinline__ dfr df_dot2(dfr a, dfr b, dfr c, dfr d, float sgn) {
  // a*b + sgn*c*d
  const float p1 = __fmul_rn(a.h, b.h);
  const float p2 = __fmul_rn(sgn * c.h, d.h);
  float e1 = __fmaf_rn(a.h, b.h, -p1);
  float e2 = __fmaf_rn(sgn * c.h, d.h, -p2);
  float s, t;
  two_sum(p1, p2, s, t);
  t = __fadd_rn(t, __fadd_rn(e1, e2));
  t = __fmaf_rn(a.h, b.l, t);
  t = __fmaf_rn(a.l, b.h, t);
  t = __fmaf_rn(sgn * c.h, d.l, t);
  t = __fmaf_rn(sgn * c.l, d.h, t);
  return fast_two_sum(s, t);
}

// ---------------------------------------------------------------------------
// arithmetic traits: reals R, complexes C (the shared-memory element)
// ---------------------------------------------------------------------------
template <typename P> struct Ar;

template <> struct Ar<double> {
  using R = double;
  using C = double2;
  __device__ __forceinline__ static R add(R a, R b) { return a + b; }
  __device__ __forceinline__ static R sub(R a, R b) { return a - b; }
  __device__ __forceinline__ static R neg(R a) { return -a; }
  __device__ __forceinline__ static R half(R a) { return 0.5 * a; }
  __device__ __forceinline__ static R mulk(R a, const Kc& k) { return a * k.d; }
  __device__ __forceinline__ static R re(C c) { return c.x; }
  __device__ __forceinline__ static R im(C c) { return c.y; }
  __device__ __forceinline__ static C mk(R r, R i) { return make_double2(r, i); }
  __device__ __forceinline__ static C cmul(C a, C w) {
    return make_double2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
  }
  __device__ __forceinline__ static C conj(C a) { return make_double2(a.x, -a.y); }
  __device__ __forceinline__ static R from_d(double x) { return x; }
  __device__ __forceinline__ static R from_f(float x) { return x; }
  __device__ __forceinline__ static double to_d(R x) { return x; }
  __device__ __forceinline__ static float to_f(R x) { return (float)x; }
  __device__ __forceinline__ static R zero() { return 0.0; }
};

template <> struct Ar<float> {
  using R = float;
  using C = float2;
  __device__ __forceinline__ static R add(R a, R b) { return a + b; }
  __device__ __forceinline__ static R sub(R a, R b) { return a - b; }
  __device__ __forceinline__ static R neg(R a) { return -a; }
  __device__ __forceinline__ static R half(R a) { return 0.5f * a; }
  __device__ __forceinline__ static R mulk(R a, const Kc& k) { return a * (float)k.d; }
  __device__ __forceinline__ static R re(C c) { return c.x; }
  __device__ __forceinline__ static R im(C c) { return c.y; }
  __device__ __forceinline__ static C mk(R r, R i) { return make_float2(r, i); }
  __device__ __forceinline__ static C cmul(C a, C w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
  }
  __device__ __forceinline__ static C conj(C a) { return make_float2(a.x, -a.y); }
  __device__ __forceinline__ static R from_d(double x) { return (float)x; }
  __device__ __forceinline__ static R from_f(float x) { return x; }
  __device__ __forceinline__ static double to_d(R x) { return x; }
  __device__ __forceinline__ static float to_f(R x) { return x; }
  __device__ __forceinline__ static R zero() { return 0.f; }
};

// complex double-float stored as float4 (re_hi, im_hi, re_lo, im_lo): the
// FMT_DF layout, so spectra move between phases without conversion
template <> struct Ar<DFP> {
  using R = dfr;
  using C = float4;
  __device__ __forceinline__ static R add(R a, R b) { return df_add(a, b); }
  __device__ __forceinline__ static R sub(R a, R b) { return df_add(a, df_neg(b)); }
  __device__ __forceinline__ static R neg(R a) { return df_neg(a); }
  __device__ __forceinline__ static R half(R a) { return dfr{0.5f * a.h, 0.5f * a.l}; }
  __device__ __forceinline__ static R mulk(R a, const Kc& k) { return df_mul(a, dfr{k.h, k.l}); }
  __device__ __forceinline__ static R re(C c) { return dfr{c.x, c.z}; }
  __device__ __forceinline__ static R im(C c) { return dfr{c.y, c.w}; }
  __device__ __forceinline__ static C mk(R r, R i) { return make_float4(r.h, i.h, r.l, i.l); }
  __device__ __forceinline__ static C cmul(C a, C w) {
    const dfr ar = re(a), ai = im(a), wr = re(w), wi = im(w);
    return mk(df_dot2(ar, wr, ai, wi, -1.f), df_dot2(ar, wi, ai, wr, 1.f));
  }
  __device__ __forceinline__ static C conj(C a) { return make_float4(a.x, -a.y, a.z, -a.w); }
  __device__ __forceinline__ static R from_d(double x) {
    const float h = (float)x;
    return dfr{h, (float)(x - (double)h)};
  }
  __device__ __forceinline__ static R from_f(float x) { return dfr{x, 0.f}; }
  __device__ __forceinline__ static double to_d(R x) { return (double)x.h + (double)x.l; }
  __device__ __forceinline__ static float to_f(R x) { return __fadd_rn(x.h, x.l); }
  __device__ __forceinline__ static R zero() { return dfr{0.f, 0.f}; }
};

// complex helpers built on the traits
template <typename P> struct Cx {
  using A = Ar<P>;
  using C = typename A::C;
  __device__ __forceinline__ static C add(C a, C b) { return A::mk(A::add(A::re(a), A::re(b)), A::add(A::im(a), A::im(b))); }
  __device__ __forceinline__ static C sub(C a, C b) { return A::mk(A::sub(A::re(a), A::re(b)), A::sub(A::im(a), A::im(b))); }
  __device__ __forceinline__ static C mulk(C a, const Kc& k) { return A::mk(A::mulk(A::re(a), k), A::mulk(A::im(a), k)); }
  // multiply by -i (forward) or +i (inverse)
  template <bool INV> __device__ __forceinline__ static C mmi(C a) {
    return INV ? A::mk(A::neg(A::im(a)), A::re(a)) : A::mk(A::im(a), A::neg(A::re(a)));
  }
};

// In-register DFT of size R: X_p = sum_q v_q exp(-+2 pi i q p / R).
template <typename P, int R, bool INV> struct Dft;

template <typename P, bool INV> struct Dft<P, 2, INV> {
  using C = typename Ar<P>::C;
  __device__ __forceinline__ static void run(C* v) {
    const C a = v[0], b = v[1];
    v[0] = Cx<P>::add(a, b);
    v[1] = Cx<P>::sub(a, b);
  }
};

template <typename P, bool INV> struct Dft<P, 3, INV> {
  using A = Ar<P>;
  using C = typename A::C;
  __device__ __forceinline__ static void run(C* v) {
    const C s = Cx<P>::add(v[1], v[2]);
    const C d = Cx<P>::mulk(Cx<P>::template mmi<INV>(Cx<P>::sub(v[1], v[2])), KS3);
    const C m = A::mk(A::sub(A::re(v[0]), A::half(A::re(s))), A::sub(A::im(v[0]), A::half(A::im(s))));
    v[0] = Cx<P>::add(v[0], s);
    v[1] = Cx<P>::add(m, d);
    v[2] = Cx<P>::sub(m, d);
  }
};

template <typename P, bool INV> struct Dft<P, 4, INV> {
  using C = typename Ar<P>::C;
  __device__ __forceinline__ static void run(C* v) {
    const C a = Cx<P>::add(v[0], v[2]), b = Cx<P>::sub(v[0], v[2]);
    const C c = Cx<P>::add(v[1], v[3]), d = Cx<P>::template mmi<INV>(Cx<P>::sub(v[1], v[3]));
    v[0] = Cx<P>::add(a, c);
    v[2] = Cx<P>::sub(a, c);
    v[1] = Cx<P>::add(b, d);
    v[3] = Cx<P>::sub(b, d);
  }
};

template <typename P, bool INV> struct Dft<P, 5, INV> {
  using C = typename Ar<P>::C;
  __device__ __forceinline__ static void run(C* v) {
    const C a1 = Cx<P>::add(v[1], v[4]), b1 = Cx<P>::sub(v[1], v[4]);
    const C a2 = Cx<P>::add(v[2], v[3]), b2 = Cx<P>::sub(v[2], v[3]);
    const C x0 = v[0];
    const C r1 = Cx<P>::add(x0, Cx<P>::add(Cx<P>::mulk(a1, KC1), Cx<P>::mulk(a2, KC2)));
    const C r2 = Cx<P>::add(x0, Cx<P>::add(Cx<P>::mulk(a1, KC2), Cx<P>::mulk(a2, KC1)));
    const C j1 = Cx<P>::template mmi<INV>(Cx<P>::add(Cx<P>::mulk(b1, KS1), Cx<P>::mulk(b2, KS2)));
    const C j2 = Cx<P>::template mmi<INV>(Cx<P>::sub(Cx<P>::mulk(b1, KS2), Cx<P>::mulk(b2, KS1)));
    v[0] = Cx<P>::add(x0, Cx<P>::add(a1, a2));
    v[1] = Cx<P>::add(r1, j1);
    v[4] = Cx<P>::sub(r1, j1);
    v[2] = Cx<P>::add(r2, j2);
    v[3] = Cx<P>::sub(r2, j2);
  }
};

template <typename P, bool INV> struct Dft<P, 8, INV> {
  using A = Ar<P>;
  using C = typename A::C;
  __device__ __forceinline__ static void run(C* v) {
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<P, 4, INV>::run(e);
    Dft<P, 4, INV>::run(o);
    // o_p *= exp(-+2 pi i p / 8): (1 -+ i)/sqrt2, -+i, (-1 -+ i)/sqrt2
    {
      const C t = Cx<P>::template mmi<INV>(o[1]);                 // -+i o1
      o[1] = Cx<P>::mulk(Cx<P>::add(o[1], t), KR2);                // (1 -+ i) o1 / sqrt2
    }
    o[2] = Cx<P>::template mmi<INV>(o[2]);
    {
      const C t = Cx<P>::template mmi<INV>(o[3]);
      o[3] = Cx<P>::mulk(Cx<P>::sub(t, o[3]), KR2);                // (-1 -+ i) o3 / sqrt2
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      v[p] = Cx<P>::add(e[p], o[p]);
      v[p + 4] = Cx<P>::sub(e[p], o[p]);
    }
  }
};

// One Stockham pass of radix R over nsig length-L signals stored back to back
// ([nsig][L]): reads `in`, writes `out`.  Butterfly j (< L/R) of a signal takes
// in[j + q L/R], applies the twiddle of its position k = j mod Ns inside the
// current sub-transform, and writes out[(j-k) R + k + q Ns].
template <typename P, int R, bool INV>
__device__ __forceinline__ void stockham_pass(const typename Ar<P>::C* __restrict__ in, typename Ar<P>::C* __restrict__ out,
                                              int L, int nsig, int Ns, const typename Ar<P>::C* __restrict__ tw) {
  using A = Ar<P>;
  using C = typename A::C;
  const int nb = L / R;
  const int tw_step = L / (Ns * R);
  for (int jt = threadIdx.x; jt < nsig * nb; jt += blockDim.x) {
    const int sig = jt / nb;
    const int j = jt - sig * nb;
    const int k = j % Ns;
    const C* src = in + sig * L;
    C* dst = out + sig * L;
    C v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = src[j + q * nb];
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        C w = tw[q * k * tw_step];
        if (INV) w = A::conj(w);
        v[q] = A::cmul(v[q], w);
      }
    }
    Dft<P, R, INV>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[base + q * Ns] = v[q];
  }
}

// FFT of the nsig signals in buf0; returns the buffer that holds the results.
template <typename P, bool INV>
__device__ typename Ar<P>::C* fft_smem(typename Ar<P>::C* buf0, typename Ar<P>::C* buf1, const FftPlan& plan, int nsig,
                                       const typename Ar<P>::C* __restrict__ tw) {
  using C = typename Ar<P>::C;
  C* in = buf0;
  C* out = buf1;
  int Ns = 1;
  for (int p = 0; p < plan.npass; ++p) {
    const int R = plan.rad[p];
    __syncthreads();
    switch (R) {
      case 2: stockham_pass<P, 2, INV>(in, out, plan.L, nsig, Ns, tw); break;
      case 3: stockham_pass<P, 3, INV>(in, out, plan.L, nsig, Ns, tw); break;
      case 4: stockham_pass<P, 4, INV>(in, out, plan.L, nsig, Ns, tw); break;
      case 5: stockham_pass<P, 5, INV>(in, out, plan.L, nsig, Ns, tw); break;
      default: stockham_pass<P, 8, INV>(in, out, plan.L, nsig, Ns, tw); break;
    }
    Ns *= R;
    C* t = in;
    in = out;
    out = t;
  }
  __syncthreads();
  return in;
}

// --- loads and stores with the phase casts --------------------------------

template <typename P, typename Tin>
__device__ __forceinline__ typename Ar<P>::R load_real(const void* p, int64_t i, bool pad_single) {
  const Tin x = __ldg(static_cast<const Tin*>(p) + i);
  if (pad_single) return Ar<P>::from_f((float)x);
  if constexpr (sizeof(Tin) == 8) return Ar<P>::from_d((double)x);
  else return Ar<P>::from_f((float)x);
}

// store one complex value (re, im) of precision P into format fmt
template <typename P>
__device__ __forceinline__ void store_cx(void* X, int64_t i, int fmt, typename Ar<P>::R re, typename Ar<P>::R im) {
  using A = Ar<P>;
  if (fmt == FMT_C128) {
    static_cast<double2*>(X)[i] = make_double2(A::to_d(re), A::to_d(im));
  } else if (fmt == FMT_C64) {
    static_cast<float2*>(X)[i] = make_float2(A::to_f(re), A::to_f(im));
  } else {
    if constexpr (std::is_same<P, double>::value) {
      // FP64 value -> hi/lo pair
      const double r = A::to_d(re), m = A::to_d(im);
      const float hr = (float)r, hm = (float)m;
      static_cast<float4*>(X)[i] = make_float4(hr, hm, (float)(r - (double)hr), (float)(m - (double)hm));
    } else if constexpr (std::is_same<P, DFP>::value) {
      static_cast<float4*>(X)[i] = Ar<DFP>::mk(re, im);
    } else {
      static_cast<float4*>(X)[i] = make_float4(A::to_f(re), A::to_f(im), 0.f, 0.f);
    }
  }
}

// load one complex value stored in format fmt into precision P
template <typename P>
__device__ __forceinline__ typename Ar<P>::C load_cx(const void* X, int64_t i, int fmt) {
  using A = Ar<P>;
  if (fmt == FMT_C128) {
    const double2 v = __ldg(static_cast<const double2*>(X) + i);
    return A::mk(A::from_d(v.x), A::from_d(v.y));
  }
  if (fmt == FMT_C64) {
    const float2 v = __ldg(static_cast<const float2*>(X) + i);
    return A::mk(A::from_f(v.x), A::from_f(v.y));
  }
  const float4 v = __ldg(static_cast<const float4*>(X) + i);
  if constexpr (std::is_same<P, DFP>::value) {
    return v;
  } else if constexpr (std::is_same<P, double>::value) {
    return A::mk((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  } else {
    return A::mk(__fadd_rn(v.x, v.z), __fadd_rn(v.y, v.w));
  }
}

// Forward: pad + real FFT; grid (row x channel group, K).  A CTA owns NP
// adjacent channel pairs (2 NP channels): consecutive threads take consecutive
// channels at one time step (loads) or one frequency (stores), so every warp
// access covers 2 NP contiguous channels.
template <typename Tin, typename P, int NP>
__global__ void __launch_bounds__(256, 3) rfft_fwd_kernel(FwdDesc d) {
  using A = Ar<P>;
  using C = typename A::C;
  using R = typename A::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = d.plan.L;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + NP * L;
  const int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  const int groups = (d.out_cols + NCH - 1) / NCH;
  const int row = blockIdx.x / groups;
  const int c0 = (blockIdx.x - row * groups) * NCH;
  const int b = blockIdx.y;
  const int64_t xo = b * d.x_ld_b + row * d.x_ld_row;
  const int64_t Xo = b * d.X_ld_b + row * d.X_ld_row;
  const bool tc = d.fmt == FMT_TC;

  // phase 1: load (cast to the pad, then the FFT precision) and zero pad;
  // channel pair p is the complex signal x_{c0+2p} + i x_{c0+2p+1}
  // (8 loads in flight per thread before the shared-memory writes: the loop is
  // latency bound otherwise)
  constexpr int U = 8;
  const int nload = d.Nt * NCH;
  for (int i0 = threadIdx.x; i0 < L * NCH; i0 += U * blockDim.x) {
    R v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      const int t = i / NCH, c = c0 + (i - t * NCH);
      v[u] = (i < nload && c < d.cols) ? load_real<P, Tin>(d.x, xo + t * d.x_ld_t + c, d.pad_single) : A::zero();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i >= L * NCH) break;
      const int t = i / NCH, cc = i - t * NCH;
      C& z = buf0[(cc >> 1) * L + t];
      if constexpr (std::is_same<P, DFP>::value) {
        if (cc & 1) { z.y = v[u].h; z.w = v[u].l; } else { z.x = v[u].h; z.z = v[u].l; }
      } else {
        if (cc & 1) z.y = v[u]; else z.x = v[u];
      }
    }
  }
  // phase 2: complex FFTs
  const C* tw = static_cast<const C*>(d.tw);
  const C* Z = fft_smem<P, false>(buf0, buf1, d.plan, NP, tw);
  // split: X_a = (Z_w + conj Z_{L-w}) / 2,  X_b = (Z_w - conj Z_{L-w}) / (2i).
  // Spectra for the tensor cores go channel-major, T[b][c][w] (FMT_TC, float2),
  // with consecutive threads on consecutive frequencies; the others go
  // frequency-major with consecutive threads on consecutive channels.
  for (int i = threadIdx.x; i < Nf * NCH; i += blockDim.x) {
    const int w = tc ? i % Nf : i / NCH;
    const int cc = tc ? i / Nf : i - w * NCH;
    const int c = c0 + cc;
    if (c >= d.out_cols) continue;
    R xr = A::zero(), xi = A::zero();
    if (c < d.cols) {
      const C z = Z[(cc >> 1) * L + w];
      const C zc = Z[(cc >> 1) * L + (w == 0 ? 0 : L - w)];
      if (cc & 1) {
        xr = A::half(A::add(A::im(z), A::im(zc)));
        xi = A::half(A::sub(A::re(zc), A::re(z)));
      } else {
        xr = A::half(A::add(A::re(z), A::re(zc)));
        xi = A::half(A::sub(A::im(z), A::im(zc)));
      }
    }
    if (tc) static_cast<float2*>(d.X)[((int64_t)b * d.out_cols + c) * Nf + w] = make_float2(A::to_f(xr), A::to_f(xi));
    else store_cx<P>(d.X, Xo + w * d.X_ld_w + c, d.fmt, xr, xi);
  }
}

template <typename Tout, typename P>
__device__ __forceinline__ void store_real(void* y, int64_t i, typename Ar<P>::R v, bool unpad_single) {
  if (unpad_single || sizeof(Tout) == 4) {
    static_cast<Tout*>(y)[i] = (Tout)Ar<P>::to_f(v);
  } else {
    static_cast<Tout*>(y)[i] = (Tout)Ar<P>::to_d(v);
  }
}

// Inverse: Hermitian assembly + inverse complex FFT + unpad; grid (channel group, K).
template <typename P, typename Tout, int NP>
__global__ void __launch_bounds__(256, 3) irfft_inv_kernel(InvDesc d) {
  using A = Ar<P>;
  using C = typename A::C;
  using R = typename A::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = d.plan.L;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + NP * L;
  const int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  const int c0 = blockIdx.x * NCH;
  const int b = blockIdx.y;
  const int64_t Xo = b * d.X_ld_b;
  // Z_w = X_a(w) + i X_b(w) over the full circle, X(L-w) = conj X(w); the DC and
  // Nyquist terms of a real signal's spectrum are taken as real.  Thread i
  // reads channel pair i % NP at frequency i / NP (two adjacent entries).
  constexpr int U = 4;   // loads in flight per thread
  const C zero = A::mk(A::zero(), A::zero());
  for (int i0 = threadIdx.x; i0 < Nf * NP; i0 += U * blockDim.x) {
    C a[U], bb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      const int w = i / NP, p = i - w * NP;
      const int ca = c0 + 2 * p, cb = ca + 1;
      const bool in = i < Nf * NP;
      a[u] = in && ca < d.cols ? load_cx<P>(d.X, Xo + w * d.X_ld_w + ca, d.in_fmt) : zero;
      bb[u] = in && cb < d.cols ? load_cx<P>(d.X, Xo + w * d.X_ld_w + cb, d.in_fmt) : zero;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i >= Nf * NP) break;
      const int w = i / NP, p = i - w * NP;
      C* z = buf0 + p * L;
      if (w == 0 || w == Nf - 1) {
        z[w] = A::mk(A::re(a[u]), A::re(bb[u]));
      } else {
        z[w] = A::mk(A::sub(A::re(a[u]), A::im(bb[u])), A::add(A::im(a[u]), A::re(bb[u])));
        z[L - w] = A::mk(A::add(A::re(a[u]), A::im(bb[u])), A::sub(A::re(bb[u]), A::im(a[u])));
      }
    }
  }
  const C* tw = static_cast<const C*>(d.tw);
  const C* z = fft_smem<P, true>(buf0, buf1, d.plan, NP, tw);
  const Kc inv_L{d.inv_L, d.inv_L_hi, d.inv_L_lo};
  for (int i = threadIdx.x; i < d.Nt * NCH; i += blockDim.x) {
    const int t = i / NCH, cc = i - t * NCH;
    const int c = c0 + cc;
    if (c >= d.cols) continue;
    const C zt = z[(cc >> 1) * L + t];
    const R v = A::mulk((cc & 1) ? A::im(zt) : A::re(zt), inv_L);
    store_real<Tout, P>(d.y, b * d.y_ld_b + t * d.y_ld_t + c, v, d.unpad_single);
  }
}

template <typename K>
cudaError_t prep(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

// channel pairs per CTA: the most (up to 8) whose two buffers fit in kFftSmemCap
constexpr size_t kFftSmemCap = 100 * 1024;
template <typename P>
int pairs_per_cta(int L) {
  const size_t per_pair = 2 * (size_t)L * sizeof(typename Ar<P>::C);
  int np = 8;
  while (np > 1 && np * per_pair > kFftSmemCap) np /= 2;
  return np;
}

template <typename Tin, typename P, int NP>
cudaError_t fwd_launch_np(const FwdDesc& d, cudaStream_t s) {
  const int groups = (d.out_cols + 2 * NP - 1) / (2 * NP);
  dim3 grid(d.rows * groups, d.K);
  const size_t smem = 2 * (size_t)NP * d.plan.L * sizeof(typename Ar<P>::C);
  cudaError_t e = prep(rfft_fwd_kernel<Tin, P, NP>, smem);
  if (e != cudaSuccess) return e;
  rfft_fwd_kernel<Tin, P, NP><<<grid, 256, smem, s>>>(d);
  return cudaGetLastError();
}

template <typename Tin, typename P>
cudaError_t fwd_launch(const FwdDesc& d, cudaStream_t s) {
  switch (pairs_per_cta<P>(d.plan.L)) {
    case 8: return fwd_launch_np<Tin, P, 8>(d, s);
    case 4: return fwd_launch_np<Tin, P, 4>(d, s);
    case 2: return fwd_launch_np<Tin, P, 2>(d, s);
    default: return fwd_launch_np<Tin, P, 1>(d, s);
  }
}

template <typename P, typename Tout, int NP>
cudaError_t inv_launch_np(const InvDesc& d, cudaStream_t s) {
  dim3 grid((d.cols + 2 * NP - 1) / (2 * NP), d.K);
  const size_t smem = 2 * (size_t)NP * d.plan.L * sizeof(typename Ar<P>::C);
  cudaError_t e = prep(irfft_inv_kernel<P, Tout, NP>, smem);
  if (e != cudaSuccess) return e;
  irfft_inv_kernel<P, Tout, NP><<<grid, 256, smem, s>>>(d);
  return cudaGetLastError();
}

template <typename P, typename Tout>
cudaError_t inv_launch(const InvDesc& d, cudaStream_t s) {
  switch (pairs_per_cta<P>(d.plan.L)) {
    case 8: return inv_launch_np<P, Tout, 8>(d, s);
    case 4: return inv_launch_np<P, Tout, 4>(d, s);
    case 2: return inv_launch_np<P, Tout, 2>(d, s);
    default: return inv_launch_np<P, Tout, 1>(d, s);
  }
}

}  // namespace

size_t fft_smem_bytes(int L, int prec) { return 2 * (size_t)L * (prec == FFT_F32 ? sizeof(float2) : 16); }

int fft_max_length(int prec) {
  const size_t cap = 227 * 1024;
  return (int)(cap / (2 * (prec == FFT_F32 ? sizeof(float2) : 16)));
}

cudaError_t launch_rfft_fwd(const FwdDesc& d, bool in_f32, int prec, cudaStream_t s) {
  if (d.rows == 0 || d.out_cols == 0 || d.K == 0) return cudaSuccess;
  if (!in_f32) {
    if (prec == FFT_F64) return fwd_launch<double, double>(d, s);
    if (prec == FFT_DF) return fwd_launch<double, DFP>(d, s);
    return fwd_launch<double, float>(d, s);
  }
  if (prec == FFT_F64) return fwd_launch<float, double>(d, s);
  if (prec == FFT_DF) return fwd_launch<float, DFP>(d, s);
  return fwd_launch<float, float>(d, s);
}

cudaError_t launch_irfft_inv(const InvDesc& d, int prec, bool out_f32, cudaStream_t s) {
  if (d.cols == 0 || d.K == 0) return cudaSuccess;
  if (!out_f32) {
    if (prec == FFT_F64) return inv_launch<double, double>(d, s);
    if (prec == FFT_DF) return inv_launch<DFP, double>(d, s);
    return inv_launch<float, double>(d, s);
  }
  if (prec == FFT_F64) return inv_launch<double, float>(d, s);
  if (prec == FFT_DF) return inv_launch<DFP, float>(d, s);
  return inv_launch<float, float>(d, s);
}

}  // namespace fftmv
