// Batched real FFTs along time for the block-Toeplitz matvec (Section 2.4,
// phases 1-2 and 4-5 of the paper's algorithm), written for sm_103a.
//
// A CTA transforms NP pairs of real channels; pair (c, c+1) is the complex
// signal z = x_c + i x_{c+1}, and the real-to-complex split is done in the
// epilogue (forward) or the Hermitian assembly in the prologue (inverse).  The
// complex FFT of length L = 2^a 3^b 5^c is a Stockham auto-sort sequence of
// radix-2, 3, 4, 5, 8 passes, so the result lands in natural order with no bit
// reversal.  The passes run in place on one shared-memory buffer (each thread
// holds its butterflies in registers across a barrier), which leaves room for
// 2 NP channels per CTA: a time step of them is 32 to 64 contiguous bytes of
// HBM.  Twiddles come from a per-length table exp(-2 pi i j / L) built once on
// the host.
//
// Zero padding (phase 1) and unpadding (phase 5) are fused into the first and
// last radix passes: samples t >= Nt are never read from HBM, and only t < Nt
// is written back.  Casts between the I/O dtype, the pad/unpad precision and the
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
//            is the accuracy an FFT's normwise error analysis needs.  The FFT
//            phases run it with lazy renormalisation (DFL, below): the same
//            normwise accuracy with a quarter fewer operations.

#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fftmv_internal.h"

namespace fftmv {
namespace {

struct DFP {};  // precision tag: double-float on the FP32 pipe
struct DFL {};  // the same format with lazy renormalisation (Ar<DFL>)

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

// Double-float with lazy renormalisation: a sum keeps TwoSum's exact error of
// the hi parts and adds the lo parts to it (8 operations), a product keeps the
// FMA-exact TwoProd with the cross terms (4), with no Fast2Sum at the end.  So
// hi + lo is no longer normalised (after a cancellation lo can be several ulp
// of hi), but it is exact to within the lo parts' own FP32 roundings, which
// are of order u^2 times the operands' magnitudes: the normwise accuracy an
// FFT's error analysis asks of each operation, as for DFP.  The only term a
// product drops, lo*lo, stays below u^2 of the operands' magnitudes with an
// unnormalised lo as well.  Stores to the FMT_DF format renormalise (TwoSum,
// as |lo| <= |hi| no longer holds).
__device__ __forceinline__ dfr dfl_add(dfr a, dfr b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return dfr{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ dfr dfl_mul(dfr a, dfr b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dfr{p, e};
}
// a*b + sgn*c*d
__device__ __forceinline__ dfr dfl_dot2(dfr a, dfr b, dfr c, dfr d, float sgn) {
  const float p1 = __fmul_rn(a.h, b.h);
  const float p2 = __fmul_rn(sgn * c.h, d.h);
  const float e1 = __fmaf_rn(a.h, b.h, -p1);
  const float e2 = __fmaf_rn(sgn * c.h, d.h, -p2);
  float s, t;
  two_sum(p1, p2, s, t);
  t = __fadd_rn(t, __fadd_rn(e1, e2));
  t = __fmaf_rn(a.h, b.l, t);
  t = __fmaf_rn(a.l, b.h, t);
  t = __fmaf_rn(sgn * c.h, d.l, t);
  t = __fmaf_rn(sgn * c.l, d.h, t);
  return dfr{s, t};
}
__device__ __forceinline__ dfr dfl_norm(dfr a) {
  float s, e;
  two_sum(a.h, a.l, s, e);
  return dfr{s, e};
}
template <> struct Ar<DFL> {
  using R = dfr;
  using C = float4;
  __device__ __forceinline__ static R add(R a, R b) { return dfl_add(a, b); }
  __device__ __forceinline__ static R sub(R a, R b) { return dfl_add(a, df_neg(b)); }
  __device__ __forceinline__ static R neg(R a) { return df_neg(a); }
  __device__ __forceinline__ static R half(R a) { return dfr{0.5f * a.h, 0.5f * a.l}; }
  __device__ __forceinline__ static R mulk(R a, const Kc& k) { return dfl_mul(a, dfr{k.h, k.l}); }
  __device__ __forceinline__ static R re(C c) { return dfr{c.x, c.z}; }
  __device__ __forceinline__ static R im(C c) { return dfr{c.y, c.w}; }
  __device__ __forceinline__ static C mk(R r, R i) { return make_float4(r.h, i.h, r.l, i.l); }
  __device__ __forceinline__ static C cmul(C a, C w) {
    const dfr ar = re(a), ai = im(a), wr = re(w), wi = im(w);
    return mk(dfl_dot2(ar, wr, ai, wi, -1.f), dfl_dot2(ar, wi, ai, wr, 1.f));
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

// the double-float arithmetic of the FFT phases: lazy renormalisation (DFL)
// unless FFTMV_DF_LAZY=0 (DFP, every result renormalised)
#ifndef FFTMV_DF_LAZY
#define FFTMV_DF_LAZY 1
#endif
using DFA = std::conditional<FFTMV_DF_LAZY != 0, DFL, DFP>::type;

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
    // (x0 + a1 c1) + a2 c2: two fused multiply-adds per real part in FP32 and FP64
    const C r1 = Cx<P>::add(Cx<P>::add(x0, Cx<P>::mulk(a1, KC1)), Cx<P>::mulk(a2, KC2));
    const C r2 = Cx<P>::add(Cx<P>::add(x0, Cx<P>::mulk(a1, KC2)), Cx<P>::mulk(a2, KC1));
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

// The same DFTs when the upper half of the inputs (q >= R/2) is zero: the
// first forward pass, whose inputs t >= L/2 >= Nt are padding.
template <typename P, int R, bool INV> struct DftHalf {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) { Dft<P, R, INV>::run(v); }
};
template <typename P, bool INV> struct DftHalf<P, 2, INV> {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) { v[1] = v[0]; }
};
template <typename P, bool INV> struct DftHalf<P, 4, INV> {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) {
    const typename Ar<P>::C a = v[0], c = v[1], d = Cx<P>::template mmi<INV>(v[1]);
    v[0] = Cx<P>::add(a, c);
    v[2] = Cx<P>::sub(a, c);
    v[1] = Cx<P>::add(a, d);
    v[3] = Cx<P>::sub(a, d);
  }
};
template <typename P, bool INV> struct DftHalf<P, 8, INV> {
  using A = Ar<P>;
  using C = typename A::C;
  __device__ __forceinline__ static void run(C* v) {
    C e[4] = {v[0], v[2], v[4], v[6]};   // v[4], v[6] are zero
    C o[4] = {v[1], v[3], v[5], v[7]};
    DftHalf<P, 4, INV>::run(e);
    DftHalf<P, 4, INV>::run(o);
    {
      const C t = Cx<P>::template mmi<INV>(o[1]);
      o[1] = Cx<P>::mulk(Cx<P>::add(o[1], t), KR2);
    }
    o[2] = Cx<P>::template mmi<INV>(o[2]);
    {
      const C t = Cx<P>::template mmi<INV>(o[3]);
      o[3] = Cx<P>::mulk(Cx<P>::sub(t, o[3]), KR2);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      v[p] = Cx<P>::add(e[p], o[p]);
      v[p + 4] = Cx<P>::sub(e[p], o[p]);
    }
  }
};

// --- composite radices in registers -----------------------------------------
// cos and sin of 2 pi m / n at compile time: quadrant reduction (exact: the
// quadrant's cosine and sine are 0 and +-1), then Taylor series on
// |x| <= pi/4, whose 14 terms leave an error below 1e-30.
__host__ __device__ constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
// (cos, sin) of 2 pi m / n: quadrant q = round(4 m / n), x = 2 pi (m/n - q/4)
__host__ __device__ constexpr double cos_2pi(int m, int n) {
  const int r = ((m % n) + n) % n;
  const int q = (8 * r + n) / (2 * n);                  // nearest quadrant, 0..4
  const double x = 2.0 * 3.14159265358979323846264338327950288 * ((double)(4 * r - q * n) / (4.0 * n));
  switch (q & 3) {
    case 0: return taylor_cos(x);
    case 1: return -taylor_sin(x);
    case 2: return -taylor_cos(x);
    default: return taylor_sin(x);
  }
}
__host__ __device__ constexpr double sin_2pi(int m, int n) {
  const int r = ((m % n) + n) % n;
  const int q = (8 * r + n) / (2 * n);
  const double x = 2.0 * 3.14159265358979323846264338327950288 * ((double)(4 * r - q * n) / (4.0 * n));
  switch (q & 3) {
    case 0: return taylor_sin(x);
    case 1: return taylor_cos(x);
    case 2: return -taylor_sin(x);
    default: return -taylor_cos(x);
  }
}
__host__ __device__ constexpr Kc kc_of(double v) { return Kc{v, (float)v, (float)(v - (double)(float)v)}; }

// W_R^m = exp(-2 pi i m / R) for m < R, in every precision
template <int R> struct TwTab {
  Kc c[R], s[R];
};
template <int R>
__host__ __device__ constexpr TwTab<R> make_twtab() {
  TwTab<R> t{};
  for (int m = 0; m < R; ++m) {
    t.c[m] = kc_of(cos_2pi(m, R));
    t.s[m] = kc_of(sin_2pi(m, R));
  }
  return t;
}
__device__ constexpr TwTab<16> kTw16 = make_twtab<16>();
__device__ constexpr TwTab<25> kTw25 = make_twtab<25>();
template <int R> __device__ __forceinline__ const TwTab<R>& twtab();
template <> __device__ __forceinline__ const TwTab<16>& twtab<16>() { return kTw16; }
template <> __device__ __forceinline__ const TwTab<25>& twtab<25>() { return kTw25; }

// DFT of size R = R1 R2 in registers (Cooley-Tukey with constant twiddles):
//   X[k1 + R1 k2] = sum_n2 W_R2^(n2 k2) W_R^(n2 k1) sum_n1 W_R1^(n1 k1) x[n1 R2 + n2]
// HALF: inputs n >= R/2 are zero, i.e. n1 >= R1/2 in every inner DFT.
template <typename P, int R1, int R2, bool INV, bool HALF> struct DftComp {
  using A = Ar<P>;
  using C = typename A::C;
  static constexpr int R = R1 * R2;
  __device__ __forceinline__ static void run(C* v) {
    const TwTab<R>& tt = twtab<R>();
    C y[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      C u[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[n1] = v[n1 * R2 + n2];
      if constexpr (HALF) DftHalf<P, R1, INV>::run(u);
      else Dft<P, R1, INV>::run(u);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int m = (n2 * k1) % R;
        if (m == 0) {
          y[n2 * R1 + k1] = u[k1];
        } else if constexpr (std::is_same<P, float>::value || std::is_same<P, double>::value) {
          // u * (c -+ i s) with fused multiply-adds: c and s of the table are
          // the cosine and sine of 2 pi m / R
          using Rl = typename A::R;
          const Rl re = A::re(u[k1]), im = A::im(u[k1]);
          const Rl c = (Rl)tt.c[m].d, sn = (Rl)tt.s[m].d;
          y[n2 * R1 + k1] = INV ? A::mk(fma(re, c, -(im * sn)), fma(im, c, re * sn))
                                : A::mk(fma(re, c, im * sn), fma(im, c, -(re * sn)));
        } else {   // u * (c -+ i s)
          const typename A::R re = A::re(u[k1]), im = A::im(u[k1]);
          const typename A::R cr = A::mulk(re, tt.c[m]), ci = A::mulk(im, tt.c[m]);
          const typename A::R sr = A::mulk(re, tt.s[m]), si = A::mulk(im, tt.s[m]);
          y[n2 * R1 + k1] = INV ? A::mk(A::sub(cr, si), A::add(ci, sr)) : A::mk(A::add(cr, si), A::sub(ci, sr));
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C w[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[n2] = y[n2 * R1 + k1];
      Dft<P, R2, INV>::run(w);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = w[k2];
    }
  }
};
template <typename P, bool INV> struct Dft<P, 16, INV> {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) { DftComp<P, 4, 4, INV, false>::run(v); }
};
template <typename P, bool INV> struct Dft<P, 25, INV> {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) { DftComp<P, 5, 5, INV, false>::run(v); }
};
template <typename P, bool INV> struct DftHalf<P, 16, INV> {
  __device__ __forceinline__ static void run(typename Ar<P>::C* v) { DftComp<P, 4, 4, INV, true>::run(v); }
};

// Shared-memory layout: the NP complex signals of a CTA are interleaved,
// element t of signal p at t * NP + p, so one time step (or frequency) of all
// the CTA's channels is contiguous, like a row of the HBM arrays.  16-byte
// chunks are XOR-swizzled inside each 128-byte line (chunk ^= line mod 8):
// the strided rows of a first radix pass then fall on distinct banks.
template <typename C>
__device__ __forceinline__ int swz(int e) {
  if constexpr (sizeof(C) == 8) return e ^ ((e >> 3) & 14);
  else return e ^ ((e >> 3) & 7);
}
template <typename C, int NP>
__device__ __forceinline__ int sidx(int t, int p) { return swz<C>(t * NP + p); }

// One Stockham pass of radix R over the CTA's NP signals of length L.
// Butterfly j (< L/R) of signal p takes elements j + q L/R (q < R), applies the
// twiddles exp(-+2 pi i q k / (Ns R)) of its position k = j mod Ns inside the
// current sub-transform, and hands its R outputs to `dst` at (j - k) R + k + q Ns.
// KMODE: 0 the first forward pass (Ns = 1, no twiddles; for even R the inputs
// q >= R/2 lie at t >= L/2 >= Nt, in the padding, and are neither read nor
// added), 1 a middle pass (k from a
// multiply-high by the plan's magic constant), 2 the last pass (Ns = L/R, so
// k = j).  A thread keeps all its butterflies (at most E / R, rounded up) in
// registers, so with SYNC_MID the pass runs in place on one shared buffer:
// every read, a barrier, then every write.  `src(t, p, e)` gets the input
// position t = j + q L/R, the signal and the interleaved element index
// e = t NP + p; `dst(t, p, e, v)` the same for an output.
template <typename P, int R, bool INV, int NP, int E, int KMODE, bool SYNC_MID, class Src, class Dst>
__device__ __forceinline__ void radix_pass(int T, int L, int Ns, int tws, unsigned magic,
                                           const typename Ar<P>::C* __restrict__ tw, Src src, Dst dst) {
  using A = Ar<P>;
  using C = typename A::C;
  constexpr int IT = (E + R - 1) / R;
  const int nb = L / R, nbt = nb * NP;
  C v[IT][R];
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int jt = threadIdx.x + i * T;
    if (jt < nbt) {
      const int j = jt / NP, p = jt % NP;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if (KMODE == 0 && R % 2 == 0 && q >= R / 2) v[i][q] = A::mk(A::zero(), A::zero());
        else v[i][q] = src(j + q * nb, p, jt + q * nbt);
      }
    }
  }
  if constexpr (SYNC_MID) __syncthreads();
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int jt = threadIdx.x + i * T;
    if (jt < nbt) {
      const int j = jt / NP, p = jt % NP;
      int k = 0;
      if constexpr (KMODE == 2) k = j;
      else if constexpr (KMODE == 1) k = Ns > 1 ? j - (int)__umulhi((unsigned)j, magic) * Ns : 0;
      if (KMODE != 0 && k > 0) {
        const int kt = k * tws;
#pragma unroll
        for (int q = 1; q < R; ++q) {
          C w = tw[q * kt];
          if (INV) w = A::conj(w);
          v[i][q] = A::cmul(v[i][q], w);
        }
      }
      if constexpr (KMODE == 0 && R % 2 == 0) DftHalf<P, R, INV>::run(v[i]);
      else Dft<P, R, INV>::run(v[i]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int t = base + q * Ns;
        dst(t, p, t * NP + p, v[i][q]);
      }
    }
  }
}

template <typename P, bool INV, int NP, int E, int KMODE, bool SYNC_MID, class Src, class Dst>
__device__ __forceinline__ void any_pass(const FftPlan& plan, int ps, const typename Ar<P>::C* __restrict__ tw, Src src,
                                         Dst dst) {
  const int L = plan.L, Ns = plan.ns[ps], tws = plan.tws[ps];
  const unsigned mg = plan.magic[ps];
  switch (plan.rad[ps]) {
    case 2: radix_pass<P, 2, INV, NP, E, KMODE, SYNC_MID>(blockDim.x, L, Ns, tws, mg, tw, src, dst); break;
    case 3: radix_pass<P, 3, INV, NP, E, KMODE, SYNC_MID>(blockDim.x, L, Ns, tws, mg, tw, src, dst); break;
    case 4: radix_pass<P, 4, INV, NP, E, KMODE, SYNC_MID>(blockDim.x, L, Ns, tws, mg, tw, src, dst); break;
    case 5: radix_pass<P, 5, INV, NP, E, KMODE, SYNC_MID>(blockDim.x, L, Ns, tws, mg, tw, src, dst); break;
    default: radix_pass<P, 8, INV, NP, E, KMODE, SYNC_MID>(blockDim.x, L, Ns, tws, mg, tw, src, dst); break;
  }
}

// Passes [p0, p1) of the plan in place in shared memory, each followed by a
// barrier.  make_plan groups the radices in the order 8, 4, 2, 5, 3; every
// group runs in a loop of its own (one inlined pass body per loop keeps the
// register allocation of each radix separate).
template <typename P, bool INV, int NP, int E, class Src, class Dst>
__device__ __forceinline__ void inplace_passes(const FftPlan& plan, int p0, int p1,
                                               const typename Ar<P>::C* __restrict__ tw, Src src, Dst dst) {
  int ps = p0;
#define FFTMV_RADIX_LOOP(RR)                                                                          \
  for (; ps < p1 && plan.rad[ps] == RR; ++ps) {                                                       \
    radix_pass<P, RR, INV, NP, E, 1, true>(blockDim.x, plan.L, plan.ns[ps], plan.tws[ps], plan.magic[ps], tw, src, dst); \
    __syncthreads();                                                                                  \
  }
  FFTMV_RADIX_LOOP(8)
  FFTMV_RADIX_LOOP(4)
  FFTMV_RADIX_LOOP(2)
  FFTMV_RADIX_LOOP(5)
  FFTMV_RADIX_LOOP(3)
#undef FFTMV_RADIX_LOOP
}

// complex elements a thread holds during a pass: FP32 complexes take two
// registers, FP64 and double-float ones four
#ifndef FFTMV_FFT_E32
#define FFTMV_FFT_E32 16
#endif
#ifndef FFTMV_FFT_E64
#define FFTMV_FFT_E64 8
#endif
template <typename P> constexpr int kFftE = std::is_same<P, float>::value ? FFTMV_FFT_E32 : FFTMV_FFT_E64;

// Channel pairs per CTA: the most (up to 8) whose signals fit in 64 KB, so
// that two CTAs share an SM; threads: enough for E elements each.
#ifndef FFTMV_FFT_TILE_KB
#define FFTMV_FFT_TILE_KB 64
#endif
constexpr size_t kFftTileBytes = FFTMV_FFT_TILE_KB * 1024;
template <typename P>
__host__ __device__ constexpr int fft_pairs(int L) {
  int np = 8;
  while (np > 1 && (size_t)np * L * sizeof(typename Ar<P>::C) > kFftTileBytes) np /= 2;
  return np;
}
template <typename P>
__host__ __device__ constexpr int fft_nthreads(int np, int L, int e = kFftE<P>) {
  const int t = ((np * L + e - 1) / e + 31) / 32 * 32;
  return t < 64 ? 64 : t;
}

// --- lengths known at compile time ------------------------------------------
// The workloads' lengths get kernels of their own (FFTMV_FIXED_LENGTHS below):
// with L constant the plan, the pass sequence, the thread count and every
// index computation fold into constants.  Other lengths take the runtime plan.
struct CPlan {
  int npass;
  int rad[kMaxPasses];
  int ns[kMaxPasses];
};
// FP64 and double-float: the same radix order as make_plan (8, 4, 2, 5, 3).
// FP32 keeps up to 25 complexes per thread in registers, so its plans use the
// composite radices 16 and 25 and need fewer passes through shared memory:
// 2000 = 16 5 25, 1000 = 8 5 25, 256 = 16 16, 128 = 16 8.
template <typename P>
__host__ __device__ constexpr CPlan cplan(int L) {
  CPlan p{};
  int np = 0;
  if (std::is_same<P, float>::value && (L == 2000 || L == 1000 || L == 256 || L == 128)) {
    const int r2000[3] = {16, 5, 25}, r1000[3] = {8, 5, 25}, r256[2] = {16, 16}, r128[2] = {16, 8};
    const int* r = L == 2000 ? r2000 : L == 1000 ? r1000 : L == 256 ? r256 : r128;
    np = (L >= 1000) ? 3 : 2;
    for (int i = 0; i < np; ++i) p.rad[i] = r[i];
  } else {
    int n = L;
    const int order[5] = {8, 4, 2, 5, 3};
    for (int o = 0; o < 5; ++o)
      while (n % order[o] == 0) {
        p.rad[np++] = order[o];
        n /= order[o];
      }
  }
  p.npass = np;
  int ns = 1;
  for (int i = 0; i < np; ++i) {
    p.ns[i] = ns;
    ns *= p.rad[i];
  }
  return p;
}
// complex elements a thread holds during a pass of the length-L kernel
template <typename P>
__host__ __device__ constexpr int fft_elems(int L) {
  return (std::is_same<P, float>::value && (L == 2000 || L == 1000)) ? 25 : kFftE<P>;
}
// launch bounds of the length-L kernel: its exact thread count; 25-element
// threads get up to 65536 / (threads * CTAs per SM) registers (about 100),
// the others 64
template <typename P>
__host__ __device__ constexpr int fft_bound_threads(int NP, int LC) {
  return LC > 0 && fft_elems<P>(LC) == 25 ? fft_nthreads<P>(NP, LC, 25) : 1024;
}
template <typename P>
__host__ __device__ constexpr int fft_bound_blocks(int NP, int LC) {
  return LC > 0 && fft_elems<P>(LC) == 25 ? (fft_bound_threads<P>(NP, LC) <= 320 ? 2 : 1) : 1;
}
// loads in flight per thread for the inverse's spectrum assembly of a
// compile-time length: items / threads rounded up, capped by the register budget
__host__ __device__ constexpr int fft_inv_loads(int csize, int e, int nf, int np, int threads) {
  const int want = (nf * np + threads - 1) / threads;
  const int cap = csize == 8 ? (e == 25 ? 16 : 8) : 8;
  return want < cap ? want : cap;
}
__host__ __device__ constexpr unsigned cmagic(int ns) {
  return ns > 1 ? (unsigned)((((unsigned long long)1 << 32) + (unsigned long long)ns - 1) / (unsigned long long)ns) : 0u;
}

// pass PS of the length-L plan
template <typename P, bool INV, int NP, int E, int L, int PS, int KMODE, bool SYNC_MID, class Src, class Dst>
__device__ __forceinline__ void cpass(int T, const typename Ar<P>::C* __restrict__ tw, Src src, Dst dst) {
  constexpr CPlan pl = cplan<P>(L);
  constexpr int R = pl.rad[PS], Ns = pl.ns[PS];
  radix_pass<P, R, INV, NP, E, KMODE, SYNC_MID>(T, L, Ns, L / (Ns * R), cmagic(Ns), tw, src, dst);
}
// passes [PS, PE) in place, each followed by a barrier
template <typename P, bool INV, int NP, int E, int L, int PS, int PE, class Src, class Dst>
__device__ __forceinline__ void cpasses(int T, const typename Ar<P>::C* __restrict__ tw, Src src, Dst dst) {
  if constexpr (PS < PE) {
    cpass<P, INV, NP, E, L, PS, 1, true>(T, tw, src, dst);
    __syncthreads();
    cpasses<P, INV, NP, E, L, PS + 1, PE>(T, tw, src, dst);
  }
}

// --- loads and stores with the phase casts --------------------------------

template <typename P, typename Tin>
__device__ __forceinline__ typename Ar<P>::R cvt_real(Tin x, bool pad_single) {
  if (pad_single) return Ar<P>::from_f((float)x);
  if constexpr (sizeof(Tin) == 8) return Ar<P>::from_d((double)x);
  else return Ar<P>::from_f((float)x);
}
template <typename P, typename Tin>
__device__ __forceinline__ typename Ar<P>::R load_real(const void* p, int64_t i, bool pad_single) {
  return cvt_real<P, Tin>(__ldg(static_cast<const Tin*>(p) + i), pad_single);
}
// the same cast after an exact power-of-two scale `sc` in FP64 (range scaling:
// the value then fits the FP32 exponent range of the double-float format)
template <typename P, typename Tin>
__device__ __forceinline__ typename Ar<P>::R cvt_real_scaled(Tin x, bool pad_single, double sc) {
  const double v = pad_single ? (double)(float)x : (double)x;
  return Ar<P>::from_d(v * sc);
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
    } else if constexpr (std::is_same<P, DFL>::value) {
      static_cast<float4*>(X)[i] = Ar<DFL>::mk(dfl_norm(re), dfl_norm(im));
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
  if constexpr (std::is_same<P, DFP>::value || std::is_same<P, DFL>::value) {
    return v;
  } else if constexpr (std::is_same<P, double>::value) {
    return A::mk((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  } else {
    return A::mk(__fadd_rn(v.x, v.z), __fadd_rn(v.y, v.w));
  }
}

// an FP64 (FMT_C128) spectrum value times the power of two sc, loaded into precision P
template <typename P>
__device__ __forceinline__ typename Ar<P>::C load_cx_scaled(const void* X, int64_t i, double sc) {
  using A = Ar<P>;
  const double2 v = __ldg(static_cast<const double2*>(X) + i);
  return A::mk(A::from_d(v.x * sc), A::from_d(v.y * sc));
}

// Forward: pad + real FFT; grid (row x channel group, K).  A CTA owns NP
// adjacent channel pairs (2 NP channels); pair p is the complex signal
// x_{c0+2p} + i x_{c0+2p+1}.  The first radix pass reads the samples straight
// from HBM (zero padding and the pad cast fused: t >= Nt is never read), the
// other passes run in place in shared memory, then the real/imaginary split
// writes the spectra.
template <typename Tin, typename P, int NP, int LC>
__global__ void __launch_bounds__(fft_bound_threads<P>(NP, LC), fft_bound_blocks<P>(NP, LC)) rfft_fwd_kernel(FwdDesc d) {
  using A = Ar<P>;
  using C = typename A::C;
  using R = typename A::R;
  constexpr int E = LC > 0 ? fft_elems<P>(LC) : kFftE<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int L = LC > 0 ? LC : d.plan.L;
  const int T = LC > 0 ? fft_nthreads<P>(NP, LC, fft_elems<P>(LC)) : (int)blockDim.x;
  const int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  const int groups = (d.out_cols + NCH - 1) / NCH;
  const int row = blockIdx.x / groups;
  const int c0 = (blockIdx.x - row * groups) * NCH;
  const int b = blockIdx.y;
  const int64_t xo = b * d.x_ld_b + row * d.x_ld_row;
  const C* tw = static_cast<const C*>(d.tw);
  const C zero = A::mk(A::zero(), A::zero());

  // range scaling: right-hand side b is divided by 2^e_b as it loads
  const int in_exp = d.in_absmax != nullptr ? range_exp(d.in_absmax[b]) : 0;
  const bool scaled = in_exp != 0;
  const double insc = scaled ? ldexp(1.0, -in_exp) : 1.0;
  // sample t of channel pair p, the pad cast fused; SC: range-scaled (the
  // first pass is instantiated once per case, so the unscaled one carries no
  // scaling code)
  auto gsrc_of = [&](auto sc_t) {
    constexpr bool SC = decltype(sc_t)::value;
    return [&](int t, int p, int) -> C {
      const int c = c0 + 2 * p;
      if (t >= d.Nt || c >= d.cols) return zero;
      const int64_t o = xo + t * d.x_ld_t + c;
      if (d.pair_ok && c + 1 < d.cols) {   // both channels in one 8- or 16-byte load
        using V = typename std::conditional<sizeof(Tin) == 4, float2, double2>::type;
        const V v = __ldg(reinterpret_cast<const V*>(static_cast<const Tin*>(d.x) + o));
        if constexpr (SC)
          return A::mk(cvt_real_scaled<P, Tin>(v.x, d.pad_single, insc), cvt_real_scaled<P, Tin>(v.y, d.pad_single, insc));
        else
          return A::mk(cvt_real<P, Tin>(v.x, d.pad_single), cvt_real<P, Tin>(v.y, d.pad_single));
      }
      const Tin* xp = static_cast<const Tin*>(d.x) + o;
      const Tin xa = __ldg(xp), xb = c + 1 < d.cols ? __ldg(xp + 1) : Tin(0);
      if constexpr (SC)
        return A::mk(cvt_real_scaled<P, Tin>(xa, d.pad_single, insc), cvt_real_scaled<P, Tin>(xb, d.pad_single, insc));
      else
        return A::mk(cvt_real<P, Tin>(xa, d.pad_single), cvt_real<P, Tin>(xb, d.pad_single));
    };
  };
  auto sdst = [&](int, int, int e, C v) { buf[swz<C>(e)] = v; };
  auto ssrc = [&](int, int, int e) -> C { return buf[swz<C>(e)]; };
  auto first = [&](auto gsrc) {
    if constexpr (LC > 0) cpass<P, false, NP, E, LC, 0, 0, false>(T, tw, gsrc, sdst);
    else any_pass<P, false, NP, E, 0, false>(d.plan, 0, tw, gsrc, sdst);
  };
  if (scaled) first(gsrc_of(std::true_type{}));
  else first(gsrc_of(std::false_type{}));
  __syncthreads();
  if constexpr (LC > 0) cpasses<P, false, NP, E, LC, 1, cplan<P>(LC).npass>(T, tw, ssrc, sdst);
  else inplace_passes<P, false, NP, E>(d.plan, 1, d.plan.npass, tw, ssrc, sdst);

  // split: X_a = (Z_w + conj Z_{L-w}) / 2,  X_b = (Z_w - conj Z_{L-w}) / (2i)
  auto split = [&](int w, int cc, R& xr, R& xi) {
    const C z = buf[sidx<C, NP>(w, cc >> 1)];
    const C zc = buf[sidx<C, NP>(w == 0 ? 0 : L - w, cc >> 1)];
    if (cc & 1) {
      xr = A::half(A::add(A::im(z), A::im(zc)));
      xi = A::half(A::sub(A::re(zc), A::re(z)));
    } else {
      xr = A::half(A::add(A::re(z), A::re(zc)));
      xi = A::half(A::sub(A::im(z), A::im(zc)));
    }
  };
  if (d.fmt == FMT_TC) {
    // bf16 hi/lo B planes [2][J][ldb/g][Nf][g] (ldb = out_cols, g = 2^tc_group_log2):
    // a thread takes one frequency and G adjacent channels, and writes them as
    // one 2G-byte run into each of the four rows (Re, Im) x (hi, lo);
    // consecutive threads take consecutive frequencies (adjacent runs for g = 8)
    constexpr int G = NCH < 8 ? NCH : 8;
    constexpr int NG = NCH / G;
    using Vec = typename std::conditional<G == 8, uint4, typename std::conditional<G == 4, uint2, uint32_t>::type>::type;
    unsigned short* B = static_cast<unsigned short*>(d.X);
    const bool f16 = d.tc_inv_scale != nullptr;
    // the FP16 path's power-of-two scale; the split's 1/2 is applied by the
    // contraction's epilogue (the planes hold 2 X)
    const float hsc = f16 ? d.tc_inv_scale[b] : 1.f;
    const int ch = b / d.tc_KC, q = b - ch * d.tc_KC;
    const int64_t jr = (int64_t)ch * d.tc_N + q, ji = jr + d.tc_KC;
    const int64_t row_el = (int64_t)d.out_cols * Nf;   // bf16 per B row
    const int64_t plane_el = (int64_t)d.tc_J * row_el;
    for (int i = threadIdx.x; i < Nf * NG; i += T) {
      const int w = i / NG, g = i % NG;
      const int cg = g * G, c = c0 + cg;
      if (c >= d.out_cols) continue;
      // the G/2 signals of this thread at w and L - w: 16-byte chunks (the
      // swizzle moves whole chunks), so a warp reads rows conflict-free
      C zw[G / 2], zc[G / 2];
      const int wc = w == 0 ? 0 : L - w;
      if constexpr (sizeof(C) == 8 && G >= 4) {
#pragma unroll
        for (int u = 0; u < G / 2; u += 2) {
          const float4 a = *reinterpret_cast<const float4*>(buf + swz<C>(w * NP + cg / 2 + u));
          const float4 bq = *reinterpret_cast<const float4*>(buf + swz<C>(wc * NP + cg / 2 + u));
          zw[u] = A::mk(a.x, a.y);
          zw[u + 1] = A::mk(a.z, a.w);
          zc[u] = A::mk(bq.x, bq.y);
          zc[u + 1] = A::mk(bq.z, bq.w);
        }
      } else {
#pragma unroll
        for (int u = 0; u < G / 2; ++u) {
          zw[u] = buf[swz<C>(w * NP + cg / 2 + u)];
          zc[u] = buf[swz<C>(wc * NP + cg / 2 + u)];
        }
      }
      __align__(16) unsigned short h[4][G];   // rows: Re hi, Re lo, Im hi, Im lo (bf16 or FP16 bits)
#pragma unroll
      for (int u = 0; u < G; ++u) {
        float fr = 0.f, fi = 0.f;
        if (c + u < d.cols) {
          const C z = zw[u >> 1], y = zc[u >> 1];
          R xr, xi;
          if (u & 1) {
            xr = A::add(A::im(z), A::im(y));
            xi = A::sub(A::re(y), A::re(z));
          } else {
            xr = A::add(A::re(z), A::re(y));
            xi = A::sub(A::im(z), A::im(y));
          }
          fr = A::to_f(xr) * hsc;
          fi = A::to_f(xi) * hsc;
        }
        if (f16) {   // x = hi + lo in FP16 after the power-of-two scale
          const __half rh = __float2half_rn(fr), ih = __float2half_rn(fi);
          h[0][u] = __half_as_ushort(rh);
          h[1][u] = __half_as_ushort(__float2half_rn(fr - __half2float(rh)));
          h[2][u] = __half_as_ushort(ih);
          h[3][u] = __half_as_ushort(__float2half_rn(fi - __half2float(ih)));
        } else {
          const __nv_bfloat16 rh = __float2bfloat16(fr), ih = __float2bfloat16(fi);
          h[0][u] = __bfloat16_as_ushort(rh);
          h[1][u] = __bfloat16_as_ushort(__float2bfloat16(fr - __bfloat162float(rh)));
          h[2][u] = __bfloat16_as_ushort(ih);
          h[3][u] = __bfloat16_as_ushort(__float2bfloat16(fi - __bfloat162float(ih)));
        }
      }
      const int sh = d.tc_group_log2;
      const int64_t off = (((int64_t)(c >> sh) * Nf + w) << sh) + (c & ((1 << sh) - 1));
      *reinterpret_cast<Vec*>(B + jr * row_el + off) = *reinterpret_cast<const Vec*>(h[0]);
      *reinterpret_cast<Vec*>(B + plane_el + jr * row_el + off) = *reinterpret_cast<const Vec*>(h[1]);
      *reinterpret_cast<Vec*>(B + ji * row_el + off) = *reinterpret_cast<const Vec*>(h[2]);
      *reinterpret_cast<Vec*>(B + plane_el + ji * row_el + off) = *reinterpret_cast<const Vec*>(h[3]);
    }
    return;
  }
  // frequency-major spectra X[b][w][row][col]: consecutive threads on consecutive channels
  const int64_t Xo = b * d.X_ld_b + row * d.X_ld_row;
  for (int i = threadIdx.x; i < Nf * NCH; i += T) {
    const int w = i / NCH, cc = i - w * NCH;
    const int c = c0 + cc;
    if (c >= d.out_cols) continue;
    R xr = A::zero(), xi = A::zero();
    if (c < d.cols) split(w, cc, xr, xi);
    store_cx<P>(d.X, Xo + w * d.X_ld_w + c, d.fmt, xr, xi);
  }
}

// v (the scaled result) in FP64 times s1 s2, then the output cast
template <typename Tout, typename P>
__device__ __forceinline__ void store_real_scaled(void* y, int64_t i, typename Ar<P>::R v, bool unpad_single, double s1,
                                                  double s2) {
  const double r = Ar<P>::to_d(v) * s1 * s2;
  if (unpad_single || sizeof(Tout) == 4) static_cast<Tout*>(y)[i] = (Tout)(float)r;
  else static_cast<Tout*>(y)[i] = (Tout)r;
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
// The assembly loads the half spectra into shared memory, the passes run in
// place, and the last pass writes t < Nt straight to HBM (1/L scale, unpad and
// output cast fused).
template <typename P, typename Tout, int NP, int LC>
__global__ void __launch_bounds__(fft_bound_threads<P>(NP, LC), fft_bound_blocks<P>(NP, LC)) irfft_inv_kernel(InvDesc d) {
  using A = Ar<P>;
  using C = typename A::C;
  constexpr int E = LC > 0 ? fft_elems<P>(LC) : kFftE<P>;
  constexpr int T_LC = LC > 0 ? fft_nthreads<P>(NP, LC, E) : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int L = LC > 0 ? LC : d.plan.L;
  const int T = LC > 0 ? fft_nthreads<P>(NP, LC, fft_elems<P>(LC)) : (int)blockDim.x;
  const int Nf = L / 2 + 1;
  constexpr int NCH = 2 * NP;
  const int c0 = blockIdx.x * NCH;
  const int b = blockIdx.y;
  const int64_t Xo = b * d.X_ld_b;
  // Z_w = X_a(w) + i X_b(w) over the full circle, X(L-w) = conj X(w); the DC and
  // Nyquist terms of a real signal's spectrum are taken as real.  Thread i
  // reads channel pair i % NP at frequency i / NP (two adjacent entries).
  // Loads in flight per thread.  The compile-time kernels take enough for all
  // Nf NP of them to issue in one round, up to what their registers hold (16
  // FP32 complexes in the 25-element kernels, 8 otherwise): at L = 2000 the
  // FP32 F* at K = 64 takes 2.76 ms against 3.06 with 4.  The runtime-length
  // kernels take 8 FP32 complexes (4 with one pair per CTA) or 4 wider ones.
  constexpr int U = LC > 0 ? fft_inv_loads(sizeof(C), E, LC / 2 + 1, NP, T_LC)
                           : (sizeof(C) == 8 && NP >= 2 ? 8 : 4);
  const C zero = A::mk(A::zero(), A::zero());
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
        buf[sidx<C, NP>(w, p)] = A::mk(A::re(a[u]), A::re(bb[u]));
      } else {
        buf[sidx<C, NP>(w, p)] = A::mk(A::sub(A::re(a[u]), A::im(bb[u])), A::add(A::im(a[u]), A::re(bb[u])));
        buf[sidx<C, NP>(L - w, p)] = A::mk(A::add(A::re(a[u]), A::im(bb[u])), A::sub(A::re(bb[u]), A::im(a[u])));
      }
    }
  }
  __syncthreads();
  const C* tw = static_cast<const C*>(d.tw);
  auto sdst = [&](int, int, int e, C v) { buf[swz<C>(e)] = v; };
  auto ssrc = [&](int, int, int e) -> C { return buf[swz<C>(e)]; };
  if constexpr (LC > 0) cpasses<P, true, NP, E, LC, 0, cplan<P>(LC).npass - 1>(T, tw, ssrc, sdst);
  else inplace_passes<P, true, NP, E>(d.plan, 0, d.plan.npass - 1, tw, ssrc, sdst);
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
  // the last pass writes t < Nt straight to HBM; SC: range-scaled outputs (one
  // instantiation of the pass per case)
  auto gdst_of = [&](auto sc_t) {
    constexpr bool SC = decltype(sc_t)::value;
    return [&](int t, int p, int, C v) {
      const int c = c0 + 2 * p;
      if (t >= d.Nt || c >= d.cols) return;
      const int64_t o = b * d.y_ld_b + t * d.y_ld_t + c;
      if constexpr (SC) {
        store_real_scaled<Tout, P>(d.y, o, A::mulk(A::re(v), inv_L), d.unpad_single, s1, s2);
        if (c + 1 < d.cols) store_real_scaled<Tout, P>(d.y, o + 1, A::mulk(A::im(v), inv_L), d.unpad_single, s1, s2);
      } else {
        store_real<Tout, P>(d.y, o, A::mulk(A::re(v), inv_L), d.unpad_single);
        if (c + 1 < d.cols) store_real<Tout, P>(d.y, o + 1, A::mulk(A::im(v), inv_L), d.unpad_single);
      }
    };
  };
  auto last = [&](auto gdst) {
    if constexpr (LC > 0) cpass<P, true, NP, E, LC, cplan<P>(LC).npass - 1, 2, false>(T, tw, ssrc, gdst);
    else any_pass<P, true, NP, E, 2, false>(d.plan, d.plan.npass - 1, tw, ssrc, gdst);
  };
  if (scaled) last(gdst_of(std::true_type{}));
  else last(gdst_of(std::false_type{}));
}

template <typename K>
cudaError_t prep(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}


template <typename Tin, typename P, int NP, int LC>
cudaError_t fwd_launch_np(const FwdDesc& d, cudaStream_t s) {
  const int groups = (d.out_cols + 2 * NP - 1) / (2 * NP);
  dim3 grid(d.rows * groups, d.K);
  const size_t smem = (size_t)NP * d.plan.L * sizeof(typename Ar<P>::C);
  const int threads = LC > 0 ? fft_nthreads<P>(NP, LC, fft_elems<P>(LC)) : fft_nthreads<P>(NP, d.plan.L);
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = prep(rfft_fwd_kernel<Tin, P, NP, LC>, smem);
  if (e != cudaSuccess) return e;
  rfft_fwd_kernel<Tin, P, NP, LC><<<grid, threads, smem, s>>>(d);
  return cudaGetLastError();
}

template <typename P, typename Tout, int NP, int LC>
cudaError_t inv_launch_np(const InvDesc& d, cudaStream_t s) {
  dim3 grid((d.cols + 2 * NP - 1) / (2 * NP), d.K);
  const size_t smem = (size_t)NP * d.plan.L * sizeof(typename Ar<P>::C);
  const int threads = LC > 0 ? fft_nthreads<P>(NP, LC, fft_elems<P>(LC)) : fft_nthreads<P>(NP, d.plan.L);
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = prep(irfft_inv_kernel<P, Tout, NP, LC>, smem);
  if (e != cudaSuccess) return e;
  irfft_inv_kernel<P, Tout, NP, LC><<<grid, threads, smem, s>>>(d);
  return cudaGetLastError();
}

// the lengths with kernels of their own: L = 2 Nt for Nt = 64, 128, 256, 500, 1000
#define FFTMV_FIXED_LENGTHS(X) X(128) X(256) X(512) X(1000) X(2000)

// SMs of the current device, looked up once per device
inline int fft_sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

// Channel pairs per CTA for a grid of `groups(np)` CTAs: the shared-memory
// tile's share (fft_pairs).  In native FP64 it is halved while the grid would
// cover fewer SMs than the GPU has: the FP64 arithmetic of a whole CTA shares
// one SM's FP64 pipe (about 2 DFMA per clock), so spreading the pairs over
// more SMs shortens a small transform.  FP32 and double-float CTAs are bound
// by their threads' dependency chains, which do not shorten with fewer pairs,
// and keep the compile-time kernels.
template <typename P, class Groups>
int fft_pairs_for_grid(int L, Groups groups) {
  int np = fft_pairs<P>(L);
  if constexpr (std::is_same<P, double>::value) {
    const int64_t sms = fft_sm_count();
    while (np > 1 && groups(np) < sms) np /= 2;
  }
  return np;
}

}  // namespace
}  // namespace fftmv
