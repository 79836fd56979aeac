// Per-frequency complex block matvec (Section 2.4, phase 3; Section 3.1.1's
// short-and-wide strided-batched GEMV), written for sm_103a.
//
// For every frequency w the operator block F-hat_w is Nd x Nm complex with
// Nd << Nm, stored row-major with a padded row length ldn (a multiple of 8).
// Both directions stream F-hat exactly once per pass of right-hand sides: N
// through a bulk-copy pipeline into shared memory, H with 16-byte vector loads:
//
//  N (F):  d-hat_w[r] = sum_n F_w[r, n] m-hat_w[n].  A CTA owns R rows of one
//          frequency and sweeps the whole row length; each thread keeps R
//          private accumulators over a strided set of columns, and one block
//          reduction per row finishes the dot products.  No split-K, no
//          scratch, no atomics: results do not depend on scheduling.
//  H (F*): m-hat_w[n] = sum_r conj(F_w[r, n]) d-hat_w[r].  A CTA owns a run of
//          columns of one frequency; d-hat_w sits in shared memory and each
//          thread accumulates its own columns over all Nd rows: no reduction.
//
// Arithmetic kinds:
//  GEMV_F64: FP64 F-hat (16 B per entry), FP64 FMA.
//  GEMV_DF:  FP64-class.  F-hat stored as FP32 hi/lo pairs (16 B per entry,
//            about 48 significant bits); products by TwoProd (FMA), sums by
//            TwoSum, all on the FP32 pipe.  GB300's FP64 FMA rate (about 1.2
//            TFLOP/s measured) cannot keep up with HBM for a 0.5 flop/byte
//            GEMV; the FP32 pipe can.
//  GEMV_F32: FP32 F-hat (8 B per entry), FP32 FMA.

#include <type_traits>

#include "fftmv_internal.h"
#include "pipe.cuh"

namespace fftmv {
namespace {

// ---------------------------------------------------------------------------
// error-free transformations (Knuth's TwoSum, FMA-based TwoProd)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += p exactly in hi, with the rounding error folded into lo.
__device__ __forceinline__ void df_acc(float& hi, float& lo, float p) {
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// (hi, lo) -> hi' + lo' with |lo'| <= ulp(hi')/2, exact whatever the magnitudes (TwoSum)
__device__ __forceinline__ float2 renorm(float hi, float lo) {
  float s, e;
  two_sum(hi, lo, s, e);
  return make_float2(s, e);
}

// (a_hi, a_lo) + (b_hi, b_lo), renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  const float l = __fsub_rn(e, __fsub_rn(h, s));
  return make_float2(h, l);
}

// ---------------------------------------------------------------------------
// arithmetic kinds
// ---------------------------------------------------------------------------
struct KindF64 {
  using Pack = double2;  // one complex entry
  using Elem = double2;  // one complex vector element (H input)
  using Acc = double2;
  static constexpr int P = 1;
  __device__ __forceinline__ static Acc zero() { return make_double2(0.0, 0.0); }
  __device__ __forceinline__ static Pack ldF(const Pack* p) { return __ldcs(p); }
  // acc += f * x
  __device__ __forceinline__ static void mac_n(Acc& a, Pack f, Pack x) {
    a.x = fma(f.x, x.x, fma(-f.y, x.y, a.x));
    a.y = fma(f.x, x.y, fma(f.y, x.x, a.y));
  }
  // acc += conj(f) * x
  __device__ __forceinline__ static void mac_h(Acc* a, Pack f, Elem x) {
    a[0].x = fma(f.x, x.x, fma(f.y, x.y, a[0].x));
    a[0].y = fma(f.x, x.y, fma(-f.y, x.x, a[0].y));
  }
  __device__ __forceinline__ static Acc add(Acc a, Acc b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ __forceinline__ static Acc shfl_xor(Acc a, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
  __device__ __forceinline__ static void store(void* y, int64_t i, Acc a) { static_cast<double2*>(y)[i] = a; }
};

struct KindDF {
  using Pack = float4;  // (re_hi, im_hi, re_lo, im_lo)
  using Elem = float4;
  using Acc = float4;   // (re_hi, re_lo, im_hi, im_lo)
  static constexpr int P = 1;
  __device__ __forceinline__ static Acc zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ static Pack ldF(const Pack* p) { return __ldcs(p); }
  // acc += (fr + i fi) * (xr + i xi) with s = +1, or conj(f) * x with s = -1,
  // each operand a hi/lo pair.  The four hi*hi products are split exactly by
  // TwoProd and their hi parts enter the accumulators through TwoSum; the
  // TwoProd errors and the hi*lo cross terms (lo*lo is below 2^-48) are
  // summed into the lo accumulators.
  template <int S>
  __device__ __forceinline__ static void cmac(Acc& a, Pack f, Elem x) {
    const float fr = f.x, fi = S * f.y, frl = f.z, fil = S * f.w;
    const float xr = x.x, xi = x.y, xrl = x.z, xil = x.w;
    // real part: fr*xr - fi*xi
    const float p1 = __fmul_rn(fr, xr), p2 = __fmul_rn(-fi, xi);
    float lre = __fmaf_rn(fr, xr, -p1);
    lre = __fadd_rn(lre, __fmaf_rn(-fi, xi, -p2));
    lre = __fmaf_rn(fr, xrl, lre);
    lre = __fmaf_rn(frl, xr, lre);
    lre = __fmaf_rn(-fi, xil, lre);
    lre = __fmaf_rn(-fil, xi, lre);
    // imaginary part: fr*xi + fi*xr
    const float p3 = __fmul_rn(fr, xi), p4 = __fmul_rn(fi, xr);
    float lim = __fmaf_rn(fr, xi, -p3);
    lim = __fadd_rn(lim, __fmaf_rn(fi, xr, -p4));
    lim = __fmaf_rn(fr, xil, lim);
    lim = __fmaf_rn(frl, xi, lim);
    lim = __fmaf_rn(fi, xrl, lim);
    lim = __fmaf_rn(fil, xr, lim);
    df_acc(a.x, a.y, p1);
    df_acc(a.x, a.y, p2);
    a.y = __fadd_rn(a.y, lre);
    df_acc(a.z, a.w, p3);
    df_acc(a.z, a.w, p4);
    a.w = __fadd_rn(a.w, lim);
  }
  __device__ __forceinline__ static void mac_n(Acc& a, Pack f, Pack x) { cmac<1>(a, f, x); }
  __device__ __forceinline__ static void mac_h(Acc* a, Pack f, Elem x) { cmac<-1>(a[0], f, x); }
  __device__ __forceinline__ static Acc add(Acc a, Acc b) {
    const float2 r = df_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 i = df_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(r.x, r.y, i.x, i.y);
  }
  __device__ __forceinline__ static Acc shfl_xor(Acc a, int m) {
    return make_float4(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m),
                       __shfl_xor_sync(0xffffffffu, a.z, m), __shfl_xor_sync(0xffffffffu, a.w, m));
  }
  // FMT_DF: (re_hi, im_hi, re_lo, im_lo), read as is by the double-float FFT
  __device__ __forceinline__ static void store(void* y, int64_t i, Acc a) {
    const float2 r = renorm(a.x, a.y), m = renorm(a.z, a.w);
    static_cast<float4*>(y)[i] = make_float4(r.x, m.x, r.y, m.y);
  }
};

struct KindF32 {
  using Pack = float4;   // two adjacent complex entries (n, n+1)
  using Elem = float2;   // one complex vector element (H input)
  using Acc = float2;
  static constexpr int P = 2;
  __device__ __forceinline__ static Acc zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static Pack ldF(const Pack* p) { return __ldcs(p); }
  __device__ __forceinline__ static void mac_n(Acc& a, Pack f, Pack x) {
    a.x = fmaf(f.x, x.x, fmaf(-f.y, x.y, a.x));
    a.y = fmaf(f.x, x.y, fmaf(f.y, x.x, a.y));
    a.x = fmaf(f.z, x.z, fmaf(-f.w, x.w, a.x));
    a.y = fmaf(f.z, x.w, fmaf(f.w, x.z, a.y));
  }
  __device__ __forceinline__ static void mac_h(Acc* a, Pack f, Elem x) {
    a[0].x = fmaf(f.x, x.x, fmaf(f.y, x.y, a[0].x));
    a[0].y = fmaf(f.x, x.y, fmaf(-f.y, x.x, a[0].y));
    a[1].x = fmaf(f.z, x.x, fmaf(f.w, x.y, a[1].x));
    a[1].y = fmaf(f.z, x.y, fmaf(-f.w, x.x, a[1].y));
  }
  __device__ __forceinline__ static Acc add(Acc a, Acc b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ __forceinline__ static Acc shfl_xor(Acc a, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
  __device__ __forceinline__ static void store(void* y, int64_t i, Acc a) { static_cast<float2*>(y)[i] = a; }
};

// ---------------------------------------------------------------------------
// N direction: grid (ceil(Nd / R), Nf, ceil(K / KB)).  Warp-specialised
// bulk-copy pipeline: warp 0 (one elected thread) streams each CW-pack segment
// of the R rows of F-hat_w and the matching segments of KB right-hand sides
// m-hat_w into a ring of STAGES shared-memory stages with cp.async.bulk,
// completion counted on the stage's "full" mbarrier; NCW consumer warps
// compute from shared memory (consumer thread tc owns pack tc of every segment,
// so its columns are tc, tc + CW, ...) and release the stage through its
// "empty" mbarrier.  Every F-hat pack serves all KB right-hand sides, so K of
// them cost ceil(K / KB) passes over F-hat.  Bytes stay in flight while the
// consumers do their (double-float) arithmetic.
// ---------------------------------------------------------------------------
template <class Kd, int R, int KB, int NCW, int STAGES, int V = 1>
__global__ void __launch_bounds__(32 * (NCW + 1), 2) gemv_n_kernel(GemvDesc d) {
  using Pack = typename Kd::Pack;
  using Acc = typename Kd::Acc;
  constexpr int NC = 32 * NCW;   // consumer threads
  constexpr int CW = NC * V;     // packs per row segment (V per consumer thread)
  constexpr int STAGE = (R + KB) * CW;
  static_assert(R * KB <= NC, "one consumer thread per output");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Pack* stage = reinterpret_cast<Pack*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(stage + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  Acc* red = reinterpret_cast<Acc*>(empty + STAGES);   // [NCW][R][KB]

  const int w = blockIdx.y, b0 = blockIdx.z * KB;
  const int nbk = min(KB, d.K - b0);
  const int r0 = blockIdx.x * R;
  const int nr = min(R, d.Nd - r0);
  const int ldp = d.ldn / Kd::P;                        // packs per row
  const int nseg = (ldp + CW - 1) / CW;
  const Pack* F = static_cast<const Pack*>(d.F) + ((int64_t)w * d.Nd + r0) * ldp;
  const Pack* x = static_cast<const Pack*>(d.x) + (b0 * d.x_ld_b + (int64_t)w * d.ldn) / Kd::P;
  const int64_t xb = d.x_ld_b / Kd::P;                   // packs between right-hand sides

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (warp == 0) {  // producer
    if (lane == 0) {
      const uint64_t policy = l2_evict_first_policy();
      bool ok = true;
      int c = 0;
      for (; c < nseg; ++c) {
        const int s = c % STAGES;
        if (c >= STAGES && !mbar_wait(&empty[s], ((c / STAGES) & 1) ^ 1)) {
          ok = false;
          break;
        }
        const int p0 = c * CW;
        const uint32_t bytes = (uint32_t)min(CW, ldp - p0) * (uint32_t)sizeof(Pack);
        mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)(nr + nbk));
        Pack* st = stage + s * STAGE;
        for (int r = 0; r < nr; ++r) bulk_g2s_hint(st + r * CW, F + (int64_t)r * ldp + p0, bytes, &full[s], policy);
        for (int k = 0; k < nbk; ++k) bulk_g2s(st + (R + k) * CW, x + k * xb + p0, bytes, &full[s]);
      }
      // no copy may outlive the CTA: wait for the last issued stages to land
      for (int cc = max(0, c - STAGES); cc < c; ++cc)
        if (!mbar_wait(&full[cc % STAGES], (cc / STAGES) & 1)) ok = false;
      if (!ok) atomicOr(d.status, kStatusWaitTimeout);
    }
    return;
  }

  // consumers
  const int tc = threadIdx.x - 32;
  Acc acc[R][KB];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < KB; ++k) acc[r][k] = Kd::zero();
  for (int c = 0; c < nseg; ++c) {
    const int s = c % STAGES;
    if (!mbar_wait(&full[s], (c / STAGES) & 1)) {
      atomicOr(d.status, kStatusWaitTimeout);
      break;
    }
    const Pack* st = stage + s * STAGE;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int q = tc + NC * v;   // pack of the segment
      if (q < ldp - c * CW) {
        // rows r >= nr and right-hand sides k >= nbk (last blocks only) hold
        // stale shared memory; their accumulators are never stored
        Pack xv[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) xv[k] = st[(R + k) * CW + q];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const Pack f = st[r * CW + q];
#pragma unroll
          for (int k = 0; k < KB; ++k) Kd::mac_n(acc[r][k], f, xv[k]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  // reduction over the consumer threads: warp shuffles, then across warps
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) acc[r][k] = Kd::add(acc[r][k], Kd::shfl_xor(acc[r][k], m));
  const int cw = warp - 1;
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < KB; ++k) red[(cw * R + r) * KB + k] = acc[r][k];
  }
  named_bar_sync(1, NC);
  const int r = tc / KB, k = tc % KB;
  if (tc < R * KB && r < nr && k < nbk) {
    Acc sum = red[r * KB + k];
#pragma unroll
    for (int q = 1; q < NCW; ++q) sum = Kd::add(sum, red[(q * R + r) * KB + k]);
    Kd::store(d.y, (b0 + k) * d.y_ld_b + (int64_t)w * d.Nd + r0 + r, sum);
  }
}

// ---------------------------------------------------------------------------
// H direction: grid (ceil(ldp / (T V)), Nf, ceil(K / KB)).  d-hat_w of KB
// right-hand sides sits in shared memory; every F-hat pack loaded from HBM
// serves all KB of them, so K right-hand sides cost ceil(K / KB) passes over
// F-hat instead of K.
// ---------------------------------------------------------------------------
template <class Kd, int V, int T, int U, int KB>
__global__ void __launch_bounds__(T) gemv_h_kernel(GemvDesc d) {
  using Pack = typename Kd::Pack;
  using Elem = typename Kd::Elem;
  using Acc = typename Kd::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Elem* xs = reinterpret_cast<Elem*>(smem_raw);   // [KB][Nd]
  const int w = blockIdx.y;
  const int b0 = blockIdx.z * KB;
  const int nb = min(KB, d.K - b0);
  const int ldp = d.ldn / Kd::P;
  for (int i = threadIdx.x; i < KB * d.Nd; i += T) {
    const int kb = i / d.Nd, r = i - kb * d.Nd;
    const Elem* __restrict__ x = static_cast<const Elem*>(d.x) + (b0 + kb) * d.x_ld_b + (int64_t)w * d.Nd;
    if (kb < nb) xs[i] = x[r];
    else xs[i] = Elem{};  // right-hand sides past K: zeros, results not stored
  }
  __syncthreads();

  const Pack* __restrict__ F = static_cast<const Pack*>(d.F) + (int64_t)w * d.Nd * ldp;
  int pc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int p = blockIdx.x * (T * V) + v * T + threadIdx.x;
    pc[v] = p < ldp ? p : ldp - 1;  // out-of-range columns re-read the last one; not stored
  }
  Acc acc[KB][V][Kd::P];
#pragma unroll
  for (int kb = 0; kb < KB; ++kb)
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int e = 0; e < Kd::P; ++e) acc[kb][v][e] = Kd::zero();

  int r = 0;
  for (; r + U <= d.Nd; r += U) {
    Pack fv[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < V; ++v) fv[u][v] = Kd::ldF(F + (int64_t)(r + u) * ldp + pc[v]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        const Elem xr = xs[kb * d.Nd + r + u];
#pragma unroll
        for (int v = 0; v < V; ++v) Kd::mac_h(acc[kb][v], fv[u][v], xr);
      }
    }
  }
  for (; r < d.Nd; ++r) {
    Pack fv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) fv[v] = Kd::ldF(F + (int64_t)r * ldp + pc[v]);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const Elem xr = xs[kb * d.Nd + r];
#pragma unroll
      for (int v = 0; v < V; ++v) Kd::mac_h(acc[kb][v], fv[v], xr);
    }
  }
#pragma unroll
  for (int kb = 0; kb < KB; ++kb) {
    if (kb >= nb) break;
    const int64_t yo = (b0 + kb) * d.y_ld_b + (int64_t)w * d.ldn;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int p = blockIdx.x * (T * V) + v * T + threadIdx.x;
      if (p < ldp) {
#pragma unroll
        for (int e = 0; e < Kd::P; ++e) Kd::store(d.y, yo + (int64_t)p * Kd::P + e, acc[kb][v][e]);
      }
    }
  }
}

// H direction, one right-hand side, bulk-copy pipelined: grid (ceil(ldp /
// CW), Nf).  Warp 0 (one elected thread) streams the CTA's run of CW packs of
// RS rows of F-hat_w at a time into a ring of STAGES shared-memory stages with
// cp.async.bulk (one contiguous copy per row); NCW consumer warps own V packs
// each (consumer thread tc: packs tc + NC v) and accumulate them over every
// row with d-hat_w from shared memory, releasing each stage through its
// "empty" mbarrier.  As the N kernel, bytes stay in flight while the
// consumers do their double-float arithmetic.
template <class Kd, int V, int NCW, int RS, int STAGES, int KB>
__global__ void __launch_bounds__(32 * (NCW + 1)) gemv_h_pipe_kernel(GemvDesc d) {
  using Pack = typename Kd::Pack;
  using Elem = typename Kd::Elem;
  using Acc = typename Kd::Acc;
  constexpr int NC = 32 * NCW;
  constexpr int CW = NC * V;         // packs per row run
  constexpr int STAGE = RS * CW;     // packs per stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Pack* stage = reinterpret_cast<Pack*>(smem_raw);
  Elem* xs = reinterpret_cast<Elem*>(stage + STAGES * STAGE);   // [KB][Nd]
  uint64_t* full = reinterpret_cast<uint64_t*>(xs + KB * d.Nd);
  uint64_t* empty = full + STAGES;

  const int w = blockIdx.y;
  const int b0 = blockIdx.z * KB;
  const int nb = min(KB, d.K - b0);
  const int ldp = d.ldn / Kd::P;     // packs per row
  const int p0 = blockIdx.x * CW;
  const int np = min(CW, ldp - p0);
  const int nseg = (d.Nd + RS - 1) / RS;
  const Pack* F = static_cast<const Pack*>(d.F) + (int64_t)w * d.Nd * ldp + p0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    mbar_init_fence();
  }
  for (int i = threadIdx.x; i < KB * d.Nd; i += blockDim.x) {
    const int k = i / d.Nd, r = i - k * d.Nd;
    const Elem* x = static_cast<const Elem*>(d.x) + (b0 + k) * d.x_ld_b + (int64_t)w * d.Nd;
    if (k < nb) xs[i] = x[r];
    else xs[i] = Elem{};   // right-hand sides past K: zeros, results not stored
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (warp == 0) {  // producer
    if (lane == 0) {
      const uint64_t policy = l2_evict_first_policy();
      const uint32_t bytes = (uint32_t)np * (uint32_t)sizeof(Pack);
      bool ok = true;
      int c = 0;
      for (; c < nseg; ++c) {
        const int s = c % STAGES;
        if (c >= STAGES && !mbar_wait(&empty[s], ((c / STAGES) & 1) ^ 1)) {
          ok = false;
          break;
        }
        const int r0 = c * RS, nr = min(RS, d.Nd - r0);
        mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)nr);
        Pack* st = stage + s * STAGE;
        for (int r = 0; r < nr; ++r)
          bulk_g2s_hint(st + r * CW, F + (int64_t)(r0 + r) * ldp, bytes, &full[s], policy);
      }
      // no copy may outlive the CTA: wait for the last issued stages to land
      for (int cc = max(0, c - STAGES); cc < c; ++cc)
        if (!mbar_wait(&full[cc % STAGES], (cc / STAGES) & 1)) ok = false;
      if (!ok) atomicOr(d.status, kStatusWaitTimeout);
    }
    return;
  }

  // consumers
  const int tc = threadIdx.x - 32;
  Acc acc[V][KB][Kd::P];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
      for (int e = 0; e < Kd::P; ++e) acc[v][k][e] = Kd::zero();
  for (int c = 0; c < nseg; ++c) {
    const int s = c % STAGES;
    if (!mbar_wait(&full[s], (c / STAGES) & 1)) {
      atomicOr(d.status, kStatusWaitTimeout);
      break;
    }
    const Pack* st = stage + s * STAGE;
    const int r0 = c * RS, nr = min(RS, d.Nd - r0);
    // packs past np (last column run only) hold stale shared memory; their
    // accumulators are never stored
#pragma unroll
    for (int r = 0; r < RS; ++r) {
      if (r < nr) {
        Pack f[V];
#pragma unroll
        for (int v = 0; v < V; ++v) f[v] = st[r * CW + tc + NC * v];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const Elem xv = xs[k * d.Nd + r0 + r];
#pragma unroll
          for (int v = 0; v < V; ++v) Kd::mac_h(acc[v][k], f[v], xv);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (k >= nb) break;
    const int64_t yo = (b0 + k) * d.y_ld_b + (int64_t)w * d.ldn + (int64_t)p0 * Kd::P;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int p = tc + NC * v;
      if (p < np) {
#pragma unroll
        for (int e = 0; e < Kd::P; ++e) Kd::store(d.y, yo + (int64_t)p * Kd::P + e, acc[v][k][e]);
      }
    }
  }
}

// master FP64 F-hat -> stored kind.  The double-float form holds F-hat times
// the power of two `mul` (exact), which brings its largest entry into [1, 2):
// FP32 hi/lo pairs have FP32's exponent range, so this keeps every operator
// whose entries fit FP64 representable, and the inverse FFT multiplies back.
__global__ void convert_df_kernel(const double2* __restrict__ in, float4* __restrict__ out, size_t n, double mul) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 v = in[i];
    v.x *= mul;
    v.y *= mul;
    const float hr = (float)v.x, hi = (float)v.y;
    out[i] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
  }
}
__global__ void convert_f32_kernel(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

// N, one right-hand side: rows per CTA, consumer warps, pipeline stages.
// Double-float: FFTMV_NDF_* below (2.45 ms with 8 rows and 8 warps); FP32 and
// FP64 keep 8 rows and 8 warps, their best.
constexpr int kNR = 8, kNW = 8, kNS = 3;
// double-float: 2 rows, 4 consumer warps with 2 packs each per segment (4 KB
// row runs), 2 stages: 2.25 ms at the paper shape; with 3 stages 2.26, with 4
// stages 2.43; 2.29 for 4 rows and one pack (2 KB runs), 2.34 for 4 rows and
// two packs, 2.33 / 2.69 for 4 rows and four packs with 2 / 3 stages, 2.27 for
// 2 rows and four packs, 2.39 for one row and four packs, 2.30 with 2 consumer
// warps
#ifndef FFTMV_NDF_R
#define FFTMV_NDF_R 2
#endif
#ifndef FFTMV_NDF_W
#define FFTMV_NDF_W 4
#endif
#ifndef FFTMV_NDF_ST
#define FFTMV_NDF_ST 2
#endif
#ifndef FFTMV_NDF_V
#define FFTMV_NDF_V 2
#endif
constexpr int kHV = 2, kHT = 256, kHU = 4;   // H: packs per thread, threads, rows in flight

template <class Kd, int R, int KB, int NCW, int STAGES, int V = 1>
cudaError_t run_n_cfg(const GemvDesc& d, cudaStream_t s) {
  auto kernel = gemv_n_kernel<Kd, R, KB, NCW, STAGES, V>;
  const size_t smem = (size_t)STAGES * (R + KB) * (32 * NCW * V) * sizeof(typename Kd::Pack) +
                      2 * STAGES * sizeof(uint64_t) + (size_t)NCW * R * KB * sizeof(typename Kd::Acc);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((d.Nd + R - 1) / R, d.Nf, (d.K + KB - 1) / KB);
  kernel<<<grid, 32 * (NCW + 1), smem, s>>>(d);
  return cudaGetLastError();
}

template <class Kd>
cudaError_t run_n(const GemvDesc& d, cudaStream_t s) {
  if constexpr (std::is_same<Kd, KindDF>::value)
    return run_n_cfg<Kd, FFTMV_NDF_R, 1, FFTMV_NDF_W, FFTMV_NDF_ST, FFTMV_NDF_V>(d, s);
  else return run_n_cfg<Kd, kNR, 1, kNW, kNS>(d, s);
}

template <class Kd, int KB>
cudaError_t run_h_kb(const GemvDesc& d, cudaStream_t s) {
  // (packs per thread, threads): double-float, one RHS: 4 x 128 (2.33 ms against
  // 2.36 for 2 x 256 at the paper shape); double-float, 4 RHS: 1 x 256 (6.5 against
  // 7.0 ms); FP32, eight RHS: 2 x 512 (1.85 against 2.64 ms); otherwise 2 x 256
  constexpr bool df1 = std::is_same<Kd, KindDF>::value && KB == 1;
  constexpr bool f8 = std::is_same<Kd, KindF32>::value && KB == 8;
  constexpr bool dfk = std::is_same<Kd, KindDF>::value && KB > 1;   // double-float, several RHS: 1 x 256
  constexpr int V = df1 ? 4 : dfk ? 1 : kHV, T = df1 ? 128 : f8 ? 512 : kHT;
  const int ldp = d.ldn / Kd::P;
  dim3 grid((ldp + T * V - 1) / (T * V), d.Nf, (d.K + KB - 1) / KB);
  const size_t smem = (size_t)KB * d.Nd * sizeof(typename Kd::Elem);
  auto kernel = gemv_h_kernel<Kd, V, T, kHU, KB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, T, smem, s>>>(d);
  return cudaGetLastError();
}

// right-hand sides per CTA: up to 8 for FP32 (8-byte entries), 4 otherwise
// one right-hand side in double-float or FP32: the bulk-copy pipeline (V
// packs per consumer thread, NCW consumer warps, RS rows per stage, STAGES
// stages)
#ifndef FFTMV_HPIPE
#define FFTMV_HPIPE 1
#endif
#ifndef FFTMV_HPIPE_V
#define FFTMV_HPIPE_V 4
#endif
#ifndef FFTMV_HPIPE_W
#define FFTMV_HPIPE_W 4
#endif
#ifndef FFTMV_HPIPE_RS
#define FFTMV_HPIPE_RS 4
#endif
#ifndef FFTMV_HPIPE_ST
#define FFTMV_HPIPE_ST 3
#endif
#ifndef FFTMV_HPIPE_F32
#define FFTMV_HPIPE_F32 1
#endif
#ifndef FFTMV_HPIPE_MULTI
#define FFTMV_HPIPE_MULTI 1
#endif
template <class Kd, int KB, int V>
cudaError_t run_h_pipe(const GemvDesc& d, cudaStream_t s) {
  constexpr int NCW = FFTMV_HPIPE_W, RS = FFTMV_HPIPE_RS, STAGES = FFTMV_HPIPE_ST;
  constexpr int CW = 32 * NCW * V;
  using Pack = typename Kd::Pack;
  using Elem = typename Kd::Elem;
  auto kernel = gemv_h_pipe_kernel<Kd, V, NCW, RS, STAGES, KB>;
  const size_t smem = (size_t)STAGES * RS * CW * sizeof(Pack) + (size_t)KB * d.Nd * sizeof(Elem) +
                      2 * STAGES * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((d.ldn / Kd::P + CW - 1) / CW, d.Nf, (d.K + KB - 1) / KB);
  kernel<<<grid, 32 * (NCW + 1), smem, s>>>(d);
  return cudaGetLastError();
}

template <class Kd>
cudaError_t run_h(const GemvDesc& d, cudaStream_t s) {
#if FFTMV_HPIPE
  if constexpr (!std::is_same<Kd, KindF64>::value) {
    // one right-hand side: V = FFTMV_HPIPE_V packs per thread; several: up to 8
    // (FP32) or 4 (double-float) per pass over F-hat with 2 packs per thread,
    // so the accumulators stay in registers
    const size_t el = sizeof(typename Kd::Elem);
    if (d.K == 1 && (size_t)d.Nd * el <= 64 * 1024 && (FFTMV_HPIPE_F32 || std::is_same<Kd, KindDF>::value))
      return run_h_pipe<Kd, 1, FFTMV_HPIPE_V>(d, s);
    if (FFTMV_HPIPE_MULTI && d.K > 1) {
      constexpr int kmaxp = Kd::P == 2 ? 8 : 4;
      if (d.K >= kmaxp && (size_t)kmaxp * d.Nd * el <= 64 * 1024) return run_h_pipe<Kd, kmaxp, 2>(d, s);
      if (d.K >= 4 && (size_t)4 * d.Nd * el <= 64 * 1024) return run_h_pipe<Kd, 4, 2>(d, s);
      if ((size_t)2 * d.Nd * el <= 64 * 1024) return run_h_pipe<Kd, 2, 2>(d, s);
    }
  }
#endif
  const int kmax = Kd::P == 2 ? 8 : 4;
  if (d.K >= 8 && kmax >= 8) return run_h_kb<Kd, 8>(d, s);
  if (d.K >= 4) return run_h_kb<Kd, 4>(d, s);
  if (d.K >= 2) return run_h_kb<Kd, 2>(d, s);
  return run_h_kb<Kd, 1>(d, s);
}

}  // namespace

int gemv_in_fmt(int kind) {
  switch (kind) {
    case GEMV_F64: return FMT_C128;
    case GEMV_DF: return FMT_DF;
    case GEMV_TC: return FMT_TC;
    default: return FMT_C64;
  }
}
int gemv_out_fmt(int kind) {
  switch (kind) {
    case GEMV_F64: return FMT_C128;
    case GEMV_DF: return FMT_DF;
    default: return FMT_C64;  // GEMV_F32 and GEMV_TC write float2
  }
}
size_t fmt_bytes(int fmt) { return fmt == FMT_C64 ? 8 : 16; }

cudaError_t launch_gemv_n(int kind, const GemvDesc& d, cudaStream_t s) {
  if (d.Nf == 0 || d.Nd == 0 || d.K == 0) return cudaSuccess;
  switch (kind) {
    // one right-hand side: 8 rows per CTA; several: every F-hat pack feeds
    // KB of them (FP64 stays at one: its FMA rate, not HBM, bounds it)
    case GEMV_F64: return run_n<KindF64>(d, s);
    // double-float, several RHS: 4 rows x 4 RHS, 4 warps (4 RHS: 8.4 ms against 9.2 for 2 rows)
    case GEMV_DF: return d.K == 1 ? run_n<KindDF>(d, s) : run_n_cfg<KindDF, 4, 4, 4, 3>(d, s);
    // FP32, several RHS: 8 rows x 8 RHS, 4 consumer warps, 2 stages (8 RHS at the
    // paper shape: 2.14 ms against 2.89 for 4 rows x 8 RHS with 3 stages)
    default: return d.K == 1 ? run_n<KindF32>(d, s) : run_n_cfg<KindF32, 8, 8, 4, 2>(d, s);
  }
}

cudaError_t launch_gemv_h(int kind, const GemvDesc& d, cudaStream_t s) {
  if (d.Nf == 0 || d.ldn == 0 || d.K == 0) return cudaSuccess;
  switch (kind) {
    case GEMV_F64: return run_h<KindF64>(d, s);
    case GEMV_DF: return run_h<KindDF>(d, s);
    default: return run_h<KindF32>(d, s);
  }
}

cudaError_t launch_convert_fhat(int kind, const double2* master, void* out, size_t n, int fexp, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)((n + threads - 1) / threads < (size_t)152 * 32 ? (n + threads - 1) / threads : 152 * 32);
  if (kind == GEMV_DF) convert_df_kernel<<<blocks, threads, 0, s>>>(master, static_cast<float4*>(out), n, ldexp(1.0, -fexp));
  else convert_f32_kernel<<<blocks, threads, 0, s>>>(master, static_cast<float2*>(out), n);
  return cudaGetLastError();
}

namespace {

// max |x| over the n values of right-hand side blockIdx.y, as the bits of a
// non-negative double (their integer order is the order of the values); a
// block reduction, then one atomicMax per CTA
template <typename T>
__global__ void __launch_bounds__(512) absmax_kernel(const T* __restrict__ x, int64_t n,
                                                     unsigned long long* __restrict__ absmax) {
  __shared__ double red[16];
  const T* p = x + (int64_t)blockIdx.y * n;
  double m0 = 0.0, m1 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {   // two loads in flight
    m0 = fmax(m0, fabs((double)__ldcs(p + i)));
    m1 = fmax(m1, fabs((double)__ldcs(p + i + stride)));
  }
  if (i < n) m0 = fmax(m0, fabs((double)__ldcs(p + i)));
  double mx = fmax(m0, m1);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) atomicMax(absmax + blockIdx.y, (unsigned long long)__double_as_longlong(mx));
  }
}

}  // namespace

cudaError_t launch_absmax(const void* x, bool x_f32, int K, int64_t n, unsigned long long* absmax, cudaStream_t s) {
  if (K == 0) return cudaSuccess;
  // about four CTAs of 512 threads per SM over all right-hand sides, at least 32 values a thread
  int64_t bx = (4 * 152 + K - 1) / K;
  const int64_t most = (n + 512 * 32 - 1) / (512 * 32);
  bx = bx > most ? most : bx;
  bx = bx < 1 ? 1 : bx;
  dim3 grid((unsigned)bx, K);
  if (x_f32) absmax_kernel<float><<<grid, 512, 0, s>>>(static_cast<const float*>(x), n, absmax);
  else absmax_kernel<double><<<grid, 512, 0, s>>>(static_cast<const double*>(x), n, absmax);
  return cudaGetLastError();
}

}  // namespace fftmv
