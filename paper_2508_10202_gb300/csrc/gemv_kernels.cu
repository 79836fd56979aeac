// Per-frequency complex block matvec (Section 2.4, phase 3; Section 3.1.1's
// short-and-wide strided-batched GEMV), written for sm_103a.
//
// For every frequency w the operator block F-hat_w is Nd x Nm complex with
// Nd << Nm, stored row-major with a padded row length ldn (a multiple of 8).
// Both directions stream F-hat exactly once with 16-byte vector loads:
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

#include "fftmv_internal.h"

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
  __device__ __forceinline__ static Pack ldX(const Pack* p) { return __ldg(p); }
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
  __device__ __forceinline__ static Pack ldX(const Pack* p) { return __ldg(p); }
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
  __device__ __forceinline__ static Pack ldX(const Pack* p) { return __ldg(p); }
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
// N direction: grid (ceil(Nd / R), Nf, K), T threads, U column steps in flight
// ---------------------------------------------------------------------------
template <class Kd, int R, int T, int U>
__global__ void __launch_bounds__(T) gemv_n_kernel(GemvDesc d) {
  using Pack = typename Kd::Pack;
  using Acc = typename Kd::Acc;
  __shared__ Acc red[T / 32][R];
  const int w = blockIdx.y, b = blockIdx.z;
  const int r0 = blockIdx.x * R;
  const int ldp = d.ldn / Kd::P;  // packs per row
  const Pack* __restrict__ F = static_cast<const Pack*>(d.F) + ((int64_t)w * d.Nd + r0) * ldp;
  const Pack* __restrict__ x =
      static_cast<const Pack*>(d.x) + (b * d.x_ld_b + (int64_t)w * d.ldn) / Kd::P;
  // rows past Nd (last block only) re-read row r0 and are discarded
  const Pack* rowp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) rowp[r] = (r0 + r < d.Nd) ? F + (int64_t)r * ldp : F;

  Acc acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = Kd::zero();

  int p = threadIdx.x;
  for (; p + (U - 1) * T < ldp; p += U * T) {
    Pack xv[U], fv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = Kd::ldX(x + p + u * T);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) fv[u][r] = Kd::ldF(rowp[r] + p + u * T);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) Kd::mac_n(acc[r], fv[u][r], xv[u]);
  }
  for (; p < ldp; p += T) {
    const Pack xv = Kd::ldX(x + p);
#pragma unroll
    for (int r = 0; r < R; ++r) Kd::mac_n(acc[r], Kd::ldF(rowp[r] + p), xv);
  }
  // block reduction: warp shuffles, then across warps through shared memory
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc[r] = Kd::add(acc[r], Kd::shfl_xor(acc[r], m));
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < R; ++r) red[warp][r] = acc[r];
  }
  __syncthreads();
  if (threadIdx.x < R && r0 + (int)threadIdx.x < d.Nd) {
    Acc s = red[0][threadIdx.x];
#pragma unroll
    for (int q = 1; q < T / 32; ++q) s = Kd::add(s, red[q][threadIdx.x]);
    Kd::store(d.y, b * d.y_ld_b + (int64_t)w * d.Nd + r0 + threadIdx.x, s);
  }
}

// ---------------------------------------------------------------------------
// H direction: grid (ceil(ldp / (T V)), Nf, K); d-hat_w in shared memory
// ---------------------------------------------------------------------------
template <class Kd, int V, int T, int U>
__global__ void __launch_bounds__(T) gemv_h_kernel(GemvDesc d) {
  using Pack = typename Kd::Pack;
  using Elem = typename Kd::Elem;
  using Acc = typename Kd::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Elem* xs = reinterpret_cast<Elem*>(smem_raw);
  const int w = blockIdx.y, b = blockIdx.z;
  const int ldp = d.ldn / Kd::P;
  const Elem* __restrict__ x = static_cast<const Elem*>(d.x) + b * d.x_ld_b + (int64_t)w * d.Nd;
  for (int r = threadIdx.x; r < d.Nd; r += T) xs[r] = x[r];
  __syncthreads();

  const Pack* __restrict__ F = static_cast<const Pack*>(d.F) + (int64_t)w * d.Nd * ldp;
  int pc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int p = blockIdx.x * (T * V) + v * T + threadIdx.x;
    pc[v] = p < ldp ? p : ldp - 1;  // out-of-range columns re-read the last one; not stored
  }
  Acc acc[V][Kd::P];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int e = 0; e < Kd::P; ++e) acc[v][e] = Kd::zero();

  int r = 0;
  for (; r + U <= d.Nd; r += U) {
    Pack fv[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < V; ++v) fv[u][v] = Kd::ldF(F + (int64_t)(r + u) * ldp + pc[v]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const Elem xr = xs[r + u];
#pragma unroll
      for (int v = 0; v < V; ++v) Kd::mac_h(acc[v], fv[u][v], xr);
    }
  }
  for (; r < d.Nd; ++r) {
    const Elem xr = xs[r];
#pragma unroll
    for (int v = 0; v < V; ++v) Kd::mac_h(acc[v], Kd::ldF(F + (int64_t)r * ldp + pc[v]), xr);
  }
  const int64_t yo = b * d.y_ld_b + (int64_t)w * d.ldn;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int p = blockIdx.x * (T * V) + v * T + threadIdx.x;
    if (p < ldp) {
#pragma unroll
      for (int e = 0; e < Kd::P; ++e) Kd::store(d.y, yo + (int64_t)p * Kd::P + e, acc[v][e]);
    }
  }
}

// master FP64 F-hat -> stored kind
__global__ void convert_df_kernel(const double2* __restrict__ in, float4* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
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

constexpr int kNR = 8, kNT = 256, kNU = 2;   // N: rows per CTA, threads, column steps
constexpr int kHV = 2, kHT = 256, kHU = 4;   // H: packs per thread, threads, rows in flight

template <class Kd>
cudaError_t run_n(const GemvDesc& d, cudaStream_t s) {
  dim3 grid((d.Nd + kNR - 1) / kNR, d.Nf, d.K);
  gemv_n_kernel<Kd, kNR, kNT, kNU><<<grid, kNT, 0, s>>>(d);
  return cudaGetLastError();
}

template <class Kd>
cudaError_t run_h(const GemvDesc& d, cudaStream_t s) {
  const int ldp = d.ldn / Kd::P;
  dim3 grid((ldp + kHT * kHV - 1) / (kHT * kHV), d.Nf, d.K);
  const size_t smem = (size_t)d.Nd * sizeof(typename Kd::Elem);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gemv_h_kernel<Kd, kHV, kHT, kHU>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gemv_h_kernel<Kd, kHV, kHT, kHU><<<grid, kHT, smem, s>>>(d);
  return cudaGetLastError();
}

}  // namespace

int gemv_in_fmt(int kind) { return kind == GEMV_F64 ? FMT_C128 : kind == GEMV_DF ? FMT_DF : FMT_C64; }
int gemv_out_fmt(int kind) { return kind == GEMV_F32 ? FMT_C64 : kind == GEMV_DF ? FMT_DF : FMT_C128; }
size_t fmt_bytes(int fmt) { return fmt == FMT_C64 ? 8 : 16; }

cudaError_t launch_gemv_n(int kind, const GemvDesc& d, cudaStream_t s) {
  if (d.Nf == 0 || d.Nd == 0 || d.K == 0) return cudaSuccess;
  switch (kind) {
    case GEMV_F64: return run_n<KindF64>(d, s);
    case GEMV_DF: return run_n<KindDF>(d, s);
    default: return run_n<KindF32>(d, s);
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

cudaError_t launch_convert_fhat(int kind, const double2* master, void* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)((n + threads - 1) / threads < (size_t)152 * 32 ? (n + threads - 1) / threads : 152 * 32);
  if (kind == GEMV_DF) convert_df_kernel<<<blocks, threads, 0, s>>>(master, static_cast<float4*>(out), n);
  else convert_f32_kernel<<<blocks, threads, 0, s>>>(master, static_cast<float2*>(out), n);
  return cudaGetLastError();
}

}  // namespace fftmv
