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

#include "fftmv_internal.h"

namespace fftmv {
namespace {

template <typename T> struct CxT;
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return {a.x * s, a.y * s}; }

// Constants of the small DFTs (cos/sin of 2 pi / 5, 4 pi / 5, pi / 3, pi / 4).
#define K_C1 0.30901699437494742410
#define K_C2 (-0.80901699437494742410)
#define K_S1 0.95105651629515357212
#define K_S2 0.58778525229247312917
#define K_S3 0.86602540378443864676
#define K_R2 0.70710678118654752440

// In-register DFT of size R: X_p = sum_q v_q exp(-+2 pi i q p / R).
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 2, INV> {
  using C = typename CxT<T>::type;
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename T, bool INV> struct Dft<T, 3, INV> {
  using C = typename CxT<T>::type;
  __device__ __forceinline__ static void run(C* v) {
    C s = cadd(v[1], v[2]);
    C d = mul_mi<INV>(csub(v[1], v[2]));
    C m = {v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y};
    C dd = cscale(d, T(K_S3));
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, dd);
    v[2] = csub(m, dd);
  }
};

template <typename T, bool INV> struct Dft<T, 4, INV> {
  using C = typename CxT<T>::type;
  __device__ __forceinline__ static void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <typename T, bool INV> struct Dft<T, 5, INV> {
  using C = typename CxT<T>::type;
  __device__ __forceinline__ static void run(C* v) {
    C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    C x0 = v[0];
    C r1 = {x0.x + T(K_C1) * a1.x + T(K_C2) * a2.x, x0.y + T(K_C1) * a1.y + T(K_C2) * a2.y};
    C r2 = {x0.x + T(K_C2) * a1.x + T(K_C1) * a2.x, x0.y + T(K_C2) * a1.y + T(K_C1) * a2.y};
    C j1 = mul_mi<INV>(C{T(K_S1) * b1.x + T(K_S2) * b2.x, T(K_S1) * b1.y + T(K_S2) * b2.y});
    C j2 = mul_mi<INV>(C{T(K_S2) * b1.x - T(K_S1) * b2.x, T(K_S2) * b1.y - T(K_S1) * b2.y});
    v[0] = cadd(x0, cadd(a1, a2));
    v[1] = cadd(r1, j1);
    v[4] = csub(r1, j1);
    v[2] = cadd(r2, j2);
    v[3] = csub(r2, j2);
  }
};

template <typename T, bool INV> struct Dft<T, 8, INV> {
  using C = typename CxT<T>::type;
  __device__ __forceinline__ static void run(C* v) {
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4, INV>::run(e);
    Dft<T, 4, INV>::run(o);
    // o_p *= exp(-+2 pi i p / 8)
    const T r = T(K_R2);
    o[1] = INV ? C{r * (o[1].x - o[1].y), r * (o[1].x + o[1].y)} : C{r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
    o[2] = mul_mi<INV>(o[2]);
    o[3] = INV ? C{-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y)} : C{r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      v[p] = cadd(e[p], o[p]);
      v[p + 4] = csub(e[p], o[p]);
    }
  }
};

// One Stockham pass of radix R over a length-L signal: reads `in`, writes `out`.
// Butterfly j (< L/R) takes in[j + q L/R], applies the twiddle of its position
// k = j mod Ns inside the current sub-transform, and writes out[(j-k) R + k + q Ns].
template <typename T, int R, bool INV>
__device__ __forceinline__ void stockham_pass(const typename CxT<T>::type* __restrict__ in,
                                              typename CxT<T>::type* __restrict__ out, int L, int Ns,
                                              const typename CxT<T>::type* __restrict__ tw) {
  using C = typename CxT<T>::type;
  const int nb = L / R;
  const int tw_step = L / (Ns * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = in[j + q * nb];
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        C w = tw[q * k * tw_step];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    Dft<T, R, INV>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) out[base + q * Ns] = v[q];
  }
}

// Full FFT of the signal in buf0; returns the buffer that holds the result.
template <typename T, bool INV>
__device__ typename CxT<T>::type* fft_smem(typename CxT<T>::type* buf0, typename CxT<T>::type* buf1,
                                           const FftPlan& plan, const typename CxT<T>::type* __restrict__ tw) {
  using C = typename CxT<T>::type;
  C* in = buf0;
  C* out = buf1;
  int Ns = 1;
  for (int p = 0; p < plan.npass; ++p) {
    const int R = plan.rad[p];
    __syncthreads();
    switch (R) {
      case 2: stockham_pass<T, 2, INV>(in, out, plan.L, Ns, tw); break;
      case 3: stockham_pass<T, 3, INV>(in, out, plan.L, Ns, tw); break;
      case 4: stockham_pass<T, 4, INV>(in, out, plan.L, Ns, tw); break;
      case 5: stockham_pass<T, 5, INV>(in, out, plan.L, Ns, tw); break;
      default: stockham_pass<T, 8, INV>(in, out, plan.L, Ns, tw); break;
    }
    Ns *= R;
    C* t = in;
    in = out;
    out = t;
  }
  __syncthreads();
  return in;
}

template <typename T> __device__ __forceinline__ T load_real(const void* p, int64_t i);
template <> __device__ __forceinline__ double load_real<double>(const void* p, int64_t i) {
  return __ldg(static_cast<const double*>(p) + i);
}
template <> __device__ __forceinline__ float load_real<float>(const void* p, int64_t i) {
  return __ldg(static_cast<const float*>(p) + i);
}

// Store one complex value (re, im) computed in precision T into format fmt.
template <typename T>
__device__ __forceinline__ void store_cx(void* X, int64_t i, int fmt, T re, T im) {
  if (fmt == FMT_C128) {
    static_cast<double2*>(X)[i] = make_double2((double)re, (double)im);
  } else if (fmt == FMT_C64) {
    static_cast<float2*>(X)[i] = make_float2((float)re, (float)im);
  } else {
    const float hr = (float)re, hi = (float)im;
    const float lr = (float)((double)re - (double)hr), li = (float)((double)im - (double)hi);
    static_cast<float4*>(X)[i] = make_float4(hr, hi, lr, li);
  }
}

__device__ __forceinline__ double2 load_cx(const void* X, int64_t i, int fmt) {
  if (fmt == FMT_C128) return __ldg(static_cast<const double2*>(X) + i);
  const float2 v = __ldg(static_cast<const float2*>(X) + i);
  return make_double2(v.x, v.y);
}

// Forward: pad + real FFT of channel pairs; grid (pairs, K).
template <typename Tin, typename T>
__global__ void __launch_bounds__(256) rfft_fwd_kernel(FwdDesc d) {
  using C = typename CxT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + d.plan.L;
  const int L = d.plan.L;
  const int Nf = L / 2 + 1;
  const int pairs_per_row = (d.out_cols + 1) / 2;
  const int row = blockIdx.x / pairs_per_row;
  const int ca = 2 * (blockIdx.x % pairs_per_row);
  const int cb = ca + 1;
  const int b = blockIdx.y;
  const int64_t xo = b * d.x_ld_b + row * d.x_ld_row;
  const int64_t Xo = b * d.X_ld_b + row * d.X_ld_row;
  const bool has_a = ca < d.cols, has_b = cb < d.cols;
  const bool write_b = cb < d.out_cols;

  if (!has_a) {  // a pair of padding columns: exact zeros
    for (int w = threadIdx.x; w < Nf; w += blockDim.x) {
      store_cx<T>(d.X, Xo + w * d.X_ld_w + ca, d.fmt, T(0), T(0));
      if (write_b) store_cx<T>(d.X, Xo + w * d.X_ld_w + cb, d.fmt, T(0), T(0));
    }
    return;
  }
  // phase 1: load, cast to the pad precision, then to the FFT precision; zero pad
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    T va = T(0), vb = T(0);
    if (t < d.Nt) {
      Tin a = load_real<Tin>(d.x, xo + t * d.x_ld_t + ca);
      Tin bb = has_b ? load_real<Tin>(d.x, xo + t * d.x_ld_t + cb) : Tin(0);
      if (d.pad_single) {
        a = (Tin)(float)a;
        bb = (Tin)(float)bb;
      }
      va = (T)a;
      vb = (T)bb;
    }
    buf0[t] = C{va, vb};
  }
  // phase 2: complex FFT of z = x_a + i x_b
  const C* tw = static_cast<const C*>(d.tw);
  const C* Z = fft_smem<T, false>(buf0, buf1, d.plan, tw);
  // split: X_a = (Z_w + conj Z_{L-w}) / 2,  X_b = (Z_w - conj Z_{L-w}) / (2i)
  for (int w = threadIdx.x; w < Nf; w += blockDim.x) {
    const C z = Z[w];
    const C zc = Z[w == 0 ? 0 : L - w];
    const T ar = T(0.5) * (z.x + zc.x), ai = T(0.5) * (z.y - zc.y);
    const T br = T(0.5) * (z.y + zc.y), bi = T(0.5) * (zc.x - z.x);
    store_cx<T>(d.X, Xo + w * d.X_ld_w + ca, d.fmt, ar, ai);
    if (write_b) {
      if (has_b) store_cx<T>(d.X, Xo + w * d.X_ld_w + cb, d.fmt, br, bi);
      else store_cx<T>(d.X, Xo + w * d.X_ld_w + cb, d.fmt, T(0), T(0));
    }
  }
}

template <typename T> __device__ __forceinline__ void store_real(void* y, int64_t i, T v);
template <> __device__ __forceinline__ void store_real<double>(void* y, int64_t i, double v) {
  static_cast<double*>(y)[i] = v;
}
template <> __device__ __forceinline__ void store_real<float>(void* y, int64_t i, float v) {
  static_cast<float*>(y)[i] = v;
}

// Inverse: Hermitian assembly + inverse complex FFT + unpad; grid (pairs, K).
template <typename T, typename Tout>
__global__ void __launch_bounds__(256) irfft_inv_kernel(InvDesc d) {
  using C = typename CxT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + d.plan.L;
  const int L = d.plan.L;
  const int Nf = L / 2 + 1;
  const int ca = 2 * blockIdx.x, cb = ca + 1;
  const int b = blockIdx.y;
  const bool has_b = cb < d.cols;
  const int64_t Xo = b * d.X_ld_b;
  // Z_w = X_a(w) + i X_b(w) over the full circle, X(L-w) = conj X(w);
  // the DC and Nyquist terms of a real signal's spectrum are taken as real.
  for (int w = threadIdx.x; w < Nf; w += blockDim.x) {
    double2 a = load_cx(d.X, Xo + w * d.X_ld_w + ca, d.in_fmt);
    double2 bb = has_b ? load_cx(d.X, Xo + w * d.X_ld_w + cb, d.in_fmt) : make_double2(0.0, 0.0);
    const T ax = (T)a.x, ay = (T)a.y, bx = (T)bb.x, by = (T)bb.y;
    if (w == 0 || w == Nf - 1) {
      buf0[w] = C{ax, bx};
    } else {
      buf0[w] = C{ax - by, ay + bx};
      buf0[L - w] = C{ax + by, bx - ay};
    }
  }
  const C* tw = static_cast<const C*>(d.tw);
  const C* z = fft_smem<T, true>(buf0, buf1, d.plan, tw);
  const T scale = T(1) / T(L);
  for (int t = threadIdx.x; t < d.Nt; t += blockDim.x) {
    T va = z[t].x * scale, vb = z[t].y * scale;
    if (d.unpad_single) {
      va = (T)(float)va;
      vb = (T)(float)vb;
    }
    const int64_t yo = b * d.y_ld_b + t * d.y_ld_t;
    store_real<Tout>(d.y, yo + ca, (Tout)va);
    if (has_b) store_real<Tout>(d.y, yo + cb, (Tout)vb);
  }
}

template <typename K>
cudaError_t prep(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

}  // namespace

size_t fft_smem_bytes(int L, bool fft_f32) { return 2 * (size_t)L * (fft_f32 ? sizeof(float2) : sizeof(double2)); }

int fft_max_length(bool fft_f32) {
  const size_t cap = 227 * 1024;
  return (int)(cap / (2 * (fft_f32 ? sizeof(float2) : sizeof(double2))));
}

cudaError_t launch_rfft_fwd(const FwdDesc& d, bool in_f32, bool fft_f32, cudaStream_t s) {
  const int pairs = d.rows * ((d.out_cols + 1) / 2);
  if (pairs == 0 || d.K == 0) return cudaSuccess;
  dim3 grid(pairs, d.K);
  const size_t smem = fft_smem_bytes(d.plan.L, fft_f32);
  cudaError_t e;
#define FWD_CASE(TIN, T)                                           \
  do {                                                             \
    if ((e = prep(rfft_fwd_kernel<TIN, T>, smem)) != cudaSuccess) return e; \
    rfft_fwd_kernel<TIN, T><<<grid, 256, smem, s>>>(d);            \
  } while (0)
  if (!in_f32 && !fft_f32) FWD_CASE(double, double);
  else if (!in_f32 && fft_f32) FWD_CASE(double, float);
  else if (in_f32 && !fft_f32) FWD_CASE(float, double);
  else FWD_CASE(float, float);
#undef FWD_CASE
  return cudaGetLastError();
}

cudaError_t launch_irfft_inv(const InvDesc& d, bool fft_f32, bool out_f32, cudaStream_t s) {
  const int pairs = (d.cols + 1) / 2;
  if (pairs == 0 || d.K == 0) return cudaSuccess;
  dim3 grid(pairs, d.K);
  const size_t smem = fft_smem_bytes(d.plan.L, fft_f32);
  cudaError_t e;
#define INV_CASE(T, TOUT)                                            \
  do {                                                               \
    if ((e = prep(irfft_inv_kernel<T, TOUT>, smem)) != cudaSuccess) return e; \
    irfft_inv_kernel<T, TOUT><<<grid, 256, smem, s>>>(d);            \
  } while (0)
  if (!fft_f32 && !out_f32) INV_CASE(double, double);
  else if (!fft_f32 && out_f32) INV_CASE(double, float);
  else if (fft_f32 && !out_f32) INV_CASE(float, double);
  else INV_CASE(float, float);
#undef INV_CASE
  return cudaGetLastError();
}

}  // namespace fftmv
