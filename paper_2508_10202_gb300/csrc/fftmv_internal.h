// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/fftmv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fftmv {

// Storage formats of complex arrays between phases.
enum CFmt : int {
  FMT_C128 = 0,  // double2 (re, im)
  FMT_C64 = 1,   // float2 (re, im)
  FMT_DF = 2,    // float4 (re_hi, im_hi, re_lo, im_lo): value = hi + lo, |lo| <= ulp(hi)/2
  FMT_TC = 3,    // spectra for the tensor cores, written straight into the bf16 B operand
                 // planes (TcShape, TcDesc)
};

// Arithmetic used by the per-frequency block matvec (phase 3).
enum GemvKind : int {
  GEMV_F64 = 0,   // FP64 F-hat, FP64 FMA
  GEMV_DF = 1,    // FP64-class: F-hat as FP32 hi/lo pairs, double-float arithmetic on the FP32 pipe
  GEMV_F32 = 2,   // FP32 F-hat, FP32 FMA
  GEMV_TC = 3,    // tensor cores: bf16 hi/lo F-hat and M-hat, FP32 accumulate (forward only)
};

// Arithmetic of an FFT phase.
enum FftPrec : int {
  FFT_F64 = 0,  // FP64 FMA
  FFT_F32 = 1,  // FP32
  FFT_DF = 2,   // FP64-class double-float on the FP32 pipe
};

constexpr int kMaxPasses = 16;

// A mixed-radix (2, 3, 4, 5, 8) complex FFT of length L done in shared memory.
// The passes are grouped by radix in the order 8, 4, 2, 5, 3 (the kernels rely
// on it).
struct FftPlan {
  int L;
  int npass;
  int rad[kMaxPasses];
  int ns[kMaxPasses];         // sub-transform length before pass p (product of the earlier radices)
  int tws[kMaxPasses];        // twiddle table stride L / (ns * rad)
  unsigned magic[kMaxPasses]; // ceil(2^32 / ns): j / ns = umulhi(j, magic) for j < 2^16 (ns > 1)
};

// In-place decimation-in-frequency plans of the compile-time FFT lengths
// (the FP32 kernels of fft_dif.cuh).  L = rad[0] rad[1] ... rad[n-1]; pass s
// works on blocks of M_s = L / (rad[0] ... rad[s-1]) points with butterflies
// of stride S_s = M_s / rad[s], and multiplies output q of butterfly j by
// W_{M_s}^{j q} (W_M = exp(-2 pi i / M)).  The result is left in
// digit-reversed order: frequency r_0 + rad[0] (r_1 + rad[1] (r_2 ...)) at
// position r_0 S_0 + r_1 S_1 + r_2 S_2 ...
struct DifPlan {
  int n;
  int rad[5];
};
__host__ __device__ constexpr DifPlan dif_plan(int L) {
  return L == 2000 ? DifPlan{3, {16, 5, 25, 1}}
       : L == 1000 ? DifPlan{3, {8, 5, 25, 1}}
       : L == 512  ? DifPlan{3, {8, 8, 8, 1}}
       : L == 256  ? DifPlan{2, {16, 16, 1, 1}}
       : L == 128  ? DifPlan{2, {16, 8, 1, 1}}
                   : DifPlan{0, {1, 1, 1, 1}};
}
__host__ __device__ constexpr int dif_M(int L, int s) {
  int m = L;
  for (int i = 0; i < s; ++i) m /= dif_plan(L).rad[i];
  return m;
}
__host__ __device__ constexpr int dif_S(int L, int s) { return dif_M(L, s) / dif_plan(L).rad[s]; }
// twiddle table of the plan: for every pass with S_s > 1, S_s rows of
// rad[s] - 1 entries (W_{M_s}^{j q}, q = 1 .. rad[s] - 1) padded to an even
// count, so that rows start 16-byte aligned for FP32 complexes
__host__ __device__ constexpr int dif_tw_row(int R) { return R / 2 * 2; }
__host__ __device__ constexpr int dif_tw_offset(int L, int s) {
  int off = 0;
  for (int i = 0; i < s; ++i)
    if (dif_S(L, i) > 1) off += dif_S(L, i) * dif_tw_row(dif_plan(L).rad[i]);
  return off;
}
__host__ __device__ constexpr int dif_tw_size(int L) { return dif_tw_offset(L, dif_plan(L).n); }

// Plans of the double-float in-place kernels (fft_dif_df.cuh), with the same
// conventions.  A double-float complex takes four registers, so the radices
// stay at 8 and below: 2000 = 8 2 5 5 5, 1000 = 8 5 5 5.  Their twiddle table
// has S_s rows of rad[s] - 1 entries for every pass with S_s > 1, each entry a
// double-float complex in the FMT_DF layout (re_hi, im_hi, re_lo, im_lo).
__host__ __device__ constexpr DifPlan dfd_plan(int L) {
  return L == 2000 ? DifPlan{5, {8, 2, 5, 5, 5}} : L == 1000 ? DifPlan{4, {8, 5, 5, 5, 1}} : DifPlan{0, {1, 1, 1, 1, 1}};
}
__host__ __device__ constexpr int dfd_M(int L, int s) {
  int m = L;
  for (int i = 0; i < s; ++i) m /= dfd_plan(L).rad[i];
  return m;
}
__host__ __device__ constexpr int dfd_S(int L, int s) { return dfd_M(L, s) / dfd_plan(L).rad[s]; }
__host__ __device__ constexpr int dfd_tw_offset(int L, int s) {
  int off = 0;
  for (int i = 0; i < s; ++i)
    if (dfd_S(L, i) > 1) off += dfd_S(L, i) * (dfd_plan(L).rad[i] - 1);
  return off;
}
__host__ __device__ constexpr int dfd_tw_size(int L) { return dfd_tw_offset(L, dfd_plan(L).n); }

// Forward real FFT of zero-padded channels (phases 1-2 fused).
// Channel c = (row, col) with col < cols; channels (2q, 2q+1) of a row are
// transformed together as one complex signal.  x[b][t][row][col] is read for
// t < Nt; X[b][w][row][col] is written for w < L/2+1 and col < out_cols
// (columns cols..out_cols-1 are written as zeros).
struct FwdDesc {
  FftPlan plan;
  const void* tw;          // twiddles exp(-2 pi i j / L), j < L (double2 or float2)
  const void* x;           // real input (double or float)
  void* X;                 // complex output in format fmt
  int Nt;
  int rows, cols, out_cols;
  int K;                   // right-hand sides (grid.y)
  int64_t x_ld_t, x_ld_row, x_ld_b;     // element strides of x
  int64_t X_ld_w, X_ld_row, X_ld_b;     // complex-element strides of X
  int fmt;                 // CFmt of X
  int pad_single;          // round the loaded input to FP32 (pad phase in FP32)
  int tc_KC, tc_N, tc_J;   // FMT_TC: right-hand sides per chunk, rows per chunk, rows per plane
  int tc_group_log2;       // FMT_TC: log2 of the channels per contiguous run of a B row, 3 (F) or 6 (F*)
  const float* tc_inv_scale;  // FMT_TC: null for bf16 hi/lo; else FP16 hi/lo of X * tc_inv_scale[b]
  int pair_ok;             // x and its strides allow loading channels (2q, 2q+1) as one vector
  // Range scaling of the FP64-class path (null: none).  in_absmax[b] holds the
  // bits of max |x_b| as a double; the kernel divides right-hand side b by the
  // power of two 2^e_b, e_b = range_exp(in_absmax[b]), as it loads it.
  const unsigned long long* in_absmax;
  const void* twd;         // twiddle table of the length's DifPlan (FP32 complexes), or null
  const void* twdd;        // twiddle table of the length's dfd_plan (double-float complexes), or null
};

// Inverse real FFT of Hermitian half spectra followed by unpad (phases 4-5 fused).
// X[b][w][col] (w < L/2+1, format in_fmt) -> y[b][t][col] for t < Nt, scaled by 1/L.
struct InvDesc {
  FftPlan plan;
  const void* tw;
  const void* X;
  void* y;
  int Nt;
  int cols;
  int K;
  int64_t X_ld_w, X_ld_b;  // complex-element strides
  int64_t y_ld_t, y_ld_b;  // element strides
  int in_fmt;              // FMT_C128, FMT_C64 or FMT_DF
  int unpad_single;        // round the result to FP32 before the output cast
  int pair_ok;             // FMT_C64 X and its strides allow loading channels (2q, 2q+1) as one float4
  double inv_L;            // 1/L in FP64 and as an FP32 hi/lo pair
  float inv_L_hi, inv_L_lo;
  // Range scaling (null rhs_absmax: none): FMT_C128 spectra are multiplied by
  // 2^mid_exp as they load, and every output of right-hand side b by
  // 2^(range_exp(rhs_absmax[b]) + out_exp) as it is stored (in FP64, before
  // the output cast).
  const unsigned long long* rhs_absmax;
  int mid_exp, out_exp;
  const void* twd;         // twiddle table of the length's DifPlan (FP32 complexes), or null
  const void* twdd;        // twiddle table of the length's dfd_plan (double-float complexes), or null
  int out_pair_ok;         // y and its strides allow storing channels (c, c+1) as one vector
};

// Per-frequency block matvec (phase 3) for K right-hand sides.
// F-hat is [Nf][Nd][ldn] complex in the kind's storage; ldn is a multiple of 8.
//  N (F):  y[b][w][r] = sum_n F[w][r][n] x[b][w][n]         x: [K][Nf][ldn], y: [K][Nf][Nd]
//  H (F*): y[b][w][n] = sum_r conj(F[w][r][n]) x[b][w][r]   x: [K][Nf][Nd],  y: [K][Nf][ldn]
struct GemvDesc {
  const void* F;
  const void* x;
  void* y;
  int Nf, Nd, ldn, K;
  int64_t x_ld_b, y_ld_b;  // complex-element strides between right-hand sides
  unsigned int* status;    // device status word (bits: pipe.cuh kStatus*)
};

// Tensor-core multi-RHS shape: right-hand sides go in chunks of KC <= 64;
// chunk c's B rows are [Re M (KC rows) | Im M (KC rows) | zero padding] = N rows
// (N = 2 KC rounded up to 16), so a plane has J = nch * N rows.
struct TcShape {
  int KC, N, nch, J;
};
TcShape tc_shape(int K);

struct TcDesc {
  const void* A;           // bf16 planes [Nf][4][Nd][ldn] (Re hi, Re lo, Im hi, Im lo)
  const void* B;           // bf16 planes; entry (plane, row j, frequency w, contraction index k),
                           // k < ldb = the contraction length (Nm for F, Nd for F*) rounded up to 64, at
                           //   F:  (((plane J + j) ldb/8 + k/8) Nf + w) 8 + k%8      ([2][J][ldb/8][Nf][8])
                           //   F*: (((plane J + j) ldb/64 + k/64) Nf + w) 64 + k%64  ([2][J][ldb/64][Nf][64])
  void* y;                 // FMT_C64 [K][Nf][Nd] (F) or [K][Nf][ldn] (F*)
  int Nf, Nd, Nm, ldn, ldb, K;
  int adjoint;             // 0: F (contract over n), 1: F* (contract over r, A read transposed)
  int64_t y_ld_b;
  unsigned int* status;
  const float* a_scale;    // null: bf16 planes; else FP16 planes of F-hat_w / a_scale[w] ...
  const float* b_scale;    // ... and of the spectra / b_scale[b]: results times a_scale[w] b_scale[b]
};
cudaError_t launch_tc_gemm(const TcDesc& d, cudaStream_t s);
size_t tc_operand_bytes(int K, int Nf, int ldb);   // B planes
int tc_ldb(int n);                                   // n rounded up to the 64-wide K block
cudaError_t launch_convert_bf16x2(const double2* master, void* out, int Nf, int Nd, int ldn, cudaStream_t s);
// master FP64 F-hat -> FP16 planes of F-hat_w / scale[w], scale[w] a power of two per frequency
cudaError_t launch_convert_f16x2(const double2* master, void* out, float* scale, int Nf, int Nd, int ldn, cudaStream_t s);
// per right-hand side b of x (K blocks of n values, double or float): scale[b] = 2^(ceil log2(Nt max|x_b|) - 14)
// and inv[b] = 1/scale[b] (1 for an all-zero input); absmax: K words of scratch
cudaError_t launch_rhs_scales(const void* x, bool x_f32, int K, int64_t n, int Nt, unsigned int* absmax, float* scale,
                              float* inv, cudaStream_t s);
size_t tc_smem_bytes(int N);

// Fused single-launch matvec of a small operator, all phases FP64 or all FP32
// (fused_small.cu, fused_small_f32.cu): x[b][t][Cin] -> y[b][t][Cout] (FP64 or
// FP32 I/O), F-hat [Nf][Nd][ldn] in the phases' precision.
struct FusedDesc {
  const void* x;
  void* y;
  const void* F;           // F-hat: the master (double2), or its FP32 copy (float2) when f32
  const void* tw;          // twiddles exp(-2 pi i j / L), j < L, in the same type
  int Nt, L, Nd, ldn;
  int Cin, Cout, K;
  int adjoint;             // 0: F (Cin = Nm, Cout = Nd), 1: F* (Cin = Nd, Cout = Nm)
  int io_f32;
  int f32;                 // every phase in FP32 (else every phase in FP64)
  int64_t x_ld_b, y_ld_b;  // element strides between right-hand sides
  double inv_L;
};
bool fused_small_fits(int64_t L, int64_t Cin, int64_t Cout);
cudaError_t launch_fused_small(const FusedDesc& d, cudaStream_t s);
// d.f32 set, sizes checked by the caller; cl16: the device schedules 16-CTA
// clusters of the largest FP64 fused kernel (and so of every FP32 one)
cudaError_t launch_fused_small_f32(const FusedDesc& d, bool cl16, cudaStream_t s);

cudaError_t launch_rfft_fwd(const FwdDesc& d, bool in_f32, int prec, cudaStream_t s);
cudaError_t launch_irfft_inv(const InvDesc& d, int prec, bool out_f32, cudaStream_t s);
cudaError_t launch_gemv_n(int kind, const GemvDesc& d, cudaStream_t s);
cudaError_t launch_gemv_h(int kind, const GemvDesc& d, cudaStream_t s);
// master FP64 F-hat (double2, n elements) -> kind's storage (DF float4 of F-hat * 2^-fexp, or F32 float2)
cudaError_t launch_convert_fhat(int kind, const double2* master, void* out, size_t n, int fexp, cudaStream_t s);

// Range scaling of the FP64-class path.  absmax[b] (b < K) receives the bits
// of max |x| over the n values of right-hand side b (double or float input),
// as a double; the caller zeroes it first.
cudaError_t launch_absmax(const void* x, bool x_f32, int K, int64_t n, unsigned long long* absmax, cudaStream_t s);
// The scaling exponent for the bits of a non-negative double max: 0 while
// max / 2^0 lies in [2^-40, 2^41) (data that need no scaling: F-hat and inputs
// both within it keep every double-float intermediate of an Nt, Nm <= 2^20
// operator inside FP32's range, products and lo parts included, so the common
// case runs unscaled and bit for bit as without this mechanism); otherwise e
// with max / 2^e in [1, 2): -1022 for subnormals, 1023 for inf and NaN.
constexpr int kRangeFreeExp = 40;
__host__ __device__ inline int range_exp(unsigned long long bits) {
  const int biased = (int)((bits >> 52) & 0x7FF);
  if (bits == 0) return 0;
  const int e = biased == 0 ? -1022 : biased == 0x7FF ? 1023 : biased - 1023;
  return (e >= -kRangeFreeExp && e <= kRangeFreeExp) ? 0 : e;
}

int fft_max_length(int prec);
// the input / output format each GEMV kind expects / produces
int gemv_in_fmt(int kind);
int gemv_out_fmt(int kind);
size_t fmt_bytes(int fmt);

}  // namespace fftmv
