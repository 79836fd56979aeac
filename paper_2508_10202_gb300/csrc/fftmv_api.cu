// C ABI of the block-Toeplitz matvec library: operator object, argument
// checks, scratch from a stream-ordered pool, and the phase sequence of
// Section 2.4 (pad+FFT, block matvec, IFFT+unpad) with the per-phase
// precisions of Section 3.2.  See include/fftmv.h for the contract.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "fftmv.h"
#include "fftmv_internal.h"
#include "pipe.cuh"

using namespace fftmv;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls can proceed
  return fail(e == cudaErrorMemoryAllocation ? FFTMV_ENOMEM : FFTMV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

std::mutex g_reg_mu;
std::set<const fftmv_op*> g_live;

bool smooth235(int64_t n) {
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// smallest even 2^a 3^b 5^c >= 2 Nt - 1: no circular wrap reaches outputs t < Nt
int64_t choose_length(int64_t Nt) {
  int64_t L = 2 * Nt - 1;
  if (L < 2) L = 2;
  if (L % 2) ++L;
  while (!smooth235(L)) L += 2;
  return L;
}

FftPlan make_plan(int64_t L) {
  FftPlan p{};
  p.L = (int)L;
  int64_t n = L;
  int np = 0;
  while (n % 8 == 0) { p.rad[np++] = 8; n /= 8; }
  while (n % 4 == 0) { p.rad[np++] = 4; n /= 4; }
  while (n % 2 == 0) { p.rad[np++] = 2; n /= 2; }
  while (n % 5 == 0) { p.rad[np++] = 5; n /= 5; }
  while (n % 3 == 0) { p.rad[np++] = 3; n /= 3; }
  p.npass = np;
  int64_t ns = 1;
  for (int i = 0; i < np; ++i) {
    p.ns[i] = (int)ns;
    p.tws[i] = (int)(L / (ns * p.rad[i]));
    p.magic[i] = ns > 1 ? (unsigned)(((uint64_t)1 << 32) / (uint64_t)ns + (((uint64_t)1 << 32) % (uint64_t)ns != 0)) : 0u;
    ns *= p.rad[i];
  }
  return p;
}

// page-locked host memory (cudaHostAlloc / cudaHostRegister): copies to and
// from it are truly asynchronous
bool is_pinned_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct TimingSet {
  cudaEvent_t ev[4];
  int which;
};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

struct fftmv_op {
  int device = 0;
  int64_t Nt = 0, Nd = 0, Nm = 0, L = 0, Nf = 0, ldn = 0;
  FftPlan plan{};
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  float4* twdf = nullptr;     // twiddles as FP32 hi/lo pairs
  float2* twdif32 = nullptr;  // twiddle table of the length's DifPlan (FP32), when it has one
  float4* twdfd = nullptr;    // twiddle table of the length's dfd_plan (double-float), when it has one
  double2* fhat64 = nullptr;  // master F-hat [Nf][Nd][ldn], FP64
  float4* fhat_df = nullptr;  // FP32 hi/lo pairs
  float2* fhat32 = nullptr;   // FP32
  void* fhat_bf16 = nullptr;  // bf16 planes [Nf][Re hi, Re lo, Im hi, Im lo][Nd][ldn] (tensor cores)
  void* fhat_f16 = nullptr;   // FP16 planes of F-hat_w / fscale16[w], same layout
  float* fscale16 = nullptr;  // [Nf] powers of two
  fftmv_precision prec[2]{};
  cudaMemPool_t pool = nullptr;
  unsigned int* status = nullptr;  // device status word written by bounded waits
  std::mutex mu;  // timing state
  bool timing = false;
  std::vector<TimingSet> free_sets, pending;
  double acc_ms[2][3] = {};
  int64_t calls[2] = {};
  size_t scratch_limit = 0;  // 0: kCallScratchBudget
  int fexp = 0;              // range exponent of F-hat: max |Re, Im| / 2^fexp in [1, 2)
  bool fusion = true;        // small all-FP64 or all-FP32 calls as one fused launch (fftmv_set_fusion)
};

namespace {

int check_op(const fftmv_op* op) {
  if (!op) return fail(FFTMV_EINVAL, "null operator");
  std::lock_guard<std::mutex> g(g_reg_mu);
  if (!g_live.count(op)) return fail(FFTMV_ESTATE, "operator handle is not live (freed or never created)");
  return FFTMV_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int check_prec(const fftmv_precision* p) {
  if (!p) return fail(FFTMV_EINVAL, "null precision");
  const int32_t v[5] = {p->pad, p->fft, p->gemv, p->ifft, p->unpad};
  for (int i = 0; i < 5; ++i)
    if (v[i] != FFTMV_F64 && v[i] != FFTMV_F32) return fail(FFTMV_EINVAL, "phase %d precision %d is not F64/F32", i, v[i]);
  if (p->gemv_mode != FFTMV_GEMV_NATIVE && p->gemv_mode != FFTMV_GEMV_F64X2F32 && p->gemv_mode != FFTMV_GEMV_BF16X2 &&
      p->gemv_mode != FFTMV_GEMV_F16X2)
    return fail(FFTMV_EINVAL, "gemv_mode %d unknown", p->gemv_mode);
  if (p->gemv_mode == FFTMV_GEMV_F64X2F32 && p->gemv != FFTMV_F64)
    return fail(FFTMV_EINVAL, "gemv_mode F64X2F32 needs an FP64 GEMV phase");
  if ((p->gemv_mode == FFTMV_GEMV_BF16X2 || p->gemv_mode == FFTMV_GEMV_F16X2) && p->gemv != FFTMV_F32)
    return fail(FFTMV_EINVAL, "gemv_mode %s accumulates in FP32: it needs an FP32 GEMV phase",
                p->gemv_mode == FFTMV_GEMV_BF16X2 ? "BF16X2" : "F16X2");
  if (p->fft_mode != FFTMV_GEMV_NATIVE && p->fft_mode != FFTMV_GEMV_F64X2F32)
    return fail(FFTMV_EINVAL, "fft_mode %d unknown", p->fft_mode);
  return FFTMV_OK;
}

int gemv_kind(const fftmv_precision& p) {
  if (p.gemv_mode == FFTMV_GEMV_BF16X2 || p.gemv_mode == FFTMV_GEMV_F16X2) return GEMV_TC;
  if (p.gemv == FFTMV_F32) return GEMV_F32;
  return p.gemv_mode == FFTMV_GEMV_F64X2F32 ? GEMV_DF : GEMV_F64;
}

// arithmetic of an FFT phase from its precision letter and the FP64 mode
int fft_prec(int32_t phase, int32_t mode) {
  if (phase == FFTMV_F32) return FFT_F32;
  return mode == FFTMV_GEMV_F64X2F32 ? FFT_DF : FFT_F64;
}

const void* fhat_for(const fftmv_op* op, int kind) {
  if (kind == GEMV_TC) return op->fhat_bf16;
  return kind == GEMV_F64 ? (const void*)op->fhat64 : kind == GEMV_DF ? (const void*)op->fhat_df : (const void*)op->fhat32;
}

void release(fftmv_op* op) {
  cudaFree(op->tw64);
  cudaFree(op->tw32);
  cudaFree(op->twdf);
  cudaFree(op->twdif32);
  cudaFree(op->twdfd);
  cudaFree(op->fhat64);
  cudaFree(op->fhat_df);
  cudaFree(op->fhat32);
  cudaFree(op->fhat_bf16);
  cudaFree(op->fhat_f16);
  cudaFree(op->fscale16);
  cudaFree(op->status);
  if (op->pool) cudaMemPoolDestroy(op->pool);
  for (auto& s : op->free_sets)
    for (auto e : s.ev) cudaEventDestroy(e);
  for (auto& s : op->pending)
    for (auto e : s.ev) cudaEventDestroy(e);
  cudaGetLastError();
}

// Range scaling.  The double-float format keeps FP32's exponent range, so a
// call that runs any phase in it scales its data by exact powers of two:
// F-hat by 2^-fexp (stored so), each right-hand side by 2^-e_b from its
// largest magnitude (found by one pass over the input), and the outputs back
// by 2^(e_b + fexp) in FP64 at the unpad.  Values then stay in [1, 2) at
// their largest inside the double-float phases, whatever their magnitude in
// FP64.  The tensor-core modes and all-native configurations are not scaled.
bool range_scaled(const fftmv_precision& p) {
  const int kind = gemv_kind(p);
  if (kind == GEMV_TC) return false;
  if (kind == GEMV_DF) return true;
  return p.fft_mode == FFTMV_GEMV_F64X2F32 && (p.fft == FFTMV_F64 || p.ifft == FFTMV_F64);
}

// Scratch layout of one call: the two spectra and optional host-I/O staging.
struct CallPlan {
  int kind, in_fmt, out_fmt;
  int64_t Cin, Cout;       // input / output channels
  int64_t in_ld, out_ld;   // spectral row length of the input / output side
  size_t in_hat, out_hat;  // bytes
  bool scaled;             // range scaling: K absmax words at in_hat + absmax_off
  size_t absmax_off;
  bool fused;              // one fused launch (fused_small.cu), no spectra in scratch
};

// every phase in FP32 with the FP32 copy of F-hat (the FFT mode applies to
// FP64 transforms only, so it does not matter here)
bool all_f32(const fftmv_op* op, const fftmv_precision& p) {
  return p.pad == FFTMV_F32 && p.fft == FFTMV_F32 && p.gemv == FFTMV_F32 && p.ifft == FFTMV_F32 &&
         p.unpad == FFTMV_F32 && p.gemv_mode == FFTMV_GEMV_NATIVE && op->fhat32 != nullptr;
}

// all five phases in native FP64, or all in FP32, on an operator whose
// spectra fit one cluster
bool fused_call(const fftmv_op* op, int which) {
  const fftmv_precision& p = op->prec[which];
  const bool fwd = which == FFTMV_FORWARD;
  const bool f64 = p.pad == FFTMV_F64 && p.fft == FFTMV_F64 && p.gemv == FFTMV_F64 && p.ifft == FFTMV_F64 &&
                   p.unpad == FFTMV_F64 && p.gemv_mode == FFTMV_GEMV_NATIVE && p.fft_mode == FFTMV_GEMV_NATIVE;
  return op->fusion && (f64 || all_f32(op, p)) && fused_small_fits(op->L, fwd ? op->Nm : op->Nd, fwd ? op->Nd : op->Nm);
}

CallPlan plan_call(const fftmv_op* op, int which, int64_t K) {
  CallPlan c{};
  const fftmv_precision& p = op->prec[which];
  c.kind = gemv_kind(p);
  c.in_fmt = gemv_in_fmt(c.kind);
  c.out_fmt = gemv_out_fmt(c.kind);
  const bool fwd = which == FFTMV_FORWARD;
  c.Cin = fwd ? op->Nm : op->Nd;
  c.Cout = fwd ? op->Nd : op->Nm;
  c.in_ld = fwd ? op->ldn : op->Nd;
  c.out_ld = fwd ? op->Nd : op->ldn;
  if (c.kind == GEMV_TC) {  // B operand planes (TcDesc), 2 J ldb Nf bf16
    c.in_ld = tc_ldb((int)c.Cin);
    c.in_hat = align256(tc_operand_bytes((int)K, (int)op->Nf, (int)c.in_ld));
    if (p.gemv_mode == FFTMV_GEMV_F16X2) c.in_hat += align256((size_t)K * 12);   // per-RHS max, scale, 1/scale
  } else {
    c.in_hat = align256((size_t)K * op->Nf * c.in_ld * fmt_bytes(c.in_fmt));
  }
  c.scaled = range_scaled(p);
  if (c.scaled) {
    c.absmax_off = c.in_hat;
    c.in_hat += align256((size_t)K * sizeof(unsigned long long));
  }
  c.out_hat = align256((size_t)K * op->Nf * c.out_ld * fmt_bytes(c.out_fmt));
  c.fused = fused_call(op, which) && K <= 65535;
  if (c.fused) c.in_hat = c.out_hat = 0;
  return c;
}

// The three kernel groups of one call (Section 2.4): pad+FFT -> spectrum
// in_hat, block matvec -> out_hat, IFFT+unpad -> y.  ev, when given, holds four
// events recorded around them.
cudaError_t launch_phases(const fftmv_op* op, int which, const CallPlan& c, const void* x, void* y, void* in_hat,
                          void* out_hat, int64_t K, int io, cudaStream_t s, cudaEvent_t* ev) {
  const fftmv_precision& p = op->prec[which];
  const int fprec = fft_prec(p.fft, p.fft_mode), iprec = fft_prec(p.ifft, p.fft_mode);
  const bool fwd = which == FFTMV_FORWARD;
  if (ev) cudaEventRecord(ev[0], s);
  if (c.fused) {   // the whole call is one launch; its time is reported as the first phase
    FusedDesc u{};
    u.f32 = all_f32(op, p);
    u.x = x;
    u.y = y;
    u.F = u.f32 ? (const void*)op->fhat32 : (const void*)op->fhat64;
    u.tw = u.f32 ? (const void*)op->tw32 : (const void*)op->tw64;
    u.Nt = (int)op->Nt;
    u.L = (int)op->L;
    u.Nd = (int)op->Nd;
    u.ldn = (int)op->ldn;
    u.Cin = (int)c.Cin;
    u.Cout = (int)c.Cout;
    u.K = (int)K;
    u.adjoint = !fwd;
    u.io_f32 = io == FFTMV_IO_F32;
    u.x_ld_b = op->Nt * c.Cin;
    u.y_ld_b = op->Nt * c.Cout;
    u.inv_L = 1.0 / (double)op->L;
    const cudaError_t e = launch_fused_small(u, s);
    if (ev) {
      cudaEventRecord(ev[1], s);
      cudaEventRecord(ev[2], s);
      cudaEventRecord(ev[3], s);
    }
    return e;
  }
  FwdDesc f{};
  f.plan = op->plan;
  f.tw = fprec == FFT_F32 ? (const void*)op->tw32 : fprec == FFT_DF ? (const void*)op->twdf : (const void*)op->tw64;
  f.x = x;
  f.X = in_hat;
  f.Nt = (int)op->Nt;
  f.rows = 1;
  f.cols = (int)c.Cin;
  f.out_cols = (int)c.in_ld;
  f.K = (int)K;
  f.x_ld_t = c.Cin;
  f.x_ld_row = 0;
  f.x_ld_b = op->Nt * c.Cin;
  f.X_ld_w = c.in_ld;
  f.X_ld_row = 0;
  f.X_ld_b = op->Nf * c.in_ld;
  f.fmt = c.in_fmt;
  f.pad_single = p.pad == FFTMV_F32;
  f.twd = fprec == FFT_F32 ? op->twdif32 : nullptr;
  f.twdd = fprec == FFT_DF ? op->twdfd : nullptr;
  {
    const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
    f.pair_ok = (reinterpret_cast<uintptr_t>(x) % (2 * esz) == 0) && f.x_ld_t % 2 == 0 && f.x_ld_b % 2 == 0;
  }
  cudaError_t e = cudaSuccess;
  unsigned long long* absmax = nullptr;
  if (c.scaled) {   // per-RHS largest magnitude of the input, for the range scaling
    absmax = reinterpret_cast<unsigned long long*>(static_cast<char*>(in_hat) + c.absmax_off);
    e = cudaMemsetAsync(absmax, 0, (size_t)K * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_absmax(x, io == FFTMV_IO_F32, (int)K, op->Nt * c.Cin, absmax, s);
    f.in_absmax = absmax;
  }
  const bool f16 = c.kind == GEMV_TC && p.gemv_mode == FFTMV_GEMV_F16X2;
  float* b_scale = nullptr;
  if (c.kind == GEMV_TC) {
    const TcShape t = tc_shape((int)K);
    f.tc_KC = t.KC;
    f.tc_N = t.N;
    f.tc_J = t.J;
    f.tc_group_log2 = fwd ? 3 : 6;
    const size_t bbytes = tc_operand_bytes((int)K, (int)op->Nf, (int)c.in_ld);
    // B rows no right-hand side fills (chunk padding, a short last chunk) must read as zero
    if (2 * t.KC < t.N || (int)K % t.KC != 0) e = cudaMemsetAsync(in_hat, 0, bbytes, s);
    if (f16 && e == cudaSuccess) {   // per-RHS powers of two for the FP16 spectra
      unsigned int* absmax = reinterpret_cast<unsigned int*>(static_cast<char*>(in_hat) + align256(bbytes));
      b_scale = reinterpret_cast<float*>(absmax + K);
      float* inv = b_scale + K;
      e = launch_rhs_scales(x, io == FFTMV_IO_F32, (int)K, op->Nt * c.Cin, (int)op->Nt, absmax, b_scale, inv, s);
      f.tc_inv_scale = inv;
    }
  }
  if (e == cudaSuccess) e = launch_rfft_fwd(f, io == FFTMV_IO_F32, fprec, s);
  if (ev) cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) {
    GemvDesc g{};
    g.F = fhat_for(op, c.kind);
    g.x = in_hat;
    g.y = out_hat;
    g.Nf = (int)op->Nf;
    g.Nd = (int)op->Nd;
    g.ldn = (int)op->ldn;
    g.K = (int)K;
    g.x_ld_b = op->Nf * c.in_ld;
    g.y_ld_b = op->Nf * c.out_ld;
    g.status = op->status;
    if (c.kind == GEMV_TC) {
      TcDesc t{};
      t.A = f16 ? op->fhat_f16 : op->fhat_bf16;
      t.a_scale = f16 ? op->fscale16 : nullptr;
      t.b_scale = b_scale;
      t.B = in_hat;
      t.y = out_hat;
      t.Nf = (int)op->Nf;
      t.Nd = (int)op->Nd;
      t.Nm = (int)op->Nm;
      t.ldn = (int)op->ldn;
      t.ldb = (int)c.in_ld;
      t.K = (int)K;
      t.adjoint = !fwd;
      t.y_ld_b = op->Nf * c.out_ld;
      t.status = op->status;
      e = launch_tc_gemm(t, s);
    } else {
      e = fwd ? launch_gemv_n(c.kind, g, s) : launch_gemv_h(c.kind, g, s);
    }
  }
  if (ev) cudaEventRecord(ev[2], s);
  if (e == cudaSuccess) {
    InvDesc v{};
    v.plan = op->plan;
    v.tw = iprec == FFT_F32 ? (const void*)op->tw32 : iprec == FFT_DF ? (const void*)op->twdf : (const void*)op->tw64;
    v.X = out_hat;
    v.y = y;
    v.Nt = (int)op->Nt;
    v.cols = (int)c.Cout;
    v.K = (int)K;
    v.X_ld_w = c.out_ld;
    v.X_ld_b = op->Nf * c.out_ld;
    v.y_ld_t = c.Cout;
    v.y_ld_b = op->Nt * c.Cout;
    v.in_fmt = c.out_fmt;
    v.unpad_single = p.unpad == FFTMV_F32;
    v.pair_ok = c.out_fmt == FMT_C64 && reinterpret_cast<uintptr_t>(out_hat) % 16 == 0 && v.X_ld_w % 2 == 0 &&
                v.X_ld_b % 2 == 0;
    v.inv_L = 1.0 / (double)op->L;
    v.inv_L_hi = (float)v.inv_L;
    v.inv_L_lo = (float)(v.inv_L - (double)v.inv_L_hi);
    v.twd = iprec == FFT_F32 ? op->twdif32 : nullptr;
    v.twdd = iprec == FFT_DF ? op->twdfd : nullptr;
    {
      const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
      v.out_pair_ok = reinterpret_cast<uintptr_t>(y) % (2 * esz) == 0 && v.y_ld_t % 2 == 0 && v.y_ld_b % 2 == 0;
    }
    v.rhs_absmax = absmax;
    // FP64 spectra of the native block matvec come back to the double-float
    // range before the inverse; F-hat's exponent returns at the unpad
    v.mid_exp = c.kind == GEMV_F64 ? -op->fexp : 0;
    v.out_exp = (c.kind == GEMV_F64 || c.kind == GEMV_DF) ? op->fexp : 0;
    e = launch_irfft_inv(v, iprec, io == FFTMV_IO_F32, s);
  }
  if (ev) cudaEventRecord(ev[3], s);
  return e;
}

// Scratch of one call: the two spectra plus the staging of host I/O.
size_t call_scratch(const fftmv_op* op, int which, int64_t K, size_t esz, bool stage_in, bool stage_out) {
  const CallPlan c = plan_call(op, which, K);
  size_t b = c.in_hat + c.out_hat;
  if (stage_in) b += align256((size_t)K * op->Nt * c.Cin * esz);
  if (stage_out) b += align256((size_t)K * op->Nt * c.Cout * esz);
  return b;
}

// Right-hand sides per launch sequence: all K while the scratch stays within
// kCallScratchBudget, else the most that fit (whole 64-RHS chunks on the
// tensor cores); the chunks run back to back on the stream.
constexpr size_t kCallScratchBudget = (size_t)8 << 30;
int64_t rhs_per_chunk(const fftmv_op* op, int which, int64_t K, size_t esz, bool stage_in, bool stage_out) {
  const size_t budget = op->scratch_limit ? op->scratch_limit : kCallScratchBudget;
  if (call_scratch(op, which, K, esz, stage_in, stage_out) <= budget) return K;
  int64_t lo = 1, hi = K;   // scratch grows with K
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (call_scratch(op, which, mid, esz, stage_in, stage_out) <= budget) lo = mid;
    else hi = mid - 1;
  }
  if (gemv_kind(op->prec[which]) == GEMV_TC && lo >= 64) lo = lo / 64 * 64;
  return lo;
}

// One launch sequence over K right-hand sides (no final host synchronisation).
int run_chunk(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io, cudaStream_t s, bool in_dev,
              bool out_dev) {
  const CallPlan c = plan_call(op, which, K);
  const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
  const size_t in_bytes = (size_t)K * op->Nt * c.Cin * esz;
  const size_t out_bytes = (size_t)K * op->Nt * c.Cout * esz;
  const size_t stage_in = in_dev ? 0 : align256(in_bytes);
  const size_t stage_out = out_dev ? 0 : align256(out_bytes);
  const size_t total = c.in_hat + c.out_hat + stage_in + stage_out;

  char* ws = nullptr;   // none for a fused call on device buffers
  if (total > 0) CUDA_TRY(cudaMallocFromPoolAsync((void**)&ws, total, op->pool, s));
  char* in_hat = ws;
  char* out_hat = ws + c.in_hat;
  const void* x = in;
  void* y = out;
  if (!in_dev) {
    void* st = out_hat + c.out_hat;
    cudaError_t e = cudaMemcpyAsync(st, in, in_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      if (ws) cudaFreeAsync(ws, s);
      return cuda_fail(e, "cudaMemcpyAsync(host input)");
    }
    x = st;
  }
  if (!out_dev) y = out_hat + c.out_hat + stage_in;

  TimingSet ts{};
  bool timed = false;
  if (op->timing) {
    std::lock_guard<std::mutex> g(op->mu);
    if (!op->free_sets.empty()) {
      ts = op->free_sets.back();
      op->free_sets.pop_back();
      timed = true;
    } else {
      timed = true;
      for (auto& ev : ts.ev)
        if (cudaEventCreate(&ev) != cudaSuccess) timed = false;
      cudaGetLastError();
    }
    ts.which = which;
  }
  cudaError_t e = launch_phases(op, which, c, x, y, in_hat, out_hat, K, io, s, timed ? ts.ev : nullptr);
  if (timed) {
    std::lock_guard<std::mutex> g(op->mu);
    op->pending.push_back(ts);
  }
  if (e == cudaSuccess && !out_dev) e = cudaMemcpyAsync(out, y, out_bytes, cudaMemcpyDeviceToHost, s);
  cudaError_t ef = ws ? cudaFreeAsync(ws, s) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "matvec kernels");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return FFTMV_OK;
}

int run_matvec(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io, void* stream) {
  int rc = check_op(op);
  if (rc) return rc;
  if (K < 0) return fail(FFTMV_EINVAL, "K = %lld < 0", (long long)K);
  if (io != FFTMV_IO_F64 && io != FFTMV_IO_F32) return fail(FFTMV_EINVAL, "io_dtype %d unknown", io);
  if (K == 0) return FFTMV_OK;
  if (!in || !out) return fail(FFTMV_EINVAL, "null input or output");
  if (K > 65535) return fail(FFTMV_EUNSUPPORTED, "K = %lld exceeds 65535 right-hand sides per call", (long long)K);
  DeviceGuard dg(op->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fwd = which == FFTMV_FORWARD;
  const int64_t Cin = fwd ? op->Nm : op->Nd, Cout = fwd ? op->Nd : op->Nm;
  const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
  const size_t in_rhs = (size_t)op->Nt * Cin * esz, out_rhs = (size_t)op->Nt * Cout * esz;
  {
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + K * out_rhs && b < a + K * in_rhs) return fail(FFTMV_EINVAL, "input and output overlap");
  }
  const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
  const int64_t kc = rhs_per_chunk(op, which, K, esz, !in_dev, !out_dev);
  for (int64_t k0 = 0; k0 < K; k0 += kc) {
    const int64_t k = K - k0 < kc ? K - k0 : kc;
    rc = run_chunk(op, which, static_cast<const char*>(in) + k0 * in_rhs, static_cast<char*>(out) + k0 * out_rhs, k,
                   io, s, in_dev, out_dev);
    if (rc) return rc;
  }
  // pageable host buffers: return once the result is in host memory; page-locked
  // ones stay stream ordered like device I/O
  if ((!in_dev && !is_pinned_host(in)) || (!out_dev && !is_pinned_host(out))) CUDA_TRY(cudaStreamSynchronize(s));
  return FFTMV_OK;
}

}  // namespace

extern "C" {

int fftmv_version(void) { return 100; }

const char* fftmv_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {
// The operator from its block column (F_col) or from a saved master F-hat
// (fhat, [Nf][Nd][ldn] FP64 complex); exactly one of the two is given.
int create_impl(const double* F_col, const void* fhat, int64_t Nt, int64_t Nd, int64_t Nm, void* stream,
                fftmv_op** out) {
  if (!out) return fail(FFTMV_EINVAL, "null output handle");
  *out = nullptr;
  if (!F_col && !fhat) return fail(FFTMV_EINVAL, "null block column");
  if (Nt < 1 || Nd < 1 || Nm < 1) return fail(FFTMV_EINVAL, "sizes must be >= 1 (Nt=%lld Nd=%lld Nm=%lld)",
                                              (long long)Nt, (long long)Nd, (long long)Nm);
  const int64_t L = choose_length(Nt);
  if (L > fft_max_length(FFT_F64))
    return fail(FFTMV_EUNSUPPORTED, "FFT length %lld for Nt=%lld exceeds the shared-memory FFT limit %d",
                (long long)L, (long long)Nt, fft_max_length(FFT_F64));
  const int64_t ldn = (Nm + 7) / 8 * 8;
  const int64_t Nf = L / 2 + 1;
  if (Nd * ldn > INT32_MAX || ldn > INT32_MAX / 2 || Nf * Nd > INT32_MAX)
    return fail(FFTMV_EUNSUPPORTED, "Nd * Nm too large");

  fftmv_op* op = new (std::nothrow) fftmv_op();
  if (!op) return fail(FFTMV_ENOMEM, "host allocation failed");
  op->Nt = Nt;
  op->Nd = Nd;
  op->Nm = Nm;
  op->L = L;
  op->Nf = Nf;
  op->ldn = ldn;
  op->plan = make_plan(L);
  for (auto& p : op->prec)
    p = fftmv_precision{FFTMV_F64, FFTMV_F64, FFTMV_F64, FFTMV_F64, FFTMV_F64, FFTMV_GEMV_NATIVE, FFTMV_GEMV_NATIVE};
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  auto bail = [&](int code) {
    release(op);
    delete op;
    return code;
  };
  auto cu = [&](cudaError_t e, const char* what) { return e == cudaSuccess ? 0 : bail(cuda_fail(e, what)); };
  int rc;
  if ((rc = cu(cudaGetDevice(&op->device), "cudaGetDevice"))) return rc;

  // twiddles exp(-2 pi i j / L), evaluated in long double and rounded once
  std::vector<double2> tw((size_t)L);
  std::vector<float2> tw32((size_t)L);
  std::vector<float4> twdf((size_t)L);
  for (int64_t j = 0; j < L; ++j) {
    const long double a = -2.0L * 3.141592653589793238462643383279502884L * (long double)j / (long double)L;
    const long double c = cosl(a), sn = sinl(a);
    tw[j] = make_double2((double)c, (double)sn);
    tw32[j] = make_float2((float)c, (float)sn);
    const float ch = (float)c, sh = (float)sn;
    twdf[j] = make_float4(ch, sh, (float)(c - (long double)ch), (float)(sn - (long double)sh));
  }
  if ((rc = cu(cudaMalloc(&op->tw64, L * sizeof(double2)), "cudaMalloc(twiddles)"))) return rc;
  if ((rc = cu(cudaMalloc(&op->tw32, L * sizeof(float2)), "cudaMalloc(twiddles)"))) return rc;
  if ((rc = cu(cudaMemcpy(op->tw64, tw.data(), L * sizeof(double2), cudaMemcpyHostToDevice), "twiddle copy"))) return rc;
  if ((rc = cu(cudaMemcpy(op->tw32, tw32.data(), L * sizeof(float2), cudaMemcpyHostToDevice), "twiddle copy"))) return rc;
  if ((rc = cu(cudaMalloc(&op->twdf, L * sizeof(float4)), "cudaMalloc(twiddles)"))) return rc;
  if ((rc = cu(cudaMemcpy(op->twdf, twdf.data(), L * sizeof(float4), cudaMemcpyHostToDevice), "twiddle copy"))) return rc;
  if (dif_plan((int)L).n > 0) {
    // rows of W_{M_s}^{j q} = exp(-2 pi i (L / M_s) j q / L) per pass with S_s > 1
    const DifPlan pl = dif_plan((int)L);
    std::vector<float2> twd((size_t)dif_tw_size((int)L), make_float2(1.f, 0.f));
    for (int sp = 0; sp < pl.n; ++sp) {
      const int M = dif_M((int)L, sp), S = dif_S((int)L, sp), R = pl.rad[sp];
      if (S == 1) continue;
      for (int j = 0; j < S; ++j)
        for (int q = 1; q < R; ++q) {
          const long double a = -2.0L * 3.141592653589793238462643383279502884L * (long double)(j * q) / (long double)M;
          twd[(size_t)dif_tw_offset((int)L, sp) + (size_t)j * dif_tw_row(R) + (q - 1)] =
              make_float2((float)cosl(a), (float)sinl(a));
        }
    }
    if ((rc = cu(cudaMalloc(&op->twdif32, twd.size() * sizeof(float2)), "cudaMalloc(twiddles)"))) return rc;
    if ((rc = cu(cudaMemcpy(op->twdif32, twd.data(), twd.size() * sizeof(float2), cudaMemcpyHostToDevice),
                 "twiddle copy")))
      return rc;
  }

  if (dfd_plan((int)L).n > 0) {
    // the same rows for the double-float plan, each entry hi/lo pairs of the
    // long double value
    const DifPlan pl = dfd_plan((int)L);
    std::vector<float4> twd((size_t)dfd_tw_size((int)L));
    for (int sp = 0; sp < pl.n; ++sp) {
      const int M = dfd_M((int)L, sp), S = dfd_S((int)L, sp), R = pl.rad[sp];
      if (S == 1) continue;
      for (int j = 0; j < S; ++j)
        for (int q = 1; q < R; ++q) {
          const long double a = -2.0L * 3.141592653589793238462643383279502884L * (long double)(j * q) / (long double)M;
          const long double c = cosl(a), sn = sinl(a);
          const float ch = (float)c, sh = (float)sn;
          twd[(size_t)dfd_tw_offset((int)L, sp) + (size_t)j * (R - 1) + (q - 1)] =
              make_float4(ch, sh, (float)(c - (long double)ch), (float)(sn - (long double)sh));
        }
    }
    if ((rc = cu(cudaMalloc(&op->twdfd, twd.size() * sizeof(float4)), "cudaMalloc(twiddles)"))) return rc;
    if ((rc = cu(cudaMemcpy(op->twdfd, twd.data(), twd.size() * sizeof(float4), cudaMemcpyHostToDevice),
                 "twiddle copy")))
      return rc;
  }

  if ((rc = cu(cudaMalloc(&op->status, sizeof(unsigned int)), "cudaMalloc(status)"))) return rc;
  if ((rc = cu(cudaMemset(op->status, 0, sizeof(unsigned int)), "cudaMemset(status)"))) return rc;

  const size_t fh_elems = (size_t)Nf * Nd * ldn;
  if ((rc = cu(cudaMalloc(&op->fhat64, fh_elems * sizeof(double2)), "cudaMalloc(F-hat)"))) return rc;

  FwdDesc f{};
  f.plan = op->plan;
  f.tw = op->tw64;
  f.Nt = (int)Nt;
  f.cols = (int)Nm;
  f.out_cols = (int)ldn;
  f.K = 1;
  f.x_ld_row = Nm;
  f.x_ld_b = 0;
  f.X_ld_w = Nd * ldn;
  f.X_ld_row = ldn;
  f.X_ld_b = 0;
  f.fmt = FMT_C128;
  f.pad_single = 0;
  if (fhat) {
    // a saved spectrum: copied as it is, its padding columns n >= Nm zeroed
    cudaError_t e = cudaMemcpyAsync(op->fhat64, fhat, fh_elems * sizeof(double2), cudaMemcpyDefault, s);
    if (e == cudaSuccess && ldn > Nm)
      e = cudaMemset2DAsync(op->fhat64 + Nm, ldn * sizeof(double2), 0, (ldn - Nm) * sizeof(double2), Nf * Nd, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if ((rc = cu(e, "F-hat copy"))) return rc;
  } else if (is_device_ptr(F_col)) {
    f.x = F_col;
    f.X = op->fhat64;
    f.rows = (int)Nd;
    f.x_ld_t = Nd * Nm;
    if ((rc = cu(launch_rfft_fwd(f, false, FFT_F64, s), "setup FFT"))) return rc;
  } else {
    // stage row blocks of the host block column through a bounded device buffer
    const size_t row_bytes = (size_t)Nt * Nm * sizeof(double);
    int64_t rc_rows = (int64_t)((size_t(1) << 30) / row_bytes);
    if (rc_rows < 1) rc_rows = 1;
    if (rc_rows > Nd) rc_rows = Nd;
    double* stage = nullptr;
    if ((rc = cu(cudaMalloc(&stage, rc_rows * row_bytes), "cudaMalloc(setup staging)"))) return rc;
    for (int64_t r0 = 0; r0 < Nd; r0 += rc_rows) {
      const int64_t nr = Nd - r0 < rc_rows ? Nd - r0 : rc_rows;
      cudaError_t e = cudaMemcpy2DAsync(stage, nr * Nm * sizeof(double), F_col + r0 * Nm, Nd * Nm * sizeof(double),
                                        nr * Nm * sizeof(double), Nt, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        f.x = stage;
        f.X = op->fhat64 + r0 * ldn;
        f.rows = (int)nr;
        f.x_ld_t = nr * Nm;
        e = launch_rfft_fwd(f, false, FFT_F64, s);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        cudaFree(stage);
        return bail(cuda_fail(e, "setup FFT (host block column)"));
      }
    }
    cudaFree(stage);
  }
  {  // range exponent of F-hat (largest |Re|, |Im| over all entries)
    unsigned long long* mx = nullptr;
    if ((rc = cu(cudaMalloc(&mx, sizeof *mx), "cudaMalloc(setup max)"))) return rc;
    unsigned long long bits = 0;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof *mx, s);
    if (e == cudaSuccess) e = launch_absmax(op->fhat64, false, 1, (int64_t)(Nf * Nd * ldn * 2), mx, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, mx, sizeof bits, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mx);
    if ((rc = cu(e, "setup range exponent"))) return rc;
    op->fexp = range_exp(bits);
  }

  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = op->device;
  if ((rc = cu(cudaMemPoolCreate(&op->pool, &props), "cudaMemPoolCreate"))) return rc;
  uint64_t keep = UINT64_MAX;
  if ((rc = cu(cudaMemPoolSetAttribute(op->pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool attribute"))) return rc;

  {
    std::lock_guard<std::mutex> g(g_reg_mu);
    g_live.insert(op);
  }
  *out = op;
  return FFTMV_OK;
}
}  // namespace

extern "C" {

int fftmv_create_operator(const double* F_col, int64_t Nt, int64_t Nd, int64_t Nm, void* stream, fftmv_op** out) {
  if (!F_col) {
    if (out) *out = nullptr;
    return fail(FFTMV_EINVAL, "null block column");
  }
  return create_impl(F_col, nullptr, Nt, Nd, Nm, stream, out);
}

int fftmv_create_from_fhat(const void* fhat, int64_t Nt, int64_t Nd, int64_t Nm, void* stream, fftmv_op** out) {
  if (!fhat) {
    if (out) *out = nullptr;
    return fail(FFTMV_EINVAL, "null F-hat");
  }
  return create_impl(nullptr, fhat, Nt, Nd, Nm, stream, out);
}

int fftmv_get_fhat(const fftmv_op* op, void* dst, size_t bytes, void* stream) {
  int rc = check_op(op);
  if (rc) return rc;
  if (!dst) return fail(FFTMV_EINVAL, "null destination");
  const size_t need = (size_t)op->Nf * op->Nd * op->ldn * sizeof(double2);
  if (bytes < need) return fail(FFTMV_EINVAL, "destination of %zu bytes; F-hat takes %zu", bytes, need);
  DeviceGuard dg(op->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemcpyAsync(dst, op->fhat64, need, cudaMemcpyDefault, s));
  if (!is_device_ptr(dst) && !is_pinned_host(dst)) CUDA_TRY(cudaStreamSynchronize(s));
  return FFTMV_OK;
}

int fftmv_set_precision(fftmv_op* op, int which, const fftmv_precision* prec) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if ((rc = check_prec(prec))) return rc;
  DeviceGuard dg(op->device);
  const int kind = gemv_kind(*prec);
  const size_t n = (size_t)op->Nf * op->Nd * op->ldn;
  if (kind == GEMV_DF && !op->fhat_df) {
    CUDA_TRY(cudaMalloc(&op->fhat_df, n * sizeof(float4)));
    CUDA_TRY(launch_convert_fhat(kind, op->fhat64, op->fhat_df, n, op->fexp, 0));
    CUDA_TRY(cudaStreamSynchronize(0));
  } else if (kind == GEMV_F32 && !op->fhat32) {
    CUDA_TRY(cudaMalloc(&op->fhat32, n * sizeof(float2)));
    CUDA_TRY(launch_convert_fhat(kind, op->fhat64, op->fhat32, n, 0, 0));
    CUDA_TRY(cudaStreamSynchronize(0));
  } else if (kind == GEMV_TC && prec->gemv_mode == FFTMV_GEMV_BF16X2 && !op->fhat_bf16) {
    CUDA_TRY(cudaMalloc(&op->fhat_bf16, n * 4 * 2));
    CUDA_TRY(launch_convert_bf16x2(op->fhat64, op->fhat_bf16, (int)op->Nf, (int)op->Nd, (int)op->ldn, 0));
    CUDA_TRY(cudaStreamSynchronize(0));
  } else if (kind == GEMV_TC && prec->gemv_mode == FFTMV_GEMV_F16X2 && !op->fhat_f16) {
    CUDA_TRY(cudaMalloc(&op->fhat_f16, n * 4 * 2));
    CUDA_TRY(cudaMalloc(&op->fscale16, op->Nf * sizeof(float)));
    CUDA_TRY(launch_convert_f16x2(op->fhat64, op->fhat_f16, op->fscale16, (int)op->Nf, (int)op->Nd, (int)op->ldn, 0));
    CUDA_TRY(cudaStreamSynchronize(0));
  }
  op->prec[which] = *prec;
  return FFTMV_OK;
}

int fftmv_get_precision(const fftmv_op* op, int which, fftmv_precision* out) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if (!out) return fail(FFTMV_EINVAL, "null output");
  *out = op->prec[which];
  return FFTMV_OK;
}

int fftmv_matvec(fftmv_op* op, const void* m, void* d, int64_t K, int io_dtype, void* stream) {
  return run_matvec(op, FFTMV_FORWARD, m, d, K, io_dtype, stream);
}

int fftmv_rmatvec(fftmv_op* op, const void* d, void* m, int64_t K, int io_dtype, void* stream) {
  return run_matvec(op, FFTMV_ADJOINT, d, m, K, io_dtype, stream);
}

int fftmv_workspace_bytes(const fftmv_op* op, int which, int64_t K, size_t* out) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if (K < 0 || !out) return fail(FFTMV_EINVAL, "bad K or null output");
  DeviceGuard dg(op->device);   // whether a call is fused depends on the operator's device
  const CallPlan c = plan_call(op, which, K);
  *out = c.in_hat + c.out_hat;
  return FFTMV_OK;
}

int fftmv_set_fusion(fftmv_op* op, int enable) {
  if (int rc = check_op(op)) return rc;
  op->fusion = enable != 0;
  return FFTMV_OK;
}

int fftmv_set_scratch_limit(fftmv_op* op, size_t bytes) {
  int rc = check_op(op);
  if (rc) return rc;
  op->scratch_limit = bytes;
  return FFTMV_OK;
}

int fftmv_apply_ws(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io, void* workspace,
                   size_t workspace_bytes, void* stream) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if (K < 0) return fail(FFTMV_EINVAL, "K = %lld < 0", (long long)K);
  if (io != FFTMV_IO_F64 && io != FFTMV_IO_F32) return fail(FFTMV_EINVAL, "io_dtype %d unknown", io);
  if (K == 0) return FFTMV_OK;
  if (!in || !out) return fail(FFTMV_EINVAL, "null input or output");
  if (K > 65535) return fail(FFTMV_EUNSUPPORTED, "K = %lld exceeds 65535 right-hand sides per call", (long long)K);
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(FFTMV_EINVAL, "workspace is not 256-byte aligned");
  DeviceGuard dg(op->device);
  const CallPlan c = plan_call(op, which, K);
  if (!workspace && c.in_hat + c.out_hat > 0) return fail(FFTMV_EINVAL, "null workspace");
  if (workspace_bytes < c.in_hat + c.out_hat)
    return fail(FFTMV_EINVAL, "workspace of %zu bytes; this call needs %zu", workspace_bytes, c.in_hat + c.out_hat);
  const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
  const size_t in_bytes = (size_t)K * op->Nt * c.Cin * esz;
  const size_t out_bytes = (size_t)K * op->Nt * c.Cout * esz;
  {
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + out_bytes && b < a + in_bytes) return fail(FFTMV_EINVAL, "input and output overlap");
  }
  if (!is_device_ptr(in) || !is_device_ptr(out)) return fail(FFTMV_EINVAL, "fftmv_apply_ws takes device pointers only");
  char* ws = static_cast<char*>(workspace);
  cudaError_t e = launch_phases(op, which, c, in, out, ws, ws + c.in_hat, K, io, static_cast<cudaStream_t>(stream), nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "matvec kernels");
  return FFTMV_OK;
}

int fftmv_get_info(const fftmv_op* op, fftmv_info* out) {
  int rc = check_op(op);
  if (rc) return rc;
  if (!out) return fail(FFTMV_EINVAL, "null output");
  out->Nt = op->Nt;
  out->Nd = op->Nd;
  out->Nm = op->Nm;
  out->L = op->L;
  out->Nf = op->Nf;
  out->ldn = op->ldn;
  out->device = op->device;
  const size_t n = (size_t)op->Nf * op->Nd * op->ldn;
  out->fhat_bytes = n * sizeof(double2) + (op->fhat_df ? n * sizeof(float4) : 0) + (op->fhat32 ? n * sizeof(float2) : 0) +
                    (op->fhat_bf16 ? n * 8 : 0) + (op->fhat_f16 ? n * 8 : 0);
  return FFTMV_OK;
}

int fftmv_device_status(fftmv_op* op, uint32_t* flags, int clear) {
  int rc = check_op(op);
  if (rc) return rc;
  if (!flags) return fail(FFTMV_EINVAL, "null output");
  DeviceGuard dg(op->device);
  unsigned int v = 0;
  CUDA_TRY(cudaMemcpy(&v, op->status, sizeof v, cudaMemcpyDeviceToHost));
  if (clear) CUDA_TRY(cudaMemset(op->status, 0, sizeof v));
  *flags = v;
  return FFTMV_OK;
}

}  // extern "C"

namespace {

// One warp waits on a pipeline barrier that expects one arrival, polling at
// most `polls` times, the way the copy pipelines wait for their data.  With
// `complete` that arrival happens first and the wait succeeds; otherwise
// nothing completes the phase and the wait runs out.
__global__ void bounded_wait_check_kernel(unsigned int* status, uint32_t polls, int complete) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (complete && threadIdx.x == 0) mbar_arrive(&bar);
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, polls);
  if (!ok && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

}  // namespace

extern "C" {

int fftmv_check_bounded_wait(fftmv_op* op, uint32_t polls, int complete, void* stream) {
  int rc = check_op(op);
  if (rc) return rc;
  if (polls < 1 || polls > kSpinLimit) return fail(FFTMV_EINVAL, "polls = %u outside [1, %u]", polls, kSpinLimit);
  DeviceGuard dg(op->device);
  bounded_wait_check_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(op->status, polls, complete != 0);
  CUDA_TRY(cudaGetLastError());
  return FFTMV_OK;
}

int fftmv_set_timing(fftmv_op* op, int enable) {
  int rc = check_op(op);
  if (rc) return rc;
  op->timing = enable != 0;
  return FFTMV_OK;
}

int fftmv_phase_times(fftmv_op* op, int which, double ms_out[3], int64_t* calls_out) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if (!ms_out) return fail(FFTMV_EINVAL, "null output");
  DeviceGuard dg(op->device);
  std::lock_guard<std::mutex> g(op->mu);
  for (auto& ts : op->pending) {
    CUDA_TRY(cudaEventSynchronize(ts.ev[3]));
    for (int i = 0; i < 3; ++i) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, ts.ev[i], ts.ev[i + 1]));
      op->acc_ms[ts.which][i] += ms;
    }
    op->calls[ts.which] += 1;
    op->free_sets.push_back(ts);
  }
  op->pending.clear();
  for (int i = 0; i < 3; ++i) ms_out[i] = op->acc_ms[which][i];
  if (calls_out) *calls_out = op->calls[which];
  return FFTMV_OK;
}

int fftmv_reset_timing(fftmv_op* op) {
  double tmp[3];
  int rc = fftmv_phase_times(op, FFTMV_FORWARD, tmp, nullptr);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(op->mu);
  memset(op->acc_ms, 0, sizeof op->acc_ms);
  op->calls[0] = op->calls[1] = 0;
  return FFTMV_OK;
}

int fftmv_free(fftmv_op* op) {
  if (!op) return FFTMV_OK;
  {
    std::lock_guard<std::mutex> g(g_reg_mu);
    if (!g_live.erase(op)) return fail(FFTMV_ESTATE, "operator handle is not live (double free?)");
  }
  DeviceGuard dg(op->device);
  cudaDeviceSynchronize();
  release(op);
  delete op;
  return FFTMV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of the matvec (include/fftmv.h: fftmv_apply_noalloc).
// The paper has no counterpart.  The two intermediate spectra live in this
// file-scope device array instead of the operator's pool.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char fftmv_noalloc_scratch[FFTMV_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoallocSlot {
  void* ctx = nullptr;   // the context the address belongs to
  char* addr = nullptr;
};
NoallocSlot g_noalloc[kNoallocMaxDevices];

// The current context (driver API, reached through the runtime's entry-point
// query so that the library links against the runtime only).
using CtxGetCurrentFn = int (*)(void**);
void* current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so the address
// is looked up per device and cached together with the context it belongs
// to: after a device reset the primary context, and with it the array's
// address, is new, and the lookup runs again.  The lookup may load the
// library's module, which must not happen inside a stream capture, so it is
// refused while `s` is capturing.
int noalloc_address(int device, cudaStream_t s, char** out) {
  if (device < 0 || device >= kNoallocMaxDevices)
    return fail(FFTMV_EUNSUPPORTED, "device %d beyond the %d devices the no-alloc path tracks", device,
                kNoallocMaxDevices);
  void* ctx = current_context();
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  NoallocSlot& slot = g_noalloc[device];
  if (!slot.addr || !ctx || slot.ctx != ctx) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone)
      return fail(FFTMV_ESTATE,
                  "fftmv_apply_noalloc: the first call on a device (or after a device reset) looks up the scratch "
                  "array's address; make it once before capturing the stream");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, fftmv_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fftmv_noalloc_scratch)");
    slot.addr = static_cast<char*>(p);
    slot.ctx = ctx;
  }
  *out = slot.addr;
  return FFTMV_OK;
}

}  // namespace

extern "C" int fftmv_apply_noalloc(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io,
                                   void* stream) {
  int rc = check_op(op);
  if (rc) return rc;
  if (which != FFTMV_FORWARD && which != FFTMV_ADJOINT) return fail(FFTMV_EINVAL, "which=%d is not F/F*", which);
  if (K < 0) return fail(FFTMV_EINVAL, "K = %lld < 0", (long long)K);
  if (io != FFTMV_IO_F64 && io != FFTMV_IO_F32) return fail(FFTMV_EINVAL, "io_dtype %d unknown", io);
  if (K == 0) return FFTMV_OK;
  if (!in || !out) return fail(FFTMV_EINVAL, "null input or output");
  if (K > 65535) return fail(FFTMV_EUNSUPPORTED, "K = %lld exceeds 65535 right-hand sides per call", (long long)K);
  DeviceGuard dg(op->device);
  const CallPlan c = plan_call(op, which, K);
  const size_t need = c.in_hat + c.out_hat;
  if (need > FFTMV_NOALLOC_SCRATCH_BYTES)
    return fail(FFTMV_EUNSUPPORTED, "this call needs %zu bytes of scratch; the no-alloc array holds %zu", need,
                (size_t)FFTMV_NOALLOC_SCRATCH_BYTES);
  const size_t esz = io == FFTMV_IO_F32 ? 4 : 8;
  const size_t in_bytes = (size_t)K * op->Nt * c.Cin * esz;
  const size_t out_bytes = (size_t)K * op->Nt * c.Cout * esz;
  {
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + out_bytes && b < a + in_bytes) return fail(FFTMV_EINVAL, "input and output overlap");
  }
  if (!is_device_ptr(in) || !is_device_ptr(out))
    return fail(FFTMV_EINVAL, "fftmv_apply_noalloc takes device pointers only (host I/O would need staging memory)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = nullptr;
  if ((rc = noalloc_address(op->device, s, &ws))) return rc;
  char* in_hat = ws;
  char* out_hat = ws + c.in_hat;
  cudaError_t e = launch_phases(op, which, c, in, out, in_hat, out_hat, K, io, s, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc matvec kernels");
  return FFTMV_OK;
}
