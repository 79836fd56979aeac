/*
 * fftmv.h - C ABI of the GB300 block-Toeplitz matvec library (libfftmv.so).
 *
 * Computes d = F m and m = F* d for a block lower-triangular Toeplitz matrix F
 * with Nt x Nt blocks of size Nd x Nm (Section 2.3 of Venkat et al.,
 * "Mixed-Precision Performance Portability of FFT-Based GPU-Accelerated
 * Algorithms for Block-Triangular Toeplitz Matrices", Eq. (ShiftInvariance)):
 *
 *     d_i  = sum_{j <= i} F_{i-j} m_j          (F,  i = 0..Nt-1)
 *     m*_j = sum_{i >= j} F_{i-j}^T d_i        (F*, j = 0..Nt-1)
 *
 * by the five-phase FFT algorithm of Section 2.4: zero pad in time, batched
 * real FFT, per-frequency complex block matvec against F-hat (F-hat^H for F*),
 * inverse FFT, unpad.  Every phase runs in hand-written sm_103a kernels on one
 * GPU; per-phase FP32/FP64 precision follows Section 3.2.
 *
 * Layout.  Every array is row-major, time outer and space inner (the blocks
 * of Section 2.3 laid end to end):
 *     block column  F_col[k][r][n]      k < Nt, r < Nd, n < Nm   (FP64)
 *     parameters    m[b][j][n]          b < K right-hand sides
 *     data          d[b][i][r]
 * Right-hand sides are contiguous and outermost.
 *
 * Ownership.  The operator owns F-hat in every stored form and its own
 * scratch; the caller owns F_col, m and d.  Pointers may be device pointers
 * (including managed memory) or host pointers; the library asks the CUDA
 * runtime which.  Device I/O is stream ordered and asynchronous: the caller
 * keeps the buffers alive until the stream has run the work.  Host I/O is
 * staged through device memory.  When every host buffer of a call is
 * page-locked (cudaHostAlloc / cudaHostRegister), the copies are stream
 * ordered too and the call returns at once: the result is in host memory once
 * the stream has run the work, so calls on several streams overlap one call's
 * copies with another's kernels.  With pageable host memory the call returns
 * after the result has reached host memory.
 *
 * Errors.  Every entry point returns an fftmv_status.  Nothing aborts, traps
 * or throws across the ABI.  On failure fftmv_last_error() returns a message
 * for the calling thread.  Arguments are checked before any work is queued.
 *
 * Threads and streams.  Different operators may be used from different
 * threads at once.  Calls on one operator may run on different streams at the
 * same time (each call takes its scratch from a stream-ordered pool), except
 * that fftmv_set_precision, fftmv_set_scratch_limit and fftmv_free must not
 * overlap other calls on the same operator.
 */
#ifndef FFTMV_H
#define FFTMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftmv_op fftmv_op; /* opaque operator handle */

typedef enum {
  FFTMV_OK = 0,
  FFTMV_EINVAL = -1,       /* bad argument: null pointer, size, enum value */
  FFTMV_ENOMEM = -2,       /* device or host allocation failed */
  FFTMV_EUNSUPPORTED = -3, /* valid but not supported (e.g. time length too long) */
  FFTMV_ECUDA = -4,        /* a CUDA call failed; see fftmv_last_error() */
  FFTMV_ESTATE = -5        /* operator in the wrong state (e.g. freed) */
} fftmv_status;

/* Precision of one phase (Section 3.2): each phase runs in FP32 or FP64. */
typedef enum { FFTMV_F64 = 0, FFTMV_F32 = 1 } fftmv_phase_prec;

/* How phase 3 (the per-frequency block matvec) stores F-hat and computes.
 *   NATIVE   : gemv=F64 -> F-hat FP64 (16 B/entry), FP64 FMA.
 *              gemv=F32 -> F-hat FP32 (8 B/entry), FP32 FMA.
 *   F64X2F32 : gemv=F64 only.  F-hat as FP32 hi+lo pairs (16 B/entry, about
 *              48 significant bits), double-float arithmetic on the FP32
 *              pipe.  Not native FP64: an FP64-class emulation for GPUs whose
 *              FP64 rate cannot keep pace with memory (GB300).
 *   BF16X2   : gemv=F32 only.  Many right-hand sides, F and F*, on the
 *              tensor cores (tcgen05): F-hat and the transformed inputs
 *              split into bfloat16 hi + lo parts (about 16 significant bits),
 *              hi*hi + hi*lo + lo*hi accumulated in FP32.  Pays off once K is
 *              large (tens of right-hand sides); its error is at FP32 level.
 *   F16X2    : gemv=F32 only.  As BF16X2 with FP16 hi + lo parts (about 22
 *              significant bits): F-hat scaled by a power of two per
 *              frequency, the transformed inputs by a power of two per
 *              right-hand side (from the bound |X(w)| <= Nt max|x|, found by
 *              one extra pass over the input), both scales applied in the FP32
 *              epilogue.  The same bytes and tensor work as BF16X2. */
typedef enum {
  FFTMV_GEMV_NATIVE = 0,
  FFTMV_GEMV_F64X2F32 = 1,
  FFTMV_GEMV_BF16X2 = 2,
  FFTMV_GEMV_F16X2 = 3
} fftmv_gemv_mode;

/* Per-phase precisions, in the execution order of the operation they are set
 * for (for F*: pad and FFT act on d, IFFT and unpad on the output m). */
typedef struct {
  int32_t pad;       /* fftmv_phase_prec: phase 1, zero padding (input cast)   */
  int32_t fft;       /* phase 2, forward FFT                                    */
  int32_t gemv;      /* phase 3, block matvec; also the stored F-hat precision  */
  int32_t ifft;      /* phase 4, inverse FFT                                    */
  int32_t unpad;     /* phase 5, unpadding (output cast)                        */
  int32_t gemv_mode; /* fftmv_gemv_mode                                         */
  int32_t fft_mode;  /* fftmv_gemv_mode values, for the FP64 FFT and IFFT phases:
                        NATIVE = FP64 FMA; F64X2F32 = double-float on the FP32 pipe */
} fftmv_precision;

typedef enum { FFTMV_FORWARD = 0 /* F */, FFTMV_ADJOINT = 1 /* F* */ } fftmv_which;
typedef enum { FFTMV_IO_F64 = 0, FFTMV_IO_F32 = 1 } fftmv_io_dtype;

typedef struct {
  int64_t Nt, Nd, Nm; /* block sizes */
  int64_t L;          /* FFT length: the smallest even 2^a 3^b 5^c >= 2 Nt - 1 */
  int64_t Nf;         /* frequencies kept: L / 2 + 1 */
  int64_t ldn;        /* stored row length of F-hat: Nm rounded up to 8 */
  int32_t device;     /* CUDA device the operator lives on */
  size_t fhat_bytes;  /* device bytes held by F-hat in all stored forms */
} fftmv_info;

/* Build the operator from its first block column (Section 2.4: only the first
 * block column is stored; it is zero padded to length L and Fourier
 * transformed once, always in FP64, Section 3.2).
 *   F_col  : Nt*Nd*Nm doubles, [k][r][n] row-major, host or device memory;
 *            read during the call only.
 *   Nt, Nd, Nm >= 1.  Nt is limited by the shared-memory FFT: L <= 8192
 *            (Nt <= 4096) for the FP64 and double-float FFTs, which the
 *            setup FFT always uses; EUNSUPPORTED beyond.  (The FP32 FFT
 *            itself reaches L = 16384, but an operator is only created where
 *            its FP64 setup FFT runs.)
 *   stream : cudaStream_t used for the setup work (NULL = legacy default).
 *   out    : receives the new handle.
 * Creates on the current CUDA device.  Synchronous: returns after F-hat is
 * built.  Both F and F* start in all-FP64 precision, gemv_mode and fft_mode
 * NATIVE. */
int fftmv_create_operator(const double* F_col, int64_t Nt, int64_t Nd, int64_t Nm, void* stream,
                          fftmv_op** out);

/* Checkpoint of an operator (no counterpart in the paper, which keeps only
 * output vectors): the master F-hat, [Nf][Nd][ldn] complex FP64 (re, im
 * interleaved; row length ldn = Nm rounded up to 8, padding columns zero), the
 * only state the setup FFT builds.  fftmv_get_fhat copies it to dst (host or
 * device, at least Nf*Nd*ldn*16 bytes; stream ordered, synchronous for a
 * pageable host dst).  fftmv_create_from_fhat builds an operator from such a
 * copy instead of the block column, skipping the setup FFT: fhat is host or
 * device memory read during the call (its padding columns are ignored and
 * stored as zeros), Nt, Nd, Nm as for fftmv_create_operator, and the result
 * equals the original operator's bit for bit.  Errors: EINVAL for null
 * pointers, bad sizes or a short dst; ECUDA for a failed copy. */
int fftmv_get_fhat(const fftmv_op* op, void* dst, size_t bytes, void* stream);
int fftmv_create_from_fhat(const void* fhat, int64_t Nt, int64_t Nd, int64_t Nm, void* stream, fftmv_op** out);

/* Set the per-phase precisions used by later calls for F (which=FORWARD) or
 * F* (which=ADJOINT) (Section 3.2: set at creation, changeable at runtime).
 * Builds the stored F-hat form the GEMV phase needs if it does not exist yet
 * (synchronously).  EINVAL for out-of-range values or gemv_mode F64X2F32 with
 * an FP32 GEMV phase.  fft_mode only affects phases set to FP64. */
int fftmv_set_precision(fftmv_op* op, int which, const fftmv_precision* prec);
int fftmv_get_precision(const fftmv_op* op, int which, fftmv_precision* out);

/* d = F m for K right-hand sides (Section 2.4, phases 1-5).
 *   m : K*Nt*Nm values [b][j][n]; d : K*Nt*Nd values [b][i][r].
 *   io_dtype : FFTMV_IO_F64 or FFTMV_IO_F32 for both m and d.
 *   K >= 0 (K = 0 does nothing).  m and d must not overlap.  Large K runs in
 *   chunks within the scratch bound (fftmv_set_scratch_limit). */
int fftmv_matvec(fftmv_op* op, const void* m, void* d, int64_t K, int io_dtype, void* stream);

/* m = F* d for K right-hand sides: the same phases with the conjugate
 * transpose block matvec, input and output swapped (Section 2.4).
 *   d : K*Nt*Nd values; m : K*Nt*Nm values. */
int fftmv_rmatvec(fftmv_op* op, const void* d, void* m, int64_t K, int io_dtype, void* stream);

/* Device scratch one call takes from the operator's stream-ordered pool
 * (which = FORWARD or ADJOINT), not counting host-I/O staging. */
int fftmv_workspace_bytes(const fftmv_op* op, int which, int64_t K, size_t* out);

/* Bound on the scratch one launch sequence of fftmv_matvec / fftmv_rmatvec
 * takes from the pool (spectra plus host-I/O staging).  A call whose K
 * right-hand sides need more runs them in chunks of the most that fit (whole
 * 64-RHS chunks on the tensor cores), back to back on the stream; results do
 * not depend on the chunking beyond rounding order.  bytes = 0 restores the
 * default, 8 GiB.  A single right-hand side always runs, whatever the bound.
 * Errors: EINVAL / ESTATE for a bad handle. */
int fftmv_set_scratch_limit(fftmv_op* op, size_t bytes);

/* Fused small-operator calls (Section 2.4's five phases in one launch; on by
 * default).  A call whose precision is all FP64 with native arithmetic
 * (pad, FFT, GEMV, IFFT, unpad = F64; gemv_mode = fft_mode = NATIVE) or all
 * FP32 (every phase F32, gemv_mode = NATIVE; any fft_mode), whose FFT length L
 * is 128 or 256 and whose input and output channel counts are both at most 64
 * runs as one launch per call: one thread-block cluster per right-hand side
 * (16 CTAs where the device schedules them, else 8) keeps both spectra in
 * shared memory (exchanged through distributed shared memory) and takes no
 * scratch from the pool.  Its results equal the three-kernel path's up to the
 * rounding order of the sums; with timing on, its whole duration is reported
 * as the first phase.  enable = 0 sends every call through the three-kernel
 * path.  Errors: EINVAL / ESTATE for a bad handle. */
int fftmv_set_fusion(fftmv_op* op, int enable);

/* F m (which = FFTMV_FORWARD) or F* d (FFTMV_ADJOINT) with caller-supplied
 * scratch, so a serving layer can own and account for every byte and capture
 * the call in a CUDA graph (no allocation happens inside).
 *   in, out   : device pointers (host buffers: FFTMV_EINVAL).
 *   workspace : device memory, 256-byte aligned, at least
 *               fftmv_workspace_bytes(op, which, K) bytes; used only by this
 *               call until the stream has run it.  May be null when that size
 *               is 0 (a fused call, fftmv_set_fusion).
 * Everything else as fftmv_matvec / fftmv_rmatvec. */
int fftmv_apply_ws(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io_dtype, void* workspace,
                   size_t workspace_bytes, void* stream);

int fftmv_get_info(const fftmv_op* op, fftmv_info* out);

/* Device status word of the operator.  Kernels that wait on asynchronous
 * copies bound every wait; if one runs out they set a bit here
 * (FFTMV_STATUS_WAIT_TIMEOUT), stop, and leave their outputs incomplete.
 * Reads the word after the device's pending work (synchronous); clear != 0
 * resets it. */
#define FFTMV_STATUS_WAIT_TIMEOUT 1u
int fftmv_device_status(fftmv_op* op, uint32_t* flags, int clear);

/* Self-check of that mechanism (no counterpart in the paper).  One warp
 * waits on a pipeline barrier with at most `polls` polls (1 <= polls <=
 * 2^22, the kernels' own limit).  With complete != 0 the barrier's phase is
 * completed first and the wait succeeds; with complete == 0 nothing completes
 * it, the wait runs out and FFTMV_STATUS_WAIT_TIMEOUT is raised in the
 * operator's status word, as a stalled copy pipeline would raise it.  Nothing
 * faults or hangs either way and the context stays usable.  Stream ordered;
 * EINVAL for polls out of range. */
int fftmv_check_bounded_wait(fftmv_op* op, uint32_t polls, int complete, void* stream);

/* Per-phase CUDA-event timers (the paper's per-phase timings).  While
 * enabled, every fftmv_matvec / fftmv_rmatvec call records events on its
 * stream around its three kernel groups: [0] pad+FFT, [1] block matvec,
 * [2] IFFT+unpad.  fftmv_apply_ws and fftmv_apply_noalloc calls are not
 * timed (they create no event objects).  fftmv_phase_times
 * waits for the recorded events and returns the summed milliseconds and the
 * number of calls for F or F*; reset clears them. */
int fftmv_set_timing(fftmv_op* op, int enable);
int fftmv_phase_times(fftmv_op* op, int which, double ms_out[3], int64_t* calls_out);
int fftmv_reset_timing(fftmv_op* op);

/* Size of the fixed device array behind fftmv_apply_noalloc: 64 MiB. */
#define FFTMV_NOALLOC_SCRATCH_BYTES ((size_t)64 * 1024 * 1024)

/* fftmv_apply_noalloc: F m (which = FFTMV_FORWARD) or F* d (which =
 * FFTMV_ADJOINT) like fftmv_matvec / fftmv_rmatvec, but without allocating
 * any memory.  The paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory once they are running.  Examples
 * are a process whose memory manager reserved the GPU's memory at start-up and
 * allows no further cudaMalloc, and a latency-critical loop that must not risk
 * an allocation failing, or a pool growing, in the middle of its work.
 *   in, out : device pointers only.  Host buffers would need staging memory,
 *             so they are rejected with FFTMV_EINVAL.  Layouts and dtypes as
 *             for fftmv_matvec / fftmv_rmatvec.
 *   K       : right-hand sides; the two intermediate spectra of the call must
 *             fit in FFTMV_NOALLOC_SCRATCH_BYTES (fftmv_workspace_bytes tells
 *             how much a call needs).  Larger calls are rejected with
 *             FFTMV_EUNSUPPORTED and a message giving both sizes.
 * Scratch.  The spectra live in one file-scope device array inside the
 * library.  Every GPU that loads the library holds that array until the
 * process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, and so does the
 * first call after a device reset (the address is cached per context); make
 * that first call before any stream capture: while the stream is capturing,
 * the lookup is refused with FFTMV_ESTATE.  All calls on a device share the
 * array, and it keeps the previous call's contents: the kernels overwrite
 * every scratch entry they read, or the call clears it first, so no call
 * depends on what an earlier one left.  Calls that overlap on the GPU
 * (different streams, or different operators on the same device) race on
 * the array; serialise them.
 * Timing.  These calls record no per-phase events (that would need event
 * objects): fftmv_phase_times leaves them out.
 * Errors as for fftmv_matvec.  Stream ordered and asynchronous. */
int fftmv_apply_noalloc(fftmv_op* op, int which, const void* in, void* out, int64_t K, int io_dtype,
                        void* stream);

/* Release every device resource of the operator.  NULL is a no-op.  Waits
 * for the operator's pending work. */
int fftmv_free(fftmv_op* op);

/* Message for the last failed call on this thread ("" if none). */
const char* fftmv_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int fftmv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFTMV_H */
