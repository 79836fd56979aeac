// Multi-right-hand-side block matvec on the 5th-generation tensor cores
// (tcgen05), both directions: for every frequency w
//     F:  D-hat_w (Nd x K) = F-hat_w (Nd x Nm) * M-hat_w (Nm x K)
//     F*: M-hat_w (Nm x K) = F-hat_w^H (Nm x Nd) * D-hat_w (Nd x K)   (complex)
// the per-frequency product of Section 2.4 phase 3 applied to K right-hand
// sides at once, which turns the batched GEMV into a dense contraction.
//
// Precision: F-hat and the spectra are each split into bfloat16 hi + lo parts
// (x = hi + lo + O(2^-18 |x|)); the three products hi*hi + hi*lo + lo*hi
// accumulate in FP32 in tensor memory (the lo*lo term is below 2^-16 of the
// result).  The FP16 mode splits the same way into FP16 (11-bit) parts after
// exact power-of-two scaling: F-hat_w by s_w (per frequency), the spectra of
// right-hand side b by s_b; both operands of one MMA are then FP16, and the
// epilogue multiplies each output by s_w * s_b.  The FFT hands over its
// spectra doubled (the real-to-complex split's 1/2 is left out there), so the
// epilogue also halves every output.
//
// Complex arithmetic without duplicating data: A is four planes
// (Re hi, Re lo, Im hi, Im lo) of F-hat_w, B is [Re X | Im X] (2*KC columns,
// hi and lo planes).  Two accumulators: acc1 = Re(F) * B, acc2 = Im(F) * B;
// then Re D = acc1[:, q] - acc2[:, KC + q] and Im D = acc1[:, KC + q] + acc2[:, q]
// (the acc2 signs flip for conj(F)).  F* reads the same A planes transposed
// through an MN-major descriptor.
//
// Tiles: one frequency, one chunk of KC <= 64 right-hand sides and 128 output
// rows; MMA tile M = 128 (rows past the end are zero-filled by TMA, never read
// from HBM), N = 2*KC rounded up to 16, K-step 64 16-bit values.  A is read in
// 128-byte swizzled rows (K-major for F, MN-major for F*).  B comes as the FFT
// wrote it: for F in 8-channel runs adjacent over frequency (16-byte rows,
// loaded without swizzle and described as K-major core matrices), for F* in
// 64-value rows under the 128-byte swizzle.  Persistent CTAs, one per SM, loop
// over the tiles.
// Warp roles: warp 0 issues TMA loads, warp 1 owns tensor memory and issues
// the MMAs, warps 2-9 drain the accumulators (tcgen05.ld) and write the output.
//
// Accumulation in groups: the tensor core's internal FP32 accumulation loses
// accuracy over long contractions (10^4 terms here), so the MMAs accumulate
// TC_GROUP k-blocks at a time into one of two TMEM accumulator sets; the
// epilogue warps add each finished set into FP32 registers while the MMAs fill
// the other set, and hand the set back through a "drained" mbarrier.
// Every wait is bounded (pipe.cuh); a timeout sets the status word.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fftmv_internal.h"
#include "pipe.cuh"

namespace fftmv {
namespace {

constexpr int TC_M = 128;
constexpr int TC_BK = 64;                  // bf16 per 128-byte swizzle row
constexpr int TC_STAGES = 2;
constexpr int TC_GROUP = 8;                // k-blocks accumulated in TMEM before a drain
constexpr int TC_EPI_WARPS = 8;            // two per TMEM lane quadrant
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr uint32_t TC_TMEM_COLS = 512;     // two accumulator sets of [acc1 | acc2], 128 columns each

// --- tcgen05 / TMA primitives (inline PTX) ---------------------------------

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc_sw128(const void* smem) {
  const uint64_t addr = smem_u32(smem);
  uint64_t d = (addr & 0x3FFFFull) >> 4;    // start address
  d |= (uint64_t)(16 >> 4) << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                   // descriptor version (sm_100)
  d |= (uint64_t)2 << 61;                   // layout: 128-byte swizzle
  return d;
}

// shared-memory matrix descriptor: K-major, no swizzle.  8-row x 16-byte core
// matrices (128 contiguous bytes each): the next core matrix along K is 128 B
// on (leading byte offset), the next 8-row group 1024 B on (stride byte offset).
__device__ __forceinline__ uint64_t umma_desc_kmajor_plain(const void* smem) {
  const uint64_t addr = smem_u32(smem);
  uint64_t d = (addr & 0x3FFFFull) >> 4;
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;                   // descriptor version (sm_100); layout 0: no swizzle
  return d;
}

// shared-memory matrix descriptor: MN-major, 128-byte swizzle.  A 128 x 64
// tile is two 64-wide MN halves 8 KB apart (leading byte offset), each 64 K
// rows of 128 bytes; K groups of 8 rows are 1024 B apart (stride byte offset).
__device__ __forceinline__ uint64_t umma_desc_mn_sw128(const void* smem) {
  const uint64_t addr = smem_u32(smem);
  uint64_t d = (addr & 0x3FFFFull) >> 4;
  d |= (uint64_t)(8192 >> 4) << 16;         // leading byte offset: next 64-wide MN half
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row K group
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor, kind::f16: A and B both BF16 (format 1) or both FP16
// (format 0), K-major; FP32 D; M = 128, N = n
__host__ __device__ constexpr uint32_t umma_idesc(int n, bool f16) {
  return (1u << 4)                          // D format: F32
         | ((f16 ? 0u : 1u) << 7)           // A format
         | ((f16 ? 0u : 1u) << 10)          // B format
         | ((uint32_t)(n >> 3) << 17)       // N / 8
         | ((uint32_t)(TC_M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  int Nf, M, K, KC, N, nkb;  // M: output rows (Nd for F, Nm for F*)
  const float* a_scale;      // FP16 operands: per-frequency and per-RHS scales (null: bf16)
  const float* b_scale;
  int J;                     // B rows per plane
  int nch, nmt;              // right-hand-side chunks and 128-row M tiles per frequency
  int64_t y_ld_b, y_ld_w;    // complex elements between right-hand sides / frequencies of y
  float2* y;                 // [K][Nf][rows] (FMT_C64)
  unsigned int* status;
};

// Persistent: each CTA loops over tiles (M tile, chunk, frequency), M tile
// fastest, so the CTAs working at one time share a frequency's B operand in
// L2.  Global k-block and group counters carry the pipeline phases across
// tiles: the producer runs ahead into the next tile while the epilogue drains
// the previous one from the other TMEM accumulator set.
// H = false: F, A = F-hat_w (rows r, K along n, K-major).
// H = true:  F*, A = F-hat_w^T (rows n, K along r, MN-major: the same planes read
//            transposed); the conjugate enters through the epilogue signs.
template <bool H>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tile area (the 128-byte swizzle pattern repeats every 1024 bytes)
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const int N = a.N;
  const uint32_t a_plane = TC_M * 128;               // bytes of one 128 x 64 bf16 tile
  const uint32_t b_plane = (uint32_t)N * 128;
  const uint32_t stage_bytes = 4 * a_plane + 2 * b_plane;
  unsigned char* tiles = base;
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + TC_STAGES * stage_bytes);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* ready = empty + TC_STAGES;     // [2]: accumulator set holds a finished group
  uint64_t* drained = ready + 2;           // [2]: epilogue has read the set
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 2);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ntiles = a.Nf * a.nch * a.nmt;
  const int gpt = (a.nkb + TC_GROUP - 1) / TC_GROUP;   // accumulation groups per tile
  auto decode = [&](int tile, int& w, int& ch, int& m0) {
    const int mt = tile % a.nmt, rest = tile / a.nmt;
    ch = rest % a.nch;
    w = rest / a.nch;
    m0 = mt * TC_M;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ready[s], 1);
      mbar_init(&drained[s], TC_EPI_WARPS);
    }
    mbar_init_fence();
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 1) tmem_alloc(tmem_slot, TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t it = 0;  // k-blocks issued by this CTA
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int w, ch, m0;
        decode(tile, w, ch, m0);
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const uint32_t s = it % TC_STAGES;
          if (it >= TC_STAGES && !mbar_wait(&empty[s], ((it / TC_STAGES) & 1) ^ 1)) {
            ok = false;
            break;
          }
          unsigned char* st = tiles + s * stage_bytes;
          mbar_arrive_expect_tx(&full[s], stage_bytes);
          for (int p = 0; p < 4; ++p) {
            if constexpr (H) {  // two 64 (n) x 64 (r) boxes per plane
              tma_load_4d(st + p * a_plane, &mapA, m0, kb * TC_BK, p, w, &full[s]);
              tma_load_4d(st + p * a_plane + a_plane / 2, &mapA, m0 + 64, kb * TC_BK, p, w, &full[s]);
            } else {
              tma_load_4d(st + p * a_plane, &mapA, kb * TC_BK, m0, p, w, &full[s]);
            }
          }
          for (int p = 0; p < 2; ++p) {
            if constexpr (H)   // [2][J][ldb/64][Nf][64]: N rows of 64 indices, 128-byte swizzle
              tma_load_5d(st + 4 * a_plane + p * b_plane, &mapB, 0, w, kb, ch * N, p, &full[s]);
            else               // [2][J][ldb/8][Nf][8]: 8 x 8 x 8 x N/8 core-matrix box
              tma_load_5d(st + 4 * a_plane + p * b_plane, &mapB, 0, 0, kb * (TC_BK / 8), (p * a.J + ch * N) / 8, w,
                          &full[s]);
          }
        }
      }
      // no copy may still be in flight when the CTA exits
      for (uint32_t kk = it > TC_STAGES ? it - TC_STAGES : 0; kk < it; ++kk)
        if (!mbar_wait(&full[kk % TC_STAGES], (kk / TC_STAGES) & 1)) ok = false;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = umma_idesc(N, a.a_scale != nullptr) | (H ? (1u << 15) : 0u);   // bit 15: A is MN-major
      uint32_t it = 0, G = 0;   // k-blocks consumed, groups started
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const bool first = kb % TC_GROUP == 0;
          const uint32_t set = G & 1;
          // the set was last used by group G-2: wait until the epilogue has read it
          if (first && G >= 2 && !mbar_wait(&drained[set], ((G >> 1) - 1) & 1)) {
            ok = false;
            break;
          }
          const uint32_t s = it % TC_STAGES;
          if (!mbar_wait(&full[s], (it / TC_STAGES) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc1 = tmem + 256 * set, acc2 = acc1 + 128;
          unsigned char* st = tiles + s * stage_bytes;
#pragma unroll
          for (int ks = 0; ks < TC_BK / 16; ++ks) {
            // A: K-major advances 32 B per 16 K inside the swizzled row; MN-major
            // advances two 8-row K groups (2048 B).  B: K-major.
            const uint64_t ak = H ? (uint64_t)(2048 >> 4) * ks : 2 * ks;
            const uint64_t frh = (H ? umma_desc_mn_sw128(st + 0 * a_plane) : umma_desc_sw128(st + 0 * a_plane)) + ak;
            const uint64_t frl = (H ? umma_desc_mn_sw128(st + 1 * a_plane) : umma_desc_sw128(st + 1 * a_plane)) + ak;
            const uint64_t fih = (H ? umma_desc_mn_sw128(st + 2 * a_plane) : umma_desc_sw128(st + 2 * a_plane)) + ak;
            const uint64_t fil = (H ? umma_desc_mn_sw128(st + 3 * a_plane) : umma_desc_sw128(st + 3 * a_plane)) + ak;
            // B: F* 32 B per 16 K inside the swizzled row; F two core matrices (256 B)
            const uint64_t bk = H ? 2 * ks : (uint64_t)(256 >> 4) * ks;
            const uint64_t bh = (H ? umma_desc_sw128(st + 4 * a_plane) : umma_desc_kmajor_plain(st + 4 * a_plane)) + bk;
            const uint64_t bl =
                (H ? umma_desc_sw128(st + 4 * a_plane + b_plane) : umma_desc_kmajor_plain(st + 4 * a_plane + b_plane)) + bk;
            const uint32_t acc = !(first && ks == 0);
            umma_bf16(acc1, frh, bh, idesc, acc);
            umma_bf16(acc1, frh, bl, idesc, 1);
            umma_bf16(acc1, frl, bh, idesc, 1);
            umma_bf16(acc2, fih, bh, idesc, acc);
            umma_bf16(acc2, fih, bl, idesc, 1);
            umma_bf16(acc2, fil, bh, idesc, 1);
          }
          umma_commit(&empty[s]);                                 // stage reusable
          if (kb % TC_GROUP == TC_GROUP - 1 || kb == a.nkb - 1) {  // group done
            umma_commit(&ready[set]);
            ++G;
          }
        }
      }
    }
  } else {  // epilogue: warps 2..9; TMEM lane quadrant warp % 4, half of the RHS columns each
    const int ew = warp - 2;
    const uint32_t lane_addr = (uint32_t)(32 * (warp % 4)) << 16;
    const int KC = a.KC, hw = (KC + 1) / 2;
    const int qlo = (ew / 4) * hw, qn = min(hw, KC - qlo);   // this warp's RHS columns [qlo, qlo + qn)
    uint32_t G = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      int w, ch, m0;
      decode(tile, w, ch, m0);
      const int row = m0 + 32 * (warp % 4) + lane;
      float sre[32], sim[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) sre[i] = sim[i] = 0.f;
      for (int g = 0; g < gpt; ++g, ++G) {
        const uint32_t set = G & 1;
        const bool got = mbar_wait(&ready[set], (G >> 1) & 1);
        if (!__all_sync(0xffffffffu, got)) {  // tcgen05.ld is warp-collective
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t t1 = tmem + lane_addr + 256 * set, t2 = t1 + 128;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c * 16 < qn) {
            float a1r[16], a1i[16], a2r[16], a2i[16];
            const int q0 = qlo + c * 16;
            tmem_ld16(t1 + q0, a1r);        // Re F * Re X
            tmem_ld16(t1 + KC + q0, a1i);   // Re F * Im X
            tmem_ld16(t2 + q0, a2r);        // Im F * Re X
            tmem_ld16(t2 + KC + q0, a2i);   // Im F * Im X
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if constexpr (H) {  // conj(F) X: Re = ReF ReX + ImF ImX, Im = ReF ImX - ImF ReX
                sre[c * 16 + i] += a1r[i] + a2i[i];
                sim[c * 16 + i] += a1i[i] - a2r[i];
              } else {
                sre[c * 16 + i] += a1r[i] - a2i[i];
                sim[c * 16 + i] += a1i[i] + a2r[i];
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&drained[set]);
      }
      if (ok && row < a.M) {
        const float sw = a.a_scale ? a.a_scale[w] : 1.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int q = qlo + c * 16 + i;
            const int b = ch * KC + q;
            if (c * 16 + i < qn && b < a.K) {
              // the FFT writes 2 X (the split's 1/2 lands here); powers of two: exact
              const float sc = a.a_scale ? 0.5f * sw * a.b_scale[b] : 0.5f;
              a.y[b * a.y_ld_b + (int64_t)w * a.y_ld_w + row] = make_float2(sre[c * 16 + i] * sc, sim[c * 16 + i] * sc);
            }
          }
        }
      }
    }
  }
  if (!ok) atomicOr(a.status, kStatusWaitTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

// master FP64 F-hat [Nf][Nd][ldn] -> four bf16 planes [Nf][4][Nd][ldn]: Re hi, Re lo, Im hi, Im lo
__global__ void convert_bf16x2_kernel(const double2* __restrict__ in, __nv_bfloat16* __restrict__ out, int Nd, int ldn,
                                      int64_t n) {
  const int64_t plane = (int64_t)Nd * ldn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    const int64_t w = i / plane, rem = i - w * plane;
    __nv_bfloat16* o = out + w * 4 * plane + rem;
    const __nv_bfloat16 rh = __double2bfloat16(v.x), ih = __double2bfloat16(v.y);
    o[0] = rh;
    o[plane] = __double2bfloat16(v.x - (double)__bfloat162float(rh));
    o[2 * plane] = ih;
    o[3 * plane] = __double2bfloat16(v.y - (double)__bfloat162float(ih));
  }
}

// power of two s with max / s in (2^13, 2^14]: FP16 keeps 4x headroom below its
// largest finite value, and lo parts stay normal for entries down to 2^-17 max
__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  const double m = frexp(mx, &e);       // mx = m 2^e, m in [0.5, 1)
  return ldexp(1.0, (m == 0.5 ? e - 1 : e) - 14);
}

// per frequency: scale[w] from max |Re|, |Im| of F-hat_w (one CTA per frequency)
__global__ void __launch_bounds__(1024) fhat_scale_kernel(const double2* __restrict__ in, float* __restrict__ scale,
                                                          int64_t plane) {
  __shared__ double red[32];
  const double2* p = in + blockIdx.x * plane;
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < plane; i += blockDim.x) {
    const double2 v = p[i];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) scale[blockIdx.x] = (float)pow2_scale(mx);
  }
}

// master FP64 F-hat -> four FP16 planes [Nf][4][Nd][ldn] of F-hat_w / scale[w]
__global__ void convert_f16x2_kernel(const double2* __restrict__ in, const float* __restrict__ scale,
                                     __half* __restrict__ out, int Nd, int ldn, int64_t n) {
  const int64_t plane = (int64_t)Nd * ldn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = i / plane, rem = i - w * plane;
    const double inv = 1.0 / (double)scale[w];
    const double2 v = in[i];
    const double re = v.x * inv, im = v.y * inv;
    __half* o = out + w * 4 * plane + rem;
    const __half rh = __double2half(re), ih = __double2half(im);
    o[0] = rh;
    o[plane] = __double2half(re - (double)__half2float(rh));
    o[2 * plane] = ih;
    o[3 * plane] = __double2half(im - (double)__half2float(ih));
  }
}

// per right-hand side: max |x| over its n values (float bits order like the
// values); a block reduction, then one atomic per CTA
template <typename T>
__global__ void __launch_bounds__(512) rhs_absmax_kernel(const T* __restrict__ x, int64_t n,
                                                         unsigned int* __restrict__ absmax) {
  __shared__ float red[16];
  const T* p = x + (int64_t)blockIdx.y * n;
  float m0 = 0.f, m1 = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {   // two loads in flight
    m0 = fmaxf(m0, fabsf((float)__ldcs(p + i)));
    m1 = fmaxf(m1, fabsf((float)__ldcs(p + i + stride)));
  }
  if (i < n) m0 = fmaxf(m0, fabsf((float)__ldcs(p + i)));
  float mx = fmaxf(m0, m1);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) atomicMax(absmax + blockIdx.y, __float_as_uint(mx));
  }
}

// scale[b] = power of two bounding Nt max|x_b| as above (|X(w)| <= sum_t |x_t| <= Nt max|x|)
__global__ void rhs_scale_kernel(const unsigned int* __restrict__ absmax, int K, int Nt, float* __restrict__ scale,
                                 float* __restrict__ inv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= K) return;
  // the float max may round down by half an ulp: 2^-23 of headroom more than covers it
  const double sc = pow2_scale((double)__uint_as_float(absmax[b]) * (double)Nt * (1.0 + 0x1p-20));
  scale[b] = (float)sc;
  inv[b] = (float)(1.0 / sc);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4-D bf16 map {inner, rows, planes, freqs} with a box of 64 x box_rows x 1 x 1, 128-byte swizzle
cudaError_t make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint64_t planes,
                     uint64_t freqs, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {inner, rows, planes, freqs};
  const cuuint64_t strides[3] = {inner * 2, inner * rows * 2, inner * rows * planes * 2};
  const cuuint32_t box[4] = {(cuuint32_t)TC_BK, box_rows, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// B operand maps.  F (large B, written by the costly FFT over Nm channels):
// planes [2][J][ldb/8][Nf][8] folded into 2J rows; dims {8 channels, 8 rows,
// ldb/8 channel groups, 2J/8 row groups, Nf}, box {8, 8, 8, N/8, 1}, no
// swizzle: the box lands as the K-major core-matrix layout (8 rows x 16 bytes
// per core matrix, K-neighbours 128 B apart, 8-row groups 1024 B apart) that
// umma_desc_kmajor_plain reads, and the FFT writes 16-byte runs that are
// adjacent over frequencies.  F* (small B, re-read by every M tile): planes
// [2][J][ldb/64][Nf][64]; dims {64, Nf, ldb/64, J, 2}, box {64, 1, 1, N, 1},
// 128-byte swizzle: N rows of 64 indices, one 128-byte request per row.
cudaError_t make_map_b(CUtensorMap* map, const void* base, uint64_t ldb, uint64_t J, uint64_t Nf, uint32_t box_rows,
                       bool adjoint) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUresult r;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (adjoint) {
    const cuuint64_t dims[5] = {64, Nf, ldb / 64, J, 2};
    const cuuint64_t strides[4] = {128, Nf * 128, ldb * Nf * 2, J * ldb * Nf * 2};
    const cuuint32_t box[5] = {TC_BK, 1, 1, box_rows, 1};
    r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const uint64_t row = (ldb / 8) * Nf * 16;   // bytes per B row
    const cuuint64_t dims[5] = {8, 8, ldb / 8, 2 * J / 8, Nf};
    const cuuint64_t strides[4] = {row, Nf * 16, 8 * row, 16};
    const cuuint32_t box[5] = {8, 8, TC_BK / 8, box_rows / 8, 1};
    r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

TcShape tc_shape(int K) {
  TcShape t{};
  t.KC = K < 64 ? K : 64;
  t.N = ((2 * t.KC + 15) / 16) * 16;
  t.nch = (K + t.KC - 1) / t.KC;
  t.J = t.nch * t.N;
  return t;
}

size_t tc_smem_bytes(int N) {
  const size_t stage = 4 * (size_t)TC_M * 128 + 2 * (size_t)N * 128;
  return 1024 + TC_STAGES * stage + (2 * TC_STAGES + 4) * sizeof(uint64_t) + 16;
}

cudaError_t launch_convert_f16x2(const double2* master, void* out, float* scale, int Nf, int Nd, int ldn,
                                 cudaStream_t s) {
  const int64_t plane = (int64_t)Nd * ldn, n = (int64_t)Nf * plane;
  if (n == 0) return cudaSuccess;
  fhat_scale_kernel<<<Nf, 1024, 0, s>>>(master, scale, plane);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 32 ? want : 152 * 32);
  convert_f16x2_kernel<<<blocks, threads, 0, s>>>(master, scale, static_cast<__half*>(out), Nd, ldn, n);
  return cudaGetLastError();
}

cudaError_t launch_rhs_scales(const void* x, bool x_f32, int K, int64_t n, int Nt, unsigned int* absmax, float* scale,
                              float* inv, cudaStream_t s) {
  if (K == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(absmax, 0, (size_t)K * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  // about four CTAs of 512 threads per SM over all right-hand sides, at least 32 values a thread
  int64_t bx = (4 * 152 + K - 1) / K;
  const int64_t most = (n + 512 * 32 - 1) / (512 * 32);
  bx = bx > most ? most : bx;
  bx = bx < 1 ? 1 : bx;
  dim3 grid((unsigned)bx, K);
  if (x_f32) rhs_absmax_kernel<float><<<grid, 512, 0, s>>>(static_cast<const float*>(x), n, absmax);
  else rhs_absmax_kernel<double><<<grid, 512, 0, s>>>(static_cast<const double*>(x), n, absmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  rhs_scale_kernel<<<(K + 127) / 128, 128, 0, s>>>(absmax, K, Nt, scale, inv);
  return cudaGetLastError();
}

cudaError_t launch_convert_bf16x2(const double2* master, void* out, int Nf, int Nd, int ldn, cudaStream_t s) {
  const int64_t n = (int64_t)Nf * Nd * ldn;
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 32 ? want : 152 * 32);
  convert_bf16x2_kernel<<<blocks, threads, 0, s>>>(master, static_cast<__nv_bfloat16*>(out), Nd, ldn, n);
  return cudaGetLastError();
}

size_t tc_operand_bytes(int K, int Nf, int ldb) { return (size_t)Nf * 2 * tc_shape(K).J * ldb * 2; }
int tc_ldb(int n) { return (n + TC_BK - 1) / TC_BK * TC_BK; }
cudaError_t launch_tc_gemm(const TcDesc& d, cudaStream_t s) {
  if (d.Nf == 0 || d.K == 0) return cudaSuccess;
  const TcShape t = tc_shape(d.K);
  const bool H = d.adjoint != 0;
  if (d.ldb % TC_BK != 0) return cudaErrorInvalidValue;
  CUtensorMap mapA, mapB;
  cudaError_t e = make_map(&mapA, d.A, (uint64_t)d.ldn, (uint64_t)d.Nd, 4, (uint64_t)d.Nf, H ? 64 : TC_M);
  if (e != cudaSuccess) return e;
  e = make_map_b(&mapB, d.B, (uint64_t)d.ldb, (uint64_t)t.J, (uint64_t)d.Nf, (uint32_t)t.N, H);
  if (e != cudaSuccess) return e;
  TcArgs a{};
  a.Nf = d.Nf;
  a.M = H ? d.Nm : d.Nd;
  a.K = d.K;
  a.KC = t.KC;
  a.N = t.N;
  a.nkb = d.ldb / TC_BK;
  a.nch = t.nch;
  a.J = t.J;
  a.nmt = (a.M + TC_M - 1) / TC_M;
  a.y_ld_b = d.y_ld_b;
  a.y_ld_w = H ? d.ldn : d.Nd;
  a.y = static_cast<float2*>(d.y);
  a.status = d.status;
  a.a_scale = d.a_scale;
  a.b_scale = d.b_scale;
  const size_t smem = tc_smem_bytes(t.N);
  auto kernel = H ? tc_gemm_kernel<true> : tc_gemm_kernel<false>;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)d.Nf * t.nch * a.nmt;
  const int grid = (int)(ntiles < sms ? ntiles : sms);   // one persistent CTA per SM
  kernel<<<grid, TC_THREADS, smem, s>>>(mapA, mapB, a);
  return cudaGetLastError();
}

}  // namespace fftmv
