// Sine transform along x of lines of n = 255 or n = 127 points (and along y of 3D grids with
// my = 127) as tensor-core products (tcgen05, sm_103a).
//
// The x-direction step of the shifted spatial solves (Algorithm 1 / 2, step 2: A is diagonal on
// the sine modes, Sec. 2.2) transforms every line of the half spectrum,
//   Y_k = -2i sum_{x=1}^{n} X_x sin(pi k x / (n + 1)),   k = 1..n,
// the same output as the odd-sequence FFT (k_axis, op 0). Here it is a dense contraction against
// the sine matrix, as MMAs with M = 128 outputs and K = 128 inputs:
//   * n = 255 (k_dst255_tc): the matrix is folded once. With e_x = X_x - X_{256-x} and
//     o_x = X_x + X_{256-x},
//       Y_{2k'}   = -2i sum_{x=1}^{127} e_x sin(pi k' x / 128)            (k' = 1..127)
//       Y_{2k'+1} = -2i sum_{x=1}^{128} o_x sin(pi (2k'+1) x / 256)       (o_128 = X_128, k' = 0..127)
//     (sin(pi k (256 - x) / 256) = -/+ sin(pi k x / 256) for even / odd k). Each half is a 128 x 128
//     matrix times the lines' real and imaginary parts: D = S B^T with N = 64 real rows (32
//     complex lines per tile).
//   * n = 127 (k_dst127_tc): the 127 x 127 matrix itself, padded with a zero row and column, is one
//     128 x 128 operand; no fold. N = 128 real rows (64 complex lines per tile).
//   * n = 127, strided lines (k_dst127s_tc): the y-direction transforms of 3D grids (my = 127),
//     whose lines are the columns of the (j, z) planes of my rows x mx points; a tile is up to 64
//     consecutive columns of one plane, read and written row by row (contiguous along x).
//   * n = 127, strided lines, solve (k_dst127z_tc): the z-direction solve of 3D grids (mz = 127:
//     DST-z, divide by the shifted eigenvalues, DST-z back, AxisArgs op 1) as two passes per tile,
//     the divided spectrum held in shared memory between them.
//
// Precision: FP16 operands split in two (v = hi + lo: hi of 11 significant bits by Veltkamp's
// splitting, lo = v - hi), three products per term (hi hi + hi lo + lo hi, FP32 accumulation in
// tensor memory): ~22 significant bits per operand, the accuracy of the FP32 FFT it replaces. Every
// line is scaled by a power of two (its largest |re|, |im| brought to [2^13, 2^14)) so that the
// FP16 range holds it; the matrices are scaled by 16 (their low parts stay normal numbers). Both
// scalings are exact and undone in the epilogue.
//
// Roles (one CTA per SM, persistent over tiles of lines; the resident matrices take a large part
// of its shared memory):
//   * load warp: one thread copies each tile's lines (contiguous, ~65 KB) into a raw buffer with
//     bulk asynchronous copies (cp.async.bulk, complete_tx on a shared-memory barrier), as soon as
//     the staging threads have taken the previous tile out of it (strided lines: idle);
//   * 8 staging warps: read their share of the raw tile into registers (then release the buffer;
//     strided lines: straight from global memory, coalesced along the rows),
//     reduce each line's largest magnitude, (fold,) scale and split the lines into K-chunks of 32
//     inputs in the canonical K-major layout (8-row x 16-byte core matrices, no swizzle) in a ring
//     of two stage slots, and signal each chunk on the slot's "full" barrier; after staging a tile
//     they run the previous tile's epilogue, so that a tile's MMAs overlap it;
//   * MMA warp: one thread copies the matrix operands (hi / lo, of both halves for n = 255; a
//     precomputed image of their shared-memory layout) once by bulk copies, then for each chunk
//     waits "full", issues the chunk's MMAs (M 128, N 64 or 128, K 16; three per term) and commits
//     them to the slot's "empty" barrier; after a tile's last chunk it commits the tile to its
//     accumulator buffer's barrier.
// Accumulators are double-buffered in tensor memory (2 x 128 columns: D_even and D_odd of 64
// columns each, or one D of 128); the epilogue reads them with tcgen05.ld (one output per lane:
// TMEM lane = output index), releases the buffer, unscales, applies -2i and writes the lines in
// place (every read of a tile precedes its writes).
//
// Every wait is bounded: a barrier that does not complete within ~2^31 clock cycles sets a shared
// abort flag (all roles then stop at their next wait or tile) and *err; before the CTA exits, the
// MMA thread waits (bounded) for every MMA it issued and the load thread for its last copy, and
// tensor memory is freed.
#include <cuda_fp16.h>

#include <atomic>
#include <cmath>
#include <cstdint>

#include "pint_internal.h"

namespace pint {
namespace {

// Tile geometry per line length P (compile time).
template <int P> struct TcShape {
  static_assert(P == 255 || P == 127, "line length");
  static constexpr bool kFold = P == 255;                 // folded into even / odd halves
  static constexpr int kHalves = kFold ? 2 : 1;           // D regions (and matrix operands / 2)
  static constexpr int kLines = kFold ? 32 : 64;          // complex lines per tile
  static constexpr int kN = 2 * kLines;                   // MMA N: real rows (re, then im)
  static constexpr int kChunk = 32;                       // K inputs per stage buffer
  static constexpr int kChunks = 128 / kChunk;            // stage buffers (one tile)
  static constexpr int kStageThreads = 256;               // staging / epilogue warps
  static constexpr int kItems = kLines * 16 / kStageThreads;  // items (line, pair of K inputs) per thread
  static constexpr int kVals = kFold ? 4 : 2;             // complex inputs per item and chunk
  static constexpr int kLinesPerWarp = kLines * 128 / kStageThreads;  // epilogue lines per warp
  static constexpr int kThreads = kStageThreads + 64;     // + the MMA warp and the load warp
  static constexpr int kMatBytes = 128 * 128 * 2;         // one 128 x 128 FP16 operand
  static constexpr int kABytes = 2 * kHalves * kMatBytes; // hi, lo (of each half)
  static constexpr int kOpBytes = kN * kChunk * 2;        // one B operand of one stage
  static constexpr int kStageBytes = 2 * kHalves * kOpBytes;
  static constexpr int kSlots = 2;                        // stage slots (ring of K-chunks)
  static constexpr int kLineBytes = P * 8;                // one line of complex FP32 values
  static constexpr int kRawOff = kABytes + kSlots * kStageBytes;  // the tile's lines as read
  // strided lines (P = 127): the raw buffer, unused for its lines, holds the tile's outputs on
  // their way to global memory, P rows of up to kLines columns (pitch kOutPitch float2). (The
  // smaller the shared memory, the larger the L1 that the strided kernel's global loads go through.)
  static constexpr int kOutPitch = kLines + 1;
  static constexpr int kRawBytes = kFold ? 65536 : ((P * kOutPitch * 8 + 15) / 16) * 16;
  static constexpr int kOutOff = kRawOff;
  static constexpr int kMiscOff = kRawOff + kRawBytes;
  static constexpr int kMiscBytes = kFold ? 2048 : 1664;
  static constexpr int kSmemBytes = kMiscOff + kMiscBytes;
  static constexpr int kTmemCols = 256;                   // two accumulator buffers of 128 columns
  // instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A and B FP16 (formats 0), both
  // K-major, N >> 3 at bit 17, M >> 4 at bit 24
  static constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  static_assert(kItems * kStageThreads == kLines * 16, "items");
  static_assert(kStageBytes == 16384, "stage");
  static_assert(kLines * kLineBytes <= kRawBytes, "raw tile");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};

constexpr long long kTcWaitCycles = 1ll << 31;

template <int P> struct TcMisc {
  unsigned long long bar_a;                     // matrix image copied
  unsigned long long full[2];                   // stage slot written (the staging threads arrive)
  unsigned long long empty[2];                  // stage slot's MMAs done (tcgen05.commit)
  unsigned long long raw_full;                  // the tile's lines copied (bulk copies complete)
  unsigned long long raw_empty;                 // the tile's lines read out (the staging threads arrive)
  unsigned long long acc_full[2];               // accumulator buffer complete (tcgen05.commit)
  unsigned long long acc_empty[2];              // accumulator buffer read out (256 threads arrive)
  unsigned long long fin;                       // every MMA done (tcgen05.commit, at exit)
  float pmax[4][TcShape<P>::kLines];            // per line and group of inputs: largest |re|, |im|
  float unscale[2][TcShape<P>::kLines];         // per accumulator buffer and line: 2 / (16 * 2^s)
  uint32_t tmem;                                // tensor-memory base address
  uint32_t abort;                               // a wait gave up: every role stops
};
static_assert(sizeof(TcMisc<255>) <= TcShape<255>::kMiscBytes && sizeof(TcMisc<127>) <= TcShape<127>::kMiscBytes,
              "barrier block");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start >> 4, leading (K-direction) core-matrix stride >> 4,
// stride (M/N-direction) core-matrix stride >> 4, descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <uint32_t IDESC>
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of the given parity to complete, for at most kTcWaitCycles; gives up at
// once when *abort (a shared flag, if given) is set
__device__ bool bar_wait(uint32_t bar, uint32_t parity, const uint32_t* abort) {
  const long long t0 = clock64();
  while (!bar_try(bar, parity)) {
    if (abort && *reinterpret_cast<const volatile uint32_t*>(abort)) return false;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of (row, k) in a K-major operand of `rows` rows: core matrices of 8 rows x 8 FP16,
// rows of a core matrix 16 bytes apart, core matrices along rows 128 bytes apart (SBO), along K
// rows / 8 * 128 bytes apart (LBO)
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k, int rows) {
  return (uint32_t)((k >> 3) * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// two FP16 values packed in 32 bits (a in the low half), rounded to nearest
__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// v = hi + lo with hi of 11 significant bits (Veltkamp's splitting with the factor 2^13 + 1; the
// products and sums are rounded separately, never fused), lo = v - hi exactly; both then as FP16
// (hi exactly for |v| >= 2^-14, lo rounded: ~2^-24 |v|). Returns the hi pair, *lo the lo pair.
__device__ __forceinline__ uint32_t split2(float a, float b, uint32_t* lo) {
  const float ca = __fmul_rn(a, 8193.f), cb = __fmul_rn(b, 8193.f);
  const float ha = __fsub_rn(ca, __fsub_rn(ca, a)), hb = __fsub_rn(cb, __fsub_rn(cb, b));
  *lo = pack_f16x2(__fsub_rn(a, ha), __fsub_rn(b, hb));
  return pack_f16x2(ha, hb);
}

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// the whole kernel for lines of P points (launched by k_dst255_tc / k_dst127_tc / k_dst127s_tc).
// STRIDED (P = 127): the lines are the columns of planes of P rows (a.stride points per row); a
// tile is up to 64 consecutive columns of one plane, which the staging warps read straight from
// global memory (each row's columns are contiguous) instead of through the load warp's raw buffer.
// SOLVE (strided, P = 127): per tile, the transform (pass A), the divide of AxisArgs op 1 in the
// epilogue, and the transform back (pass B, +2i) from the divided spectrum in shared memory.
template <int P, int MODE> __device__ __forceinline__ void dst_tc_body(const DstTcArgs& a) {
  using S = TcShape<P>;
  constexpr bool STRIDED = MODE >= 1, SOLVE = MODE == 2;
  static_assert(!STRIDED || P == 127, "strided lines: 127 points");
  constexpr int kLines = S::kLines, kN = S::kN, kChunk = S::kChunk, kChunks = S::kChunks;
  constexpr int kStageThreads = S::kStageThreads, kItems = S::kItems, kVals = S::kVals;
  constexpr int kLinesPerWarp = S::kLinesPerWarp, kMatBytes = S::kMatBytes, kABytes = S::kABytes;
  constexpr int kOpBytes = S::kOpBytes, kStageBytes = S::kStageBytes, kHalves = S::kHalves;
  extern __shared__ __align__(1024) unsigned char smem[];
  TcMisc<P>& ms = *reinterpret_cast<TcMisc<P>*>(smem + S::kMiscOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sA = smem_u32(smem), sB = sA + kABytes;
  // strided: tiles per plane and the tile count (lines = planes * stride)
  const int tpp = STRIDED ? (a.stride + kLines - 1) / kLines : 1;
  const int tiles = STRIDED ? (a.lines / a.stride) * tpp : (a.lines + kLines - 1) / kLines;
  const uint32_t* abort = reinterpret_cast<const uint32_t*>(&ms.abort);
  // tile tt: its first element, the element steps between lines (ls) and between points (ps) of a
  // line, and its number of lines
  struct TileGeo { float2* base; size_t ls, ps; int nl; };
  auto geo = [&](int tt) -> TileGeo {
    TileGeo g;
    if constexpr (STRIDED) {
      const int q = tt / tpp, x0 = (tt - q * tpp) * kLines;
      g.base = a.S + (size_t)q * P * a.stride + x0;
      g.ls = 1;
      g.ps = (size_t)a.stride;
      g.nl = a.stride - x0 < kLines ? a.stride - x0 : kLines;
    } else {
      const long long first = (long long)tt * kLines;
      g.base = a.S + first * P;
      g.ls = P;
      g.ps = 1;
      g.nl = (int)(a.lines - first < kLines ? a.lines - first : kLines);
    }
    return g;
  };

  if (tid == 0) {
    auto init = [](unsigned long long* b, int count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
    };
    init(&ms.bar_a, 1);
    for (int c = 0; c < S::kSlots; ++c) {
      init(&ms.full[c], kStageThreads);
      init(&ms.empty[c], 1);
    }
    init(&ms.raw_full, 1);
    init(&ms.raw_empty, kStageThreads);
    for (int b2 = 0; b2 < 2; ++b2) {
      init(&ms.acc_full[b2], 1);
      init(&ms.acc_empty[b2], kStageThreads);
    }
    init(&ms.fin, 1);
    ms.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ms.tmem)),
                 "r"(S::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = ms.tmem;

  if (warp == kStageThreads / 32) {
    // ---- MMA warp: one thread issues every MMA of the CTA ----
    if (lane == 0) {
      const uint32_t ba = smem_u32(&ms.bar_a);
      // the matrix operands: one image, copied in bulk copies of 32 KB
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba), "r"(kABytes) : "memory");
      for (int i = 0; i < 2 * kHalves; ++i)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sA + i * kMatBytes),
            "l"(reinterpret_cast<const unsigned char*>(a.tab) + (size_t)i * kMatBytes), "r"(kMatBytes),
            "r"(ba)
            : "memory");
      bool ok = bar_wait(ba, 0u, abort);
      // descriptors of the first K step (operand 2h: hi, 2h + 1: lo of half h); a later step adds
      // its byte offset >> 4 to the start field
      uint64_t dA[2 * kHalves];
#pragma unroll
      for (int i = 0; i < 2 * kHalves; ++i) dA[i] = mat_desc(sA + i * kMatBytes, 16 * 128, 128);
      // units: the tiles, or for SOLVE their two passes (accumulator buffer = pass, used once per
      // tile; otherwise buffer i & 1, used every other tile)
      constexpr int U = SOLVE ? 2 : 1;
      int i = 0;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i)
      for (int pass = 0; pass < U && ok; ++pass) {
        const int ui = i * U + pass;
        const int b2 = SOLVE ? pass : (i & 1);
        if (SOLVE ? i >= 1 : i >= 2)
          ok = bar_wait(smem_u32(&ms.acc_empty[b2]), SOLVE ? (uint32_t)((i - 1) & 1) : (uint32_t)(((i >> 1) - 1) & 1),
                        abort);
        tc_after_sync();
        const uint32_t dacc = tmem + (uint32_t)(b2 * kHalves * kN);
        for (int c = 0; c < kChunks && ok; ++c) {
          const int u = 2 * ui + (c >> 1);  // use of the chunk's slot (c & 1)
          ok = bar_wait(smem_u32(&ms.full[c & 1]), (uint32_t)(u & 1), abort);
          if (!ok) break;
          tc_after_sync();
          const uint32_t stage = sB + (c & 1) * kStageBytes;
#pragma unroll
          for (int h = 0; h < kHalves; ++h) {
            const uint32_t d = dacc + (uint32_t)(h * kN);
            const uint64_t dbh0 = mat_desc(stage + (2 * h) * kOpBytes, (kN / 8) * 128, 128);
            const uint64_t dbl0 = mat_desc(stage + (2 * h + 1) * kOpBytes, (kN / 8) * 128, 128);
#pragma unroll
            for (int ks = 0; ks < kChunk / 16; ++ks) {
              const int kg = c * (kChunk / 16) + ks;  // 16-input step within the 128 inputs
              const uint64_t aoff = (uint64_t)(kg * 2 * 16 * 128) >> 4;  // two core matrices along K
              const uint64_t boff = (uint64_t)(ks * 2 * (kN / 8) * 128) >> 4;
              mma_f16<S::kIdesc>(d, dA[2 * h] + aoff, dbh0 + boff, (c | ks) ? 1u : 0u);
              mma_f16<S::kIdesc>(d, dA[2 * h] + aoff, dbl0 + boff, 1u);
              mma_f16<S::kIdesc>(d, dA[2 * h + 1] + aoff, dbh0 + boff, 1u);
            }
          }
          mma_commit(smem_u32(&ms.empty[c & 1]));  // the slot is free once these MMAs are done
        }
        if (ok) mma_commit(smem_u32(&ms.acc_full[b2]));  // the tile's accumulators are complete
      }
      if (!ok) {
        atomicExch(&ms.abort, 1u);
        atomicExch(a.err, 1);
      }
      // the matrix image has landed and every MMA issued by this thread has completed before the
      // CTA exits and tensor memory is freed (bounded)
      bar_wait(ba, 0u, nullptr);
      const uint32_t fin = smem_u32(&ms.fin);
      mma_commit(fin);
      bar_wait(fin, 0u, nullptr);
    }
  } else if (warp == kStageThreads / 32 + 1) {
    // ---- load warp: one thread copies each tile's lines (contiguous) into the raw buffer as soon
    // as the staging threads have read the previous tile's out of it (idle for strided lines) ----
    if (!STRIDED && lane == 0) {
      const uint32_t rf = smem_u32(&ms.raw_full), sraw = sA + S::kRawOff;
      bool ok = true;
      int i = 0;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
        if (i >= 1) ok = bar_wait(smem_u32(&ms.raw_empty), (uint32_t)((i - 1) & 1), abort);
        if (!ok) break;
        const long long first = (long long)t * kLines;
        const int n = (int)(a.lines - first < kLines ? a.lines - first : kLines);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.S + first * P);
        // bulk copies move multiples of 16 bytes: an odd count of lines leaves the last value
        // of the last line (8 bytes) to a plain copy, written before the arrive that publishes it
        // (tiles start on a 16-byte boundary: a tile holds an even number of odd-length lines)
        const uint32_t bytes = (uint32_t)n * S::kLineBytes - ((n & 1) ? 8u : 0u);
        if (n & 1) {
          const float2 v = *reinterpret_cast<const float2*>(src + bytes);
          asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(sraw + bytes), "f"(v.x), "f"(v.y) : "memory");
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rf), "r"(bytes) : "memory");
        for (uint32_t off = 0; off < bytes; off += 16384u) {
          const uint32_t len = bytes - off < 16384u ? bytes - off : 16384u;
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           sraw + off),
                       "l"(src + off), "r"(len), "r"(rf)
                       : "memory");
        }
      }
      if (!ok) atomicExch(&ms.abort, 1u);
      // the last copies have landed before the CTA exits (bounded)
      if (i > 0) bar_wait(rf, (uint32_t)((i - 1) & 1), nullptr);
    }
  } else {
    // ---- staging / epilogue warps ----
    // barrier of the staging threads that also returns, to all of them, whether any saw the
    // abort flag set (one decision for all, so that they leave the loop together)
    auto ssync_abort = [&]() -> bool {
      const uint32_t f = *reinterpret_cast<volatile uint32_t*>(&ms.abort);
      uint32_t any;
      asm volatile(
          "{\n\t.reg .pred q, p;\n\tsetp.ne.u32 q, %1, 0;\n\t"
          "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(any)
          : "r"(f), "r"(kStageThreads)
          : "memory");
      return any != 0;
    };
    // item (line l, pair q, group g8) of a tile, item = tid + j * threads; for each chunk c the
    // pair covers the K inputs kk = 32 c + 8 g8 + 2 q and kk + 1, i.e. x = kk + 1 and x + 1:
    //   n = 255: X_x, X_{x+1}, X_{256-x}, X_{255-x} (folded);  n = 127: X_x, X_{x+1} (X_128 = 0)
    int il[kItems], ikl[kItems];
    uint32_t iore[kItems], ioim[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const int item = tid + j * kStageThreads;
      const int q = item & 3, rl = (item >> 2) & 7, g8 = (item >> 5) & 3, rh = item >> 7;
      il[j] = rh * 8 + rl;
      ikl[j] = g8 * 8 + 2 * q;  // K index within a chunk (even)
      iore[j] = kmajor_off(il[j], ikl[j], kN);
      ioim[j] = kmajor_off(kLines + il[j], ikl[j], kN);
    }
    const float2* raw = reinterpret_cast<const float2*>(smem + S::kRawOff);
    // epilogue of the j-th tile of this CTA (tile index tj): lanes 32 (warp % 4) .. + 31 of tensor
    // memory hold output index m; each group of four warps takes kLinesPerWarp lines
    // kind 0: the transform's output (-2i); SOLVE: kind 1 the divided spectrum (-2i, then / d) into
    // the shared buffer only, kind 2 the solution (+2i)
    auto epilogue = [&](int b2, uint32_t ph, int tj, int kind) {
      if (!bar_wait(smem_u32(&ms.acc_full[b2]), ph, abort)) atomicExch(&ms.abort, 1u);
      tc_after_sync();
      const int m = 32 * (warp & 3) + lane;
      const int l0 = kLinesPerWarp * (warp >> 2);
      const uint32_t tl = tmem + (uint32_t)(b2 * kHalves * kN) + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
      for (int h8 = 0; h8 < kLinesPerWarp; h8 += 8) {
        if constexpr (S::kFold) {
          float ere[8], eim[8], orr[8], oim8[8];
          tmem_ld8(tl + (uint32_t)(0 * kN + l0 + h8), ere);
          tmem_ld8(tl + (uint32_t)(0 * kN + kLines + l0 + h8), eim);
          tmem_ld8(tl + (uint32_t)(1 * kN + l0 + h8), orr);
          tmem_ld8(tl + (uint32_t)(1 * kN + kLines + l0 + h8), oim8);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (h8 + 8 == kLinesPerWarp) {
            tc_before_sync();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ms.acc_empty[b2])) : "memory");
          }
          if (!*reinterpret_cast<volatile uint32_t*>(&ms.abort)) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int lu = l0 + h8 + u;
              const long long line = (long long)tj * kLines + lu;
              if (line >= a.lines) break;
              const float us = ms.unscale[b2][lu];
              float2* row = a.S + line * P;
              // -2i z = (2 Im z, -2 Re z); index 2m: k = 2m + 1 (odd half), 2m + 1: k = 2m + 2 (even half)
              const float2 yo = make_float2(oim8[u] * us, -orr[u] * us);
              const float2 ye = make_float2(eim[u] * us, -ere[u] * us);
              if ((line & 1) == 0 && m < 127) {
                // even lines start on a 16-byte boundary (255 values of 8 bytes per line)
                *reinterpret_cast<float4*>(row + 2 * m) = make_float4(yo.x, yo.y, ye.x, ye.y);
              } else {
                row[2 * m] = yo;
                if (m < 127) row[2 * m + 1] = ye;
              }
            }
          }
        } else {
          float re[8], im[8];
          tmem_ld8(tl + (uint32_t)(l0 + h8), re);
          tmem_ld8(tl + (uint32_t)(kLines + l0 + h8), im);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (h8 + 8 == kLinesPerWarp) {
            tc_before_sync();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ms.acc_empty[b2])) : "memory");
          }
          if constexpr (STRIDED) {
            // output index m of the 8 lines into the transposition buffer (row m, column lu)
            if (m < P) {
              float2* so = reinterpret_cast<float2*>(smem + S::kOutOff) + m * S::kOutPitch + l0 + h8;
              if (SOLVE && kind == 1) {
                // / scale (sigma_j + lambda_other + lambda_k), k = m + 1 (as AxisArgs op 1)
                const int q = tj / tpp, x0 = (tj - q * tpp) * kLines, nl = geo(tj).nl;
                const float2 sg = a.sigma[q];
                const float lz = a.lam_axis[m];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const int lu = l0 + h8 + u;
                  const float us = ms.unscale[b2][lu];
                  const float yx = im[u] * us, yy = -re[u] * us;
                  const float lo = lu < nl ? a.lam_other[x0 + lu] : 0.f;
                  const float dx = (sg.x + lo + lz) * a.scale, dy = sg.y * a.scale;
                  const float inv = 1.f / (dx * dx + dy * dy);
                  so[u] = make_float2((yx * dx + yy * dy) * inv, (yy * dx - yx * dy) * inv);
                }
              } else if (SOLVE && kind == 2) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const float us = ms.unscale[b2][l0 + h8 + u];
                  so[u] = make_float2(-im[u] * us, re[u] * us);  // +2i z
                }
              } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const float us = ms.unscale[b2][l0 + h8 + u];
                  so[u] = make_float2(im[u] * us, -re[u] * us);
                }
              }
            }
          } else if (!*reinterpret_cast<volatile uint32_t*>(&ms.abort) && m < P) {
            const TileGeo g = geo(tj);
            float2* out = g.base + (size_t)m * g.ps;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int lu = l0 + h8 + u;
              if (lu >= g.nl) break;
              const float us = ms.unscale[b2][lu];
              // output index m: k = m + 1; -2i z = (2 Im z, -2 Re z)
              out[(size_t)lu * g.ls] = make_float2(im[u] * us, -re[u] * us);
            }
          }
        }
      }
      if constexpr (STRIDED) {
        // the buffer complete (the staging threads only), then row by row to global memory: a
        // warp stores 32 consecutive columns of a row. (The next tile's writes into the buffer
        // follow the staging threads' barrier of the next tile.)
        asm volatile("bar.sync 2, %0;" ::"r"(kStageThreads) : "memory");
        if (kind != 1 && !*reinterpret_cast<volatile uint32_t*>(&ms.abort)) {
          const TileGeo g = geo(tj);
          const float2* so = reinterpret_cast<const float2*>(smem + S::kOutOff);
          for (int idx = tid; idx < P * kLines; idx += kStageThreads) {
            const int r = idx / kLines, col = idx - r * kLines;
            if (col < g.nl) g.base[(size_t)r * g.ps + col] = so[r * S::kOutPitch + col];
          }
        }
      }
    };
    // strided lines: a tile's inputs straight from global memory into registers, point x of line
    // l at base[(x - 1) ps + l] (a warp's lanes read 8 consecutive columns of 4 rows); issued one
    // tile ahead, so that they are in flight during the previous tile's epilogue
    float2 in[kItems][kChunks][kVals];
    auto load_strided = [&](int tt) {
      if constexpr (STRIDED) {
        const TileGeo g = geo(tt);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const bool okl = il[j] < g.nl;
          const float2* col = g.base + il[j];
#pragma unroll
          for (int c = 0; c < kChunks; ++c) {
            const int x = c * kChunk + ikl[j] + 1;
            const float2 z = make_float2(0.f, 0.f);
            in[j][c][0] = okl ? col[(size_t)(x - 1) * g.ps] : z;
            in[j][c][1] = (okl && x < P) ? col[(size_t)x * g.ps] : z;  // x + 1 = 128: the zero padding
          }
        }
      }
    };
    // one unit (a tile, or a pass of a SOLVE tile) from `in`: the line maxima, the scales (unscale
    // buffer ubuf), then (fold,) scale and split chunk by chunk into the stage slots (each free once
    // the MMAs of its previous chunk are done), signalling the MMA warp; true if the CTA aborts
    // (decided for all staging threads together)
    auto stage_unit = [&](int ui, int ubuf) -> bool {
        // largest |re|, |im| of each line: over the item, its four lanes (q), the four warps
        // holding the line's groups (g8)
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          float m = 0.f;
#pragma unroll
          for (int c = 0; c < kChunks; ++c)
#pragma unroll
            for (int k = 0; k < kVals; ++k) m = fmaxf(m, fmaxf(fabsf(in[j][c][k].x), fabsf(in[j][c][k].y)));
          m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
          m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
          if ((ikl[j] & 7) == 0) ms.pmax[ikl[j] >> 3][il[j]] = m;
        }
        if (ssync_abort()) return true;
        float sc[kItems];
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const int l = il[j];
          const float m = fmaxf(fmaxf(ms.pmax[0][l], ms.pmax[1][l]), fmaxf(ms.pmax[2][l], ms.pmax[3][l]));
          // m = f 2^E, f in [0.5, 1): the scale 2^(14 - E) brings m to [2^13, 2^14)
          const int E = m > 0.f ? (int)((__float_as_uint(m) >> 23) & 0xff) - 126 : 14;
          int sh = 14 - E;
          sh = sh > 100 ? 100 : (sh < -100 ? -100 : sh);
          sc[j] = __uint_as_float((uint32_t)(127 + sh) << 23);
          if (ikl[j] == 0) ms.unscale[ubuf][l] = __uint_as_float((uint32_t)(127 - sh - 3) << 23);  // 2/(16 2^sh)
        }
        // (fold,) scale and split chunk by chunk into the stage slots (each free once the MMAs of
        // its previous chunk are done), then signal the MMA warp
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
          const int u = 2 * ui + (c >> 1);  // use of the chunk's slot (c & 1)
          if (u >= 1 && !bar_wait(smem_u32(&ms.empty[c & 1]), (uint32_t)((u - 1) & 1), abort))
            atomicExch(&ms.abort, 1u);
          const uint32_t stage = sB + (c & 1) * kStageBytes;
#pragma unroll
          for (int j = 0; j < kItems; ++j) {
            const float f = sc[j];
            uint32_t lo, hi;
            if constexpr (S::kFold) {
              const float2 a0 = in[j][c][0], a1 = in[j][c][1], b0 = in[j][c][2], b1 = in[j][c][3];
              const float2 e0 = make_float2((a0.x - b0.x) * f, (a0.y - b0.y) * f);
              const float2 e1 = make_float2((a1.x - b1.x) * f, (a1.y - b1.y) * f);
              const float2 o0 = make_float2((a0.x + b0.x) * f, (a0.y + b0.y) * f);
              const float2 o1 = make_float2((a1.x + b1.x) * f, (a1.y + b1.y) * f);
              hi = split2(e0.x, e1.x, &lo);
              sts32(stage + 0 * kOpBytes + iore[j], hi);
              sts32(stage + 1 * kOpBytes + iore[j], lo);
              hi = split2(e0.y, e1.y, &lo);
              sts32(stage + 0 * kOpBytes + ioim[j], hi);
              sts32(stage + 1 * kOpBytes + ioim[j], lo);
              hi = split2(o0.x, o1.x, &lo);
              sts32(stage + 2 * kOpBytes + iore[j], hi);
              sts32(stage + 3 * kOpBytes + iore[j], lo);
              hi = split2(o0.y, o1.y, &lo);
              sts32(stage + 2 * kOpBytes + ioim[j], hi);
              sts32(stage + 3 * kOpBytes + ioim[j], lo);
            } else {
              const float2 a0 = in[j][c][0], a1 = in[j][c][1];
              hi = split2(a0.x * f, a1.x * f, &lo);
              sts32(stage + 0 * kOpBytes + iore[j], hi);
              sts32(stage + 1 * kOpBytes + iore[j], lo);
              hi = split2(a0.y * f, a1.y * f, &lo);
              sts32(stage + 0 * kOpBytes + ioim[j], hi);
              sts32(stage + 1 * kOpBytes + ioim[j], lo);
            }
          }
          fence_async_smem();
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ms.full[c & 1])) : "memory");
        }
      return false;
    };
    if (STRIDED && blockIdx.x < tiles) load_strided(blockIdx.x);
    int i = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      const int b2 = i & 1;
      if constexpr (!STRIDED) {
        // the tile's inputs, from the raw buffer into registers; then the buffer is released
        if (!bar_wait(smem_u32(&ms.raw_full), (uint32_t)(i & 1), abort)) atomicExch(&ms.abort, 1u);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const bool okl = (long long)t * kLines + il[j] < a.lines;
          const float2* row = raw + il[j] * P;
#pragma unroll
          for (int c = 0; c < kChunks; ++c) {
            const int x = c * kChunk + ikl[j] + 1;
            const float2 z = make_float2(0.f, 0.f);
            in[j][c][0] = okl ? row[x - 1] : z;
            if constexpr (S::kFold) {
              in[j][c][1] = okl ? row[x] : z;
              in[j][c][2] = okl ? row[255 - x] : z;
              in[j][c][3] = okl ? row[254 - x] : z;
            } else {
              in[j][c][1] = (okl && x < P) ? row[x] : z;  // x + 1 = 128: the zero padding
            }
          }
        }
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ms.raw_empty)) : "memory");
      }
      if constexpr (SOLVE) {
        // pass A from the tile's rows; the divided spectrum into the shared buffer; pass B from it
        if (stage_unit(2 * i, 0)) break;
        epilogue(0, (uint32_t)(i & 1), t, 1);
        const float2* zs = reinterpret_cast<const float2*>(smem + S::kOutOff);
        const int nl = geo(t).nl;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const bool okl = il[j] < nl;
#pragma unroll
          for (int c = 0; c < kChunks; ++c) {
            const int x = c * kChunk + ikl[j] + 1;
            const float2 z = make_float2(0.f, 0.f);
            in[j][c][0] = okl ? zs[(x - 1) * S::kOutPitch + il[j]] : z;
            in[j][c][1] = (okl && x < P) ? zs[x * S::kOutPitch + il[j]] : z;
          }
        }
        // (the unit's barrier orders these reads before the buffer's next writes)
        if (stage_unit(2 * i + 1, 1)) break;
        if (t + (int)gridDim.x < tiles) load_strided(t + (int)gridDim.x);
        epilogue(1, (uint32_t)(i & 1), t, 2);
        continue;
      }
      if (stage_unit(i, b2)) break;
      // strided lines: the next tile's loads (the registers are free again)
      if (STRIDED && t + (int)gridDim.x < tiles) load_strided(t + (int)gridDim.x);
      // the previous tile's epilogue runs now, while this tile's MMAs execute
      if (i >= 1) epilogue((i - 1) & 1, (uint32_t)(((i - 1) >> 1) & 1), t - (int)gridDim.x, 0);
    }
    // the last tile's epilogue, decided once for all staging threads (the strided epilogue holds a
    // barrier of theirs)
    const bool stop = ssync_abort();
    if (!SOLVE && i >= 1 && !stop)
      epilogue((i - 1) & 1, (uint32_t)(((i - 1) >> 1) & 1), blockIdx.x + (i - 1) * (int)gridDim.x, 0);
    if (tid == 0 && *reinterpret_cast<volatile uint32_t*>(&ms.abort)) atomicExch(a.err, 1);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols) : "memory");
  }
}

__global__ void __launch_bounds__(TcShape<255>::kThreads, 1) k_dst255_tc(DstTcArgs a) { dst_tc_body<255, 0>(a); }
__global__ void __launch_bounds__(TcShape<127>::kThreads, 1) k_dst127_tc(DstTcArgs a) { dst_tc_body<127, 0>(a); }
__global__ void __launch_bounds__(TcShape<127>::kThreads, 1) k_dst127s_tc(DstTcArgs a) { dst_tc_body<127, 1>(a); }
__global__ void __launch_bounds__(TcShape<127>::kThreads, 1) k_dst127z_tc(DstTcArgs a) { dst_tc_body<127, 2>(a); }

// One FP16 operand pair (hi, lo) of a 128 x 128 matrix v(r, q) in its K-major shared-memory layout.
template <typename F> void put_matrix(unsigned short* hi_img, unsigned short* lo_img, F v) {
  for (int r = 0; r < 128; ++r)
    for (int q = 0; q < 128; ++q) {
      const double x = v(r, q);
      const __half hi = __double2half(x);
      const __half lo = __double2half(x - (double)__half2float(hi));
      const int off = (int)kmajor_off(r, q, 128) / 2;
      hi_img[off] = __half_as_ushort(hi);
      lo_img[off] = __half_as_ushort(lo);
    }
}

}  // namespace

size_t dst_tc_table_bytes(int n) {
  return n == 255 ? (size_t)TcShape<255>::kABytes : n == 127 ? (size_t)TcShape<127>::kABytes : 0;
}

// The matrix image in its shared-memory layout, FP16 K-major (row = output, K = input x - 1),
// scaled by 16.
// n = 255: [even hi | even lo | odd hi | odd lo]
//   even: row r -> k' = r + 1, column q -> x = q + 1: 16 sin(pi k' x / 128) (zero for k' = 128
//         or x = 128)
//   odd:  row r -> k' = r,     column q -> x = q + 1: 16 sin(pi (2k'+1) x / 256), halved at
//         x = 128 (the folded input there is 2 X_128)
// n = 127: [hi | lo], row r -> k = r + 1, column q -> x = q + 1: 16 sin(pi k x / 128) (zero for
//         k = 128 or x = 128)
void dst_tc_table(int n, unsigned short* img) {
  const double pi = 3.14159265358979323846;
  constexpr int half = 128 * 128;  // FP16 values per operand
  if (n == 255) {
    put_matrix(img, img + half, [&](int r, int q) {
      const int kp = r + 1, x = q + 1;
      return (kp == 128 || x == 128) ? 0.0 : 16.0 * std::sin(pi * (double)((kp * x) % 256) / 128.0);
    });
    put_matrix(img + 2 * half, img + 3 * half, [&](int r, int q) {
      const int x = q + 1;
      const double v = 16.0 * std::sin(pi * (double)(((2 * r + 1) * x) % 512) / 256.0);
      return x == 128 ? 0.5 * v : v;
    });
  } else if (n == 127) {
    put_matrix(img, img + half, [&](int r, int q) {
      const int k = r + 1, x = q + 1;
      return (k == 128 || x == 128) ? 0.0 : 16.0 * std::sin(pi * (double)((k * x) % 256) / 128.0);
    });
  }
}

cudaError_t launch_dst_tc(const DstTcArgs& a, cudaStream_t st) {
  if (a.lines <= 0) return cudaSuccess;
  if (!dst_tc_line_ok(a.n) || a.stride < 1) return cudaErrorInvalidValue;
  const bool strided = a.stride > 1, solve = a.sigma != nullptr;
  if (strided && (a.n != 127 || a.lines % a.stride != 0)) return cudaErrorInvalidValue;
  if (solve && (!strided || !a.lam_other || !a.lam_axis)) return cudaErrorInvalidValue;
  // the shared-memory attribute applies to the current device: set on every launch, as the other
  // launchers do; the SM count is queried once per device
  static std::atomic<int> sms[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int n = sms[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms[dev].store(n, std::memory_order_relaxed);
  }
  const bool l255 = a.n == 255;
  const int smem = l255 ? TcShape<255>::kSmemBytes : TcShape<127>::kSmemBytes;
  const int per_tile = l255 ? TcShape<255>::kLines : TcShape<127>::kLines;
  const int threads = l255 ? TcShape<255>::kThreads : TcShape<127>::kThreads;
  auto* kern = l255 ? k_dst255_tc : (solve ? k_dst127z_tc : (strided ? k_dst127s_tc : k_dst127_tc));
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long tiles = strided ? (long long)(a.lines / a.stride) * ((a.stride + per_tile - 1) / per_tile)
                                  : (a.lines + per_tile - 1) / per_tile;
  const int grid = tiles < n ? (int)tiles : n;
  prof_begin(solve ? "axis_solve_tc_f32" : (strided ? "dst_tc_y_f32" : "dst_tc_f32"), st);
  kern<<<grid, threads, smem, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace pint
