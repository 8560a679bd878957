// K3: grouped split-precision GEMM over the coupled sectors on the 5th-generation tensor cores.
//
// C~^c = A~^c B~^c with FP64 operands split into s BF16 slices (Ozaki-style error-free
// splitting; not part of the paper, which multiplies blocks with BLAS):
//   * every row m of A~^c gets a power-of-two scale 2^{e_m} > max_k |a_mk| and every column n
//     of B~^c a scale 2^{f_n}; a_mk 2^{-e_m} is written as s balanced base-128 digits
//     d_0..d_{s-1} to within 2^-43 + 2^-46 (|d_0| <= 128, |d_1|, |d_2| <= 64, the later ones
//     below 81), slice i holding d_i 2^{-7(i+1)} exactly in BF16;
//   * the products A_i B_j with i + j <= s - 1 run as tcgen05.mma kind::f16 (BF16 x BF16, FP32
//     accumulate in TMEM) into four accumulators by level i + j = 0, 1, 2 and >= 3.  Levels 0..2
//     are sums of integers times one power of two: per k a level-0 term is at most 128^2 = 2^14
//     in its unit, level 1 at most 2 * 128 * 64 = 2^14 and level 2 at most 2.5 * 2^12, so the FP32
//     accumulators stay exact (integers below 2^24) while K <= 1024 -- one "segment".  Longer K
//     runs in several segments whose results are added in FP64;
//   * the epilogue adds the four accumulators with error-free FP32 two-sums, converts to FP64 and
//     applies 2^{e_m + f_n}.
// With s = 6 the relative Frobenius error against FP64 is ~1e-12 on N(0,1) data.
//
// Data path: one prep launch (clusters of 4 or 8 CTAs; a 128-row operand tile takes one to eight
// of them by its depth, their scale maxima exchanged through distributed shared memory) writes the
// scales and the slices as pre-tiled 128 x 32 BF16 tiles (64-byte rows); one persistent GEMM
// launch walks a work list of (sector, 128-row tile, column tile) items, the last column tile of a
// sector as narrow as its remainder (MMA N a
// multiple of 16).  Per CTA: warp 0 issues TMA loads (cp.async.bulk.tensor, 64-byte swizzle) of
// all s A slices and all s B slices of one 32-deep k-chunk into a stage (two to four); one thread
// of warp 1 issues every slice-pair MMA from the resident stage; sixteen epilogue warps (2..17,
// four per TMEM lane quadrant) read the accumulators eight columns at a time, convert to FP64,
// store, and then hand the buffer back to the MMA warp.  With 128-column tiles the four
// accumulators fill TMEM, so the next tile's MMAs wait for that epilogue; 64-column tiles have
// two buffers and overlap it.  Every mbarrier wait is bounded: on timeout the kernel records an
// error in the context's status word, drains its own copies and MMAs (bounded again), frees
// TMEM and returns.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstring>

#include "tk_device.cuh"
#include "tk_internal.hpp"

namespace cg = cooperative_groups;

namespace tk {
namespace {

constexpr int OZ_BM = 128, OZ_BK = 32;              // k-chunk: two MMA K steps
constexpr int OZ_BN_WIDE = 128, OZ_BN_NARROW = 64;  // output tile widths (one / two TMEM buffers)
constexpr int OZ_TROWS = 128;                     // rows of a slice tile in memory (A: m, B: n)
// Two product schemes share the pipeline (template parameter MODE):
//   MODE 0, Ozaki BF16: s BF16 slices per operand, pairs i + j <= s - 1 into four level accumulators;
//   MODE 1, 3xTF32: a = hi + lo with hi, lo TF32 (FP32 containers, 13 low mantissa bits zero);
//     products hi.hi + hi.lo + lo.hi into one FP32 accumulator (about FP32 accuracy).
template <int MODE>
struct OzMode {
  static constexpr int ESZ = MODE == 0 ? 2 : 4;          // bytes per slice element
  static constexpr int ROW = OZ_BK * ESZ;                // bytes of one tile row (64 or 128)
  static constexpr int A_BYTES = OZ_BM * ROW;            // A box in shared memory
  static constexpr int MMAS = ROW / 32;                  // MMAs per k-chunk and pair (32 B of K each)
};
constexpr int OZ_MAX_STAGES = 4;                  // a stage holds all s A and s B boxes of a k-chunk
constexpr int OZ_SEG_KC = 32;                     // k-chunks per exact segment (K <= 1024)
constexpr int OZ_NACC = 4;
constexpr int OZ_TMEM_COLS = 512;                 // 4 accumulators x 128 columns, or 2 x 4 x 64
constexpr int OZ_EPI_WARPS = 16;                  // four per TMEM lane quadrant
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;  // producer warp, MMA warp, epilogue warps
constexpr int OZ_MAX_SLICES = 7;
constexpr int OZ_MAX_PAIRS = OZ_MAX_SLICES * (OZ_MAX_SLICES + 1) / 2;
constexpr int OZ_DEFAULT_SLICES = 6;
constexpr unsigned long long OZ_WAIT_NS = 2000000000ull;  // bounded waits: 2 s

struct OzSector {
  int64_t M, N, K;
  int64_t a_off, b_off, c_off;
  int64_t ta_base, tb_base;  // first tile of this sector's A / B slices
  int64_t sa_off, sb_off;    // offsets into the row / column scale arrays
  int32_t nmt, nnt, nkc, pad;  // 128-row slice tiles of A~ / B~^T, 32-deep k-chunks
};
struct OzWork {
  int32_t sector, mt, nt, nw;  // nw: columns of this tile (multiple of 16, <= the tile width)
  int32_t kc_lo, kc_hi;        // k-chunks of this item: the whole depth, or one part of a split
  int32_t part, nparts, slot, pad;  // split-K: part index, parts of the tile, tile slot (-1: no split)
};
constexpr int OZ_MAX_PARTS = 4;
struct OzJob {  // the work of one k_oz_prep CTA: its share of one 128-row tile of one operand
  int32_t sector;         // -1: an idle CTA (pads a request's list to whole clusters)
  int32_t operand;        // 0: rows of A~, 1: columns of B~
  int32_t r0;             // row tile
  int16_t gbase, gsize;   // ranks [gbase, gbase + gsize) of the cluster share the tile
};
struct OzPairs {
  int8_t i[OZ_MAX_PAIRS], j[OZ_MAX_PAIRS], lvl[OZ_MAX_PAIRS];
  int32_t n;
  int32_t first[OZ_NACC];  // index of the first pair of each level (-1 if none)
};

struct OzLayout {
  std::vector<OzSector> sectors;
  int64_t ntiles_a = 0, ntiles_b = 0, nrows_a = 0, ncols_b = 0;
  size_t off_ta = 0, off_tb = 0, off_sa = 0, off_sb = 0, bytes = 0;
  int slices = OZ_DEFAULT_SLICES;
  int mode = 0;           // 0: Ozaki BF16 slices, 1: 3xTF32
  int bn = OZ_BN_NARROW;  // output tile width of this launch
  OzPairs pairs;
  int64_t nwork = 0, nprep_ctas = 0;
  OzSector* d_sectors = nullptr;
  OzWork* d_work = nullptr;
  OzJob* d_prep_jobs = nullptr;  // one per k_oz_prep CTA, a multiple of prep_cluster
  int prep_cluster = 8;  // CTAs per k_oz_prep cluster: 4 or 8
  bool prep_img = false;  // k_oz_prep keeps each CTA's first two k-chunks in shared memory
  std::vector<int32_t> cta_work;   // work of CTA b: work[cta_work[b] .. cta_work[b + 1])
  int32_t* d_cta_work = nullptr;
  int ncta = 0;
  int32_t nslots = 0;        // split tiles
  size_t off_part = 0;       // their partial tiles in the workspace
  size_t off_cnt = 0;        // per (split tile, epilogue warp) arrival counters in the workspace
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the CTA's abort flag) if the phase did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          bool sleepy = false) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > OZ_WAIT_NS) {
      *abort_flag = 1;
      return false;
    }
    if (sleepy) __nanosleep(200);  // long waits (epilogue warps) leave the issue slots to the MMA warp
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
template <int MODE>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  if (MODE == 0)
    tc_mma_bf16(d_tmem, adesc, bdesc, idesc, accumulate);
  else
    tc_mma_tf32(d_tmem, adesc, bdesc, idesc, accumulate);
}
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, rows of ROW bytes with the matching swizzle
// (64 B: 64-byte swizzle, 128 B: 128-byte swizzle), 8-row groups 8 ROW bytes apart.
template <int ROW>
__device__ __forceinline__ uint64_t smem_desc_k(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * ROW) >> 4) << 32;         // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)(ROW == 128 ? 2 : 4) << 61;     // layout: 128-byte / 64-byte swizzle
  return d;
}
// Instruction descriptor: FP32 accumulate, both operands K-major, M x N; A and B both BF16
// (kind::f16, format 1) or both TF32 (kind::tf32, format 2).
template <int MODE>
__host__ __device__ constexpr uint32_t idesc_mma(int m, int n) {
  return (1u << 4)                                  // D format: F32
         | ((MODE == 0 ? 1u : 2u) << 7)             // A format
         | ((MODE == 0 ? 1u : 2u) << 10)            // B format
         | ((uint32_t)(n >> 3) << 17)               // N / 8
         | ((uint32_t)(m >> 4) << 24);              // M / 16
}

__device__ __noinline__ double scale_pow2_slow(double v, int e) { return ldexp(v, e); }

// (hi + lo) 2^sc in FP64 for a two-sum pair (|lo| <= ulp(hi) / 2), with no FP64 instruction (the
// FP64 pipe retires two lanes per SM per clock here, and one add per output bounded this
// epilogue).  hi's FP64 words come from its bits with 32-bit operations: the high word is hi's
// sign | ((hi's bits without the sign) >> 3) + (896 + sc) << 20 (exponent rebiased by 1023 - 127
// and raised by sc), the low word its last 3 fraction bits.  lo then moves that pattern by a whole
// number of last places of the result's binade: |lo| times 2^(179 - e_hi) (exact in FP32, at most
// 2^29) rounded to the nearest integer, added when lo has hi's sign and subtracted otherwise; when
// hi is a power of two and lo has the other sign the result lies one binade lower, where a last
// place is half as large, so the count is taken at twice the scale.  Adding to the pattern crosses
// into that binade by itself.  hi must have an FP32 exponent field in [53, 253] (the scale 2^(179 -
// e_hi), or twice it, is then a normal FP32) and sc in [-895, 2045 - e_hi] (both results normal in
// FP64); anything else clears ok and the caller takes the exact slow path.
// kexp = (896 + sc) << 20 (modulo 2^32), which the caller may have assembled from per-row and
// per-column parts.
template <bool SAFE_SC>
__device__ __forceinline__ double f32_pair_scaled(float hi, float lo, int sc, uint32_t kexp, bool& ok) {
  const uint32_t uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const uint32_t eh = (uh >> 23) & 0xFFu;
  // SAFE_SC: the caller knows |sc| <= 896, which with e_hi in [53, 253] keeps both results normal
  ok = (eh - 53u) < 201u && (SAFE_SC || (uint32_t)(sc + 895) <= (uint32_t)(2045 - (int)eh));
  const uint32_t whi = (uh & 0x80000000u) | (((uh & 0x7FFFFFFFu) >> 3) + kexp);
  const uint32_t against = (uh ^ ul) >> 31;
  const uint32_t below = against & (uint32_t)((uh & 0x7FFFFFu) == 0u);
  const float scale = __uint_as_float((306u - eh + below) << 23);  // 2^(179 - e_hi + below)
  const int off = __float2int_rn(__fmul_rn(fabsf(lo), scale));
  const long long bits = (long long)(((unsigned long long)whi << 32) | (uh << 29));
  return __longlong_as_double(bits + (against ? -(long long)off : (long long)off));
}
__device__ __noinline__ double f32_pair_scaled_slow(float hi, float lo, int sc) {
  return scale_pow2_slow(f32_to_f64(hi) + f32_to_f64(lo), sc);
}

// ------------------------------------------------------------------ scale and slice kernels
// Operand views: A~^c element (m, k) at A[a_off + m + k M]; B~^c element (k, n) at B[b_off + k + n K].

// Scale exponents 2^e > max_k |x_rk| for every row of A~^c and every column of B~^c (k_oz_prep).
constexpr int32_t kNoScale = (int32_t)0x80808080;  // the scale of an all-zero row or column
constexpr int OZ_PREP_CLUSTER = 8;                 // largest k_oz_prep cluster (4 or 8 CTAs per launch)

// e with 2^(e-1) <= mx < 2^e for a non-negative finite mx (kNoScale for 0), from the bits.
__device__ __forceinline__ int exponent_of(double mx) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(mx);
  if (b == 0) return kNoScale;
  const int ex = (int)(b >> 52);
  if (ex != 0) return ex - 1022;
  return -1074 + (64 - __clzll((long long)b));  // subnormal: highest set bit
}

// One request of a prep launch: its job list, operands, scale arrays and slice tiles;
// its jobs are blocks [block0, block0 + njobs) of the launch.
struct OzPrepSeg {
  const OzSector* secs;
  const OzJob* jobs;
  const double* A;
  const double* B;
  int32_t* sa;
  int32_t* sb;
  int* counters;
  void* ta;
  void* tb;
  int64_t block0;
  int32_t ncounters, pad;
};
template <int NSEG>
struct OzPrepT {
  OzPrepSeg seg[NSEG];
  int32_t nseg;
  int32_t img;  // each CTA keeps its first two k-chunks in shared memory (two chunk images)
};
template <int NSEG>
__device__ __forceinline__ const OzPrepSeg& prep_seg(const OzPrepT<NSEG>& P, int64_t& local) {
  int lo = 0, hi = P.nseg - 1;  // the segment with the largest block0 <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.seg[mid].block0 <= (int64_t)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  local = (int64_t)blockIdx.x - P.seg[lo].block0;
  return P.seg[lo];
}

// x = v 2^-e (|x| < 1) as hi + lo: two FP32 numbers holding the top 24 significant bits of x
// (hi: sign, exponent, 23 stored fraction bits) and the next 23 bits (lo), both exact, formed
// from the FP64 bit pattern with 32-bit integer operations (lo as a normal FP32 with those bits as
// its fraction minus the same number with a zero fraction: an exact subtraction).  The last 6
// fraction bits of v are dropped (< 2^-46 |x|), and so are parts below the FP32 normal range
// (x < 2^-126, or lo when x < 2^-103): far below the last digit, 2^-42.
__device__ __forceinline__ void scaled_split(double v, int e, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  const int ex = (int)((bh >> 20) & 0x7FFu);
  const int ef = ex - 1023 - e + 127;  // FP32 exponent field of x
  hi = lo = 0.f;
  if (ex == 0 || ef <= 0) return;
  const uint32_t sign = bh & 0x80000000u;
  hi = __uint_as_float(sign | ((uint32_t)ef << 23) | ((bh & 0xFFFFFu) << 3) | (bl >> 29));
  if (ef < 24) return;
  const uint32_t e2 = (uint32_t)(ef - 23) << 23;  // lo = bits 28..6 of the fraction, 2^-46 units
  const float l = __fsub_rn(__uint_as_float(e2 | ((bl >> 6) & 0x7FFFFFu)), __uint_as_float(e2));
  lo = __uint_as_float(__float_as_uint(l) ^ sign);
}

// v 2^-e (|v| < 2^e) as hi + lo, both TF32 values in FP32 containers (11 significant bits, the
// 13 low fraction bits zero), from the FP32 pair (h, l) above with 32-bit operations: hi is h
// rounded to 11 bits (half away from zero, on the bit pattern, so that a carry moves into the
// exponent), h - hi is exact, and lo is (h - hi) + l rounded to FP32 and then to 11 bits.  hi
// equals v 2^-e rounded to 11 bits (h holds its top 24 bits and l has h's sign); |x - hi - lo| <=
// 2^-23 |x|.  Parts below the FP32 normal range are dropped.
__device__ __forceinline__ void tf32_split(double v, int e, float& hi, float& lo) {
  float h, l;
  scaled_split(v, e, h, l);
  hi = __uint_as_float((__float_as_uint(h) + 0x1000u) & 0xFFFFE000u);
  const float t = __fadd_rn(__fsub_rn(h, hi), l);
  const uint32_t tb = (__float_as_uint(t) + 0x1000u) & 0xFFFFE000u;
  lo = (tb & 0x7F800000u) ? __uint_as_float(tb) : 0.f;
}

// The S balanced base-128 digits d_i of x = hi + lo, x ~ sum_i d_i 2^(-7 (i + 1)), in FP32 for two
// entries at once (paired FP32 instructions, each half rounded on its own as a scalar operation
// would be): with t the remainder (t = hi at first), y = 128 t is exact, d = (y + 1.5 2^23) -
// 1.5 2^23 rounds y to the nearest integer (|y| <= 128), and t = y - d is exact again, |t| <= 1/2.
// So |d_0| <= 128 and |d_1|, |d_2| <= 64 (these three make the exact levels 0..2).  After three
// digits the 24 bits of hi are used up and lo joins the remainder (lo 2^21 is exact, so the fused
// multiply-add rounds once, <= 2^-46 of the scale); the later digits (level >= 3 only, an inexact
// accumulator anyway) stay below 81.  The result is within 2^-43 + 2^-46 of x, every d_i an
// integer (exact in BF16).
template <int S>
__device__ __forceinline__ void f32_digits2(float2 hi, float2 lo, float2 (&d)[S]) {
  const float2 k128 = make_float2(128.0f, 128.0f);
  const float2 kRound = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23
  const float2 kNegRound = make_float2(-12582912.0f, -12582912.0f);
  const float2 kNegOne = make_float2(-1.0f, -1.0f);
  const float2 kLo = make_float2(2097152.0f, 2097152.0f);  // lo in the units of the 4th digit (2^21)
  float2 t = hi;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (i == 3) t = __ffma2_rn(lo, kLo, t);
    const float2 y = __fmul2_rn(t, k128);
    const float2 di = __fadd2_rn(__fadd2_rn(y, kRound), kNegRound);
    t = __ffma2_rn(di, kNegOne, y);  // y - d, exact
    d[i] = di;
  }
}

// Digits of a pair of entries, written as S packed BF16 pairs (slice i holds d_i 2^(-7 (i + 1))):
// d_i 2^(-7 (i + 1)) has at most 8 significant bits, so its BF16 pattern is the upper half of its
// FP32 pattern and two of them pack with one byte permute (no conversion instruction).
template <int S>
__device__ __forceinline__ void oz_slice_pair(double v0, double v1, int e, uint32_t* dst, int64_t stride2) {
  float h0, l0, h1, l1;
  float2 d[S];
  scaled_split(v0, e, h0, l0);
  scaled_split(v1, e, h1, l1);
  f32_digits2<S>(make_float2(h0, h1), make_float2(l0, l1), d);
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    const float sc = __int_as_float((127 - 7 * (sl + 1)) << 23);  // 2^(-7 (sl + 1)), exact
    const float2 u = __fmul2_rn(d[sl], make_float2(sc, sc));
    dst[sl * stride2] = __byte_perm(__float_as_uint(u.x), __float_as_uint(u.y), 0x7632);  // (y >> 16) << 16 | x >> 16
  }
}

// Shared staging of one k-chunk of a tile: buf[kk][r] = x(row r0 + r, k0 + kk) (for B~, r runs over
// its columns), zero outside the sector.  The padding column keeps the row-pair reads below spread
// over the banks.  A launch with chunk images holds two of them (the second also serves as the
// staging buffer of later chunks).
using PrepBuf = double[OZ_BK][OZ_TROWS + 1];
constexpr size_t OZ_PREP_SMEM = sizeof(PrepBuf);
constexpr size_t OZ_PREP_SMEM_IMG = 2 * sizeof(PrepBuf);

// One 128 x 32 (rows x k) tile (row tile rt, k-chunk kc) of one operand, all slices, with the
// rows' scale exponents in esc.  Every load of a thread is issued before any arithmetic.  A~
// (column-major, rows contiguous) is staged through shared memory so that its reads coalesce; B~
// (k contiguous) is read straight into the slicing layout.  Each thread then takes two consecutive
// k of 8 rows, so a slice of the pair is one packed 32-bit (BF16 pair) or 64-bit (TF32 pair) store
// and a half-warp writes a full 64-byte tile row.  MODE 0 writes S BF16 digit slices, MODE 1 the
// TF32 pair (hi, lo).  IMG: the chunk is already in xs (kept there by the maxima pass, zeros
// outside the sector, either operand), so nothing is loaded and no barrier is needed.  Otherwise
// called by all 256 threads of the CTA (the A path synchronises them).
template <int MODE, int S, bool IMG>
__device__ __forceinline__ void slice_tile(const OzPrepSeg& g, const OzSector& s, int op, int64_t rt, int kc,
                                           const int* esc, PrepBuf& xs) {
  constexpr int NI = OZ_TROWS / 16;  // rows per thread
  const int64_t R = op == 0 ? s.M : s.N;
  const int64_t r0 = rt * OZ_TROWS, k0 = (int64_t)kc * OZ_BK;
  const int tid = threadIdx.x;
  const int kp = (tid & 15) * 2, rw = tid >> 4;  // k pair and first row of this thread
  double v[NI][2];
  if (IMG) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      v[i][0] = xs[kp][rw + 16 * i];
      v[i][1] = xs[kp + 1][rw + 16 * i];
    }
  } else if (op == 0) {
    const int ml = tid & (OZ_TROWS - 1), kk0 = tid >> 7;
    const bool mok = r0 + ml < R;
    const double* src = g.A + s.a_off + (r0 + ml) + (k0 + kk0) * s.M;
    const int64_t step = 2 * s.M;
    double x[OZ_BK / 2];
#pragma unroll
    for (int j = 0; j < OZ_BK / 2; ++j) x[j] = (mok && k0 + kk0 + 2 * j < s.K) ? __ldg(src + j * step) : 0.0;
    __syncthreads();  // the previous tile's readers are done with xs
#pragma unroll
    for (int j = 0; j < OZ_BK / 2; ++j) xs[kk0 + 2 * j][ml] = x[j];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      v[i][0] = xs[kp][rw + 16 * i];
      v[i][1] = xs[kp + 1][rw + 16 * i];
    }
  } else {
    const int64_t k = k0 + kp;
    const double* src = g.B + s.b_off + k + (r0 + rw) * s.K;
    const int64_t step = 16 * s.K;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const bool rok = r0 + rw + 16 * i < R;
      v[i][0] = (rok && k < s.K) ? __ldg(src + i * step) : 0.0;
      v[i][1] = (rok && k + 1 < s.K) ? __ldg(src + i * step + 1) : 0.0;
    }
  }
  const int64_t nrt = op == 0 ? s.nmt : s.nnt;
  const int64_t tile0 = (op == 0 ? s.ta_base : s.tb_base) + rt * s.nkc + kc;  // slice 0
  const int64_t slice_stride = nrt * s.nkc * (int64_t)(OZ_TROWS * OZ_BK);  // elements
  void* __restrict__ tiles = op == 0 ? g.ta : g.tb;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int rl = rw + 16 * i;
    const int e = esc[rl];
    const int64_t at = tile0 * (OZ_TROWS * OZ_BK) + rl * OZ_BK + kp;  // element index of slice 0
    if constexpr (MODE == 0) {
      // at is even and tiles are 1 KB aligned: the pair is a 4-byte aligned store
      uint32_t* dst = reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_bfloat16*>(tiles) + at);
      oz_slice_pair<S>(v[i][0], v[i][1], e, dst, slice_stride / 2);
    } else {
      float h0, l0, h1, l1;
      tf32_split(v[i][0], e, h0, l0);
      tf32_split(v[i][1], e, h1, l1);
      float2* dst = reinterpret_cast<float2*>(reinterpret_cast<float*>(tiles) + at);
      dst[0] = make_float2(h0, h1);
      dst[slice_stride / 2] = make_float2(l0, l1);
    }
  }
}

// Scale and slice in one launch of thread-block clusters (4 or 8 CTAs, chosen per launch).  A
// group of g CTAs of one cluster (g set by the tile's depth, several groups per cluster when g is
// below the cluster size) owns one 128-row tile of one operand (rows of A~^c, columns of B~^c) and
// splits its k-chunks evenly among its CTAs.
//   1. Every CTA takes the maximum |x| of each of the 128 rows over its k-chunks (as FP64 bit
//      patterns, ordered as unsigned integers: no FP64 instruction).
//   2. After a cluster barrier every CTA reads the g partial maxima of its rows from its group's
//      shared memory (distributed shared memory), so all of them hold the row's power-of-two
//      scale 2^e > max_k |x| (the exponent of a maximum is the maximum of the exponents); the
//      group's first CTA writes it for the GEMM's epilogue.  A second cluster barrier keeps every
//      CTA's shared memory alive until the others have read it.
//   3. Every CTA slices its own k-chunks, re-reading them (now from L2).  In a launch with chunk
//      images (P.img, set per launch by the plan) step 1 also keeps the CTA's first two chunks in
//      shared memory, and step 3 slices those from there.
// The operands are read from HBM once instead of twice (a separate scale pass), and the scales
// need no initial fill.  The first CTA of each request also clears the GEMM's split-K counters.
template <int MODE, int NSEG, int S>
__global__ void __launch_bounds__(256, 3)
    k_oz_prep(const __grid_constant__ OzPrepT<NSEG> P) {
  extern __shared__ __align__(16) unsigned char prep_dyn[];
  PrepBuf* img = reinterpret_cast<PrepBuf*>(prep_dyn);  // P.img ? two chunk images : the staging buffer
  __shared__ unsigned long long pmax[OZ_TROWS];  // this CTA's maxima (read by the cluster)
  __shared__ unsigned long long half[OZ_TROWS];
  __shared__ int esc[OZ_TROWS];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  int64_t local;
  const OzPrepSeg& g = prep_seg(P, local);
  const int tid = threadIdx.x;
  if (local == 0)  // the GEMM's split-K arrival counters start at zero
    for (int i = tid; i < g.ncounters; i += blockDim.x) g.counters[i] = 0;
  const OzJob jb = g.jobs[local];
  if (jb.sector < 0) {  // an idle rank: it only takes part in the cluster's two barriers
    cluster.sync();
    cluster.sync();
    return;
  }
  const OzSector s = g.secs[jb.sector];
  const int op = jb.operand;
  const int64_t R = op == 0 ? s.M : s.N;
  const int64_t r0 = (int64_t)jb.r0 * OZ_TROWS;
  const int gr = rank - jb.gbase, gs = jb.gsize;  // this CTA's rank in its group, the group's size
  const int kc_lo = (int)((int64_t)gr * s.nkc / gs);
  const int kc_hi = (int)((int64_t)(gr + 1) * s.nkc / gs);
  const int nimg = P.img ? min(2, kc_hi - kc_lo) : 0;   // chunks kept in shared memory
  const int64_t k_lo = (int64_t)(kc_lo + nimg) * OZ_BK;  // the rest, read straight
  const int64_t k_hi = min(s.K, (int64_t)kc_hi * OZ_BK);
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  // ---- 1. partial maxima over this CTA's k range
  if (op == 0) {  // A~: rows contiguous; thread (row, half) walks every other column
    const int rl = tid & (OZ_TROWS - 1), h = tid >> 7;
    const int64_t m = r0 + rl;
    const bool mok = m < R;
    unsigned long long mb = 0;
    const long long* x = reinterpret_cast<const long long*>(g.A) + s.a_off + (mok ? m : 0);
    for (int c = 0; c < nimg; ++c) {  // image c: every (kk, row) written, zeros outside the sector
      const int64_t kb = (int64_t)(kc_lo + c) * OZ_BK + h;
#pragma unroll
      for (int j0 = 0; j0 < OZ_BK / 2; j0 += 8) {
        long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t k = kb + 2 * (j0 + u);
          v[u] = (mok && k < s.K) ? __ldg(x + k * s.M) : 0ll;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          mb = max(mb, (unsigned long long)v[u] & kAbs);
          img[c][h + 2 * (j0 + u)][rl] = __longlong_as_double(v[u]);
        }
      }
    }
    if (mok) {
      int64_t k = k_lo + h;
      for (; k + 14 < k_hi; k += 16) {  // eight independent loads in flight
        unsigned long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (unsigned long long)__ldg(x + (k + 2 * u) * s.M);
#pragma unroll
        for (int u = 0; u < 8; ++u) mb = max(mb, v[u] & kAbs);
      }
      for (; k < k_hi; k += 2) mb = max(mb, (unsigned long long)__ldg(x + k * s.M) & kAbs);
    }
    if (h == 1) half[rl] = mb;
    __syncthreads();
    if (h == 0) pmax[rl] = max(mb, half[rl]);
  } else {  // B~: columns contiguous along k; a warp takes four columns at a time, lanes along k
    const int warp = tid >> 5, lane = tid & 31;
    for (int cl0 = warp * 4; cl0 < OZ_TROWS; cl0 += 32) {
      const long long* x[4];
      bool nok[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        nok[u] = r0 + cl0 + u < R;
        x[u] = reinterpret_cast<const long long*>(g.B) + s.b_off + (nok[u] ? (r0 + cl0 + u) * s.K : 0);
      }
      unsigned long long mb[4] = {0, 0, 0, 0};
      for (int c = 0; c < nimg; ++c) {  // image c: lane = kk, column cl0 + u, zeros outside the sector
        const int64_t k = (int64_t)(kc_lo + c) * OZ_BK + lane;
        unsigned long long v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (nok[u] && k < s.K) ? (unsigned long long)__ldg(x[u] + k) : 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          mb[u] = max(mb[u], v[u] & kAbs);
          img[c][lane][cl0 + u] = __longlong_as_double((long long)v[u]);
        }
      }
      for (int64_t k = k_lo + lane; k < k_hi; k += 32) {  // four independent loads in flight
        unsigned long long v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = nok[u] ? (unsigned long long)__ldg(x[u] + k) : 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) mb[u] = max(mb[u], v[u] & kAbs);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          mb[u] = max(mb[u], (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mb[u], o));
      if (lane < 4) pmax[cl0 + lane] = lane == 0 ? mb[0] : lane == 1 ? mb[1] : lane == 2 ? mb[2] : mb[3];
    }
  }
  // ---- 2. the cluster's maxima -> the rows' scale exponents
  cluster.sync();
  if (tid < OZ_TROWS) {
    unsigned long long mb = pmax[tid];
    for (int q = 0; q < gs; ++q)
      if (q != gr) mb = max(mb, *cluster.map_shared_rank(&pmax[tid], jb.gbase + q));
    const int e = exponent_of(__longlong_as_double((long long)mb));
    if (gr == 0 && r0 + tid < R) (op == 0 ? g.sa + s.sa_off : g.sb + s.sb_off)[r0 + tid] = e;
    esc[tid] = e == kNoScale ? 0 : e;  // an all-zero row or column slices to zeros with any scale
  }
  cluster.sync();
  // ---- 3. slices of this CTA's k-chunks (the images were written before the cluster barriers);
  // a later chunk's A staging reuses image 1 after the slices of chunk 1 (its barrier orders them)
  for (int kc = kc_lo; kc < kc_hi; ++kc) {
    const int c = kc - kc_lo;
    if (c < nimg)
      slice_tile<MODE, S, true>(g, s, op, jb.r0, kc, esc, img[c]);
    else
      slice_tile<MODE, S, false>(g, s, op, jb.r0, kc, esc, img[nimg > 1 ? 1 : 0]);
  }
}

// ------------------------------------------------------------------ the persistent GEMM
// One request of a launch: its slice tiles (tensor maps over its workspace), tables and outputs.
// A launch serves NREQ requests of one (mode, tile width, slice count); each request's items are
// already spread over the CTAs (cta_work), and every CTA walks its share of each request in turn.
struct OzReq {
  CUtensorMap ma, mb;  // A and B slice tiles
  const OzSector* secs;
  const OzWork* work;
  const int32_t* cta_work;  // items of CTA b: work[cta_work[b] .. cta_work[b + 1]), b < ncta
  const int32_t* sa;
  const int32_t* sb;
  double* C;
  double* partials;
  int* counters;
  int32_t ncta, pad;
};
template <int NREQ>
struct OzBatchT {
  OzReq req[NREQ];
  int32_t nreq;
};
constexpr int OZ_BATCH = 32;  // requests per packed launch

struct OzSmem {
  uint64_t full[OZ_MAX_STAGES], empty[OZ_MAX_STAGES];
  uint64_t acc_full[2], acc_empty[2], drain;  // one or two TMEM buffers
  uint32_t tmem_base;
  int abort_flag;
};

// Shared memory: stages of [A_0 .. A_{s-1} | B_0 .. B_{s-1}] boxes (A 128 x 32, B BN x 32 elements
// of `row` bytes per 32), then OzSmem: as many stages as fit in 227 KB (at most four).
__host__ __device__ constexpr size_t oz_stage_bytes(int s, int bn, int row) {
  return (size_t)s * (OZ_BM + bn) * row;
}
__host__ __device__ constexpr int oz_stages(int s, int bn, int row) {
  return (int)((232448 - sizeof(OzSmem) - 1024) / oz_stage_bytes(s, bn, row)) < OZ_MAX_STAGES
             ? (int)((232448 - sizeof(OzSmem) - 1024) / oz_stage_bytes(s, bn, row))
             : OZ_MAX_STAGES;
}
__host__ __device__ constexpr size_t oz_smem_bytes(int s, int bn, int row) {
  return oz_stages(s, bn, row) * oz_stage_bytes(s, bn, row) + sizeof(OzSmem) + 1024;  // + alignment slack
}

// Every slice-pair MMA of one resident stage, unrolled for S slices: pairs grouped by
// accumulator level (0, 1, 2, >= 3); the first MMA of a level in a segment's first k-chunk
// overwrites its accumulator.  Descriptors differ from the stage's base descriptor only in the
// start-address field, so each operand offset is an added constant.
template <int S, int BN, int MODE>
__device__ __forceinline__ void oz_issue_stage(uint32_t acc0, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               bool first_kc) {
  using M = OzMode<MODE>;
  constexpr int B_BYTES = BN * M::ROW;
#pragma unroll
  for (int l = 0; l < OZ_NACC; ++l) {
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
      for (int j = 0; j < S - i; ++j) {
        // 3xTF32: every product into accumulator 0; Ozaki: level i + j (>= 3 together)
        const int lvl = MODE == 1 ? 0 : (i + j < OZ_NACC - 1 ? i + j : OZ_NACC - 1);
        if (lvl != l) continue;
        const bool first_of_level =
            MODE == 1 ? (i == 0 && j == 0) : ((l < OZ_NACC - 1) ? (i == 0) : (i == 0 && j == OZ_NACC - 1));
#pragma unroll
        for (int kk = 0; kk < M::MMAS; ++kk)
          tc_mma<MODE>(acc0 + l * BN, adesc + (uint64_t)((i * M::A_BYTES + kk * 32) >> 4),
                       bdesc + (uint64_t)((S * M::A_BYTES + j * B_BYTES + kk * 32) >> 4), idesc,
                       (first_kc && first_of_level && kk == 0) ? 0u : 1u);
      }
    }
  }
}

template <int BN, int MODE>
__device__ __forceinline__ void oz_issue(int s, uint32_t acc0, uint32_t sbase, uint32_t idesc, bool first_kc) {
  const uint64_t d = smem_desc_k<OzMode<MODE>::ROW>(sbase);
  if (MODE == 1) {  // the TF32 pair
    oz_issue_stage<2, BN, MODE>(acc0, d, d, idesc, first_kc);
    return;
  }
  switch (s) {
    case 2: oz_issue_stage<2, BN, MODE>(acc0, d, d, idesc, first_kc); break;
    case 3: oz_issue_stage<3, BN, MODE>(acc0, d, d, idesc, first_kc); break;
    case 4: oz_issue_stage<4, BN, MODE>(acc0, d, d, idesc, first_kc); break;
    case 5: oz_issue_stage<5, BN, MODE>(acc0, d, d, idesc, first_kc); break;
    case 6: oz_issue_stage<6, BN, MODE>(acc0, d, d, idesc, first_kc); break;
    default: oz_issue_stage<7, BN, MODE>(acc0, d, d, idesc, first_kc); break;
  }
}

// BN = 128: one TMEM buffer (4 x 128 columns), the MMAs wait for the epilogue between tiles;
// BN = 64: two buffers, the epilogue of one tile overlaps the MMAs of the next.
template <int BN, int MODE, int NREQ>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const __grid_constant__ OzBatchT<NREQ> L, const __grid_constant__ OzPairs pairs, int nslices,
              int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char* base = (unsigned char*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  constexpr int NBUF = OZ_TMEM_COLS / (OZ_NACC * BN);
  using MD = OzMode<MODE>;
  constexpr int B_BYTES = BN * MD::ROW;
  constexpr int SUB = OZ_TROWS / BN;  // B boxes per 128-row slice tile
  const uint32_t stage_bytes = (uint32_t)oz_stage_bytes(nslices, BN, MD::ROW);
  const uint32_t nstages = (uint32_t)oz_stages(nslices, BN, MD::ROW);
  const uint32_t b_off = (uint32_t)nslices * MD::A_BYTES;  // B boxes follow the A boxes in a stage
  OzSmem* ss = reinterpret_cast<OzSmem*>(base + nstages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &ss->abort_flag;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&ss->full[s]), 1);
      mbar_init(smem_u32(&ss->empty[s]), 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&ss->acc_full[b]), 1);
      mbar_init(smem_u32(&ss->acc_empty[b]), OZ_EPI_WARPS);
    }
    mbar_init(smem_u32(&ss->drain), 1);
    ss->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ss->tmem_base)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ss->tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int r = 0; r < L.nreq && !*abort_flag; ++r) {
        const OzReq& R = L.req[r];
        if ((int)blockIdx.x >= R.ncta) continue;  // this request has fewer work lists than CTAs
        const int w_begin = R.cta_work[blockIdx.x], w_end = R.cta_work[blockIdx.x + 1];  // this CTA's items
        const OzSector* __restrict__ secs = R.secs;
        const OzWork* __restrict__ work = R.work;
        for (int w = w_begin; w < w_end && !*abort_flag; ++w) {
          const OzWork wk = work[w];
          const OzSector s = secs[wk.sector];
          // slice tiles hold 128 rows; this item's B box is part nt % SUB of tile nt / SUB
          const int64_t ta0 = s.ta_base + (int64_t)wk.mt * s.nkc, tb0 = s.tb_base + (int64_t)(wk.nt / SUB) * s.nkc;
          const int32_t brow = (wk.nt % SUB) * BN;
          const int64_t sa_str = (int64_t)s.nmt * s.nkc, sb_str = (int64_t)s.nnt * s.nkc;  // tiles per slice
          for (int kc = wk.kc_lo; kc < wk.kc_hi && !*abort_flag; ++kc, ++it) {
            const uint32_t st = it % nstages, ph = (it / nstages) & 1;
            if (!mbar_wait(smem_u32(&ss->empty[st]), ph ^ 1, abort_flag)) break;
            const uint32_t fb = smem_u32(&ss->full[st]);
            mbar_expect_tx(fb, stage_bytes);
            const uint32_t dst = smem_u32(base + st * stage_bytes);
            for (int i = 0; i < nslices; ++i)
              tma_load_2d(dst + i * MD::A_BYTES, &R.ma, 0, (int32_t)((ta0 + i * sa_str + kc) * OZ_TROWS), fb);
            for (int j = 0; j < nslices; ++j)
              tma_load_2d(dst + b_off + j * B_BYTES, &R.mb, 0,
                          (int32_t)((tb0 + j * sb_str + kc) * OZ_TROWS + brow), fb);
          }
        }
      }
      // drain: every issued stage must have landed before this CTA may exit (bounded)
      for (uint32_t k = (it > nstages ? it - nstages : 0); k < it; ++k) {
        volatile int never = 0;
        mbar_wait(smem_u32(&ss->full[k % nstages]), (k / nstages) & 1, &never);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, seg = 0;
      for (int r = 0; r < L.nreq && !*abort_flag; ++r) {
        const OzReq& R = L.req[r];
        if ((int)blockIdx.x >= R.ncta) continue;  // this request has fewer work lists than CTAs
        const int w_begin = R.cta_work[blockIdx.x], w_end = R.cta_work[blockIdx.x + 1];  // this CTA's items
        const OzWork* __restrict__ work = R.work;
        for (int w = w_begin; w < w_end && !*abort_flag; ++w) {
          const OzWork wk = work[w];
          const uint32_t idesc = idesc_mma<MODE>(OZ_BM, wk.nw);
          for (int kc0 = wk.kc_lo; kc0 < wk.kc_hi && !*abort_flag; kc0 += OZ_SEG_KC, ++seg) {
            const int kc1 = min(wk.kc_hi, kc0 + OZ_SEG_KC);
            const uint32_t buf = seg % NBUF;
            if (!mbar_wait(smem_u32(&ss->acc_empty[buf]), ((seg / NBUF) & 1) ^ 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t acc0 = tmem + buf * (OZ_NACC * BN);
            for (int kc = kc0; kc < kc1; ++kc, ++it) {
              const uint32_t st = it % nstages, ph = (it / nstages) & 1;
              if (!mbar_wait(smem_u32(&ss->full[st]), ph, abort_flag)) break;
              tc_fence_after();
              oz_issue<BN, MODE>(nslices, acc0, smem_u32(base + st * stage_bytes), idesc, kc == kc0);
              tc_commit(smem_u32(&ss->empty[st]));  // frees the stage once these MMAs are done
            }
            tc_commit(smem_u32(&ss->acc_full[buf]));  // accumulators of this (item, segment) complete
          }
        }
      }
      // make sure no MMA is still running before TMEM is released (bounded)
      tc_commit(smem_u32(&ss->drain));
      volatile int never = 0;
      mbar_wait(smem_u32(&ss->drain), 0, &never);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..17)
    constexpr int WCOLS = BN / 4;              // columns per warp: four warps per lane quadrant
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
    const int grp = (warp - 2) >> 2;           // which quarter of the tile's columns
    const int row = quad * 32 + lane;
    // accumulators of levels without any slice pair (fewer than 4 slices) are never written
    const bool has1 = pairs.first[1] >= 0, has2 = pairs.first[2] >= 0, has3 = pairs.first[3] >= 0;
    const bool all_levels = has1 && has2 && has3;
    uint32_t seg = 0;
    for (int r = 0; r < L.nreq && !*abort_flag; ++r) {
      const OzReq& R = L.req[r];
      if ((int)blockIdx.x >= R.ncta) continue;  // this request has fewer work lists than CTAs
      const int w_begin = R.cta_work[blockIdx.x], w_end = R.cta_work[blockIdx.x + 1];  // this CTA's items
      const OzSector* __restrict__ secs = R.secs;
      const OzWork* __restrict__ work = R.work;
      const int32_t* __restrict__ scale_a = R.sa;
      const int32_t* __restrict__ scale_b = R.sb;
      double* __restrict__ C = R.C;
      double* __restrict__ partials = R.partials;
      int* __restrict__ counters = R.counters;
      for (int w = w_begin; w < w_end && !*abort_flag; ++w) {
        const OzWork wk = work[w];
        const OzSector s = secs[wk.sector];
        const int c0 = grp * WCOLS;                 // first column of this warp within the tile
        const bool active = c0 < wk.nw;             // warp-uniform
        const int64_t m = (int64_t)wk.mt * OZ_BM + row;
        const bool row_ok = m < s.M;
        int em = row_ok ? scale_a[s.sa_off + m] : 0;
        if (em == kNoScale) em = 0;
        const int64_t nb = (int64_t)wk.nt * BN + c0;
        const int64_t left = s.N - nb;
        const int ncols = left < WCOLS ? (int)left : WCOLS;  // valid columns of this warp (may be <= 0)
        int fl = (lane < ncols) ? scale_b[s.sb_off + nb + lane] : 0;  // WCOLS <= 32: one per lane
        if (fl == kNoScale) fl = 0;
        // the fast chunk body: all levels present, every scale of the warp within +-448, and the
        // warp's 32 x WCOLS part of the tile wholly inside the block (no row or column checks)
        const bool fast = all_levels && ncols >= WCOLS &&
                          __all_sync(0xffffffffu, row_ok && em >= -448 && em <= 448 && fl >= -448 && fl <= 448);
        const uint32_t kem = (uint32_t)(896 + em) << 20, kfl = (uint32_t)fl << 20;  // exponent-field parts
        // a split tile's parts go to its partial buffers (column-major 128 x BN, one per part)
        const bool split = wk.nparts > 1;
        double* const pbase = split ? partials + (int64_t)wk.slot * OZ_MAX_PARTS * (OZ_BM * BN) : nullptr;
        double* crow = split ? pbase + (int64_t)wk.part * (OZ_BM * BN) + (int64_t)c0 * OZ_BM + row
                             : C + s.c_off + nb * s.M + m;
        const int64_t ld = split ? OZ_BM : s.M;
        bool done = true;
        for (int kc0 = wk.kc_lo; kc0 < wk.kc_hi; kc0 += OZ_SEG_KC, ++seg) {
          const uint32_t buf = seg % NBUF;
          if (!mbar_wait(smem_u32(&ss->acc_full[buf]), (seg / NBUF) & 1, abort_flag, true)) {
            done = false;
            break;
          }
          tc_fence_after();
          if (active) {
            const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16) + buf * (OZ_NACC * BN) + c0;
            // one chunk of eight columns; FAST: every level accumulator was written (four or more
            // slices), every row and column scale of this warp is within +-448 and its part of the
            // tile is whole, so no level is masked, no output can leave the normal FP64 range
            // through its scale and no output needs a bounds check
            auto chunk = [&](auto fast_tag, int ch) {
              constexpr bool FAST = decltype(fast_tag)::value;
              uint32_t r0[8], r1[8], r2[8], r3[8];
              tc_ld8(lane_addr + 0 * BN + ch * 8, r0);
              tc_ld8(lane_addr + 1 * BN + ch * 8, r1);
              tc_ld8(lane_addr + 2 * BN + ch * 8, r2);
              tc_ld8(lane_addr + 3 * BN + ch * 8, r3);
              tc_wait_ld();
              // level sums, two columns per instruction: hi + lo = r0 + r1 + r2 + r3, the exact
              // levels' two-sum remainders and the inexact level r3 gathered in lo, and a last
              // two-sum leaving |lo| <= ulp(hi) / 2 for the conversion below
              float hv[8], lv[8];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float2 z = make_float2(0.f, 0.f);
                const float2 x0 = make_float2(__uint_as_float(r0[2 * q]), __uint_as_float(r0[2 * q + 1]));
                const float2 y1 = make_float2(__uint_as_float(r1[2 * q]), __uint_as_float(r1[2 * q + 1]));
                const float2 y2 = make_float2(__uint_as_float(r2[2 * q]), __uint_as_float(r2[2 * q + 1]));
                const float2 y3 = make_float2(__uint_as_float(r3[2 * q]), __uint_as_float(r3[2 * q + 1]));
                const float2 x1 = (FAST || has1) ? y1 : z;
                const float2 x2 = (FAST || has2) ? y2 : z;
                const float2 x3 = (FAST || has3) ? y3 : z;
                float2 hi, lo, e1;
                two_sum2(x0, x1, hi, lo);
                two_sum2(hi, x2, hi, e1);
                lo = __fadd2_rn(__fadd2_rn(lo, e1), x3);
                two_sum2(hi, lo, hi, lo);
                hv[2 * q] = hi.x;
                hv[2 * q + 1] = hi.y;
                lv[2 * q] = lo.x;
                lv[2 * q + 1] = lo.y;
              }
              double* dst = crow + (int64_t)(ch * 8) * ld;
#pragma unroll
              for (int j = 0; j < 8; ++j, dst += ld) {
                const float hi = hv[j], lo = lv[j];
                bool ok;
                double v;
                if constexpr (FAST) {
                  const uint32_t kfn = (uint32_t)__shfl_sync(0xffffffffu, (int)kfl, ch * 8 + j);
                  v = f32_pair_scaled<true>(hi, lo, 0, kem + kfn, ok);
                  if (!ok) v = f32_pair_scaled_slow(hi, lo, em + ((int)kfn >> 20));
                } else {
                  const int fn = __shfl_sync(0xffffffffu, fl, ch * 8 + j);
                  if (!row_ok || ch * 8 + j >= ncols) continue;
                  const int sc = em + fn;
                  v = f32_pair_scaled<false>(hi, lo, sc, (uint32_t)(896 + sc) << 20, ok);
                  if (!ok) v = f32_pair_scaled_slow(hi, lo, sc);
                }
                *dst = (kc0 == wk.kc_lo) ? v : *dst + v;
              }
            };
#pragma unroll 1
            for (int ch = 0; ch < WCOLS / 8; ++ch) {
              if (ch * 8 >= ncols) break;  // warp-uniform
              if (fast)
                chunk(std::true_type{}, ch);
              else
                chunk(std::false_type{}, ch);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&ss->acc_empty[buf]));
        }
        if (split && done && active) {
          // the warp that completes this region of the tile last adds the parts in part order
          __threadfence();
          __syncwarp();
          int* cnt = counters + (int64_t)wk.slot * OZ_EPI_WARPS + (warp - 2);
          int last = 0;
          if (lane == 0) last = atomicAdd(cnt, 1) == wk.nparts - 1;
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last) {
            __threadfence();
            if (row_ok) {
              const double* src = pbase + (int64_t)c0 * OZ_BM + row;
              double* out = C + s.c_off + nb * s.M + m;
              for (int j = 0; j < ncols; ++j, src += OZ_BM, out += s.M) {
                double v = __ldcg(src);
                for (int p = 1; p < wk.nparts; ++p) v += __ldcg(src + (int64_t)p * (OZ_BM * BN));
                *out = v;
              }
            }
            if (lane == 0) *cnt = 0;  // ready for the next launch
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (ss->abort_flag && threadIdx.x == 0) {
    atomicExch(status, 1);
    atomicExch(status + 1, 3);  // kernel tag: split-precision GEMM
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
  }
}

// Failure-path check of the bounded waits: one mbarrier that expects an arrival nobody makes,
// waited on by the same bounded wait the GEMM pipeline uses.  The wait gives up after its limit,
// the kernel records the timeout in the context's status word (tag 9) and returns; nothing is in
// flight and no TMEM is held, so the context stays usable.
__global__ void k_wait_selftest(int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, &abort_flag, true)) {
    atomicExch(status, 1);
    atomicExch(status + 1, 9);  // kernel tag: wait self-test
  }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D view [ntiles * 128 rows][32 elements] with box_rows x 32 boxes: BF16 with 64-byte swizzle
// (mode 0) or FP32 with 128-byte swizzle (mode 1).
int make_tile_map(CUtensorMap* map, void* base, int64_t ntiles, int box_rows, int mode) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return TK_ERR_CUDA;
  const int esz = mode == 0 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)OZ_BK, (cuuint64_t)(ntiles * OZ_TROWS)};
  cuuint64_t strides[1] = {(cuuint64_t)OZ_BK * esz};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  mode == 0 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TK_OK : TK_ERR_CUDA;
}

template <int BN, int MODE>
int set_smem_attr() {
  size_t most = 0;  // the largest need over every slice count this kernel accepts
  for (int sl = 2; sl <= OZ_MAX_SLICES; ++sl) most = std::max(most, oz_smem_bytes(sl, BN, OzMode<MODE>::ROW));
  return cudaFuncSetAttribute(k_oz_gemm<BN, MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) ==
                     cudaSuccess &&
                 cudaFuncSetAttribute(k_oz_gemm<BN, MODE, OZ_BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)most) == cudaSuccess
             ? TK_OK
             : TK_ERR_CUDA;
}

size_t al1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

// The k_oz_prep CTAs of one request.  A tile nkc k-chunks deep takes g = min(ceil(nkc / cpt), 8)
// CTAs of one cluster (cpt k-chunks or more each, cpt set by the launch's size): a shallow tile
// spread over a whole cluster would leave most of its CTAs without work, and the launch would run
// in many short waves.  Tiles go into clusters
// of OZ_PREP_CLUSTER CTAs deepest first, each into the open cluster with the least room that still
// holds it (best fit decreasing); the ranks a cluster leaves free become idle entries.
std::vector<OzJob> pack_prep_tiles(std::vector<OzJob> tiles, int csize) {
  std::stable_sort(tiles.begin(), tiles.end(), [](const OzJob& a, const OzJob& b) { return a.gsize > b.gsize; });
  std::vector<std::vector<OzJob>> clusters;
  std::vector<int> used;
  std::vector<int> open[OZ_PREP_CLUSTER];  // open[r]: clusters with r free ranks, 0 < r < csize
  for (OzJob t : tiles) {
    int c = -1;
    for (int r = t.gsize; r < csize && c < 0; ++r)
      if (!open[r].empty()) {
        c = open[r].back();
        open[r].pop_back();
      }
    if (c < 0) {
      c = (int)clusters.size();
      clusters.emplace_back();
      used.push_back(0);
    }
    t.gbase = (int16_t)used[(size_t)c];
    clusters[(size_t)c].push_back(t);
    used[(size_t)c] += t.gsize;
    const int left = csize - used[(size_t)c];
    if (left > 0) open[left].push_back(c);
  }
  std::vector<OzJob> ctas;
  ctas.reserve(clusters.size() * csize);
  for (size_t c = 0; c < clusters.size(); ++c) {
    for (const OzJob& t : clusters[c])
      for (int q = 0; q < t.gsize; ++q) ctas.push_back(t);
    for (int q = used[c]; q < csize; ++q) ctas.push_back(OzJob{-1, 0, 0, 0, 1});
  }
  return ctas;
}

}  // namespace

int upload_ozaki_tables(Ctx* ctx, ContractPlan& cp) {
  auto L = std::make_shared<OzLayout>();
  L->mode = cp.gemm_mode == TK_GEMM_TF32X3 ? 1 : 0;
  L->slices = L->mode == 1 ? 2 : (cp.slices > 0 ? cp.slices : OZ_DEFAULT_SLICES);
  if (L->slices < 2 || L->slices > OZ_MAX_SLICES) return TK_ERR_ARG;
  const size_t tile_bytes = (size_t)OZ_TROWS * OZ_BK * (L->mode == 0 ? 2 : 4);
  // pair list ordered by accumulator level
  OzPairs& P = L->pairs;
  std::memset(&P, 0, sizeof(P));
  for (int l = 0; l < OZ_NACC; ++l) P.first[l] = -1;
  for (int lvl = 0; lvl < OZ_NACC; ++lvl)
    for (int i = 0; i < L->slices; ++i)
      for (int j = 0; j < L->slices - i; ++j) {
        const int l = L->mode == 1 ? 0 : std::min(i + j, OZ_NACC - 1);  // 3xTF32: one accumulator
        if (l != lvl) continue;
        if (P.first[l] < 0) P.first[l] = P.n;
        P.i[P.n] = (int8_t)i;
        P.j[P.n] = (int8_t)j;
        P.lvl[P.n] = (int8_t)l;
        ++P.n;
      }
  std::vector<OzWork> work;
  std::vector<OzJob> prep_jobs, prep_tiles;
  int64_t prep_chunks = 0;
  std::vector<std::pair<double, OzWork>> wcost;
  // Tile width: measured in this kernel, a 128 x 64 x 16 MMA takes ~72 cycles and a 128 x 128 x 16
  // one ~65 (the full rate), so 128-column tiles do nearly twice the work per cycle; but they hold
  // all of TMEM, so their epilogue (~12k cycles a tile) stalls the MMAs.  They pay off once a tile
  // has a few k-chunks (average inner dimension of 128 or more).
  {
    double kw = 0, w = 0;
    for (const GemmItem& it : cp.gemms_oz) {
      const double area = (double)((it.M + OZ_BM - 1) / OZ_BM) * ((it.N + 127) / 128);
      kw += area * (double)it.K;
      w += area;
    }
    L->bn = (w > 0 && kw / w >= 128.0) ? OZ_BN_WIDE : OZ_BN_NARROW;
    if (cp.tune_oz_bn == OZ_BN_WIDE || cp.tune_oz_bn == OZ_BN_NARROW) L->bn = cp.tune_oz_bn;
  }
  const int bn = L->bn;
  for (size_t g = 0; g < cp.gemms_oz.size(); ++g) {
    const GemmItem& it = cp.gemms_oz[g];
    OzSector s;
    std::memset(&s, 0, sizeof(s));
    s.M = it.M;
    s.N = it.N;
    s.K = it.K;
    s.a_off = it.a_off;
    s.b_off = it.b_off;
    s.c_off = it.c_off;
    s.nmt = (int32_t)((it.M + OZ_TROWS - 1) / OZ_TROWS);  // 128-row slice tiles of A~ and of B~^T
    s.nnt = (int32_t)((it.N + OZ_TROWS - 1) / OZ_TROWS);
    s.nkc = (int32_t)((it.K + OZ_BK - 1) / OZ_BK);
    s.ta_base = L->ntiles_a;
    s.tb_base = L->ntiles_b;
    s.sa_off = L->nrows_a;
    s.sb_off = L->ncols_b;
    L->ntiles_a += (int64_t)L->slices * s.nmt * s.nkc;
    L->ntiles_b += (int64_t)L->slices * s.nnt * s.nkc;
    L->nrows_a += s.M;
    L->ncols_b += s.N;
    const int32_t sid = (int32_t)L->sectors.size();
    L->sectors.push_back(s);
    for (int mt = 0; mt < s.nmt; ++mt)
      for (int nt = 0; nt < (int)((s.N + bn - 1) / bn); ++nt) {  // bn-column output tiles
        const int64_t left = s.N - (int64_t)nt * bn;
        const int32_t nw = (int32_t)std::min<int64_t>(bn, (left + 15) / 16 * 16);
        // cost key: the tile depth only, so the column tiles of one row tile (which share its A
        // slices) stay adjacent in the list and run at the same time
        OzWork t;
        std::memset(&t, 0, sizeof(t));
        t.sector = sid;
        t.mt = mt;
        t.nt = nt;
        t.nw = nw;
        wcost.push_back({(double)s.nkc, t});
      }
    // the prep tiles: every 128-row tile of A~ and 128-column tile of B~ (group sizes below)
    for (int rt = 0; rt < s.nmt; ++rt) prep_tiles.push_back(OzJob{sid, 0, rt, 0, 1});
    for (int rt = 0; rt < s.nnt; ++rt) prep_tiles.push_back(OzJob{sid, 1, rt, 0, 1});
    prep_chunks += (int64_t)(s.nmt + s.nnt) * s.nkc;
  }
  {
    // k-chunks per prep CTA: one while the launch has fewer than two waves' worth of chunks (at
    // three CTAs per SM), up to three for large launches, where fewer and longer-lived CTAs lose
    // less to the per-CTA latency (job tables, two cluster barriers, first loads)
    const int64_t wave = 3 * (int64_t)std::max(ctx->num_sms, 1);
    const int cpt = (int)std::max<int64_t>(1, std::min<int64_t>(3, prep_chunks / (2 * wave)));
    // clusters of 4 where no tile needs more (or the launch is large): they pack into more of
    // the SMs (at most 51 clusters of 8 are resident on this part); else of 8, so that deep tiles
    // of small launches keep eight CTAs
    int maxg = 1;
    for (const OzJob& t : prep_tiles) {
      const int nkc = L->sectors[(size_t)t.sector].nkc;
      maxg = std::max(maxg, std::min((nkc + cpt - 1) / cpt, OZ_PREP_CLUSTER));
    }
    L->prep_cluster = (cpt >= 2 || maxg <= 4) ? 4 : OZ_PREP_CLUSTER;
    // chunk images (the first two chunks of each CTA kept in shared memory): measured faster for
    // launches at one or two chunks per CTA and slower at three, where they cover a small part of
    // a CTA's chunks.  A contraction whose double-float rows (on the second stream, beside this
    // launch and the GEMM) move more than half the bytes the preparation reads measured slower as
    // a whole with them (66 KB of shared memory per CTA leaves less room for the rows' CTAs).
    // The default takes the launches at two chunks per CTA with light rows; the autotuner tries
    // both settings.
    double rows_bytes = 0;
    for (const GemmItem& it : cp.gemms_fp64) rows_bytes += 8.0 * (double)it.M * (double)(it.K + it.N);
    const double prep_bytes = 8.0 * (double)prep_chunks * (OZ_TROWS * OZ_BK);
    L->prep_img = cp.tune_oz_img == 2   ? true
                  : cp.tune_oz_img == 1 ? false
                                        : cpt == 2 && 2.0 * rows_bytes < prep_bytes;
    for (OzJob& t : prep_tiles) {
      const int nkc = L->sectors[(size_t)t.sector].nkc;
      t.gsize = (int16_t)std::min((nkc + cpt - 1) / cpt, L->prep_cluster);
    }
  }
  prep_jobs = pack_prep_tiles(prep_tiles, L->prep_cluster);
  std::stable_sort(wcost.begin(), wcost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  // Split-K: a launch with fewer than two tiles per SM cuts deep tiles into up to OZ_MAX_PARTS
  // parts (at least 8 k-chunks each); their FP64 partial tiles are added in part order by the
  // warps that finish last.
  const int64_t sms = std::max(ctx->num_sms, 1);
  const int64_t ntiles = (int64_t)wcost.size();
  int64_t want = ntiles >= 2 * sms ? 1 : (2 * sms + ntiles - 1) / std::max<int64_t>(ntiles, 1);
  if (cp.tune_oz_split == 1) want = 1;
  if (cp.tune_oz_split == 2) want = OZ_MAX_PARTS;
  int32_t nslots = 0;
  for (auto& w : wcost) {
    OzWork t = w.second;
    const int nkc = L->sectors[t.sector].nkc;
    const int np = (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)OZ_MAX_PARTS, nkc / 8}));
    t.nparts = np;
    t.slot = np > 1 ? nslots++ : -1;
    for (int p = 0; p < np; ++p) {
      t.part = p;
      t.kc_lo = (int32_t)((int64_t)p * nkc / np);
      t.kc_hi = (int32_t)((int64_t)(p + 1) * nkc / np);
      work.push_back(t);
    }
  }
  L->nslots = nslots;
  // Static schedule: items go, longest first, to the CTA with the least work so far (LPT), the
  // cost being the item's MMAs at max(48, N/2) cycles each (a 128 x N x K-step MMA is bound by
  // shared-memory operand reads below N = 96) plus its epilogues.  Each CTA then runs its items
  // in that order, so at any time the CTAs work on items of similar rank (L2 reuse of slices).
  {
    const int mmas = L->pairs.n * (L->mode == 0 ? OzMode<0>::MMAS : OzMode<1>::MMAS);
    const int ncta = (int)std::min<int64_t>((int64_t)work.size(), sms);
    std::vector<std::pair<double, int>> cost;
    cost.reserve(work.size());
    for (size_t k = 0; k < work.size(); ++k) {
      const OzWork& x = work[k];
      const int nkc = x.kc_hi - x.kc_lo, nseg = (nkc + OZ_SEG_KC - 1) / OZ_SEG_KC;
      cost.push_back({(double)nkc * mmas * std::max(48.0, x.nw / 2.0) + 50.0 * x.nw * nseg, (int)k});
    }
    std::stable_sort(cost.begin(), cost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<std::vector<int>> lists((size_t)ncta);
    std::vector<std::pair<double, int>> heap;  // (load, cta), a min-heap
    for (int b = 0; b < ncta; ++b) heap.push_back({0.0, b});
    auto later = [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
      return a.first != b.first ? a.first > b.first : a.second > b.second;
    };
    std::make_heap(heap.begin(), heap.end(), later);
    for (const auto& c : cost) {
      std::pop_heap(heap.begin(), heap.end(), later);
      heap.back().first += c.first;
      lists[(size_t)heap.back().second].push_back(c.second);
      std::push_heap(heap.begin(), heap.end(), later);
    }
    std::vector<OzWork> ordered;
    ordered.reserve(work.size());
    L->cta_work.assign((size_t)ncta + 1, 0);
    for (int b = 0; b < ncta; ++b) {
      L->cta_work[(size_t)b] = (int32_t)ordered.size();
      for (int k : lists[(size_t)b]) ordered.push_back(work[(size_t)k]);
    }
    L->cta_work[(size_t)ncta] = (int32_t)ordered.size();
    L->ncta = ncta;
    work.swap(ordered);
  }
  L->nwork = (int64_t)work.size();
  L->nprep_ctas = (int64_t)prep_jobs.size();
  // workspace layout: A tiles | B tiles | row scales | column scales | split-K partial tiles
  L->off_ta = 0;
  L->off_tb = al1k((size_t)L->ntiles_a * tile_bytes);
  L->off_sa = L->off_tb + al1k((size_t)L->ntiles_b * tile_bytes);
  L->off_sb = L->off_sa + al1k((size_t)L->nrows_a * 4);
  L->off_part = L->off_sb + al1k((size_t)L->ncols_b * 4);
  L->off_cnt = L->off_part + al1k((size_t)nslots * OZ_MAX_PARTS * OZ_BM * bn * sizeof(double));
  L->bytes = L->off_cnt + al1k((size_t)nslots * OZ_EPI_WARPS * sizeof(int));
  int rc = TK_OK;
  if (!L->sectors.empty()) {
    if ((rc = dev_upload(ctx, (void**)&L->d_sectors, L->sectors.data(), L->sectors.size() * sizeof(OzSector))) != TK_OK ||
        (rc = dev_upload(ctx, (void**)&L->d_work, work.data(), work.size() * sizeof(OzWork))) != TK_OK ||
        (rc = dev_upload(ctx, (void**)&L->d_prep_jobs, prep_jobs.data(), prep_jobs.size() * sizeof(OzJob))) != TK_OK ||
        (rc = dev_upload(ctx, (void**)&L->d_cta_work, L->cta_work.data(), L->cta_work.size() * sizeof(int32_t))) != TK_OK)
      return rc;
  }
  cp.d_oz = {L->d_sectors, L->d_work, L->d_prep_jobs, L->d_cta_work};
  cp.oz_nwork = L->nwork;
  cp.oz_bytes = L->bytes;
  cp.oz = L;
  return TK_OK;
}

namespace {
template <typename K>
bool prep_attr(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_PREP_SMEM_IMG) ==
         cudaSuccess;
}
template <int NSEG>
int set_prep_attrs() {
  return prep_attr(k_oz_prep<1, NSEG, 2>) && prep_attr(k_oz_prep<0, NSEG, 2>) && prep_attr(k_oz_prep<0, NSEG, 3>) &&
                 prep_attr(k_oz_prep<0, NSEG, 4>) && prep_attr(k_oz_prep<0, NSEG, 5>) &&
                 prep_attr(k_oz_prep<0, NSEG, 6>) && prep_attr(k_oz_prep<0, NSEG, 7>)
             ? TK_OK
             : TK_ERR_CUDA;
}
int ensure_smem_attrs(Ctx* ctx) {
  static bool attr_set[64] = {false};
  if (ctx->device < 64 && !attr_set[ctx->device]) {
    if (set_smem_attr<OZ_BN_WIDE, 0>() != TK_OK || set_smem_attr<OZ_BN_NARROW, 0>() != TK_OK ||
        set_smem_attr<OZ_BN_WIDE, 1>() != TK_OK || set_smem_attr<OZ_BN_NARROW, 1>() != TK_OK ||
        set_prep_attrs<1>() != TK_OK || set_prep_attrs<OZ_BATCH>() != TK_OK) {
      ctx->last_error = "cannot reserve shared memory for the split-precision GEMM";
      return TK_ERR_CUDA;
    }
    attr_set[ctx->device] = true;
  }
  return TK_OK;
}

// Describe one request for the prep launch and the GEMM launch.
int describe_ozaki_request(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                           OzPrepSeg& P, OzReq& R) {
  const OzLayout* L = static_cast<const OzLayout*>(cp.oz.get());
  if (((uintptr_t)ws & 15) != 0) {
    ctx->last_error = "split-precision workspace must be 16-byte aligned";
    return TK_ERR_WORKSPACE;
  }
  char* w = (char*)ws;
  void* ta = w + L->off_ta;
  void* tb = w + L->off_tb;
  int32_t* sa = (int32_t*)(w + L->off_sa);
  int32_t* sb = (int32_t*)(w + L->off_sb);
  std::memset(&R, 0, sizeof(R));
  if (make_tile_map(&R.ma, ta, L->ntiles_a, OZ_BM, L->mode) != TK_OK ||
      make_tile_map(&R.mb, tb, L->ntiles_b, L->bn, L->mode) != TK_OK) {
    ctx->last_error = "cuTensorMapEncodeTiled failed";
    return TK_ERR_CUDA;
  }
  int* counters = (int*)(w + L->off_cnt);  // cleared by k_oz_prep
  std::memset(&P, 0, sizeof(P));
  P.secs = L->d_sectors;
  P.A = (const double*)a;
  P.B = (const double*)b;
  P.sa = sa;
  P.sb = sb;
  P.counters = counters;
  P.ncounters = (int32_t)(L->nslots * OZ_EPI_WARPS);
  P.ta = ta;
  P.tb = tb;
  R.secs = L->d_sectors;
  R.work = L->d_work;
  R.cta_work = L->d_cta_work;
  R.sa = sa;
  R.sb = sb;
  R.C = (double*)c;
  R.partials = (double*)(w + L->off_part);
  R.counters = counters;
  R.ncta = L->ncta;
  return TK_OK;
}

// Scale and slice the operands of every request of one batch: one launch of k_oz_prep clusters.
template <int NSEG>
int launch_oz_prep(Ctx* ctx, const OzLayout* const* lay, OzPrepT<NSEG>& P, int mode, int nslices, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int64_t blocks = 0;
  P.img = 1;  // chunk images only if every request of the launch asks for them
  for (int i = 0; i < P.nseg; ++i) {  // every segment starts on a cluster boundary
    P.seg[i].block0 = blocks;
    P.seg[i].jobs = lay[i]->d_prep_jobs;
    blocks += lay[i]->nprep_ctas;
    if (!lay[i]->prep_img) P.img = 0;
  }
  if (blocks == 0) return TK_OK;
  ProfScope prof(ctx, "k_oz_prep", stream);
  // a thread-block-cluster launch: every segment's CTA list is a whole number of clusters of the
  // launch's size (the requests of one launch share it)
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = P.img ? OZ_PREP_SMEM_IMG : OZ_PREP_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  std::memset(&attr, 0, sizeof(attr));
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)lay[0]->prep_cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (mode == 1) {
    e = cudaLaunchKernelEx(&cfg, k_oz_prep<1, NSEG, 2>, P);
  } else {
    switch (nslices) {
      case 2: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 2>, P); break;
      case 3: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 3>, P); break;
      case 4: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 4>, P); break;
      case 5: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 5>, P); break;
      case 6: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 6>, P); break;
      default: e = cudaLaunchKernelEx(&cfg, k_oz_prep<0, NSEG, 7>, P); break;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string("k_oz_prep launch: ") + cudaGetErrorString(e);
    return TK_ERR_CUDA;
  }
  ctx->launches += 1;
  return TK_OK;
}

template <int NREQ>
int launch_oz_gemm(Ctx* ctx, const OzLayout* L, const OzBatchT<NREQ>& B, int grid, void* stream) {
  const size_t smem = oz_smem_bytes(L->slices, L->bn, L->mode == 0 ? OzMode<0>::ROW : OzMode<1>::ROW);
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope prof(ctx, "k_oz_gemm", stream);
  if (L->mode == 0) {
    if (L->bn == OZ_BN_WIDE)
      k_oz_gemm<OZ_BN_WIDE, 0, NREQ><<<grid, OZ_THREADS, smem, s>>>(B, L->pairs, L->slices, ctx->d_status);
    else
      k_oz_gemm<OZ_BN_NARROW, 0, NREQ><<<grid, OZ_THREADS, smem, s>>>(B, L->pairs, L->slices, ctx->d_status);
  } else {
    if (L->bn == OZ_BN_WIDE)
      k_oz_gemm<OZ_BN_WIDE, 1, NREQ><<<grid, OZ_THREADS, smem, s>>>(B, L->pairs, L->slices, ctx->d_status);
    else
      k_oz_gemm<OZ_BN_NARROW, 1, NREQ><<<grid, OZ_THREADS, smem, s>>>(B, L->pairs, L->slices, ctx->d_status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string("k_oz_gemm launch: ") + cudaGetErrorString(e);
    return TK_ERR_CUDA;
  }
  ctx->launches += 1;
  return TK_OK;
}
}  // namespace

int launch_gemm_ozaki(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                      void* stream) {
  const OzLayout* L = static_cast<const OzLayout*>(cp.oz.get());
  if (!L) {
    ctx->last_error = "split-precision tables missing";
    return TK_ERR_UNSUPPORTED;
  }
  if (L->nwork == 0) return TK_OK;
  int rc = ensure_smem_attrs(ctx);
  if (rc != TK_OK) return rc;
  OzBatchT<1> B;
  OzPrepT<1> P;
  std::memset(&B, 0, sizeof(B));
  std::memset(&P, 0, sizeof(P));
  if ((rc = describe_ozaki_request(ctx, cp, a, b, c, ws, P.seg[0], B.req[0])) != TK_OK)
    return rc;
  B.nreq = 1;
  P.nseg = 1;
  const OzLayout* lay[1] = {L};
  if ((rc = launch_oz_prep<1>(ctx, lay, P, L->mode, L->slices, stream)) != TK_OK) return rc;
  return launch_oz_gemm<1>(ctx, L, B, L->ncta, stream);
}

int launch_gemm_ozaki_batch(Ctx* ctx, int n, const ContractPlan* const* plans, const void* const* a,
                            const void* const* b, void* const* c, void* const* ws, void* stream) {
  int rc = ensure_smem_attrs(ctx);
  if (rc != TK_OK) return rc;
  // requests that share the launch parameters (mode, tile width, slice count) share a launch
  std::vector<int> todo;
  for (int i = 0; i < n; ++i) {
    const OzLayout* L = static_cast<const OzLayout*>(plans[i]->oz.get());
    if (L && L->nwork > 0) todo.push_back(i);
  }
  static thread_local OzBatchT<OZ_BATCH> B;  // ~12 KB of kernel parameters
  static thread_local OzPrepT<OZ_BATCH> P;   // ~3 KB
  while (!todo.empty()) {
    const OzLayout* L0 = static_cast<const OzLayout*>(plans[todo[0]]->oz.get());
    std::vector<int> rest;
    std::memset(&B, 0, sizeof(B));
    std::memset(&P, 0, sizeof(P));
    const OzLayout* lay[OZ_BATCH];
    int grid = 0;
    for (int i : todo) {
      const OzLayout* L = static_cast<const OzLayout*>(plans[i]->oz.get());
      if (B.nreq < OZ_BATCH && L->mode == L0->mode && L->bn == L0->bn && L->slices == L0->slices &&
          L->prep_cluster == L0->prep_cluster) {
        if ((rc = describe_ozaki_request(ctx, *plans[i], a[i], b[i], c[i], ws[i], P.seg[B.nreq], B.req[B.nreq])) !=
            TK_OK)
          return rc;
        lay[B.nreq] = L;
        grid = std::max(grid, L->ncta);
        B.nreq += 1;
      } else {
        rest.push_back(i);
      }
    }
    P.nseg = B.nreq;
    if ((rc = launch_oz_prep<OZ_BATCH>(ctx, lay, P, L0->mode, L0->slices, stream)) != TK_OK) return rc;
    if ((rc = launch_oz_gemm<OZ_BATCH>(ctx, L0, B, grid, stream)) != TK_OK) return rc;
    todo.swap(rest);
  }
  return TK_OK;
}

int launch_wait_selftest(Ctx* ctx, void* stream) {
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status);
  if (cudaGetLastError() != cudaSuccess) return TK_ERR_CUDA;
  ctx->launches += 1;
  return TK_OK;
}

}  // namespace tk
