// Device kernels of the contraction path (sm_103a):
//   K1 k_permute   -- fusion-tree permute: every destination reduced array is a
//                     coefficient-weighted sum of strided transposes of source reduced arrays
//                     (Algorithm 10; Algorithm 6 for abelian symmetries, one source, weight 1);
//                     the input permute launch also zero-fills the output blocks of coupled
//                     sectors whose inner dimension is empty and clears the split-K counters.
//   K2 k_gemm_f64  -- grouped FP64 GEMM over the coupled sectors (Algorithm 8, step 2).
//   k_zero_batch   -- the zero fill of many requests of one packed batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "tk_device.cuh"
#include "tk_internal.hpp"

namespace tk {

// ------------------------------------------------------------------ helpers
ProfScope::ProfScope(Ctx* c, const char* n, void* s) : ctx(c), name(n), stream(s) {
  if (!ctx->profiling) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) == cudaSuccess && cudaEventRecord(e, (cudaStream_t)s) == cudaSuccess) start = e;
}

ProfScope::~ProfScope() {
  if (!start) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) == cudaSuccess && cudaEventRecord(e, (cudaStream_t)stream) == cudaSuccess)
    ctx->prof.push_back(Ctx::Rec{name, start, (void*)e});
}

PermutePlan::~PermutePlan() {
  dev_free(d_tasks);
  dev_free(d_rtasks);
  dev_free(d_runs);
  dev_free(d_srcs);
  dev_free(d_tile_task);
}

ContractPlan::~ContractPlan() {
  dev_free(d_gemm_items);
  dev_free(d_gemm_tiles);
  dev_free(d_zero);
  for (void* p : d_oz) dev_free(p);
}

namespace {

template <typename T>
struct Elem;
template <>
struct Elem<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double conj(double v) { return v; }
  __device__ static void fma(double& acc, double c, double v) { acc = fma_(c, v, acc); }
  __device__ static double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ static double scale(double c, double v) { return c * v; }
};
template <>
struct Elem<double2> {
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double2 conj(double2 v) { return make_double2(v.x, -v.y); }
  __device__ static void fma(double2& acc, double c, double2 v) {
    acc.x = __fma_rn(c, v.x, acc.x);
    acc.y = __fma_rn(c, v.y, acc.y);
  }
  __device__ static double2 scale(double c, double2 v) { return make_double2(c * v.x, c * v.y); }
};

// Weighted sum over the sources of one destination element.  The common abelian case (one
// source, weight exactly 1) is a plain copy with no floating-point operation.
template <typename T>
__device__ __forceinline__ T gather(const PermSrc* __restrict__ srcs, int nsrc, int src_begin,
                                    const T* __restrict__ in, int64_t ir, int64_t ic, int conj = 0) {
  const PermSrc s0 = srcs[src_begin];
  T v = __ldg(in + s0.in_off + ir + ic * s0.ld);
  if (conj) v = Elem<T>::conj(v);  // adjoint tasks: one source, weight 1
  if (nsrc == 1 && s0.coef == 1.0) return v;
  T acc = Elem<T>::scale(s0.coef, v);
  for (int s = 1; s < nsrc; ++s) {
    const PermSrc si = srcs[src_begin + s];
    Elem<T>::fma(acc, si.coef, __ldg(in + si.in_off + ir + ic * si.ld));
  }
  return acc;
}

constexpr int kTaskWords = (int)(sizeof(PermTask) / sizeof(int64_t));
static_assert(sizeof(PermTask) % sizeof(int64_t) == 0, "PermTask must be 8-byte multiple");

// One launch serves up to four segments (the run list and the tile list of up to two permutes,
// e.g. both operands of a contraction); each segment owns a contiguous range of blocks.
struct PermSeg {
  int32_t kind;    // 0: contiguous runs, 1: tiles, 2: fill nwork ints at out (split-K counters,
                   // scale arrays), 3: zero fill of the ZeroItems at in (nwork = items x chunks)
  int32_t group;   // runs: lanes per run (32, or 16 when the runs are short); fills: the value;
                   // zero fill: the number of items
  int64_t block0, nblocks, nwork;  // blocks [block0, block0 + nblocks); runs or tiles to do
  const PermRun* runs;
  const PermTask* tasks;  // run tasks (kind 0) or tile tasks (kind 1)
  const int32_t* tile_task;  // tiles: owning task of every tile
  const PermSrc* srcs;
  const void* in;
  void* out;
};
constexpr int kMaxPermSegs = 7;       // one contraction: runs + tiles of two operands, fills, zero fill
constexpr int kZeroChunk = 2048;      // elements of a zero-fill unit
constexpr int kBatchSegs = 160;       // a packed launch over many requests (about 13 KB of parameters)
template <int NSEG>
struct PermLaunchT {
  PermSeg seg[NSEG];
  int32_t nseg;
};
using PermLaunch = PermLaunchT<kMaxPermSegs>;

// Segment owning block b: segments are sorted by their first block.
template <typename Seg>
__device__ __forceinline__ int find_seg(const Seg* segs, int nseg, int64_t b) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].block0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Outer offsets of one tile: the dims other than the tiled ones, decoded from o (32-bit: a task
// has fewer than 2^31 elements).
__device__ __forceinline__ void tile_outer(const PermTask& t, int kfirst, int skip1, int skip2, int o, int64_t& ob,
                                           int64_t& irb, int64_t& icb) {
  ob = t.out_off;
  irb = 0;
  icb = 0;
  for (int k = kfirst; k < t.ndim; ++k) {
    if (k == skip1 || k == skip2) continue;
    const int x = o % t.ext[k];
    o /= t.ext[k];
    ob += (int64_t)x * t.ostr[k];
    irb += (int64_t)x * t.irs[k];
    icb += (int64_t)x * t.ics[k];
  }
}

// Short-vector transpose tile (mode 3): dim 0 (E elements) is contiguous on both sides and moves
// as a unit; dim 1 follows it in the destination, dim td in the source.  A tile is 16 (dim 1) x
// 16 (dim td) vectors: loads run along (dim 0, dim td), stores along (dim 0, dim 1).
template <typename T, int E>
__device__ __forceinline__ void permute_vec_tile(const PermTask& t, int local, const PermSrc* __restrict__ srcs,
                                                 const T* __restrict__ in, T* __restrict__ out, T* s) {
  constexpr int SPAN = 16 * E, ROW = SPAN + 1;  // s: [16 b][16 E + 1]
  const int tid = threadIdx.x;
  const int td = t.tdim, ea = t.ext[1], eb = t.ext[td];
  const int nba = (ea + 15) / 16, nbb = (eb + 15) / 16;
  const int ba = local % nba, rest = local / nba;
  const int bb = rest % nbb;
  int64_t ob, irb, icb;
  tile_outer(t, 2, td, td, rest / nbb, ob, irb, icb);
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int idx = tid + 256 * q;
    const int wb = idx % SPAN, al = idx / SPAN;  // along the source: (w, b) contiguous
    const int w = wb % E, bl = wb / E;
    const int a = ba * 16 + al, b = bb * 16 + bl;
    if (a < ea && b < eb)
      s[bl * ROW + al * E + w] =
          gather<T>(srcs, t.nsrc, t.src_begin, in, irb + (int64_t)a * t.irs[1] + (int64_t)b * E + w,
                    icb + (int64_t)a * t.ics[1], t.conj);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int idx = tid + 256 * q;
    const int wa = idx % SPAN, bl = idx / SPAN;  // along the destination: (w, a) contiguous
    const int a = ba * 16 + wa / E, b = bb * 16 + bl;
    if (a < ea && b < eb) out[ob + (int64_t)b * t.ostr[td] + (int64_t)ba * 16 * E + wa] = s[bl * ROW + wa];
  }
}

template <typename T>
__device__ __forceinline__ void permute_tiles(const PermSeg& g, int64_t bid, T (*tile)[33], int64_t* task_words) {
  const PermTask& t = *reinterpret_cast<const PermTask*>(task_words);
  const PermTask* __restrict__ tasks = g.tasks;
  const int32_t* __restrict__ tile_task = g.tile_task;
  const PermSrc* __restrict__ srcs = g.srcs;
  const T* __restrict__ in = (const T*)g.in;
  T* __restrict__ out = (T*)g.out;
  const int tid = threadIdx.x;
  for (int64_t tidx = bid; tidx < g.nwork; tidx += g.nblocks) {
    const int task = __ldg(tile_task + tidx);  // the task owning this tile
    __syncthreads();  // previous iteration finished with task_words / tile
    if (tid < kTaskWords) task_words[tid] = __ldg(reinterpret_cast<const int64_t*>(tasks + task) + tid);
    __syncthreads();
    const int local = (int)(tidx - t.tile_begin);
    if (t.mode == 1) {
      const int td = t.tdim;
      const int e0 = t.ext[0], et = t.ext[td];
      const int nb0 = (e0 + 31) / 32, nbt = (et + 31) / 32;
      const int b0 = local % nb0, rest = local / nb0;
      const int bt = rest % nbt;
      int64_t ob, irb, icb;
      tile_outer(t, 1, td, td, rest / nbt, ob, irb, icb);
      const int lx = tid & 31, ly = tid >> 5;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int j0 = ly + 8 * r;
        const int i0 = b0 * 32 + j0, it = bt * 32 + lx;
        if (i0 < e0 && it < et) {
          const int64_t ir = irb + (int64_t)i0 * t.irs[0] + it;  // irs[td] = 1
          const int64_t ic = icb + (int64_t)i0 * t.ics[0];       // ics[td] = 0
          tile[j0][lx] = gather<T>(srcs, t.nsrc, t.src_begin, in, ir, ic, t.conj);
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int jt = ly + 8 * r;
        const int i0 = b0 * 32 + lx, it = bt * 32 + jt;
        if (i0 < e0 && it < et) out[ob + i0 + (int64_t)it * t.ostr[td]] = tile[lx][jt];
      }
    } else if (t.mode == 3) {
      T* s = &tile[0][0];
      if (t.ext[0] == 2)
        permute_vec_tile<T, 2>(t, local, srcs, in, out, s);
      else if (t.ext[0] == 3)
        permute_vec_tile<T, 3>(t, local, srcs, in, out, s);
      else
        permute_vec_tile<T, 4>(t, local, srcs, in, out, s);
    } else {
      int total = 1;
      for (int k = 0; k < t.ndim; ++k) total *= t.ext[k];
      int e = local * 256 + tid;
      if (e < total) {
        int64_t oa = t.out_off, ir = 0, ic = 0;
        for (int k = 0; k < t.ndim; ++k) {
          const int x = e % t.ext[k];
          e /= t.ext[k];
          oa += (int64_t)x * t.ostr[k];
          ir += (int64_t)x * t.irs[k];
          ic += (int64_t)x * t.ics[k];
        }
        out[oa] = gather<T>(srcs, t.nsrc, t.src_begin, in, ir, ic, t.conj);
      }
    }
  }
}

// Contiguous runs (destination and sources share their fastest leg): one warp per run, lanes
// along the run, U elements per lane in flight.  Copy runs (one source, weight 1) carry their
// source offset, so the next run's record is the only load before the data; it is fetched while
// the current run is copied.  SU(2) runs sum their weighted sources in FP64.
// Contiguous runs, G lanes per run (a warp, or half a warp when the runs are short so that two
// runs' loads are in flight per warp), U loads in flight per lane; the next run's descriptor is
// fetched while the current run is copied.
template <typename T, int G>
__device__ __forceinline__ void permute_runs(const PermSeg& g, int64_t bid) {
  constexpr int U = 4;
  const PermRun* __restrict__ runs = g.runs;
  const PermTask* __restrict__ tasks = g.tasks;
  const PermSrc* __restrict__ srcs = g.srcs;
  const T* __restrict__ in = (const T*)g.in;
  T* __restrict__ out = (T*)g.out;
  constexpr int LG = G == 16 ? 4 : 5;
  const int sub = threadIdx.x & (G - 1);  // lane within the run's group
  const int64_t ngroups = (g.nblocks * blockDim.x) >> LG;
  int64_t r = (bid * blockDim.x + threadIdx.x) >> LG;
  PermRun next;
  if (r < g.nwork) next = runs[r];
  for (; r < g.nwork; r += ngroups) {
    const PermRun run = next;
    if (r + ngroups < g.nwork) next = runs[r + ngroups];
    T* dst = out + run.dst;
    if (run.task < 0) {
      const T* src = in + run.ir;
      if (run.task == -2) {  // adjoint: conjugating copy
        for (int e = sub; e < run.len; e += G) dst[e] = Elem<T>::conj(__ldg(src + e));
        continue;
      }
      for (int e = sub; e < run.len; e += G * U) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e + G * u < run.len) v[u] = __ldg(src + e + G * u);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e + G * u < run.len) dst[e + G * u] = v[u];
      }
      continue;
    }
    const int nsrc = __ldg(&tasks[run.task].nsrc);
    const int sb = __ldg(&tasks[run.task].src_begin);
    for (int e = sub; e < run.len; e += G)
      dst[e] = gather<T>(srcs, nsrc, sb, in, run.ir + e, run.ic);
  }
}

template <typename T, int NSEG>
__global__ void __launch_bounds__(256, 4) k_permute(const __grid_constant__ PermLaunchT<NSEG> L) {
  __shared__ T tile[32][33];
  __shared__ int64_t task_words[kTaskWords];
  const PermSeg& g = L.seg[find_seg(L.seg, L.nseg, (int64_t)blockIdx.x)];
  const int64_t bid = (int64_t)blockIdx.x - g.block0;
  if (g.kind == 0) {
    if constexpr (sizeof(T) == 8) {  // complex runs move 16 B per element: always a warp per run
      if (g.group == 16) {
        permute_runs<T, 16>(g, bid);
        return;
      }
    }
    permute_runs<T, 32>(g, bid);
  } else if (g.kind == 1) {
    permute_tiles<T>(g, bid, tile, task_words);
  } else if (g.kind == 2) {
    int* p = (int*)g.out;
    for (int64_t i = bid * blockDim.x + threadIdx.x; i < g.nwork; i += g.nblocks * blockDim.x) p[i] = g.group;
  } else {  // unit u: chunk u / nitems of item u % nitems
    const ZeroItem* __restrict__ items = (const ZeroItem*)g.in;
    T* __restrict__ c = (T*)g.out;
    for (int64_t u = bid; u < g.nwork; u += g.nblocks) {
      const ZeroItem z = items[u % g.group];
      const int64_t e0 = (u / g.group) * kZeroChunk, e1 = min(z.n, e0 + kZeroChunk);
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) c[z.off + e] = Elem<T>::zero();
    }
  }
}

// ------------------------------------------------------------------ K2 grouped FP64 GEMM
// Work list of output tiles over all sector GEMMs of one contraction, each tile tagged with one
// of three shapes chosen on the host: 64x64 (4x4 per thread), 32x32 (2x2 per thread) when the
// 64x64 tiles are too few to fill 152 SMs, and a row kernel for N <= 8 (one output row per
// thread; the skinny MPO products).  Tiles are sorted by cost (M_t N_t K) descending.
struct GemmTile {
  int32_t item, m0, n0, cfg;
  int32_t k0, k1;       // inner-dimension range of this tile
  int32_t slot, part;   // split-K: output tile slot and this tile's part (slot < 0: no split)
  int32_t nsplit, rpt;  // rpt: rows per thread of a row block (N <= 8 products)
  int64_t poff;         // split-K: first element of this slot's partials (nsplit parts of one tile)
  int32_t nblk, pad1;   // row blocks: consecutive 256 x rpt row groups walked by one CTA (>= 1)
};
constexpr int SPLIT_MAX = 8;

enum { CFG_64 = 0, CFG_32 = 1, CFG_ROWS = 2, CFG_ROWS_DF = 3 };
constexpr int BK = 16;
constexpr int ROWS_NMAX = 8, ROWS_KCHUNK = 256;
// Rows per thread of an N <= 8 row block over a long product (real data): four groups of four
// loads and the accumulators stay within the three-CTAs-per-SM register budget.  Row blocks of
// shorter products, and all complex ones, take one row per thread (more CTAs).  A row block
// covers 256 x rpt rows.
__host__ __device__ constexpr int rows_rpt(int nt) { return nt <= 2 ? 4 : nt <= 4 ? 2 : 1; }
// The double-float rows run with four CTAs per SM (64 registers): at most two rows per thread.
__host__ __device__ constexpr int rows_rpt_df(int nt) { return nt <= 4 ? 2 : 1; }

__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename T>
struct Mac;
template <>
struct Mac<double> {
  __device__ static void mac(double& acc, double a, double b) { acc = __fma_rn(a, b, acc); }
};
template <>
struct Mac<double2> {
  __device__ static void mac(double2& acc, double2 a, double2 b) {
    acc.x = __fma_rn(a.x, b.x, acc.x);
    acc.x = __fma_rn(-a.y, b.y, acc.x);
    acc.y = __fma_rn(a.x, b.y, acc.y);
    acc.y = __fma_rn(a.y, b.x, acc.y);
  }
};

// One BMxBN tile with 256 threads in a 16x16 grid, TMxTN outputs per thread (BM = 16 TM).
template <typename T, int BM, int BN, int TM, int TN>
__device__ __forceinline__ void gemm_tile(const GemmItem& it, const GemmTile& tl,
                                          const T* __restrict__ A, const T* __restrict__ B,
                                          T* __restrict__ C, T* smem, T* __restrict__ partials,
                                          int* __restrict__ counters) {
  const int64_t m0 = tl.m0, n0 = tl.n0;
  T(*As)[BM + 1] = reinterpret_cast<T(*)[BM + 1]>(smem);
  T(*Bs)[BN + 1] = reinterpret_cast<T(*)[BN + 1]>(smem + BK * (BM + 1));
  const int64_t M = it.M, N = it.N, K = it.K;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Elem<T>::zero();
  const T* Ab = A + it.a_off;
  const T* Bb = B + it.b_off;
  const int64_t kend = tl.k1;
  // The next k-chunk's operands are loaded into registers while the current chunk is multiplied
  // out of shared memory, so each chunk's global-load latency overlaps the previous chunk's FMAs.
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;
  T ra[LA], rb[LB];
  auto load = [&](int64_t k0, int kmax) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q, mm = e % BM, kk = e / BM;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[q] = (gm < M && kk < kmax) ? Ab[gm + gk * M] : Elem<T>::zero();
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q, kb = e % BK, nn = e / BK;
      const int64_t gk = k0 + kb, gn = n0 + nn;
      rb[q] = (kb < kmax && gn < N) ? Bb[gk + gn * K] : Elem<T>::zero();
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[e / BM][e % BM] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[e % BK][e / BK] = rb[q];
    }
  };
  int64_t k0 = tl.k0;
  int kmax = (int)((kend - k0) < BK ? (kend - k0) : BK);
  if (k0 < kend) {
    load(k0, kmax);
    store();
  }
  __syncthreads();
  while (k0 < kend) {
    const int64_t kn = k0 + BK;
    const int kmaxn = kn < kend ? (int)((kend - kn) < BK ? (kend - kn) : BK) : 0;
    if (kn < kend) load(kn, kmaxn);
#pragma unroll 4
    for (int kk = 0; kk < kmax; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) Mac<T>::mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
    if (kn < kend) store();
    __syncthreads();
    k0 = kn;
    kmax = kmaxn;
  }
  T* Cb = C + it.c_off;
  if (tl.slot >= 0) {
    // split-K: publish this part; the CTA that completes the slot sums the parts in a fixed order
    __shared__ int s_last;
    T* mine = partials + tl.poff + (int64_t)tl.part * (BM * BN);
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < TM; ++i) mine[(tx + 16 * i) + (ty + 16 * j) * BM] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&counters[tl.slot], 1) == tl.nsplit - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const T* base = partials + tl.poff;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + ty + 16 * j;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + tx + 16 * i;
        T v = Elem<T>::zero();
        for (int p = 0; p < tl.nsplit; ++p) v = add(v, __ldcg(base + p * (BM * BN) + (tx + 16 * i) + (ty + 16 * j) * BM));
        if (gm < M && gn < N) Cb[gm + gn * M] = v;
      }
    }
    if (tid == 0) counters[tl.slot] = 0;  // ready for the next launch
    return;
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t gn = n0 + ty + 16 * j;
    if (gn >= N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + tx + 16 * i;
      if (gm < M) Cb[gm + gn * M] = acc[i][j];
    }
  }
}

// Split-K epilogue shared by the row kernels: publish this part's (256 RPT) x NT partial sums; the
// CTA that completes the slot adds the parts in part order (deterministic) and writes C.  Thread
// tid owns rows m0 + tid + 256 r, r < RPT.
template <typename T, int NT, int RPT>
__device__ __forceinline__ void rows_store(const GemmItem& it, const GemmTile& tl, int64_t m0,
                                           const T (&acc)[RPT][NT], T* __restrict__ C,
                                           T* __restrict__ partials, int* __restrict__ counters) {
  const int64_t M = it.M;
  const int tid = threadIdx.x;
  T* Cb = C + it.c_off;
  if (tl.slot < 0) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t m = m0 + r * 256 + tid;
      if (m < M) {
#pragma unroll
        for (int j = 0; j < NT; ++j) Cb[m + j * M] = acc[r][j];
      }
    }
    return;
  }
  constexpr int PS = 256 * RPT * NT;  // elements of one part
  __shared__ int s_last;
  T* mine = partials + tl.poff + (int64_t)tl.part * PS;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int j = 0; j < NT; ++j) mine[r * 256 + tid + 256 * RPT * j] = acc[r][j];
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&counters[tl.slot], 1) == tl.nsplit - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const T* base = partials + tl.poff;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int64_t m = m0 + r * 256 + tid;
    if (m < M) {
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        T v = Elem<T>::zero();
        for (int p = 0; p < tl.nsplit; ++p) v = add(v, __ldcg(base + p * PS + r * 256 + tid + 256 * RPT * j));
        Cb[m + j * M] = v;
      }
    }
  }
  if (tid == 0) counters[tl.slot] = 0;  // ready for the next launch
}

// N <= 8 products (the skinny MPO steps): streams over A's rows.  Thread tid owns RPT rows
// (m0 + tid + 256 r) and walks K in groups of four (4 RPT independent loads in flight) plus a
// guarded tail; B is broadcast from shared memory in K chunks.  The code is instantiated for each
// N (NT), so every FMA issued is one of the product's M K N.
template <typename T, int NT, int RPT>
__device__ __forceinline__ void gemm_rows_n(const GemmItem& it, const GemmTile& tl, const T* __restrict__ A,
                                            const T* __restrict__ B, T* __restrict__ C, T* smem,
                                            T* __restrict__ partials, int* __restrict__ counters) {
  T(*Bs)[NT] = reinterpret_cast<T(*)[NT]>(smem);
  const int64_t M = it.M, K = it.K;
  const int tid = threadIdx.x;
  // one K chunk: B is staged once for all of this CTA's row groups
  const bool one_chunk = tl.k1 - tl.k0 <= ROWS_KCHUNK;
  const T* Bb = B + it.b_off;
  for (int sb = 0; sb < tl.nblk; ++sb) {
    const int64_t m0 = (int64_t)tl.m0 + (int64_t)sb * 256 * RPT;
    if (m0 >= M) break;
    bool live[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) live[r] = m0 + r * 256 + tid < M;
    T acc[RPT][NT];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int j = 0; j < NT; ++j) acc[r][j] = Elem<T>::zero();
    for (int64_t k0 = tl.k0; k0 < tl.k1; k0 += ROWS_KCHUNK) {
      const int kmax = (int)((tl.k1 - k0) < ROWS_KCHUNK ? (tl.k1 - k0) : ROWS_KCHUNK);
      if (sb == 0 || !one_chunk) {
        for (int e = tid; e < kmax * NT; e += 256) {
          const int kk = e % kmax, nn = e / kmax;
          Bs[kk][nn] = Bb[(k0 + kk) + nn * K];
        }
        __syncthreads();
      }
      const T* Ak = A + it.a_off + m0 + tid + k0 * M;  // column k0 of this thread's first row
      int kk = 0;
      for (; kk + 4 <= kmax; kk += 4, Ak += 4 * M) {
        T a[4][RPT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int r = 0; r < RPT; ++r) a[u][r] = live[r] ? Ak[u * M + r * 256] : Elem<T>::zero();
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const T b = Bs[kk + u][j];
#pragma unroll
            for (int r = 0; r < RPT; ++r) Mac<T>::mac(acc[r][j], a[u][r], b);
          }
      }
      if (kk < kmax) {  // 1..3 left; the branches are uniform over the block
        const int left = kmax - kk;
        T a[3][RPT];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int r = 0; r < RPT; ++r) a[u][r] = (live[r] && u < left) ? Ak[u * M + r * 256] : Elem<T>::zero();
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < left) {
#pragma unroll
            for (int j = 0; j < NT; ++j) {
              const T b = Bs[kk + u][j];
#pragma unroll
              for (int r = 0; r < RPT; ++r) Mac<T>::mac(acc[r][j], a[u][r], b);
            }
          }
      }
      if (!one_chunk) __syncthreads();
    }
    rows_store<T, NT, RPT>(it, tl, m0, acc, C, partials, counters);
  }
}

template <typename T>
__device__ __forceinline__ void gemm_rows(const GemmItem& it, const GemmTile& tl, const T* __restrict__ A,
                                          const T* __restrict__ B, T* __restrict__ C, T* smem,
                                          T* __restrict__ partials, int* __restrict__ counters) {
  constexpr bool CX = sizeof(T) == 16;
#define TK_ROWS_CASE(NT)                                                                                  \
  if (CX || tl.rpt == 1)                                                                                  \
    gemm_rows_n<T, NT, 1>(it, tl, A, B, C, smem, partials, counters);                                     \
  else                                                                                                    \
    gemm_rows_n<T, NT, CX ? 1 : rows_rpt(NT)>(it, tl, A, B, C, smem, partials, counters);
  switch (it.N) {
    case 1: TK_ROWS_CASE(1) break;
    case 2: TK_ROWS_CASE(2) break;
    case 3: TK_ROWS_CASE(3) break;
    case 4: TK_ROWS_CASE(4) break;
    case 5: TK_ROWS_CASE(5) break;
    case 6: TK_ROWS_CASE(6) break;
    case 7: TK_ROWS_CASE(7) break;
    default: TK_ROWS_CASE(8) break;
  }
#undef TK_ROWS_CASE
}

// Split-precision mode only: the N <= 8 row kernel in double-float arithmetic (pairs of FP32
// with error-free products and sums), ~2^-44 relative per term, on the FP32 pipe.
// a = hi + lo to within 2^-46 |a|, by integer operations on the FP64 bit pattern: hi keeps the
// sign, the exponent and the top 23 stored mantissa bits; lo is the next 23 bits, formed as a
// normal FP32 with those bits as its fraction minus the same number with a zero fraction (an
// exact subtraction), so no conversion instruction runs.  The pair arithmetic keeps its precision
// while every product and its error term stay normal FP32: each A value in [2^-58, 2^96) and each
// B value (the MPO side) in [2^-20, 2^20) give products in [2^-78, 2^116) (and sums of up to 2^10
// of them below 2^127).  A nonzero value outside its window (FP64 subnormals included) counts as
// zero here and marks the block; the block flags its tile, and the launch after it redoes the
// flagged tiles' output rows in plain FP64 (rows_df_redo).  The window test is the exponent branch
// every value takes anyway; only the rare values pay for more.
__shared__ int s_df_oor;  // the block met an out-of-range value (cleared at the block's start)
__device__ __noinline__ void df_split_rare(double a, float& hi, float& lo) {
  if (__double_as_longlong(a) << 1) s_df_oor = 1;  // zero is in range
  hi = 0.f;
  lo = 0.f;
}
// EMIN, EMAX: the window [2^EMIN, 2^EMAX) of magnitudes split here.
template <int EMIN, int EMAX>
__device__ __forceinline__ void df_split(double a, float& hi, float& lo) {
  static_assert(EMIN >= -103 && EMAX <= 127, "the window must keep hi and lo normal FP32");
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int ef = ex - 1023 + 127;
  if ((unsigned int)(ef - (127 + EMIN)) >= (unsigned int)(EMAX - EMIN)) {
    df_split_rare(a, hi, lo);  // out of line
    return;
  }
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  hi = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu));
  // mantissa bits 28..6 as t: lo = t 2^(ex-1069) = (1 + t 2^-23) 2^(ef-150) - 2^(ef-150)
  const unsigned int e2 = (unsigned int)(ef - 23) << 23;
  const float l = __fsub_rn(__uint_as_float(e2 | ((unsigned int)(b >> 6) & 0x7FFFFFu)), __uint_as_float(e2));
  lo = __uint_as_float(__float_as_uint(l) ^ sign);
}
constexpr int DF_A_EMIN = -58, DF_A_EMAX = 96, DF_B_EMIN = -20, DF_B_EMAX = 20;
// Double-float multiply-add on two output columns at once with the packed FP32 pair instructions
// (one instruction per pair): (sh, sl) += a * b, a = ah + al, b = bh + bl; no operation is
// contracted.
__device__ __forceinline__ void df_mac2(float2& sh, float2& sl, float ah, float al, float2 bh, float2 bl) {
  const float2 a2 = make_float2(ah, ah), l2 = make_float2(al, al);
  const float2 p = __fmul2_rn(a2, bh);
  const float2 pe = __ffma2_rn(a2, bh, make_float2(-p.x, -p.y));  // exact error of ah*bh
  const float2 cross = __ffma2_rn(a2, bl, __ffma2_rn(l2, bh, pe));
  float2 s, e;
  two_sum2(sh, p, s, e);
  sl = __fadd2_rn(sl, __fadd2_rn(e, cross));
  sh = s;
}
template <int NP, int RPT>
__device__ __forceinline__ void df_rows_group(float2 (&sh)[RPT][NP], float2 (&sl)[RPT][NP], const double (&a)[RPT],
                                              const float2* bh, const float2* bl) {
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    float ah, al;
    df_split<DF_A_EMIN, DF_A_EMAX>(a[r], ah, al);
#pragma unroll
    for (int q = 0; q < NP; ++q) df_mac2(sh[r][q], sl[r][q], ah, al, bh[q], bl[q]);
  }
}
// Columns are processed in pairs (NP = ceil(NT / 2)); for odd NT the last pair's second column
// multiplies a zero B column and is not stored.
template <int NT, int RPT>
__device__ __forceinline__ void gemm_rows_df_n(const GemmItem& it, const GemmTile& tl, const double* __restrict__ A,
                                               const double* __restrict__ B, double* __restrict__ C,
                                               double* smem, double* __restrict__ partials,
                                               int* __restrict__ counters) {
  constexpr int NP = (NT + 1) / 2;
  float2(*Bh)[NP] = reinterpret_cast<float2(*)[NP]>(smem);
  float2(*Bl)[NP] = reinterpret_cast<float2(*)[NP]>(reinterpret_cast<float2*>(smem) + ROWS_KCHUNK * NP);
  const int64_t M = it.M, K = it.K;
  const int tid = threadIdx.x;
  const bool one_chunk = tl.k1 - tl.k0 <= ROWS_KCHUNK;  // then B is staged once for all row groups
  const double* Bb = B + it.b_off;
  for (int sb = 0; sb < tl.nblk; ++sb) {
    const int64_t m0 = (int64_t)tl.m0 + (int64_t)sb * 256 * RPT;
    if (m0 >= M) break;
    bool live[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) live[r] = m0 + r * 256 + tid < M;
    float2 sh[RPT][NP], sl[RPT][NP];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int q = 0; q < NP; ++q) sh[r][q] = sl[r][q] = make_float2(0.f, 0.f);
    for (int64_t k0 = tl.k0; k0 < tl.k1; k0 += ROWS_KCHUNK) {
      const int kmax = (int)((tl.k1 - k0) < ROWS_KCHUNK ? (tl.k1 - k0) : ROWS_KCHUNK);
      if (sb == 0 || !one_chunk) {
        for (int e = tid; e < kmax * NP; e += 256) {
          const int kk = e % kmax, q = e / kmax;
          float h0, l0, h1 = 0.f, l1 = 0.f;
          df_split<DF_B_EMIN, DF_B_EMAX>(Bb[(k0 + kk) + (2 * q) * K], h0, l0);
          if (2 * q + 1 < NT) df_split<DF_B_EMIN, DF_B_EMAX>(Bb[(k0 + kk) + (2 * q + 1) * K], h1, l1);
          Bh[kk][q] = make_float2(h0, h1);
          Bl[kk][q] = make_float2(l0, l1);
        }
        __syncthreads();
      }
      const double* Ak = A + it.a_off + m0 + tid + k0 * M;
      int kk = 0;
      for (; kk + 4 <= kmax; kk += 4, Ak += 4 * M) {
        double a[4][RPT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int r = 0; r < RPT; ++r) a[u][r] = live[r] ? Ak[u * M + r * 256] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) df_rows_group<NP, RPT>(sh, sl, a[u], Bh[kk + u], Bl[kk + u]);
      }
      if (kk < kmax) {  // 1..3 left; the branches are uniform over the block
        const int left = kmax - kk;
        double a[3][RPT];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int r = 0; r < RPT; ++r) a[u][r] = (live[r] && u < left) ? Ak[u * M + r * 256] : 0.0;
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < left) df_rows_group<NP, RPT>(sh, sl, a[u], Bh[kk + u], Bl[kk + u]);
      }
      if (!one_chunk) __syncthreads();
    }
    double acc[RPT][NT];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const float2 h = sh[r][j / 2], l = sl[r][j / 2];
        acc[r][j] = (j & 1) ? f32_to_f64(h.y) + f32_to_f64(l.y) : f32_to_f64(h.x) + f32_to_f64(l.x);
      }
    rows_store<double, NT, RPT>(it, tl, m0, acc, C, partials, counters);
  }
}

__device__ __forceinline__ void gemm_rows_df(const GemmItem& it, const GemmTile& tl, const double* __restrict__ A,
                                             const double* __restrict__ B, double* __restrict__ C, double* smem,
                                             double* __restrict__ partials, int* __restrict__ counters) {
#define TK_ROWS_DF_CASE(NT)                                                   \
  if (tl.rpt == 1)                                                            \
    gemm_rows_df_n<NT, 1>(it, tl, A, B, C, smem, partials, counters);         \
  else                                                                        \
    gemm_rows_df_n<NT, rows_rpt_df(NT)>(it, tl, A, B, C, smem, partials, counters);
  switch (it.N) {
    case 1: TK_ROWS_DF_CASE(1) break;
    case 2: TK_ROWS_DF_CASE(2) break;
    case 3: TK_ROWS_DF_CASE(3) break;
    case 4: TK_ROWS_DF_CASE(4) break;
    case 5: TK_ROWS_DF_CASE(5) break;
    case 6: TK_ROWS_DF_CASE(6) break;
    case 7: TK_ROWS_DF_CASE(7) break;
    default: TK_ROWS_DF_CASE(8) break;
  }
#undef TK_ROWS_DF_CASE
}

// One launch per contraction for every FP64-list product: 64x64 / 32x32 tiles and the N <= 8
// row blocks share the grid (their shared-memory needs overlap in one buffer).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 1) k_gemm_f64(const GemmItem* __restrict__ items,
                                                                        const GemmTile* __restrict__ tiles,
                                                                        const T* __restrict__ A,
                                                                        const T* __restrict__ B, T* __restrict__ C,
                                                                        T* __restrict__ partials,
                                                                        int* __restrict__ counters) {
  constexpr int kTileElems = BK * 65 * 2, kRowElems = ROWS_KCHUNK * ROWS_NMAX;
  __shared__ T smem[kTileElems > kRowElems ? kTileElems : kRowElems];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmItem it = items[tl.item];
  if (tl.cfg == CFG_64)
    gemm_tile<T, 64, 64, 4, 4>(it, tl, A, B, C, smem, partials, counters);
  else if (tl.cfg == CFG_32)
    gemm_tile<T, 32, 32, 2, 2>(it, tl, A, B, C, smem, partials, counters);
  else
    gemm_rows<T>(it, tl, A, B, C, smem, partials, counters);
}

// Split-precision modes: every product left to the CUDA cores is an N <= 8 row block in
// double-float (the planner cuts wider thin products into such blocks), so this launch runs the
// row code alone, with the registers of four CTAs per SM.
// The double-float launch's exact fallback, run after it: the output rows of every tile whose
// flag is set (a value out of range), again in plain FP64 over the whole inner dimension, straight
// to C (the launch, split-K sums included, has finished; two flagged parts of one split tile write
// the same values).  Each block reads 256 flags at a time, one per thread, so a launch with no
// flag set costs one load round; the flagged tiles of the round are then redone one by one.
__device__ __noinline__ void rows_df_redo(const GemmItem* __restrict__ items, const GemmTile* __restrict__ tiles,
                                          int64_t ntiles, const double* __restrict__ A,
                                          const double* __restrict__ B, double* __restrict__ C,
                                          const int* __restrict__ flags, int64_t block, int64_t nblocks) {
  __shared__ int64_t list[256];
  __shared__ int count;
  for (int64_t t0 = block * 256; t0 < ntiles; t0 += nblocks * 256) {
    const int64_t t = t0 + threadIdx.x;
    const int f = t < ntiles ? *(volatile const int*)&flags[t] : 0;
    if (!__syncthreads_or(f)) continue;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    if (f) list[atomicAdd(&count, 1)] = t;
    __syncthreads();
    for (int i = 0; i < count; ++i) {
      const GemmTile tl = tiles[list[i]];
      const GemmItem it = items[tl.item];
      const int64_t rows = (int64_t)256 * tl.rpt * tl.nblk;
      for (int64_t m = tl.m0 + threadIdx.x; m < min(it.M, (int64_t)tl.m0 + rows); m += blockDim.x)
        for (int64_t j = 0; j < it.N; ++j) {
          double s = 0.0;
          for (int64_t k = 0; k < it.K; ++k) s = __fma_rn(A[it.a_off + m + k * it.M], B[it.b_off + k + j * it.K], s);
          C[it.c_off + m + j * it.M] = s;
        }
    }
    __syncthreads();  // list and count are reused by the next round
  }
}
// Start of a double-float block: clear its out-of-range mark before any value is split.
__device__ __forceinline__ void rows_df_clear_mark() {
  if (threadIdx.x == 0) s_df_oor = 0;
  __syncthreads();
}
// End of a double-float block: flag its tile if the block met an out-of-range value.
__device__ __forceinline__ void rows_df_mark(int* flag) {
  __syncthreads();
  if (threadIdx.x == 0 && s_df_oor) *flag = 1;
}
// A small launch after a double-float launch (one block per 256 tiles, one SM's worth at most):
// the exact fallback for the flagged tiles, else nothing.
__global__ void __launch_bounds__(256) k_rows_df_fixup(const GemmItem* __restrict__ items,
                                                       const GemmTile* __restrict__ tiles, int64_t ntiles,
                                                       const double* __restrict__ A, const double* __restrict__ B,
                                                       double* __restrict__ C, const int* flags) {
  rows_df_redo(items, tiles, ntiles, A, B, C, flags, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256, 4) k_gemm_rows_df(const GemmItem* __restrict__ items,
                                                         const GemmTile* __restrict__ tiles,
                                                         const double* __restrict__ A, const double* __restrict__ B,
                                                         double* __restrict__ C, double* __restrict__ partials,
                                                         int* __restrict__ counters, int* guard) {
  __shared__ double smem[ROWS_KCHUNK * ROWS_NMAX];  // B of one K chunk as double-float pairs
  const GemmTile tl = tiles[blockIdx.x];
  const GemmItem it = items[tl.item];
  rows_df_clear_mark();
  gemm_rows_df(it, tl, A, B, C, smem, partials, counters);
  rows_df_mark(guard + blockIdx.x);
}

// Packed FP64 GEMM over many requests: each segment carries one request's work list and buffers.
struct GemmSeg {
  const GemmItem* items;
  const GemmTile* tiles;
  const void *A, *B;
  void *C, *partials;
  int* counters;
  int* guard;  // double-float launches: one out-of-range flag per tile
  int64_t block0, ntiles;
};
struct GemmBatch {
  GemmSeg seg[kBatchSegs];
  int32_t nseg;
};

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 1) k_gemm_batch(const __grid_constant__ GemmBatch L) {
  constexpr int kTileElems = BK * 65 * 2, kRowElems = ROWS_KCHUNK * ROWS_NMAX;
  __shared__ T smem[kTileElems > kRowElems ? kTileElems : kRowElems];
  const GemmSeg& g = L.seg[find_seg(L.seg, L.nseg, (int64_t)blockIdx.x)];
  const GemmTile tl = g.tiles[blockIdx.x - g.block0];
  const GemmItem it = g.items[tl.item];
  const T* A = (const T*)g.A;
  const T* B = (const T*)g.B;
  T* C = (T*)g.C;
  T* P = (T*)g.partials;
  if (tl.cfg == CFG_64)
    gemm_tile<T, 64, 64, 4, 4>(it, tl, A, B, C, smem, P, g.counters);
  else if (tl.cfg == CFG_32)
    gemm_tile<T, 32, 32, 2, 2>(it, tl, A, B, C, smem, P, g.counters);
  else
    gemm_rows<T>(it, tl, A, B, C, smem, P, g.counters);
}

// Packed double-float row blocks (split-precision batches): as k_gemm_batch, row code only.
__global__ void __launch_bounds__(256, 4) k_gemm_rows_df_batch(const __grid_constant__ GemmBatch L) {
  __shared__ double smem[ROWS_KCHUNK * ROWS_NMAX];
  const GemmSeg& g = L.seg[find_seg(L.seg, L.nseg, (int64_t)blockIdx.x)];
  const GemmTile tl = g.tiles[blockIdx.x - g.block0];
  const GemmItem it = g.items[tl.item];
  rows_df_clear_mark();
  gemm_rows_df(it, tl, (const double*)g.A, (const double*)g.B, (double*)g.C, smem, (double*)g.partials,
               g.counters);
  rows_df_mark(g.guard + (blockIdx.x - g.block0));
}
// After a packed double-float launch: blocks (x, s) run the exact fallback for segment s's flagged
// tiles, block x reading rounds x, x + gridDim.x, ... of 256 flags.
__global__ void __launch_bounds__(256) k_rows_df_fixup_batch(const __grid_constant__ GemmBatch L) {
  const GemmSeg& g = L.seg[blockIdx.y];
  rows_df_redo(g.items, g.tiles, g.ntiles, (const double*)g.A, (const double*)g.B, (double*)g.C, g.guard, blockIdx.x,
               gridDim.x);
}

// Packed zero fill: block row y belongs to the segment whose first item index is the largest <= y.
struct ZeroSeg {
  const ZeroItem* items;
  void* c;
  int64_t block0;  // first global item index of this segment (named for find_seg)
  int64_t nitems;
};
struct ZeroBatch {
  ZeroSeg seg[kBatchSegs];
  int32_t nseg;
};
template <typename T>
__global__ void k_zero_batch(const __grid_constant__ ZeroBatch L, int64_t total_items) {
  for (int64_t i = blockIdx.y; i < total_items; i += gridDim.y) {
    const ZeroSeg& g = L.seg[find_seg(L.seg, L.nseg, i)];
    const ZeroItem z = g.items[i - g.block0];
    T* c = (T*)g.c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < z.n; e += (int64_t)gridDim.x * blockDim.x)
      c[z.off + e] = Elem<T>::zero();
  }
}

int check_launch(Ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return TK_ERR_CUDA;
  }
  ctx->launches += 1;
  return TK_OK;
}

}  // namespace

namespace {
// Segments (runs and tiles) of the non-identity permutes among jobs, with their natural block counts.
void perm_segments(const PermJob* jobs, int njobs, std::vector<PermSeg>& segs, std::vector<int64_t>& natural,
                   int& dtype) {
  // Tile segments first: blocks start in index order, and a launch holds about two waves of them,
  // so the transposes (the slower work per block) start in the first wave and the runs fill in
  // around them instead of queueing the transposes behind every run.
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < njobs; ++j) {
      const PermutePlan& pp = *jobs[j].plan;
      if (pp.identity) continue;
      dtype = pp.dtype;
      if (pass == 1 && !pp.runs.empty()) {
        PermSeg g;
        std::memset(&g, 0, sizeof(g));
        g.kind = 0;
        g.group = pp.dtype == TK_C128 ? 32 : pp.run_group;
        g.nwork = (int64_t)pp.runs.size();
        g.runs = pp.d_runs;
        g.tasks = pp.d_rtasks;
        g.srcs = pp.d_srcs;
        g.in = jobs[j].in;
        g.out = jobs[j].out;
        segs.push_back(g);
        const int64_t per_block = 256 / g.group;  // runs in flight per block
        natural.push_back((g.nwork + per_block - 1) / per_block);
      }
      if (pass == 0 && !pp.tasks.empty() && pp.total_tiles > 0) {
        PermSeg g;
        std::memset(&g, 0, sizeof(g));
        g.kind = 1;
        g.nwork = pp.total_tiles;
        g.tasks = pp.d_tasks;
        g.tile_task = pp.d_tile_task;
        g.srcs = pp.d_srcs;
        g.in = jobs[j].in;
        g.out = jobs[j].out;
        segs.push_back(g);
        natural.push_back(g.nwork);
      }
    }
}

// Blocks per segment: natural counts, or a share of 8 blocks per SM in proportion to the work when
// the total exceeds that.
template <int NSEG>
int64_t fill_perm_launch(PermLaunchT<NSEG>& L, const PermSeg* segs, const int64_t* natural, int n, int64_t cap) {
  std::memset(&L, 0, sizeof(L));
  int64_t total = 0;
  for (int i = 0; i < n; ++i) total += natural[i];
  int64_t b0 = 0;
  for (int i = 0; i < n; ++i) {
    int64_t nb = natural[i];
    if (total > cap) nb = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)((double)cap * natural[i] / total)));
    L.seg[i] = segs[i];
    L.seg[i].block0 = b0;
    L.seg[i].nblocks = nb;
    b0 += nb;
  }
  L.nseg = n;
  return b0;
}
}  // namespace

int launch_permutes(Ctx* ctx, const PermJob* jobs, int njobs, void* stream, const IntClear* clears, int nclears,
                    const ZeroJob* zero) {
  std::vector<PermSeg> segs;
  std::vector<int64_t> natural;
  int dtype = TK_F64;
  perm_segments(jobs, njobs, segs, natural, dtype);
  if (zero) dtype = zero->dtype;  // the same as the permutes' (one contraction)
  if (segs.empty() && zero) {  // nothing to permute: the zero fill takes its own launch
    const int64_t units = zero->nitems * ((zero->maxn + kZeroChunk - 1) / kZeroChunk);
    if (units > 0) {
      PermSeg g;
      std::memset(&g, 0, sizeof(g));
      g.kind = 3;
      g.group = (int32_t)zero->nitems;
      g.nwork = units;
      g.in = zero->items;
      g.out = zero->c;
      segs.push_back(g);
      natural.push_back(units);
      zero = nullptr;
    }
  }
  if (segs.empty()) {  // nothing to permute: clear with plain memsets
    for (int i = 0; i < nclears; ++i)
      if (cudaMemsetAsync(clears[i].p, clears[i].fill & 0xFF, (size_t)clears[i].n * sizeof(int), (cudaStream_t)stream) !=
          cudaSuccess)
        return TK_ERR_CUDA;
    return TK_OK;
  }
  for (int i = 0; i < nclears; ++i) {  // ride along in the permute launch that precedes the GEMM
    PermSeg g;
    std::memset(&g, 0, sizeof(g));
    g.kind = 2;
    g.group = clears[i].fill;
    g.nwork = clears[i].n;
    g.out = clears[i].p;
    segs.push_back(g);
    natural.push_back(1);
  }
  if (zero) {  // zero fill of the GEMM output's empty blocks rides along too
    const int64_t units = zero->nitems * ((zero->maxn + kZeroChunk - 1) / kZeroChunk);
    if (units > 0) {
      PermSeg g;
      std::memset(&g, 0, sizeof(g));
      g.kind = 3;
      g.group = (int32_t)zero->nitems;
      g.nwork = units;
      g.in = zero->items;
      g.out = zero->c;
      segs.push_back(g);
      natural.push_back(units);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t cap = (int64_t)std::max(ctx->num_sms, 1) * 8;
  ProfScope prof(ctx, "k_permute", stream);
  if ((int)segs.size() <= kMaxPermSegs) {  // one contraction: small parameter block
    PermLaunch L;
    const int64_t blocks = fill_perm_launch(L, segs.data(), natural.data(), (int)segs.size(), cap);
    if (dtype == TK_C128)
      k_permute<double2, kMaxPermSegs><<<(unsigned)blocks, 256, 0, s>>>(L);
    else
      k_permute<double, kMaxPermSegs><<<(unsigned)blocks, 256, 0, s>>>(L);
    return check_launch(ctx, "k_permute");
  }
  static thread_local PermLaunchT<kBatchSegs> big;  // ~13 KB: not on the stack
  for (size_t first = 0; first < segs.size(); first += kBatchSegs) {
    const int n = (int)std::min<size_t>(kBatchSegs, segs.size() - first);
    const int64_t blocks = fill_perm_launch(big, segs.data() + first, natural.data() + first, n, cap);
    if (dtype == TK_C128)
      k_permute<double2, kBatchSegs><<<(unsigned)blocks, 256, 0, s>>>(big);
    else
      k_permute<double, kBatchSegs><<<(unsigned)blocks, 256, 0, s>>>(big);
    int rc = check_launch(ctx, "k_permute");
    if (rc != TK_OK) return rc;
  }
  return TK_OK;
}

int launch_permute(Ctx* ctx, const PermutePlan& pp, const void* in, void* out, void* stream) {
  const PermJob job{&pp, in, out};
  return launch_permutes(ctx, &job, 1, stream, nullptr, 0);
}

int upload_gemm_tables(Ctx* ctx, ContractPlan& cp) {
  // Shapes: the rows kernel for N <= 8, 64x64 or 32x32 tiles otherwise.  A launch that would give
  // the SMs too few CTAs cuts the inner dimension into up to SPLIT_MAX parts (split-K); the parts
  // of one output tile are added in part order by the CTA that finishes last (deterministic).
  const int64_t sms = std::max(ctx->num_sms, 1);
  int64_t tiles64 = 0, tiles32 = 0, split64 = 0;
  double pad64 = 0, pad32 = 0;
  for (const GemmItem& g : cp.gemms_fp64) {
    if (g.N <= ROWS_NMAX) continue;
    const int64_t t64 = ((g.M + 63) / 64) * ((g.N + 63) / 64), t32 = ((g.M + 31) / 32) * ((g.N + 31) / 32);
    tiles64 += t64;
    tiles32 += t32;
    split64 += t64 * std::max<int64_t>(1, std::min<int64_t>(SPLIT_MAX, g.K / 64));
    pad64 += 4096.0 * t64 * g.K;
    pad32 += 1024.0 * t32 * g.K;
  }
  // 64x64 tiles reuse registers twice as well as 32x32 ones; take them unless padding to 64 costs
  // more than a fifth extra work, or they are too few even after splitting K
  const bool use64 = cp.tune_tile == 64 ? true
                    : cp.tune_tile == 32 ? false
                                         : (tiles64 >= 3 * sms || (pad64 <= 1.2 * pad32 && split64 >= 3 * sms));
  const int bm = use64 ? 64 : 32;
  // A product whose N exceeds a multiple of the tile width by at most ROWS_NMAX columns gives those
  // last columns to the rows kernel (B and C are column-major: their trailing columns are a
  // contiguous sub-matrix with the same leading dimension) instead of padding a whole tile column.
  std::vector<GemmItem> gl;
  gl.reserve(cp.gemms_fp64.size() * 2);
  for (const GemmItem& g : cp.gemms_fp64) {
    if (cp.gemm_mode != TK_GEMM_FP64 && g.N > ROWS_NMAX) {
      // split-precision modes: the thin products left to this kernel run in double-float as
      // row blocks of at most ROWS_NMAX columns (B and C are column-major: a column range is a
      // contiguous sub-matrix with the same leading dimension)
      for (int64_t n0 = 0; n0 < g.N; n0 += ROWS_NMAX) {
        GemmItem part = g;
        part.N = std::min<int64_t>(ROWS_NMAX, g.N - n0);
        part.b_off = g.b_off + n0 * g.K;
        part.c_off = g.c_off + n0 * g.M;
        gl.push_back(part);
      }
      continue;
    }
    const int64_t rem = g.N % bm;
    if (g.N > bm && rem > 0 && rem <= ROWS_NMAX) {
      GemmItem main = g, tail = g;
      main.N = g.N - rem;
      tail.N = rem;
      tail.b_off = g.b_off + main.N * g.K;
      tail.c_off = g.c_off + main.N * g.M;
      gl.push_back(main);
      gl.push_back(tail);
    } else {
      gl.push_back(g);
    }
  }
  // several rows per thread only where the product is long enough to give eight waves of
  // one-row blocks at three CTAs per SM (fewer, longer-lived threads then lose nothing)
  const bool cplx = cp.dtype == TK_C128;
  const bool df = cp.gemm_mode != TK_GEMM_FP64;
  auto rows_per_thread = [&](const GemmItem& g) {
    if (cplx || (g.M + 255) / 256 < 8 * 3 * sms) return 1;
    return df ? rows_rpt_df((int)g.N) : rows_rpt((int)g.N);
  };
  auto rows_block = [&](const GemmItem& g) { return (int64_t)256 * rows_per_thread(g); };
  int64_t rows_ctas = 0;
  tiles64 = tiles32 = 0;
  for (const GemmItem& g : gl) {
    if (g.N <= ROWS_NMAX)
      rows_ctas += (g.M + rows_block(g) - 1) / rows_block(g);
    else
      (use64 ? tiles64 : tiles32) += ((g.M + bm - 1) / bm) * ((g.N + bm - 1) / bm);
  }
  const int64_t ntiles = use64 ? tiles64 : tiles32;
  int64_t want_tiles = ntiles >= 3 * sms ? 1 : (4 * sms + ntiles - 1) / std::max<int64_t>(ntiles, 1);
  int64_t want_rows = rows_ctas >= 2 * sms ? 1 : (4 * sms + rows_ctas - 1) / std::max<int64_t>(rows_ctas, 1);
  if (cp.tune_split == 1) want_tiles = want_rows = 1;           // no split-K
  if (cp.tune_split == 2) want_tiles = want_rows = SPLIT_MAX;   // as many parts as K allows
  int32_t nslots = 0;
  int64_t poff = 0;
  struct Cand {
    GemmTile t;
    double cost;
  };
  std::vector<Cand> cands;
  // one output tile as nsplit parts over [0, K), each part's depth a multiple of kalign
  auto emit = [&](int32_t item, int64_t m0, int64_t n0, int32_t cfg, int64_t K, int nsplit, int kalign,
                  int64_t part_elems, double area, int rpt, int nblk) {
    const int64_t kstep = ((K + nsplit - 1) / nsplit + kalign - 1) / kalign * kalign;
    nsplit = (int)std::max<int64_t>(1, (K + kstep - 1) / kstep);  // no empty parts after rounding
    const int32_t slot = nsplit > 1 ? nslots++ : -1;
    for (int p = 0; p < nsplit; ++p) {
      const int64_t k0 = std::min<int64_t>(K, p * kstep), k1 = std::min<int64_t>(K, k0 + kstep);
      GemmTile t;
      std::memset(&t, 0, sizeof(t));
      t.item = item;
      t.m0 = (int32_t)m0;
      t.n0 = (int32_t)n0;
      t.cfg = cfg;
      t.k0 = (int32_t)k0;
      t.k1 = (int32_t)k1;
      t.slot = slot;
      t.part = p;
      t.nsplit = nsplit;
      t.rpt = rpt;
      t.nblk = nblk;
      t.poff = nsplit > 1 ? poff : 0;
      cands.push_back({t, area * (double)(k1 - k0)});
    }
    if (nsplit > 1) poff += (int64_t)nsplit * part_elems;
  };
  for (size_t i = 0; i < gl.size(); ++i) {
    const GemmItem& g = gl[i];
    if (g.N <= ROWS_NMAX) {
      const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want_rows, (int64_t)SPLIT_MAX, g.K / 8}));
      const int32_t cfg = cp.gemm_mode == TK_GEMM_FP64 ? CFG_ROWS : CFG_ROWS_DF;
      const int rpt = rows_per_thread(g);
      // a CTA walks several row groups of a product that needs one K chunk and no split: four
      // of a long product, two of a shorter one when the launch has at least four one-group
      // blocks per SM (so at least two paired blocks per SM remain)
      const int nblk = (nsplit == 1 && g.K <= ROWS_KCHUNK) ? (rpt > 1 ? 4 : rows_ctas >= 4 * sms ? 2 : 1) : 1;
      const int64_t rb = 256 * rpt * nblk;
      for (int64_t m0 = 0; m0 < g.M; m0 += rb)
        emit((int32_t)i, m0, 0, cfg, g.K, nsplit, 8, (int64_t)256 * rpt * g.N,
             (double)std::min<int64_t>(rb, g.M - m0) * g.N, rpt, nblk);
      continue;
    }
    const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want_tiles, (int64_t)SPLIT_MAX, g.K / 64}));
    for (int64_t n0 = 0; n0 < g.N; n0 += bm)
      for (int64_t m0 = 0; m0 < g.M; m0 += bm)
        emit((int32_t)i, m0, n0, use64 ? CFG_64 : CFG_32, g.K, nsplit, BK, (int64_t)bm * bm, (double)bm * bm, 1, 1);
  }
  cp.split_slots = nslots;
  if (cp.gemm_mode != TK_GEMM_FP64)  // the split-precision launch runs row blocks only
    for (const Cand& c : cands)
      if (c.t.cfg != CFG_ROWS_DF) {
        ctx->last_error = "split-precision plan with a non-row CUDA-core tile";
        return TK_ERR_UNSUPPORTED;
      }
  // Row blocks first (they are latency-bound: a serial walk over K), then tiles by cost, largest
  // first, so the short tiles fill the tail.
  std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) {
    const bool ra = a.t.cfg >= CFG_ROWS, rb = b.t.cfg >= CFG_ROWS;
    if (ra != rb) return ra;
    return a.cost > b.cost;
  });
  std::vector<GemmTile> tiles;
  for (auto& c : cands) tiles.push_back(c.t);
  cp.n_gemm_tiles = (int64_t)tiles.size();
  int rc = dev_upload(ctx, &cp.d_gemm_items, gl.data(), gl.size() * sizeof(GemmItem));
  if (rc != TK_OK) return rc;
  rc = dev_upload(ctx, &cp.d_gemm_tiles, tiles.data(), tiles.size() * sizeof(GemmTile));
  if (rc != TK_OK) return rc;
  if (!cp.zeros.empty()) {
    rc = dev_upload(ctx, &cp.d_zero, cp.zeros.data(), cp.zeros.size() * sizeof(ZeroItem));
    if (rc != TK_OK) return rc;
  }
  if (nslots > 0) cp.partials_bytes = (size_t)poff * (cp.dtype == TK_C128 ? 16 : 8);
  return TK_OK;
}

int launch_gemm_fp64(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c,
                     void* partials, int* counters, void* stream) {
  if (cp.n_gemm_tiles == 0) return TK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const GemmItem* items = (const GemmItem*)cp.d_gemm_items;
  const GemmTile* tiles = (const GemmTile*)cp.d_gemm_tiles;
  const unsigned grid = (unsigned)cp.n_gemm_tiles;
  if (cp.dtype != TK_C128 && cp.gemm_mode != TK_GEMM_FP64) {
    ProfScope prof(ctx, "k_gemm_rows_df", stream);
    k_gemm_rows_df<<<grid, 256, 0, s>>>(items, tiles, (const double*)a, (const double*)b, (double*)c,
                                        (double*)partials, counters, counters + cp.split_slots);
    int rc = check_launch(ctx, "k_gemm_rows_df");
    if (rc != TK_OK) return rc;
    const unsigned fix_grid = (unsigned)std::min<int64_t>((cp.n_gemm_tiles + 255) / 256, std::max(ctx->num_sms, 1));
    k_rows_df_fixup<<<fix_grid, 256, 0, s>>>(items, tiles, cp.n_gemm_tiles, (const double*)a, (const double*)b,
                                             (double*)c, counters + cp.split_slots);
    return check_launch(ctx, "k_rows_df_fixup");
  }
  ProfScope prof(ctx, "k_gemm_f64", stream);
  if (cp.dtype == TK_C128)
    k_gemm_f64<double2><<<grid, 256, 0, s>>>(items, tiles, (const double2*)a, (const double2*)b, (double2*)c,
                                             (double2*)partials, counters);
  else
    k_gemm_f64<double><<<grid, 256, 0, s>>>(items, tiles, (const double*)a, (const double*)b, (double*)c,
                                            (double*)partials, counters);
  return check_launch(ctx, "k_gemm_f64");
}

namespace {
// Complex operands of a split-precision plan: real and imaginary parts into separate arrays, and
// the four real products back into one complex result.
__global__ void k_cx_split(const double2* __restrict__ a, double* __restrict__ ar, double* __restrict__ ai,
                           int64_t na, const double2* __restrict__ b, double* __restrict__ br,
                           double* __restrict__ bi, int64_t nb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na + nb; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < na) {
      const double2 v = a[i];
      ar[i] = v.x;
      ai[i] = v.y;
    } else {
      const double2 v = b[i - na];
      br[i - na] = v.x;
      bi[i - na] = v.y;
    }
  }
}
// c = (rr - ii) + i (ri + ir)
__global__ void k_cx_join(const double* __restrict__ rr, const double* __restrict__ ii,
                          const double* __restrict__ ri, const double* __restrict__ ir, double2* __restrict__ c,
                          int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    c[k] = make_double2(rr[k] - ii[k], ri[k] + ir[k]);
}
}  // namespace

// Workspace of a complex split-precision plan: Re A | Im A | Re B | Im B | four real results |
// the real plan's workspace.
struct CxLayout {
  double *ar, *ai, *br, *bi, *t[4];
  char* ws_re;
};
static CxLayout cx_layout(const ContractPlan& cp, void* ws) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* w = (char*)ws;
  CxLayout L;
  L.ar = (double*)w;
  w += al((size_t)cp.cx_na * 8);
  L.ai = (double*)w;
  w += al((size_t)cp.cx_na * 8);
  L.br = (double*)w;
  w += al((size_t)cp.cx_nb * 8);
  L.bi = (double*)w;
  w += al((size_t)cp.cx_nb * 8);
  for (int k = 0; k < 4; ++k) {
    L.t[k] = (double*)w;
    w += al((size_t)cp.cx_nc * 8);
  }
  L.ws_re = w;
  return L;
}

int run_contract_cx_split(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                          void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const CxLayout L = cx_layout(cp, ws);
  const int64_t nab = cp.cx_na + cp.cx_nb;
  const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nab + 255) / 256, (int64_t)ctx->num_sms * 16));
  {
    ProfScope prof(ctx, "k_cx_split", stream);
    k_cx_split<<<g1, 256, 0, s>>>((const double2*)a, L.ar, L.ai, cp.cx_na, (const double2*)b, L.br, L.bi, cp.cx_nb);
    int rc = check_launch(ctx, "k_cx_split");
    if (rc != TK_OK) return rc;
  }
  const double* ops[4][2] = {{L.ar, L.br}, {L.ai, L.bi}, {L.ar, L.bi}, {L.ai, L.br}};
  for (int k = 0; k < 4; ++k) {
    int rc = run_contract(ctx, *cp.re, ops[k][0], ops[k][1], L.t[k], L.ws_re, stream);
    if (rc != TK_OK) return rc;
  }
  const unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cp.cx_nc + 255) / 256, (int64_t)ctx->num_sms * 16));
  ProfScope prof(ctx, "k_cx_join", stream);
  k_cx_join<<<g2, 256, 0, s>>>(L.t[0], L.t[1], L.t[2], L.t[3], (double2*)c, cp.cx_nc);
  return check_launch(ctx, "k_cx_join");
}

int run_contract(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                 void* stream) {
  if (cp.re) return run_contract_cx_split(ctx, cp, a, b, c, ws, stream);
  char* w = (char*)ws;
  const void* at = cp.pa->identity ? a : (const void*)(w + cp.ws_at);
  const void* bt = cp.pb->identity ? b : (const void*)(w + cp.ws_bt);
  void* ct = cp.pc ? (void*)(w + cp.ws_ct) : c;
  int rc;
  const PermJob in_jobs[2] = {{cp.pa.get(), a, (void*)at}, {cp.pb.get(), b, (void*)bt}};
  IntClear clears[1];
  int nclears = 0;
  const int64_t nclear = (int64_t)cp.split_slots + df_guard_words(cp);  // split-K counters, rows guard
  if (nclear > 0) clears[nclears++] = IntClear{(int*)(w + cp.ws_counters), nclear};
  // both operands in one launch, which also clears the split-K counters and zero-fills the output
  // blocks with an empty inner dimension
  ZeroJob zj{(const ZeroItem*)cp.d_zero, (int64_t)cp.zeros.size(), 0, ct, cp.dtype};
  for (const ZeroItem& z : cp.zeros) zj.maxn = std::max(zj.maxn, z.n);
  if ((rc = launch_permutes(ctx, in_jobs, 2, stream, clears, nclears, cp.zeros.empty() ? nullptr : &zj)) != TK_OK)
    return rc;
  if (!cp.gemms_fp64.empty() && !cp.gemms_oz.empty() && ctx->side) {
    // split precision with CUDA-core products too: those run on the side stream beside the
    // prep / tensor-core launches.  They write other C blocks (or other columns of a
    // block), their own split-K partials and counters, and read only the permuted operands.
    cudaStream_t s = (cudaStream_t)stream, side = (cudaStream_t)ctx->side;
    std::lock_guard<std::mutex> lk(ctx->side_mu);
    if (cudaEventRecord((cudaEvent_t)ctx->ev_fork, s) != cudaSuccess ||
        cudaStreamWaitEvent(side, (cudaEvent_t)ctx->ev_fork, 0) != cudaSuccess)
      return TK_ERR_CUDA;
    if ((rc = launch_gemm_fp64(ctx, cp, at, bt, ct, w + cp.ws_partials, (int*)(w + cp.ws_counters), side)) != TK_OK)
      return rc;
    if (cudaEventRecord((cudaEvent_t)ctx->ev_join, side) != cudaSuccess) return TK_ERR_CUDA;
    rc = launch_gemm_ozaki(ctx, cp, at, bt, ct, w + cp.ws_slices, stream);
    if (cudaStreamWaitEvent(s, (cudaEvent_t)ctx->ev_join, 0) != cudaSuccess) return TK_ERR_CUDA;  // join first
    if (rc != TK_OK) return rc;
  } else {
    if (!cp.gemms_fp64.empty() &&
        (rc = launch_gemm_fp64(ctx, cp, at, bt, ct, w + cp.ws_partials, (int*)(w + cp.ws_counters), stream)) != TK_OK)
      return rc;
    if (!cp.gemms_oz.empty() && (rc = launch_gemm_ozaki(ctx, cp, at, bt, ct, w + cp.ws_slices, stream)) != TK_OK)
      return rc;
  }
  if (cp.pc && (rc = launch_permute(ctx, *cp.pc, ct, c, stream)) != TK_OK) return rc;
  return TK_OK;
}

int run_contract_batch(Ctx* ctx, int n, const ContractPlan* const* plans, const void* const* a,
                       const void* const* b, void* const* c, void* const* ws, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const bool cplx = plans[0]->dtype == TK_C128;
  const bool split = plans[0]->gemm_mode != TK_GEMM_FP64;  // a batch has one gemm mode (checked by the ABI)
  std::vector<const void*> at((size_t)n), bt((size_t)n);
  std::vector<void*> ct((size_t)n);
  std::vector<PermJob> in_jobs, out_jobs;
  std::vector<IntClear> clears;
  for (int i = 0; i < n; ++i) {
    const ContractPlan& cp = *plans[i];
    char* w = (char*)ws[i];
    at[i] = cp.pa->identity ? a[i] : (const void*)(w + cp.ws_at);
    bt[i] = cp.pb->identity ? b[i] : (const void*)(w + cp.ws_bt);
    ct[i] = cp.pc ? (void*)(w + cp.ws_ct) : c[i];
    in_jobs.push_back({cp.pa.get(), a[i], (void*)at[i]});
    in_jobs.push_back({cp.pb.get(), b[i], (void*)bt[i]});
    if (cp.pc) out_jobs.push_back({cp.pc.get(), ct[i], c[i]});
    const int64_t nclear = (int64_t)cp.split_slots + df_guard_words(cp);
    if (nclear > 0) clears.push_back({(int*)(w + cp.ws_counters), nclear});
  }
  int rc = launch_permutes(ctx, in_jobs.data(), (int)in_jobs.size(), stream, clears.data(), (int)clears.size());
  if (rc != TK_OK) return rc;
  // zero fill of blocks with an empty inner dimension, all requests in one launch per 160
  {
    static thread_local ZeroBatch zb;
    int64_t total = 0, maxn = 0;
    zb.nseg = 0;
    auto flush = [&]() -> int {
      if (zb.nseg == 0) return TK_OK;
      dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((maxn + 255) / 256, 1024)),
                (unsigned)std::min<int64_t>(total, 65535));
      ProfScope prof(ctx, "k_zero", stream);
      if (cplx)
        k_zero_batch<double2><<<grid, 256, 0, s>>>(zb, total);
      else
        k_zero_batch<double><<<grid, 256, 0, s>>>(zb, total);
      zb.nseg = 0;
      total = maxn = 0;
      return check_launch(ctx, "k_zero");
    };
    for (int i = 0; i < n; ++i) {
      const ContractPlan& cp = *plans[i];
      if (cp.zeros.empty()) continue;
      ZeroSeg& g = zb.seg[zb.nseg++];
      g.items = (const ZeroItem*)cp.d_zero;
      g.c = ct[i];
      g.block0 = total;
      g.nitems = (int64_t)cp.zeros.size();
      total += g.nitems;
      for (const ZeroItem& z : cp.zeros) maxn = std::max(maxn, z.n);
      if (zb.nseg == kBatchSegs && (rc = flush()) != TK_OK) return rc;
    }
    if ((rc = flush()) != TK_OK) return rc;
  }
  // every GEMM tile of every request in one grouped launch per 160 requests
  {
    static thread_local GemmBatch gb;
    int64_t blocks = 0;
    gb.nseg = 0;
    auto flush = [&]() -> int {
      if (gb.nseg == 0) return TK_OK;
      if (split) {
        ProfScope prof(ctx, "k_gemm_rows_df", stream);
        k_gemm_rows_df_batch<<<(unsigned)blocks, 256, 0, s>>>(gb);
        int rc2 = check_launch(ctx, "k_gemm_rows_df_batch");
        if (rc2 != TK_OK) return rc2;
        k_rows_df_fixup_batch<<<dim3(4, (unsigned)gb.nseg), 256, 0, s>>>(gb);
        gb.nseg = 0;
        blocks = 0;
        return check_launch(ctx, "k_rows_df_fixup");
      }
      ProfScope prof(ctx, "k_gemm_f64", stream);
      if (cplx)
        k_gemm_batch<double2><<<(unsigned)blocks, 256, 0, s>>>(gb);
      else
        k_gemm_batch<double><<<(unsigned)blocks, 256, 0, s>>>(gb);
      gb.nseg = 0;
      blocks = 0;
      return check_launch(ctx, "k_gemm_batch");
    };
    for (int i = 0; i < n; ++i) {
      const ContractPlan& cp = *plans[i];
      if (cp.n_gemm_tiles == 0) continue;
      char* w = (char*)ws[i];
      GemmSeg& g = gb.seg[gb.nseg++];
      g.items = (const GemmItem*)cp.d_gemm_items;
      g.tiles = (const GemmTile*)cp.d_gemm_tiles;
      g.A = at[i];
      g.B = bt[i];
      g.C = ct[i];
      g.partials = w + cp.ws_partials;
      g.counters = (int*)(w + cp.ws_counters);
      g.guard = g.counters + cp.split_slots;
      g.block0 = blocks;
      g.ntiles = cp.n_gemm_tiles;
      blocks += cp.n_gemm_tiles;
      if (gb.nseg == kBatchSegs && (rc = flush()) != TK_OK) return rc;
    }
    if ((rc = flush()) != TK_OK) return rc;
  }
  if (split) {  // the tensor-core products of every request, packed
    std::vector<void*> wsl((size_t)n);
    for (int i = 0; i < n; ++i) wsl[(size_t)i] = (char*)ws[i] + plans[i]->ws_slices;
    if ((rc = launch_gemm_ozaki_batch(ctx, n, plans, at.data(), bt.data(), ct.data(), wsl.data(), stream)) != TK_OK)
      return rc;
  }
  return launch_permutes(ctx, out_jobs.data(), (int)out_jobs.size(), stream, nullptr, 0);
}

}  // namespace tk
