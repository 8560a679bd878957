// Device kernels of the contraction path (sm_103a):
//   K1 k_permute   -- fusion-tree permute: every destination reduced array is a
//                     coefficient-weighted sum of strided transposes of source reduced arrays
//                     (Algorithm 10; Algorithm 6 for abelian symmetries, one source, weight 1).
//   K2 k_gemm_f64  -- grouped FP64 GEMM over the coupled sectors (Algorithm 8, step 2).
//   k_zero         -- zero blocks of coupled sectors whose inner dimension is empty.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "tk_internal.hpp"

namespace tk {

// ------------------------------------------------------------------ helpers
int dev_upload(Ctx* ctx, void** dst, const void* src, size_t bytes) {
  if (bytes == 0) {
    *dst = nullptr;
    return TK_OK;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return TK_ERR_CUDA;
  if (cudaMalloc(dst, bytes) != cudaSuccess) return TK_ERR_OOM;
  if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return TK_ERR_CUDA;
  return TK_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

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
  dev_free(d_tile_starts);
}

ContractPlan::~ContractPlan() {
  dev_free(d_gemm_items);
  dev_free(d_gemm_tiles);
  dev_free(d_gemm_rows);
  dev_free(d_split_counters);
  dev_free(d_zero);
  for (void* p : d_oz) dev_free(p);
}

namespace {

template <typename T>
struct Elem;
template <>
struct Elem<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static void fma(double& acc, double c, double v) { acc = fma_(c, v, acc); }
  __device__ static double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ static double scale(double c, double v) { return c * v; }
};
template <>
struct Elem<double2> {
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
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
                                    const T* __restrict__ in, int64_t ir, int64_t ic) {
  const PermSrc s0 = srcs[src_begin];
  T v = __ldg(in + s0.in_off + ir + ic * s0.ld);
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

template <typename T>
__global__ void __launch_bounds__(256) k_permute(const PermTask* __restrict__ tasks, int ntasks,
                                                 const int64_t* __restrict__ tile_starts,
                                                 const PermSrc* __restrict__ srcs,
                                                 int64_t total_tiles, const T* __restrict__ in,
                                                 T* __restrict__ out) {
  __shared__ T tile[32][33];
  __shared__ int64_t task_words[kTaskWords];
  const PermTask& t = *reinterpret_cast<const PermTask*>(task_words);
  const int tid = threadIdx.x;
  for (int64_t tidx = blockIdx.x; tidx < total_tiles; tidx += gridDim.x) {
    // locate the task owning this tile
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(tile_starts + mid) <= tidx)
        lo = mid;
      else
        hi = mid - 1;
    }
    __syncthreads();  // previous iteration finished with task_words / tile
    if (tid < kTaskWords) task_words[tid] = reinterpret_cast<const int64_t*>(tasks + lo)[tid];
    __syncthreads();
    const int64_t local = tidx - t.tile_begin;
    const int nd = t.ndim;
    if (t.mode == 1) {
      const int td = t.tdim;
      const int e0 = t.ext[0], et = t.ext[td];
      const int64_t nb0 = (e0 + 31) / 32, nbt = (et + 31) / 32;
      const int64_t b0 = local % nb0;
      int64_t rest = local / nb0;
      const int64_t bt = rest % nbt;
      int64_t o = rest / nbt;
      int64_t ob = t.out_off, irb = 0, icb = 0;
      for (int k = 1; k < nd; ++k) {
        if (k == td) continue;
        const int64_t x = o % t.ext[k];
        o /= t.ext[k];
        ob += x * t.ostr[k];
        irb += x * t.irs[k];
        icb += x * t.ics[k];
      }
      const int lx = tid & 31, ly = tid >> 5;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int j0 = ly + 8 * r;
        const int64_t i0 = b0 * 32 + j0, it = bt * 32 + lx;
        if (i0 < e0 && it < et) {
          const int64_t ir = irb + i0 * t.irs[0] + it * t.irs[td];
          const int64_t ic = icb + i0 * t.ics[0] + it * t.ics[td];
          tile[j0][lx] = gather<T>(srcs, t.nsrc, t.src_begin, in, ir, ic);
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int jt = ly + 8 * r;
        const int64_t i0 = b0 * 32 + lx, it = bt * 32 + jt;
        if (i0 < e0 && it < et) out[ob + i0 + it * t.ostr[td]] = tile[lx][jt];
      }
    } else {
      int64_t total = 1;
      for (int k = 0; k < nd; ++k) total *= t.ext[k];
      int64_t e = local * 256 + tid;
      if (e < total) {
        int64_t oa = t.out_off, ir = 0, ic = 0;
        for (int k = 0; k < nd; ++k) {
          const int64_t x = e % t.ext[k];
          e /= t.ext[k];
          oa += x * t.ostr[k];
          ir += x * t.irs[k];
          ic += x * t.ics[k];
        }
        out[oa] = gather<T>(srcs, t.nsrc, t.src_begin, in, ir, ic);
      }
    }
  }
}

// Contiguous runs (destination and sources share their fastest leg): one warp per run, lanes
// along the run, four elements per lane in flight.  Abelian runs (one source, weight 1) are plain
// copies; SU(2) runs sum their weighted sources in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_permute_runs(const PermRun* __restrict__ runs, int64_t nruns,
                                                      const PermTask* __restrict__ tasks,
                                                      const PermSrc* __restrict__ srcs,
                                                      const T* __restrict__ in, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nruns; r += nwarps) {
    const PermRun run = runs[r];
    const int nsrc = __ldg(&tasks[run.task].nsrc);
    const int sb = __ldg(&tasks[run.task].src_begin);
    const PermSrc s0 = srcs[sb];
    T* dst = out + run.dst;
    if (nsrc == 1 && s0.coef == 1.0) {
      const T* src = in + s0.in_off + run.ir + run.ic * s0.ld;
      for (int e = lane; e < run.len; e += 128) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (e + 32 * u < run.len) v[u] = __ldg(src + e + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (e + 32 * u < run.len) dst[e + 32 * u] = v[u];
      }
    } else {
      for (int e = lane; e < run.len; e += 32)
        dst[e] = gather<T>(srcs, nsrc, sb, in, run.ir + e, run.ic);
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
  int32_t nsplit, pad0, pad1, pad2;
};
constexpr int SPLIT_MAX = 8;

enum { CFG_64 = 0, CFG_32 = 1, CFG_ROWS = 2, CFG_ROWS_DF = 3 };
constexpr int BK = 16;
constexpr int ROWS_PER_THREAD = 1, ROWS_PER_CTA = 256 * ROWS_PER_THREAD, ROWS_NMAX = 8, ROWS_KCHUNK = 256;

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
  for (int64_t k0 = tl.k0; k0 < kend; k0 += BK) {
    const int kmax = (int)((kend - k0) < BK ? (kend - k0) : BK);
    for (int e = tid; e < BM * BK; e += 256) {
      const int mm = e % BM, kk = e / BM;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && kk < kmax) ? Ab[gm + gk * M] : Elem<T>::zero();
    }
    for (int e = tid; e < BN * BK; e += 256) {
      const int kb = e % BK, nn = e / BK;
      const int64_t gk = k0 + kb, gn = n0 + nn;
      Bs[kb][nn] = (kb < kmax && gn < N) ? Bb[gk + gn * K] : Elem<T>::zero();
    }
    __syncthreads();
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
  }
  T* Cb = C + it.c_off;
  if (tl.slot >= 0) {
    // split-K: publish this part; the CTA that completes the slot sums the parts in a fixed order
    __shared__ int s_last;
    T* mine = partials + ((int64_t)tl.slot * SPLIT_MAX + tl.part) * (BM * BN);
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
    const T* base = partials + (int64_t)tl.slot * SPLIT_MAX * (BM * BN);
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

// N <= 8: thread t owns row m0 + t, B streamed through shared memory in K chunks.
template <typename T>
__device__ __forceinline__ void gemm_rows(const GemmItem& it, int64_t m0, const T* __restrict__ A,
                                          const T* __restrict__ B, T* __restrict__ C, T* smem) {
  T(*Bs)[ROWS_NMAX] = reinterpret_cast<T(*)[ROWS_NMAX]>(smem);
  const int64_t M = it.M, N = it.N, K = it.K;
  const int tid = threadIdx.x;
  T acc[ROWS_PER_THREAD][ROWS_NMAX];
#pragma unroll
  for (int r = 0; r < ROWS_PER_THREAD; ++r)
#pragma unroll
    for (int j = 0; j < ROWS_NMAX; ++j) acc[r][j] = Elem<T>::zero();
  const T* Ab = A + it.a_off;
  const T* Bb = B + it.b_off;
  for (int64_t k0 = 0; k0 < K; k0 += ROWS_KCHUNK) {
    const int kmax = (int)((K - k0) < ROWS_KCHUNK ? (K - k0) : ROWS_KCHUNK);
    for (int e = tid; e < kmax * ROWS_NMAX; e += 256) {
      const int kk = e % kmax, nn = e / kmax;
      Bs[kk][nn] = (nn < N) ? Bb[(k0 + kk) + nn * K] : Elem<T>::zero();
    }
    __syncthreads();
    for (int kk = 0; kk < kmax; ++kk) {
      T a[ROWS_PER_THREAD];
#pragma unroll
      for (int r = 0; r < ROWS_PER_THREAD; ++r) {
        const int64_t m = m0 + tid + 256 * r;
        a[r] = (m < M) ? Ab[m + (k0 + kk) * M] : Elem<T>::zero();
      }
#pragma unroll
      for (int j = 0; j < ROWS_NMAX; ++j) {
        if (j < N) {
          const T b = Bs[kk][j];
#pragma unroll
          for (int r = 0; r < ROWS_PER_THREAD; ++r) Mac<T>::mac(acc[r][j], a[r], b);
        }
      }
    }
    __syncthreads();
  }
  T* Cb = C + it.c_off;
#pragma unroll
  for (int r = 0; r < ROWS_PER_THREAD; ++r) {
    const int64_t m = m0 + tid + 256 * r;
    if (m < M) {
#pragma unroll
      for (int j = 0; j < ROWS_NMAX; ++j)
        if (j < N) Cb[m + j * M] = acc[r][j];
    }
  }
}

// Split-precision mode only: the N <= 8 row kernel in double-float arithmetic (pairs of FP32
// with error-free products and sums), ~2^-44 relative per term, on the FP32 pipe.
// a = hi + lo to ~2^-53, by integer operations on the FP64 bit pattern: hi keeps the sign, the
// exponent and the top 23 stored mantissa bits; lo is the remaining 29 bits converted to FP32.
// Values outside the normal FP32 range take the conversion instructions.
__device__ __forceinline__ void df_split(double a, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) {  // zero or FP64 subnormal (far below FP32)
    hi = 0.f;
    lo = 0.f;
    return;
  }
  const int ef = ex - 1023 + 127;
  if (ef <= 52 || ef >= 255) {  // lo's scale 2^(ex-1075) must be a normal FP32
    hi = __double2float_rn(a);
    lo = __double2float_rn(a - (double)hi);
    return;
  }
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  hi = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu));
  const unsigned int low = (unsigned int)(b & 0x1FFFFFFFu);  // value low * 2^(ex-1075)
  // low < 2^29: its FP32 rounding loses at most 2^-24 of lo, i.e. ~2^-53 of a
  const float lf = __uint2float_rn(low);
  lo = __fmul_rn(lf, __uint_as_float((unsigned int)(ef - 52) << 23)) * (sign ? -1.f : 1.f);
}
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  // __fmul_rn / __fadd_rn are never contracted into FMAs, which keeps the transformations exact
  const float p = __fmul_rn(ah, bh);
  const float pe = fmaf(ah, bh, -p);                 // exact error of ah*bh
  const float cross = fmaf(ah, bl, fmaf(al, bh, pe));
  const float s = __fadd_rn(sh, p);                  // two-sum of sh + p
  const float bb = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sl = __fadd_rn(sl, __fadd_rn(e, cross));
  sh = s;
}
__device__ __forceinline__ void gemm_rows_df(const GemmItem& it, int64_t m0, const double* __restrict__ A,
                                             const double* __restrict__ B, double* __restrict__ C,
                                             double* smem) {
  float(*Bh)[ROWS_NMAX] = reinterpret_cast<float(*)[ROWS_NMAX]>(smem);
  float(*Bl)[ROWS_NMAX] = reinterpret_cast<float(*)[ROWS_NMAX]>(reinterpret_cast<float*>(smem) + ROWS_KCHUNK * ROWS_NMAX);
  const int64_t M = it.M, N = it.N, K = it.K;
  const int tid = threadIdx.x;
  float sh[ROWS_PER_THREAD][ROWS_NMAX], sl[ROWS_PER_THREAD][ROWS_NMAX];
#pragma unroll
  for (int r = 0; r < ROWS_PER_THREAD; ++r)
#pragma unroll
    for (int j = 0; j < ROWS_NMAX; ++j) sh[r][j] = sl[r][j] = 0.f;
  const double* Ab = A + it.a_off;
  const double* Bb = B + it.b_off;
  for (int64_t k0 = 0; k0 < K; k0 += ROWS_KCHUNK) {
    const int kmax = (int)((K - k0) < ROWS_KCHUNK ? (K - k0) : ROWS_KCHUNK);
    for (int e = tid; e < kmax * ROWS_NMAX; e += 256) {
      const int kk = e % kmax, nn = e / kmax;
      float h = 0.f, l = 0.f;
      if (nn < N) df_split(Bb[(k0 + kk) + nn * K], h, l);
      Bh[kk][nn] = h;
      Bl[kk][nn] = l;
    }
    __syncthreads();
    for (int kk = 0; kk < kmax; ++kk) {
      float ah[ROWS_PER_THREAD], al[ROWS_PER_THREAD];
#pragma unroll
      for (int r = 0; r < ROWS_PER_THREAD; ++r) {
        const int64_t m = m0 + tid + 256 * r;
        df_split((m < M) ? Ab[m + (k0 + kk) * M] : 0.0, ah[r], al[r]);
      }
#pragma unroll
      for (int j = 0; j < ROWS_NMAX; ++j) {
        if (j < N) {
          const float bh = Bh[kk][j], bl = Bl[kk][j];
#pragma unroll
          for (int r = 0; r < ROWS_PER_THREAD; ++r) df_mac(sh[r][j], sl[r][j], ah[r], al[r], bh, bl);
        }
      }
    }
    __syncthreads();
  }
  double* Cb = C + it.c_off;
#pragma unroll
  for (int r = 0; r < ROWS_PER_THREAD; ++r) {
    const int64_t m = m0 + tid + 256 * r;
    if (m < M) {
#pragma unroll
      for (int j = 0; j < ROWS_NMAX; ++j)
        if (j < N) Cb[m + j * M] = (double)sh[r][j] + (double)sl[r][j];
    }
  }
}

template <typename T>
__device__ __forceinline__ void gemm_rows_df_dispatch(const GemmItem& it, int64_t m0, const T* A, const T* B, T* C,
                                                      T* smem) {
  gemm_rows<T>(it, m0, A, B, C, smem);  // complex tensors never take the split-precision path
}
template <>
__device__ __forceinline__ void gemm_rows_df_dispatch<double>(const GemmItem& it, int64_t m0, const double* A,
                                                              const double* B, double* C, double* smem) {
  gemm_rows_df(it, m0, A, B, C, smem);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_f64(const GemmItem* __restrict__ items,
                                                  const GemmTile* __restrict__ tiles,
                                                  const T* __restrict__ A,
                                                  const T* __restrict__ B, T* __restrict__ C,
                                                  T* __restrict__ partials, int* __restrict__ counters) {
  __shared__ T smem[BK * 65 * 2];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmItem it = items[tl.item];
  if (tl.cfg == CFG_64)
    gemm_tile<T, 64, 64, 4, 4>(it, tl, A, B, C, smem, partials, counters);
  else
    gemm_tile<T, 32, 32, 2, 2>(it, tl, A, B, C, smem, partials, counters);
}

// The N <= 8 products in a launch of their own (their register needs differ from the tiles').
template <typename T, bool DF>
__global__ void __launch_bounds__(256) k_gemm_rows(const GemmItem* __restrict__ items,
                                                   const GemmTile* __restrict__ tiles,
                                                   const T* __restrict__ A, const T* __restrict__ B,
                                                   T* __restrict__ C) {
  __shared__ T smem[ROWS_KCHUNK * ROWS_NMAX];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmItem it = items[tl.item];
  if (DF)
    gemm_rows_df_dispatch<T>(it, tl.m0, A, B, C, smem);
  else
    gemm_rows<T>(it, tl.m0, A, B, C, smem);
}

template <typename T>
__global__ void k_zero(const ZeroItem* __restrict__ items, int nitems, T* __restrict__ c) {
  for (int i = blockIdx.y; i < nitems; i += gridDim.y) {
    const ZeroItem z = items[i];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < z.n;
         e += (int64_t)gridDim.x * blockDim.x)
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

int launch_permute(Ctx* ctx, const PermutePlan& pp, const void* in, void* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!pp.runs.empty()) {
    const int64_t nruns = (int64_t)pp.runs.size();
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((nruns + 7) / 8, (int64_t)ctx->num_sms * 8));
    ProfScope prof(ctx, "k_permute", stream);
    if (pp.dtype == TK_C128)
      k_permute_runs<double2><<<(unsigned)grid, 256, 0, s>>>(pp.d_runs, nruns, pp.d_rtasks, pp.d_srcs,
                                                             (const double2*)in, (double2*)out);
    else
      k_permute_runs<double><<<(unsigned)grid, 256, 0, s>>>(pp.d_runs, nruns, pp.d_rtasks, pp.d_srcs,
                                                            (const double*)in, (double*)out);
    int rc = check_launch(ctx, "k_permute_runs");
    if (rc != TK_OK) return rc;
  }
  if (!pp.tasks.empty()) {
    const int ntasks = (int)pp.tasks.size();
    int64_t grid = std::min<int64_t>(pp.total_tiles, (int64_t)ctx->num_sms * 8);
    if (grid < 1) grid = 1;
    ProfScope prof(ctx, "k_permute", stream);
    if (pp.dtype == TK_C128)
      k_permute<double2><<<(unsigned)grid, 256, 0, s>>>(pp.d_tasks, ntasks, pp.d_tile_starts, pp.d_srcs,
                                                        pp.total_tiles, (const double2*)in, (double2*)out);
    else
      k_permute<double><<<(unsigned)grid, 256, 0, s>>>(pp.d_tasks, ntasks, pp.d_tile_starts, pp.d_srcs,
                                                       pp.total_tiles, (const double*)in, (double*)out);
    return check_launch(ctx, "k_permute");
  }
  return TK_OK;
}

int upload_gemm_tables(Ctx* ctx, ContractPlan& cp) {
  // shape choice: rows kernel for N <= 8; 64x64 tiles unless they give fewer than ~3 CTAs per
  // SM over the whole launch, then 32x32
  const std::vector<GemmItem>& gl = cp.gemms_fp64;
  int64_t tiles64 = 0;
  for (const GemmItem& g : gl)
    if (g.N > ROWS_NMAX) tiles64 += ((g.M + 63) / 64) * ((g.N + 63) / 64);
  const bool small_tiles = tiles64 < 3 * (int64_t)std::max(ctx->num_sms, 1);
  int64_t tiles32 = 0;
  for (const GemmItem& g : gl)
    if (g.N > ROWS_NMAX) tiles32 += ((g.M + 31) / 32) * ((g.N + 31) / 32);
  int32_t nslots = 0;
  struct Cand {
    GemmTile t;
    double cost;
  };
  std::vector<Cand> cands;
  for (size_t i = 0; i < gl.size(); ++i) {
    const GemmItem& g = gl[i];
    if (g.N <= ROWS_NMAX) {
      for (int64_t m0 = 0; m0 < g.M; m0 += ROWS_PER_CTA) {
        GemmTile t;
        std::memset(&t, 0, sizeof(t));
        t.item = (int32_t)i;
        t.m0 = (int32_t)m0;
        t.cfg = cp.gemm_mode == TK_GEMM_FP64 ? CFG_ROWS : CFG_ROWS_DF;
        t.k1 = (int32_t)g.K;
        t.slot = -1;
        t.nsplit = 1;
        cands.push_back({t, (double)std::min<int64_t>(ROWS_PER_CTA, g.M - m0) * g.N * g.K});
      }
      continue;
    }
    const int bm = small_tiles ? 32 : 64, bn = bm;
    // split-K (32x32 tiles only): enough parts to give ~6 CTAs per SM, each part >= 64 deep
    int nsplit = 1;
    if (small_tiles) {
      const int64_t want = (6 * (int64_t)std::max(ctx->num_sms, 1) + tiles32 - 1) / std::max<int64_t>(tiles32, 1);
      nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)SPLIT_MAX, g.K / 64}));
    }
    for (int64_t n0 = 0; n0 < g.N; n0 += bn)
      for (int64_t m0 = 0; m0 < g.M; m0 += bm) {
        const int32_t slot = nsplit > 1 ? nslots++ : -1;
        const int64_t kstep = ((g.K + nsplit - 1) / nsplit + BK - 1) / BK * BK;
        for (int p = 0; p < nsplit; ++p) {
          const int64_t k0 = p * kstep, k1 = std::min<int64_t>(g.K, k0 + kstep);
          GemmTile t;
          std::memset(&t, 0, sizeof(t));
          t.item = (int32_t)i;
          t.m0 = (int32_t)m0;
          t.n0 = (int32_t)n0;
          t.cfg = small_tiles ? CFG_32 : CFG_64;
          t.k0 = (int32_t)k0;
          t.k1 = (int32_t)std::max<int64_t>(k0, k1);
          t.slot = slot;
          t.part = p;
          t.nsplit = nsplit;
          cands.push_back({t, (double)bm * bn * (double)(t.k1 - t.k0)});
        }
      }
  }
  cp.split_slots = nslots;
  std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.cost > b.cost; });
  std::vector<GemmTile> tiles, rows;
  for (auto& c : cands) (c.t.cfg >= CFG_ROWS ? rows : tiles).push_back(c.t);
  cp.n_gemm_tiles = (int64_t)tiles.size();
  cp.n_gemm_rows = (int64_t)rows.size();
  int rc = dev_upload(ctx, &cp.d_gemm_items, gl.data(), gl.size() * sizeof(GemmItem));
  if (rc != TK_OK) return rc;
  rc = dev_upload(ctx, &cp.d_gemm_tiles, tiles.data(), tiles.size() * sizeof(GemmTile));
  if (rc != TK_OK) return rc;
  rc = dev_upload(ctx, &cp.d_gemm_rows, rows.data(), rows.size() * sizeof(GemmTile));
  if (rc != TK_OK) return rc;
  if (!cp.zeros.empty()) {
    rc = dev_upload(ctx, &cp.d_zero, cp.zeros.data(), cp.zeros.size() * sizeof(ZeroItem));
    if (rc != TK_OK) return rc;
  }
  if (nslots > 0) {
    std::vector<int> zeros((size_t)nslots, 0);
    rc = dev_upload(ctx, &cp.d_split_counters, zeros.data(), zeros.size() * sizeof(int));
    if (rc != TK_OK) return rc;
    cp.partials_bytes = (size_t)nslots * SPLIT_MAX * 32 * 32 * (cp.dtype == TK_C128 ? 16 : 8);
  }
  return TK_OK;
}

int launch_gemm_fp64(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c,
                     void* partials, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const GemmItem* items = (const GemmItem*)cp.d_gemm_items;
  if (cp.n_gemm_tiles > 0) {
    ProfScope prof(ctx, "k_gemm_f64", stream);
    const GemmTile* tiles = (const GemmTile*)cp.d_gemm_tiles;
    int* counters = (int*)cp.d_split_counters;
    if (cp.dtype == TK_C128)
      k_gemm_f64<double2><<<(unsigned)cp.n_gemm_tiles, 256, 0, s>>>(items, tiles, (const double2*)a, (const double2*)b,
                                                                    (double2*)c, (double2*)partials, counters);
    else
      k_gemm_f64<double><<<(unsigned)cp.n_gemm_tiles, 256, 0, s>>>(items, tiles, (const double*)a, (const double*)b,
                                                                   (double*)c, (double*)partials, counters);
    int rc = check_launch(ctx, "k_gemm_f64");
    if (rc != TK_OK) return rc;
  }
  if (cp.n_gemm_rows > 0) {
    ProfScope prof(ctx, "k_gemm_rows", stream);
    const GemmTile* rows = (const GemmTile*)cp.d_gemm_rows;
    if (cp.dtype == TK_C128)
      k_gemm_rows<double2, false><<<(unsigned)cp.n_gemm_rows, 256, 0, s>>>(items, rows, (const double2*)a,
                                                                           (const double2*)b, (double2*)c);
    else if (cp.gemm_mode == TK_GEMM_FP64)
      k_gemm_rows<double, false><<<(unsigned)cp.n_gemm_rows, 256, 0, s>>>(items, rows, (const double*)a,
                                                                          (const double*)b, (double*)c);
    else
      k_gemm_rows<double, true><<<(unsigned)cp.n_gemm_rows, 256, 0, s>>>(items, rows, (const double*)a,
                                                                         (const double*)b, (double*)c);
    return check_launch(ctx, "k_gemm_rows");
  }
  return TK_OK;
}

int launch_zero(Ctx* ctx, const ContractPlan& cp, void* c, void* stream) {
  if (cp.zeros.empty()) return TK_OK;
  int64_t maxn = 0;
  for (auto& z : cp.zeros) maxn = std::max(maxn, z.n);
  dim3 grid((unsigned)std::min<int64_t>((maxn + 255) / 256, 1024), (unsigned)std::min<size_t>(cp.zeros.size(), 65535));
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope prof(ctx, "k_zero", stream);
  if (cp.dtype == TK_C128)
    k_zero<double2><<<grid, 256, 0, s>>>((const ZeroItem*)cp.d_zero, (int)cp.zeros.size(), (double2*)c);
  else
    k_zero<double><<<grid, 256, 0, s>>>((const ZeroItem*)cp.d_zero, (int)cp.zeros.size(), (double*)c);
  return check_launch(ctx, "k_zero");
}

int run_contract(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                 void* stream) {
  char* w = (char*)ws;
  const void* at = cp.pa->identity ? a : (const void*)(w + cp.ws_at);
  const void* bt = cp.pb->identity ? b : (const void*)(w + cp.ws_bt);
  void* ct = cp.pc ? (void*)(w + cp.ws_ct) : c;
  int rc;
  if (!cp.pa->identity && (rc = launch_permute(ctx, *cp.pa, a, (void*)at, stream)) != TK_OK) return rc;
  if (!cp.pb->identity && (rc = launch_permute(ctx, *cp.pb, b, (void*)bt, stream)) != TK_OK) return rc;
  if ((rc = launch_zero(ctx, cp, ct, stream)) != TK_OK) return rc;
  if (!cp.gemms_fp64.empty() && (rc = launch_gemm_fp64(ctx, cp, at, bt, ct, w + cp.ws_partials, stream)) != TK_OK)
    return rc;
  if (!cp.gemms_oz.empty() && (rc = launch_gemm_ozaki(ctx, cp, at, bt, ct, w + cp.ws_slices, stream)) != TK_OK)
    return rc;
  if (cp.pc && (rc = launch_permute(ctx, *cp.pc, ct, c, stream)) != TK_OK) return rc;
  return TK_OK;
}

}  // namespace tk
