// Block singular value decomposition of a symmetric tensor map and its truncation (the
// decomposition after the two-site step, Algorithm 12 with Algorithm 9).
//
// For t : cod <- dom every coupled sector c carries one block t_c (rows: splitting trees of cod,
// columns: fusion trees of dom).  With orthonormal canonical trees the SVD of t is the SVD of
// each block: t = U S V^dagger with the bond space W = sum_c (c, r_c), r_c = min(rows_c, cols_c),
// U : cod <- W (block c: rows_c x r_c), S diagonal on W and V^dagger : W <- dom (block c:
// r_c x cols_c).
//
// All blocks are factorised in one launch, one CTA per block, by one-sided Jacobi (Hestenes):
// the columns of a working copy G (the block, or its adjoint when it has fewer rows than columns,
// so that G is M x N with M >= N) are made mutually orthogonal by plane rotations, which are
// accumulated in an N x N matrix Q (G_final = G_0 Q).  Then the singular values are the column
// norms of G_final, its normalised columns are the left vectors of G_0 and Q holds the right
// vectors.  A sweep visits every column pair once, in the round-robin (circle) order: each round
// is N/2 disjoint pairs, one per warp, so the rounds of a sweep need no other synchronisation
// than a CTA barrier between them.  A pair (i, j) with Gram entries a = |g_i|^2, b = |g_j|^2,
// g = g_i^H g_j is rotated when |g| > tol sqrt(a b), tol = sqrt(M) eps: with g = |g| e^{i phi},
// the phase e^{-i phi} on column j makes the 2 x 2 Gram matrix real, and the Jacobi rotation
// [[c, s], [-s, c]] with t = s / c = sign(z) / (|z| + sqrt(1 + z^2)), z = (b - a) / (2 |g|)
// diagonalises it.  The sweeps stop when a sweep rotates no pair (or after kMaxSweeps).
// Singular values are then ordered descending within the block by rank counting.
//
// Truncation keeps, per sector, the leading k_c <= r_c singular triplets: the first k_c columns
// of U's block (a contiguous prefix, column-major) and the first k_c rows of V^dagger's block (a
// strided 2-D copy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "tk_device.cuh"
#include "tk_internal.hpp"

namespace tk {

SvdPlan::~SvdPlan() { dev_free(d_jobs); }

namespace {

constexpr int kSvdThreads = 512;  // 16 warps: 16 column pairs rotated at a time
constexpr int kSvdGroup = 512;    // pairs of one round handled per three-step group
constexpr size_t kSvdSmemG = 180 * 1024;  // a block whose G fits in this many bytes keeps G in shared memory
constexpr int kMaxSweeps = 60;

struct SvdJob {       // one block's factorisation, device side
  int64_t m, n;       // block rows, columns
  int64_t a_off, u_off, vh_off, s_off;
  int64_t g_off, q_off, norm_off;  // working arrays in the workspace (elements of T / doubles)
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// scalar helpers for double and interleaved complex double
__device__ __forceinline__ double cj(double x) { return x; }
__device__ __forceinline__ double2 cj(double2 x) { return make_double2(x.x, -x.y); }
__device__ __forceinline__ double abs2(double x) { return x * x; }
__device__ __forceinline__ double abs2(double2 x) { return x.x * x.x + x.y * x.y; }
// x^H y accumulated into acc
__device__ __forceinline__ void dot_acc(double& acc, double x, double y) { acc = fma(x, y, acc); }
__device__ __forceinline__ void dot_acc(double2& acc, double2 x, double2 y) {
  acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
  acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }
__device__ __forceinline__ double mag(double g) { return fabs(g); }
__device__ __forceinline__ double mag(double2 g) { return hypot(g.x, g.y); }
// e^{-i phi} for g = |g| e^{i phi} (|g| > 0)
__device__ __forceinline__ double unit_conj_phase(double g, double) { return g >= 0.0 ? 1.0 : -1.0; }
__device__ __forceinline__ double2 unit_conj_phase(double2 g, double ag) { return make_double2(g.x / ag, -g.y / ag); }
__device__ __forceinline__ double2 mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ T zero_of();
template <>
__device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <>
__device__ __forceinline__ double2 zero_of<double2>() { return make_double2(0.0, 0.0); }
template <typename T>
__device__ __forceinline__ T one_of();
template <>
__device__ __forceinline__ double one_of<double>() { return 1.0; }
template <>
__device__ __forceinline__ double2 one_of<double2>() { return make_double2(1.0, 0.0); }

// The plane rotation of columns x, y (n entries, one warp, lanes along the column):
// x' = c x - s ph y, y' = s x + c ph y.  For real data ph = +-1 is folded into the coefficients
// (four FP64 operations per entry instead of five).
__device__ __forceinline__ void rotate_columns(double* x, double* y, int64_t n, double c, double sn, double ph,
                                               int lane) {
  const double sp = sn * ph, cp = c * ph;
  for (int64_t e = lane; e < n; e += 32) {
    const double a = x[e], b = y[e];
    x[e] = fma(-sp, b, c * a);
    y[e] = fma(cp, b, sn * a);
  }
}
__device__ __forceinline__ void rotate_columns(double2* x, double2* y, int64_t n, double c, double sn, double2 ph,
                                               int lane) {
  for (int64_t e = lane; e < n; e += 32) {
    const double2 a = x[e], b = mul(y[e], ph);
    x[e] = add(scale(a, c), scale(b, -sn));
    y[e] = add(scale(a, sn), scale(b, c));
  }
}

// Column p of the round-robin schedule in round r (positions 0 .. np-1, np even): position 0 is
// fixed, the others rotate; pair k of round r is (pos(k), pos(np - 1 - k)).
__device__ __forceinline__ int64_t rr_column(int64_t pos, int64_t r, int64_t np) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (np - 1)) + 1;
}

template <typename T>
__global__ void __launch_bounds__(kSvdThreads) k_svd_jacobi(const SvdJob* __restrict__ jobs, const T* __restrict__ a,
                                                            T* __restrict__ u, double* __restrict__ s,
                                                            T* __restrict__ vh, T* __restrict__ ws,
                                                            double* __restrict__ wsd, size_t g_smem) {
  extern __shared__ __align__(16) unsigned char svd_dyn[];
  const SvdJob jb = jobs[blockIdx.x];
  const bool tall = jb.m >= jb.n;
  const int64_t M = tall ? jb.m : jb.n, N = tall ? jb.n : jb.m;  // G is M x N, M >= N
  // G in shared memory when the launch gave enough (the largest fitting block sets the size), else
  // in the workspace; Q always in the workspace
  T* G = (size_t)jb.m * (size_t)jb.n * sizeof(T) <= g_smem ? reinterpret_cast<T*>(svd_dyn) : ws + jb.g_off;
  T* Q = ws + jb.q_off;
  double* nrm = wsd + jb.norm_off;
  const T* A = a + jb.a_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kSvdThreads / 32;
  // G = A (tall) or A^H (wide); Q = identity
  for (int64_t e = tid; e < M * N; e += kSvdThreads) {
    const int64_t i = e % M, j = e / M;
    G[e] = tall ? A[i + j * jb.m] : cj(A[j + i * jb.m]);
  }
  for (int64_t e = tid; e < N * N; e += kSvdThreads) Q[e] = (e % N == e / N) ? one_of<T>() : zero_of<T>();
  __syncthreads();
  const double tol = sqrt((double)M) * 2.220446049250313e-16;
  const int64_t np = N + (N & 1);  // even number of positions (an odd N has one idle position)
  // A round's disjoint pairs go in groups of up to kSvdGroup, in three steps: every warp forms
  // the Gram entries of its pairs (lane sums), one thread per pair turns them into the rotation
  // (the square roots and divisions, done once per pair instead of once per lane), and every warp
  // rotates its pairs' columns of G and Q.  On this part the FP64 pipe retires two lanes per SM
  // per clock, and the per-pair scalar work done by all 32 lanes of a warp cost about as much as
  // the column arithmetic.
  __shared__ double s_al[kSvdGroup], s_be[kSvdGroup], s_c[kSvdGroup], s_sn[kSvdGroup];
  __shared__ T s_ga[kSvdGroup], s_ph[kSvdGroup];
  __shared__ int rotated;
  for (int sweep = 0; sweep < kMaxSweeps && N > 1; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int64_t r = 0; r < np - 1; ++r) {
      for (int64_t k0 = 0; k0 < np / 2; k0 += kSvdGroup) {
        const int64_t kn = min((int64_t)kSvdGroup, np / 2 - k0);
        // 1. Gram entries |g_i|^2, |g_j|^2, g_i^H g_j of each pair (an idle pair gets zeros)
        for (int64_t k = warp; k < kn; k += nwarps) {
          int64_t i = rr_column(k0 + k, r, np), j = rr_column(np - 1 - (k0 + k), r, np);
          if (i > j) {
            const int64_t t = i;
            i = j;
            j = t;
          }
          double al = 0.0, be = 0.0;
          T ga = zero_of<T>();
          if (j < N) {
            const T* gi = G + i * M;
            const T* gj = G + j * M;
            for (int64_t e = lane; e < M; e += 32) {
              const T x = gi[e], y = gj[e];
              al += abs2(x);
              be += abs2(y);
              dot_acc(ga, x, y);
            }
            al = warp_sum(al);
            be = warp_sum(be);
            ga = warp_sum(ga);
          }
          if (lane == 0) {
            s_al[k] = al;
            s_be[k] = be;
            s_ga[k] = ga;
          }
        }
        __syncthreads();
        // 2. one thread per pair: the rotation, or c = 0 marking "leave this pair alone"
        for (int64_t k = tid; k < kn; k += kSvdThreads) {
          const double al = s_al[k], be = s_be[k];
          const T ga = s_ga[k];
          const double ag = mag(ga);
          double c = 0.0, sn = 0.0;
          T ph = zero_of<T>();
          if (ag > tol * sqrt(al * be)) {  // not yet orthogonal to working precision
            const double z = (be - al) / (2.0 * ag);
            const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = c * t;
            ph = unit_conj_phase(ga, ag);  // e^{-i phi}
            rotated = 1;                   // every writer writes 1
          }
          s_c[k] = c;
          s_sn[k] = sn;
          s_ph[k] = ph;
        }
        __syncthreads();
        // 3. the rotations of G's and Q's columns
        for (int64_t k = warp; k < kn; k += nwarps) {
          const double c = s_c[k], sn = s_sn[k];
          if (c == 0.0) continue;  // warp-uniform: nothing to rotate (c = 1/sqrt(1 + t^2) > 0 otherwise)
          const T ph = s_ph[k];
          int64_t i = rr_column(k0 + k, r, np), j = rr_column(np - 1 - (k0 + k), r, np);
          if (i > j) {
            const int64_t t = i;
            i = j;
            j = t;
          }
          rotate_columns(G + i * M, G + j * M, M, c, sn, ph, lane);
          rotate_columns(Q + i * N, Q + j * N, N, c, sn, ph, lane);
        }
        __syncthreads();  // the next group reuses the shared arrays; the next round reads these columns
      }
    }
    __syncthreads();
    if (!rotated) break;
    __syncthreads();
  }
  // singular values: column norms of G, ordered descending (ties by column index)
  for (int64_t j = warp; j < N; j += nwarps) {
    double acc = 0.0;
    for (int64_t e = lane; e < M; e += 32) acc += abs2(G[e + j * M]);
    acc = warp_sum(acc);
    if (lane == 0) nrm[j] = sqrt(acc);
  }
  __syncthreads();
  const int64_t r = N;  // = min(m, n)
  for (int64_t j = tid; j < N; j += kSvdThreads) {
    const double sj = nrm[j];
    int64_t rank = 0;
    for (int64_t k = 0; k < N; ++k) {
      const double sk = nrm[k];
      rank += (sk > sj || (sk == sj && k < j)) ? 1 : 0;
    }
    s[jb.s_off + rank] = sj;
    nrm[N + j] = (double)rank;  // the column's place in the output
  }
  __syncthreads();
  T* U = u + jb.u_off;   // m x r
  T* VH = vh + jb.vh_off;  // r x n
  for (int64_t e = tid; e < M * N; e += kSvdThreads) {
    const int64_t i = e % M, j = e / M;
    const int64_t rk = (int64_t)nrm[N + j];
    const double sj = nrm[j];
    const T g = sj > 0.0 ? scale(G[e], 1.0 / sj) : G[e];
    if (tall) U[i + rk * jb.m] = g;      // left vectors of A
    else VH[rk + i * r] = cj(g);         // G = A^H: its left vectors are A's right vectors
  }
  for (int64_t e = tid; e < N * N; e += kSvdThreads) {
    const int64_t i = e % N, j = e / N;
    const int64_t rk = (int64_t)nrm[N + j];
    if (tall) VH[rk + i * r] = cj(Q[e]);  // V^dagger row rk = (column j of Q)^H
    else U[i + rk * jb.m] = Q[e];
  }
}

}  // namespace

std::shared_ptr<SvdPlan> make_svd_plan(Ctx* ctx, std::shared_ptr<Structure> in, int dtype) {
  auto sp = std::make_shared<SvdPlan>();
  sp->in = in;
  sp->dtype = dtype;
  Space w;
  w.sym = in->sym;
  for (const Block& b : in->blocks) {
    const int64_t r = std::min(b.rows, b.cols);
    if (r == 0) continue;
    w.sectors.push_back(b.c);
    w.mults.push_back(r);
  }
  w.dual = false;
  w.finalize();
  sp->bond = w;
  sp->u = build_structure(in->sym, in->cod, {w});
  sp->vh = build_structure(in->sym, {w}, in->dom);
  int64_t s_off = 0;
  for (const Block& b : in->blocks) {
    const int64_t r = std::min(b.rows, b.cols);
    if (r == 0) continue;
    SvdBlock k;
    k.c = b.c;
    k.m = b.rows;
    k.n = b.cols;
    k.r = r;
    k.a_off = b.offset;
    k.u_off = sp->u->blocks[sp->u->block_of(b.c)].offset;
    k.vh_off = sp->vh->blocks[sp->vh->block_of(b.c)].offset;
    k.s_off = s_off;
    s_off += r;
    sp->blocks.push_back(k);
  }
  sp->nvalues = s_off;
  // workspace: per block G (M x N) and Q (N x N) in the element type, then 2 N doubles (norms and
  // output ranks); largest blocks first in the job list so they start first
  const size_t es = dtype == TK_C128 ? 16 : 8;
  std::vector<SvdJob> jobs;
  int64_t elems = 0, dbl = 0;
  std::vector<size_t> order(sp->blocks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const SvdBlock &p = sp->blocks[x], &q = sp->blocks[y];
    return p.m * p.n * p.r > q.m * q.n * q.r;
  });
  for (size_t i : order) {
    const SvdBlock& k = sp->blocks[i];
    const int64_t M = std::max(k.m, k.n), N = std::min(k.m, k.n);
    SvdJob j{k.m, k.n, k.a_off, k.u_off, k.vh_off, k.s_off, elems, elems + M * N, dbl};
    elems += M * N + N * N;
    dbl += 2 * N;
    jobs.push_back(j);
  }
  sp->ws_solver = align256((size_t)elems * es);          // G and Q of every block
  sp->lwork = dbl;
  sp->ws_total = sp->ws_solver + align256((size_t)dbl * 8);
  sp->d_jobs = nullptr;
  sp->njobs = (int64_t)jobs.size();
  if (ctx && ctx->device >= 0 && !jobs.empty()) {
    int rc = dev_upload(ctx, &sp->d_jobs, jobs.data(), jobs.size() * sizeof(SvdJob));
    if (rc != TK_OK) throw Error{rc, "uploading the SVD job table failed"};
  }
  return sp;
}

int run_svd(Ctx* ctx, const SvdPlan& sp, const void* a, void* u, double* s, void* vh, void* ws, void* stream) {
  if (sp.njobs == 0) return TK_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double* wsd = (double*)((char*)ws + sp.ws_solver);
  // dynamic shared memory: the largest G (m n elements) that fits in kSvdSmemG
  const size_t es = sp.dtype == TK_C128 ? 16 : 8;
  size_t g_smem = 0;
  for (const SvdBlock& k : sp.blocks) {
    const size_t b = (size_t)k.m * (size_t)k.n * es;
    if (b <= kSvdSmemG) g_smem = std::max(g_smem, b);
  }
  static bool attr_set[64][2] = {};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device][es == 16]) {
    const cudaError_t e = es == 16 ? cudaFuncSetAttribute(k_svd_jacobi<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)kSvdSmemG)
                                   : cudaFuncSetAttribute(k_svd_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)kSvdSmemG);
    if (e != cudaSuccess) {
      ctx->last_error = "cannot reserve shared memory for the block SVD";
      return TK_ERR_CUDA;
    }
    attr_set[ctx->device][es == 16] = true;
  }
  {
    ProfScope prof(ctx, "k_svd_jacobi", stream);
    if (sp.dtype == TK_C128)
      k_svd_jacobi<double2><<<(unsigned)sp.njobs, kSvdThreads, g_smem, st>>>(
          (const SvdJob*)sp.d_jobs, (const double2*)a, (double2*)u, s, (double2*)vh, (double2*)ws, wsd, g_smem);
    else
      k_svd_jacobi<double><<<(unsigned)sp.njobs, kSvdThreads, g_smem, st>>>(
          (const SvdJob*)sp.d_jobs, (const double*)a, (double*)u, s, (double*)vh, (double*)ws, wsd, g_smem);
  }
  if (cudaGetLastError() != cudaSuccess) {
    ctx->last_error = "block SVD launch failed";
    return TK_ERR_CUDA;
  }
  ctx->launches += 1;
  return TK_OK;
}

int run_svd_truncate(Ctx* ctx, const SvdPlan& sp, const int64_t* keep, const void* u, const double* s, const void* vh,
                     void* ut, double* st_out, void* vht, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = sp.dtype == TK_C128 ? 16 : 8;
  int64_t uo = 0, so = 0, vo = 0;  // offsets in the truncated U, S, V^dagger (sector order)
  for (size_t i = 0; i < sp.blocks.size(); ++i) {
    const SvdBlock& k = sp.blocks[i];
    const int64_t kc = keep[i];
    if (kc < 0 || kc > k.r) {
      ctx->last_error = "keep count outside 0..min(rows, cols)";
      return TK_ERR_ARG;
    }
    if (kc == 0) continue;
    if (cudaMemcpyAsync((char*)ut + (size_t)uo * es, (const char*)u + (size_t)k.u_off * es, (size_t)(k.m * kc) * es,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(st_out + so, s + k.s_off, (size_t)kc * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess ||
        cudaMemcpy2DAsync((char*)vht + (size_t)vo * es, (size_t)kc * es, (const char*)vh + (size_t)k.vh_off * es,
                          (size_t)k.r * es, (size_t)kc * es, (size_t)k.n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return TK_ERR_CUDA;
    uo += k.m * kc;
    so += kc;
    vo += kc * k.n;
  }
  return TK_OK;
}

}  // namespace tk
