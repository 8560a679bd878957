// Block singular value decomposition of a symmetric tensor map and its truncation (the
// decomposition after the two-site step, Algorithm 12 with Algorithm 9).
//
// For t : cod <- dom every coupled sector c carries one block t_c (rows: splitting trees of cod,
// columns: fusion trees of dom).  With orthonormal canonical trees the SVD of t is the SVD of
// each block: t = U S V^dagger with the bond space W = sum_c (c, r_c), r_c = min(rows_c, cols_c),
// U : cod <- W (block c: rows_c x r_c), S diagonal on W and V^dagger : W <- dom (block c:
// r_c x cols_c).  Each block is factorised by cuSOLVER's Jacobi SVD (gesvdj, economy size) on a
// copy in the caller's workspace; V is turned into V^dagger by a transpose kernel (conjugating
// complex data).  Truncation keeps, per sector, the leading k_c <= r_c singular triplets: the
// first k_c columns of U's block (a contiguous prefix, column-major) and the first k_c rows of
// V^dagger's block (a strided 2-D copy).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cstring>

#include "tk_internal.hpp"

namespace tk {

SvdPlan::~SvdPlan() = default;

void* solver_handle(Ctx* ctx) {
  if (!ctx || ctx->device < 0) return nullptr;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->solver) {
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return nullptr;
    ctx->solver = h;
  }
  return ctx->solver;
}

void destroy_solver_handle(Ctx* ctx) {
  if (ctx && ctx->solver) {
    cusolverDnDestroy((cusolverDnHandle_t)ctx->solver);
    ctx->solver = nullptr;
  }
}

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
  int64_t s_off = 0, amax = 0;
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
    amax = std::max(amax, b.rows * b.cols + b.cols * r);  // A copy + V (n x r)
    sp->blocks.push_back(k);
  }
  sp->nvalues = s_off;
  // workspace: the largest block's A copy and V, then the solver's work array and info word
  const size_t es = dtype == TK_C128 ? 16 : 8;
  sp->ws_solver = ((size_t)amax * es + 255) & ~(size_t)255;
  sp->lwork = 0;
  if (ctx && ctx->device >= 0 && !sp->blocks.empty()) {
    cusolverDnHandle_t h = (cusolverDnHandle_t)solver_handle(ctx);
    if (!h) throw Error{TK_ERR_CUDA, "cusolverDnCreate failed"};
    gesvdjInfo_t params;
    if (cusolverDnCreateGesvdjInfo(&params) != CUSOLVER_STATUS_SUCCESS) throw Error{TK_ERR_CUDA, "gesvdj info"};
    for (const SvdBlock& k : sp->blocks) {
      int lw = 0;
      cusolverStatus_t st;
      if (dtype == TK_C128)
        st = cusolverDnZgesvdj_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)k.m, (int)k.n, nullptr, (int)k.m,
                                          nullptr, nullptr, (int)k.m, nullptr, (int)k.n, &lw, params);
      else
        st = cusolverDnDgesvdj_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)k.m, (int)k.n, nullptr, (int)k.m,
                                          nullptr, nullptr, (int)k.m, nullptr, (int)k.n, &lw, params);
      if (st != CUSOLVER_STATUS_SUCCESS) {
        cusolverDnDestroyGesvdjInfo(params);
        throw Error{TK_ERR_CUDA, "gesvdj buffer size query failed"};
      }
      sp->lwork = std::max<int64_t>(sp->lwork, lw);
    }
    cusolverDnDestroyGesvdjInfo(params);
  }
  sp->ws_total = sp->ws_solver + (((size_t)sp->lwork * es + 255) & ~(size_t)255) + 256;
  return sp;
}

namespace {

// V (n x r, column-major) -> V^dagger (r x n, column-major), conjugated for complex data.
template <typename T>
__global__ void k_adjoint_copy(const T* __restrict__ v, T* __restrict__ vh, int64_t n, int64_t r) {
  __shared__ T tile[32][33];
  const int64_t bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // bi over n, bj over r
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int y = ty; y < 32; y += 8) {
    const int64_t i = bi + tx, j = bj + y;
    if (i < n && j < r) tile[y][tx] = v[i + j * n];
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int64_t j = bj + tx, i = bi + y;
    if (i < n && j < r) {
      T x = tile[tx][y];
      if constexpr (sizeof(T) == 16) x.y = -x.y;
      vh[j + i * r] = x;
    }
  }
}

}  // namespace

int run_svd(Ctx* ctx, const SvdPlan& sp, const void* a, void* u, double* s, void* vh, void* ws, void* stream) {
  if (sp.blocks.empty()) return TK_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cusolverDnHandle_t h = (cusolverDnHandle_t)solver_handle(ctx);
  if (!h || cusolverDnSetStream(h, st) != CUSOLVER_STATUS_SUCCESS) {
    ctx->last_error = "cuSOLVER handle unavailable";
    return TK_ERR_CUDA;
  }
  gesvdjInfo_t params;
  if (cusolverDnCreateGesvdjInfo(&params) != CUSOLVER_STATUS_SUCCESS) return TK_ERR_CUDA;
  const size_t es = sp.dtype == TK_C128 ? 16 : 8;
  char* w = (char*)ws;
  void* acopy = w;
  void* work = w + sp.ws_solver;
  int* info = (int*)(w + sp.ws_total - 256);
  int rc = TK_OK;
  ProfScope prof(ctx, "svd_gesvdj", stream);
  for (const SvdBlock& k : sp.blocks) {
    char* vbuf = (char*)acopy + (size_t)k.m * k.n * es;  // V (n x r) after the A copy
    if (cudaMemcpyAsync(acopy, (const char*)a + (size_t)k.a_off * es, (size_t)k.m * k.n * es, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess) {
      rc = TK_ERR_CUDA;
      break;
    }
    cusolverStatus_t cs;
    if (sp.dtype == TK_C128)
      cs = cusolverDnZgesvdj(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)k.m, (int)k.n, (cuDoubleComplex*)acopy, (int)k.m,
                             s + k.s_off, (cuDoubleComplex*)u + k.u_off, (int)k.m, (cuDoubleComplex*)vbuf, (int)k.n,
                             (cuDoubleComplex*)work, (int)sp.lwork, info, params);
    else
      cs = cusolverDnDgesvdj(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)k.m, (int)k.n, (double*)acopy, (int)k.m, s + k.s_off,
                             (double*)u + k.u_off, (int)k.m, (double*)vbuf, (int)k.n, (double*)work, (int)sp.lwork,
                             info, params);
    if (cs != CUSOLVER_STATUS_SUCCESS) {
      ctx->last_error = "gesvdj failed";
      rc = TK_ERR_CUDA;
      break;
    }
    const dim3 grid((unsigned)((k.n + 31) / 32), (unsigned)((k.r + 31) / 32)), block(32, 8);
    if (sp.dtype == TK_C128)
      k_adjoint_copy<double2><<<grid, block, 0, st>>>((const double2*)vbuf, (double2*)vh + k.vh_off, k.n, k.r);
    else
      k_adjoint_copy<double><<<grid, block, 0, st>>>((const double*)vbuf, (double*)vh + k.vh_off, k.n, k.r);
    if (cudaGetLastError() != cudaSuccess) {
      rc = TK_ERR_CUDA;
      break;
    }
    ctx->launches += 1;
  }
  cusolverDnDestroyGesvdjInfo(params);
  return rc;
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
