// extern "C" boundary of libtk: handles, argument checking, error mapping, execution order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <exception>
#include <new>

#include "abi_handles.hpp"

namespace {

int fail(tk_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->c.last_error = msg;
  return code;
}

template <typename F>
int guarded(tk_ctx* ctx, F&& f) {
  try {
    return f();
  } catch (const tk::Error& e) {
    return fail(ctx, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(ctx, TK_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ctx, TK_ERR_ARG, e.what());
  } catch (...) {
    return fail(ctx, TK_ERR_ARG, "unknown error");
  }
}

bool read_perm(int np, const int* p, int nq, const int* q, std::vector<int>& vp, std::vector<int>& vq) {
  if (np < 0 || nq < 0 || np + nq > 8) return false;
  if ((np > 0 && !p) || (nq > 0 && !q)) return false;
  vp.assign(p, p + np);
  vq.assign(q, q + nq);
  return true;
}

int set_device(tk_ctx* ctx) {
  if (ctx->c.device < 0) return fail(ctx, TK_ERR_NO_DEVICE, "execution call on a host-only context");
  if (cudaSetDevice(ctx->c.device) != cudaSuccess) return fail(ctx, TK_ERR_CUDA, "cudaSetDevice failed");
  return TK_OK;
}

// An execution call given a NULL stream runs on the context's stream.
void* use_stream(const tk_ctx* ctx, void* stream) { return stream ? stream : ctx->c.stream; }

// A buffer may be NULL only when its tensor map has no elements (nothing is read or written).
bool have(const void* p, int64_t numel) { return p != nullptr || numel == 0; }

bool operands_present(const tk::ContractPlan& cp, const void* a, const void* b, const void* c) {
  return have(a, cp.pa->in->numel) && have(b, cp.pb->in->numel) && have(c, cp.c->numel);
}

}  // namespace

extern "C" {

int tk_version(void) { return 100; }

const char* tk_status_string(int s) {
  switch (s) {
    case TK_OK: return "ok";
    case TK_ERR_ARG: return "invalid argument";
    case TK_ERR_SPACE_MISMATCH: return "space mismatch";
    case TK_ERR_PERM: return "invalid permutation";
    case TK_ERR_SECTOR: return "invalid sector";
    case TK_ERR_OOM: return "out of memory";
    case TK_ERR_CUDA: return "CUDA error";
    case TK_ERR_UNSUPPORTED: return "unsupported";
    case TK_ERR_TIMEOUT: return "device wait timed out";
    case TK_ERR_WORKSPACE: return "workspace too small";
    case TK_ERR_NO_DEVICE: return "host-only context";
    case TK_ERR_BUDGET: return "device memory budget exceeded";
  }
  return "unknown status";
}

int tk_ctx_create(int device, void* stream, tk_alloc_fn alloc, tk_free_fn release, void* alloc_user,
                  tk_ctx** out) {
  if (!out) return TK_ERR_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (release == nullptr)) return TK_ERR_ARG;  // both hooks or neither
  tk_ctx* ctx = new (std::nothrow) tk_ctx();
  if (!ctx) return TK_ERR_OOM;
  ctx->c.device = device < 0 ? -1 : device;
  ctx->c.stream = device < 0 ? nullptr : stream;
  ctx->c.mem = std::make_shared<tk::DeviceMemory>();
  ctx->c.mem->device = ctx->c.device;
  ctx->c.mem->alloc = alloc;
  ctx->c.mem->release = release;
  ctx->c.mem->user = alloc_user;
  if (device >= 0) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) {
      delete ctx;
      return TK_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->c.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      delete ctx;
      return TK_ERR_CUDA;
    }
    void* st = nullptr;
    int rc = tk::dev_alloc(&ctx->c, &st, sizeof(int) * 4);
    if (rc != TK_OK) {
      delete ctx;
      return rc;
    }
    ctx->c.d_status = (int*)st;
    cudaStream_t side = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemsetAsync(ctx->c.d_status, 0, sizeof(int) * 4, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
      if (side) cudaStreamDestroy(side);
      if (e0) cudaEventDestroy(e0);
      tk::dev_free(ctx->c.d_status);
      delete ctx;
      return TK_ERR_CUDA;
    }
    ctx->c.side = side;
    ctx->c.ev_fork = e0;
    ctx->c.ev_join = e1;
  }
  *out = ctx;
  return TK_OK;
}

void tk_ctx_destroy(tk_ctx* ctx) {
  if (!ctx) return;
  if (ctx->c.device >= 0) {
    cudaSetDevice(ctx->c.device);
    ctx->c.perm_cache.clear();
    ctx->c.contract_cache.clear();
    tk::dev_free(ctx->c.d_status);
    if (ctx->c.side) cudaStreamDestroy((cudaStream_t)ctx->c.side);
    if (ctx->c.ev_fork) cudaEventDestroy((cudaEvent_t)ctx->c.ev_fork);
    if (ctx->c.ev_join) cudaEventDestroy((cudaEvent_t)ctx->c.ev_join);
  }
  delete ctx;
}

int tk_ctx_set_budget(tk_ctx* ctx, size_t bytes) {
  if (!ctx) return TK_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->c.mem->mu);
  ctx->c.mem->budget = bytes;
  return TK_OK;
}

int tk_ctx_reserve(tk_ctx* ctx, size_t bytes) {
  if (!ctx) return TK_ERR_ARG;
  tk::DeviceMemory& m = *ctx->c.mem;
  std::lock_guard<std::mutex> lk(m.mu);
  if (m.budget && m.in_use + m.reserved + bytes > m.budget) {
    ctx->c.last_error = "reserving " + std::to_string(bytes) + " bytes would exceed the budget of " +
                        std::to_string(m.budget) + " (library " + std::to_string(m.in_use) + ", reserved " +
                        std::to_string(m.reserved) + ")";
    return TK_ERR_BUDGET;
  }
  m.reserved += bytes;
  return TK_OK;
}

int tk_ctx_release(tk_ctx* ctx, size_t bytes) {
  if (!ctx) return TK_ERR_ARG;
  tk::DeviceMemory& m = *ctx->c.mem;
  std::lock_guard<std::mutex> lk(m.mu);
  if (bytes > m.reserved) return fail(ctx, TK_ERR_ARG, "releasing more than was reserved");
  m.reserved -= bytes;
  return TK_OK;
}

int tk_ctx_memory(tk_ctx* ctx, size_t* library_bytes, size_t* reserved_bytes, size_t* budget_bytes,
                  int64_t* allocations) {
  if (!ctx) return TK_ERR_ARG;
  tk::DeviceMemory& m = *ctx->c.mem;
  std::lock_guard<std::mutex> lk(m.mu);
  if (library_bytes) *library_bytes = m.in_use;
  if (reserved_bytes) *reserved_bytes = m.reserved;
  if (budget_bytes) *budget_bytes = m.budget;
  if (allocations) *allocations = (int64_t)m.allocations;
  return TK_OK;
}

int tk_ctx_alloc(tk_ctx* ctx, size_t bytes, void** out) {
  if (!ctx || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  rc = tk::dev_alloc(&ctx->c, out, bytes);
  if (rc == TK_ERR_BUDGET) return fail(ctx, rc, "allocation of " + std::to_string(bytes) + " bytes exceeds the budget");
  if (rc != TK_OK) return fail(ctx, rc, "device allocation failed");
  return TK_OK;
}

int tk_ctx_free(tk_ctx* ctx, void* ptr) {
  if (!ctx) return TK_ERR_ARG;
  if (!ptr) return TK_OK;
  if (!tk::dev_owns(ptr)) return fail(ctx, TK_ERR_ARG, "not an allocation of the library");
  if (ctx->c.device >= 0) cudaSetDevice(ctx->c.device);
  tk::dev_free(ptr);
  return TK_OK;
}

const char* tk_ctx_last_error(const tk_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

int tk_ctx_sync(tk_ctx* ctx, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx) return TK_ERR_ARG;
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(ctx, TK_ERR_CUDA, std::string("stream sync: ") + cudaGetErrorString(e));
  int status[4] = {0, 0, 0, 0};
  if (cudaMemcpy(status, ctx->c.d_status, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "reading device status failed");
  if (status[0] != 0) {
    cudaMemset(ctx->c.d_status, 0, sizeof(int) * 4);
    return fail(ctx, TK_ERR_TIMEOUT, "a bounded device-side wait gave up (kernel tag " +
                                         std::to_string(status[1]) + ")");
  }
  return TK_OK;
}

int64_t tk_ctx_launch_count(const tk_ctx* ctx) { return ctx ? ctx->c.launches : -1; }

int tk_ctx_selftest_timeout(tk_ctx* ctx, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx) return TK_ERR_ARG;
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  return guarded(ctx, [&] { return launch_wait_selftest(&ctx->c, stream); });
}

int tk_ctx_profile(tk_ctx* ctx, int enable) {
  if (!ctx) return TK_ERR_ARG;
  if (ctx->c.device < 0) return fail(ctx, TK_ERR_NO_DEVICE, "profiling needs a device context");
  ctx->c.profiling = enable != 0;
  return TK_OK;
}

int tk_ctx_profile_read(tk_ctx* ctx, int max, char* names, int64_t* counts, double* total_ms, int* n_out) {
  if (!ctx || max < 0 || (max > 0 && (!names || !counts || !total_ms)) || !n_out) return TK_ERR_ARG;
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  std::vector<std::string> keys;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  int status = TK_OK;
  for (auto& r : ctx->c.prof) {
    float t = 0.f;
    cudaEvent_t s = (cudaEvent_t)r.start, e = (cudaEvent_t)r.end;
    if (cudaEventSynchronize(e) != cudaSuccess || cudaEventElapsedTime(&t, s, e) != cudaSuccess)
      status = TK_ERR_CUDA;
    cudaEventDestroy(s);
    cudaEventDestroy(e);
    size_t i = 0;
    while (i < keys.size() && keys[i] != r.name) ++i;
    if (i == keys.size()) {
      keys.push_back(r.name);
      cnt.push_back(0);
      ms.push_back(0.0);
    }
    cnt[i] += 1;
    ms[i] += t;
  }
  ctx->c.prof.clear();
  *n_out = (int)keys.size();
  for (int i = 0; i < (int)keys.size() && i < max; ++i) {
    std::memset(names + 32 * i, 0, 32);
    std::strncpy(names + 32 * i, keys[i].c_str(), 31);
    counts[i] = cnt[i];
    total_ms[i] = ms[i];
  }
  if (status != TK_OK) return fail(ctx, status, "reading profile events failed");
  return TK_OK;
}

int tk_space_create(tk_ctx* ctx, int sym, int nsec, const int32_t* sectors, const int64_t* mults,
                    int is_dual, tk_space** out) {
  if (!out) return fail(ctx, TK_ERR_ARG, "null out");
  *out = nullptr;
  if (sym < 0 || sym > TK_SYM_Z2_U1) return fail(ctx, TK_ERR_ARG, "unknown symmetry");
  if (nsec <= 0 || !sectors || !mults) return fail(ctx, TK_ERR_ARG, "a space needs at least one sector");
  return guarded(ctx, [&]() {
    std::vector<std::pair<int32_t, int64_t>> v;
    for (int i = 0; i < nsec; ++i) {
      if (!tk::sector_valid(sym, sectors[i])) return fail(ctx, TK_ERR_SECTOR, "invalid sector label");
      if (mults[i] <= 0) return fail(ctx, TK_ERR_ARG, "multiplicities must be positive");
      v.push_back({sectors[i], mults[i]});
    }
    std::sort(v.begin(), v.end());
    for (size_t i = 1; i < v.size(); ++i)
      if (v[i].first == v[i - 1].first) return fail(ctx, TK_ERR_ARG, "duplicate sector");
    auto* s = new tk_space();
    s->s.sym = sym;
    for (auto& kv : v) {
      s->s.sectors.push_back(kv.first);
      s->s.mults.push_back(kv.second);
    }
    s->s.dual = is_dual != 0;
    s->s.finalize();
    *out = s;
    return TK_OK;
  });
}

int tk_space_dual(tk_ctx* ctx, const tk_space* v, tk_space** out) {
  if (!v || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  return guarded(ctx, [&]() {
    auto* s = new tk_space();
    s->s = v->s.flipped();
    *out = s;
    return TK_OK;
  });
}

void tk_space_destroy(tk_space* v) { delete v; }
int64_t tk_space_dim(const tk_space* v) { return v ? v->s.dim() : -1; }
int64_t tk_space_reduced_dim(const tk_space* v) { return v ? v->s.reduced_dim() : -1; }

int tk_tmap_create(tk_ctx* ctx, int n_cod, const tk_space* const* cod, int n_dom,
                   const tk_space* const* dom, tk_tmap** out) {
  if (!out) return fail(ctx, TK_ERR_ARG, "null out");
  *out = nullptr;
  if (n_cod < 0 || n_dom < 0 || n_cod + n_dom < 1 || n_cod + n_dom > 8)
    return fail(ctx, TK_ERR_ARG, "a tensor map has 1 to 8 legs");
  if ((n_cod && !cod) || (n_dom && !dom)) return fail(ctx, TK_ERR_ARG, "null space array");
  return guarded(ctx, [&]() {
    std::vector<tk::Space> c, d;
    int sym = -1;
    for (int i = 0; i < n_cod; ++i) {
      if (!cod[i]) return fail(ctx, TK_ERR_ARG, "null space");
      c.push_back(cod[i]->s);
    }
    for (int i = 0; i < n_dom; ++i) {
      if (!dom[i]) return fail(ctx, TK_ERR_ARG, "null space");
      d.push_back(dom[i]->s);
    }
    for (auto& s : c) sym = sym < 0 ? s.sym : sym;
    for (auto& s : d) sym = sym < 0 ? s.sym : sym;
    for (auto& s : c)
      if (s.sym != sym) return fail(ctx, TK_ERR_ARG, "mixed symmetries");
    for (auto& s : d)
      if (s.sym != sym) return fail(ctx, TK_ERR_ARG, "mixed symmetries");
    auto* t = new tk_tmap();
    t->st = tk::build_structure(sym, c, d);
    *out = t;
    return TK_OK;
  });
}

void tk_tmap_destroy(tk_tmap* t) { delete t; }
int64_t tk_tmap_numel(const tk_tmap* t) { return t ? t->st->numel : -1; }
uint64_t tk_tmap_hash(const tk_tmap* t) { return t ? t->st->hash : 0; }

int tk_tmap_nlegs(const tk_tmap* t, int* n_cod, int* n_dom) {
  if (!t) return TK_ERR_ARG;
  if (n_cod) *n_cod = (int)t->st->cod.size();
  if (n_dom) *n_dom = (int)t->st->dom.size();
  return TK_OK;
}

int tk_tmap_leg(tk_ctx* ctx, const tk_tmap* t, int leg, tk_space** out) {
  if (!t || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  int n1 = (int)t->st->cod.size();
  if (leg < 0 || leg >= t->st->nleg()) return fail(ctx, TK_ERR_ARG, "leg out of range");
  auto* s = new (std::nothrow) tk_space();
  if (!s) return TK_ERR_OOM;
  s->s = leg < n1 ? t->st->cod[leg] : t->st->dom[leg - n1];
  *out = s;
  return TK_OK;
}

int tk_tmap_nblocks(const tk_tmap* t) { return t ? (int)t->st->blocks.size() : -1; }

int tk_tmap_block(const tk_tmap* t, int i, int32_t* sector, int64_t* rows, int64_t* cols, int64_t* offset) {
  if (!t || i < 0 || i >= (int)t->st->blocks.size()) return TK_ERR_ARG;
  const tk::Block& b = t->st->blocks[i];
  if (sector) *sector = b.c;
  if (rows) *rows = b.rows;
  if (cols) *cols = b.cols;
  if (offset) *offset = b.offset;
  return TK_OK;
}

int64_t tk_tmap_ntreepairs(const tk_tmap* t) { return t ? (int64_t)t->st->pairs.size() : -1; }

int tk_tmap_treepair(const tk_tmap* t, int64_t i, int32_t* labels, int64_t* offset, int64_t* ld,
                     int64_t* dims) {
  if (!t || i < 0 || i >= (int64_t)t->st->pairs.size()) return TK_ERR_ARG;
  const tk::Structure& st = *t->st;
  const tk::TreePair& p = st.pairs[i];
  const tk::Block& b = st.blocks[p.block];
  const tk::Tree& s = st.split_trees[b.split[p.s]];
  const tk::Tree& f = st.fuse_trees[b.fuse[p.f]];
  if (labels) {
    int k = 0;
    for (auto x : s.unc) labels[k++] = x;
    for (auto x : f.unc) labels[k++] = x;
    for (auto x : s.inner) labels[k++] = x;
    labels[k++] = b.c;
    for (auto x : f.inner) labels[k++] = x;
  }
  if (offset) *offset = p.offset;
  if (ld) *ld = b.rows;
  if (dims) {
    std::vector<int64_t> d;
    st.pair_dims(p, d);
    for (size_t k = 0; k < d.size(); ++k) dims[k] = d[k];
  }
  return TK_OK;
}

int tk_permute_plan(tk_ctx* ctx, const tk_tmap* a, int np, const int* p, int nq, const int* q,
                    int dtype, tk_plan** out) {
  if (!ctx || !a || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  std::vector<int> vp, vq;
  if (!read_perm(np, p, nq, q, vp, vq) || np + nq != a->st->nleg())
    return fail(ctx, TK_ERR_PERM, "(p, q) must list every leg once");
  return guarded(ctx, [&]() {
    if (ctx->c.device >= 0 && cudaSetDevice(ctx->c.device) != cudaSuccess)
      return fail(ctx, TK_ERR_CUDA, "cudaSetDevice failed");
    auto pl = new tk_plan();
    pl->kind = 0;
    try {
      pl->perm = tk::make_permute_plan(&ctx->c, a->st, vp, vq, dtype);
    } catch (...) {
      delete pl;
      throw;
    }
    *out = pl;
    return TK_OK;
  });
}

int tk_adjoint_plan(tk_ctx* ctx, const tk_tmap* a, int dtype, tk_plan** out) {
  if (!ctx || !a || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  return guarded(ctx, [&]() {
    if (ctx->c.device >= 0 && cudaSetDevice(ctx->c.device) != cudaSuccess)
      return fail(ctx, TK_ERR_CUDA, "cudaSetDevice failed");
    auto pl = new tk_plan();
    pl->kind = 0;
    try {
      pl->perm = tk::make_adjoint_plan(&ctx->c, a->st, dtype);
    } catch (...) {
      delete pl;
      throw;
    }
    *out = pl;
    return TK_OK;
  });
}

int tk_contract_plan(tk_ctx* ctx, const tk_tmap* a, int npa, const int* pa, int nqa, const int* qa,
                     const tk_tmap* b, int npb, const int* pb, int nqb, const int* qb, int npab,
                     const int* pab, int nqab, const int* qab, int dtype, int gemm_mode, int slices,
                     tk_plan** out) {
  if (!ctx || !a || !b || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  if (gemm_mode < TK_GEMM_FP64 || gemm_mode > TK_GEMM_TF32X3) return fail(ctx, TK_ERR_ARG, "unknown gemm mode");
  if (slices < 0 || slices > 8) return fail(ctx, TK_ERR_ARG, "slices must be in [0, 8]");
  std::vector<int> vpa, vqa, vpb, vqb, vpab, vqab;
  if (!read_perm(npa, pa, nqa, qa, vpa, vqa) || npa + nqa != a->st->nleg() ||
      !read_perm(npb, pb, nqb, qb, vpb, vqb) || npb + nqb != b->st->nleg() ||
      !read_perm(npab, pab, nqab, qab, vpab, vqab))
    return fail(ctx, TK_ERR_PERM, "permutation tuples must list every leg once");
  if (npab + nqab != npa + nqb) return fail(ctx, TK_ERR_PERM, "(pab, qab) must list the legs of A~ o B~");
  return guarded(ctx, [&]() {
    if (ctx->c.device >= 0 && cudaSetDevice(ctx->c.device) != cudaSuccess)
      return fail(ctx, TK_ERR_CUDA, "cudaSetDevice failed");
    auto pl = new tk_plan();
    pl->kind = 1;
    try {
      pl->con = tk::make_contract_plan(&ctx->c, a->st, vpa, vqa, b->st, vpb, vqb, vpab, vqab, dtype,
                                       gemm_mode, slices);
    } catch (...) {
      delete pl;
      throw;
    }
    *out = pl;
    return TK_OK;
  });
}

int tk_compose_plan(tk_ctx* ctx, const tk_tmap* a, const tk_tmap* b, int dtype, int gemm_mode, int slices,
                    tk_plan** out) {
  if (!ctx || !a || !b || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  // A o B = the contraction of A's domain with B's codomain, legs kept in place (Sec. 2.3)
  const int n1a = (int)a->st->cod.size(), n2a = (int)a->st->dom.size();
  const int n1b = (int)b->st->cod.size(), n2b = (int)b->st->dom.size();
  std::vector<int> pa(n1a), qa(n2a), pb(n1b), qb(n2b), pab(n1a), qab(n2b);
  for (int i = 0; i < n1a; ++i) pa[i] = pab[i] = i;
  for (int i = 0; i < n2a; ++i) qa[i] = n1a + i;
  for (int i = 0; i < n1b; ++i) pb[i] = i;
  for (int i = 0; i < n2b; ++i) {
    qb[i] = n1b + i;
    qab[i] = n1a + i;
  }
  return tk_contract_plan(ctx, a, n1a, pa.data(), n2a, qa.data(), b, n1b, pb.data(), n2b, qb.data(), n1a,
                          pab.data(), n2b, qab.data(), dtype, gemm_mode, slices, out);
}

void tk_plan_destroy(tk_plan* plan) { delete plan; }

int tk_plan_output(tk_ctx* ctx, const tk_plan* plan, tk_tmap** out) {
  if (!plan || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  auto* t = new (std::nothrow) tk_tmap();
  if (!t) return TK_ERR_OOM;
  t->st = plan->kind == 0 ? plan->perm->out : plan->kind == 1 ? plan->con->c : plan->svd->u;
  *out = t;
  return TK_OK;
}

size_t tk_plan_workspace_bytes(const tk_plan* plan) {
  if (!plan) return 0;
  if (plan->kind == 2) return plan->svd->ws_total;
  if (plan->kind != 1) return 0;
  return tk::contract_ws_bytes(*plan->con);
}

double tk_plan_flops(const tk_plan* plan) {
  if (!plan || plan->kind != 1) return 0.0;
  return plan->con->flops;
}

double tk_plan_tensor_flops(const tk_plan* plan) {
  if (!plan || plan->kind != 1) return 0.0;
  const tk::ContractPlan& cp = plan->con->re ? *plan->con->re : *plan->con;
  double f = 0;
  for (const tk::GemmItem& g : cp.gemms_oz) f += 2.0 * (double)g.M * (double)g.N * (double)g.K;
  return plan->con->re ? 4.0 * f : f;  // a complex plan runs four real products
}

double tk_plan_permute_bytes(const tk_plan* plan) {
  if (!plan) return 0.0;
  if (plan->kind == 0) return plan->perm->identity ? 0.0 : plan->perm->bytes;
  double b = 0;
  const auto& c = plan->con->re ? *plan->con->re : *plan->con;
  if (!c.pa->identity) b += c.pa->bytes;
  if (!c.pb->identity) b += c.pb->bytes;
  if (c.pc) b += c.pc->bytes;
  return plan->con->re ? 4.0 * b : b;  // a complex plan runs four real products
}

static const tk::PermutePlan* which_perm(const tk_plan* plan, int which) {
  if (!plan) return nullptr;
  if (plan->kind == 0) return which == 0 ? plan->perm.get() : nullptr;
  const auto& c = *plan->con;
  const tk::PermutePlan* p = which == 0 ? c.pa.get() : which == 1 ? c.pb.get() : which == 2 ? c.pc.get() : nullptr;
  if (p && p->identity) return nullptr;
  return p;
}

int64_t tk_plan_ntransform(const tk_plan* plan, int which) {
  const tk::PermutePlan* p = which_perm(plan, which);
  return p ? (int64_t)p->terms.size() : -1;
}

int tk_plan_transform(const tk_plan* plan, int which, int64_t k, int64_t* src_offset,
                      int64_t* dst_offset, double* coef) {
  const tk::PermutePlan* p = which_perm(plan, which);
  if (!p || k < 0 || k >= (int64_t)p->terms.size()) return TK_ERR_ARG;
  const tk::TransformTerm& t = p->terms[k];
  if (src_offset) *src_offset = p->in->pairs[t.src_pair].offset;
  if (dst_offset) *dst_offset = p->out->pairs[t.dst_pair].offset;
  if (coef) *coef = t.coef;
  return TK_OK;
}

int tk_plan_permute_stats(const tk_plan* plan, int which, int64_t* stats) {
  const tk::PermutePlan* p = which_perm(plan, which);
  if (!p || !stats) return TK_ERR_ARG;
  for (int i = 0; i < 8; ++i) stats[i] = 0;
  auto elems = [](const tk::PermTask& t) {
    int64_t n = 1;
    for (int k = 0; k < t.ndim; ++k) n *= t.ext[k];
    return n;
  };
  for (const auto& t : p->rtasks) {
    stats[0] += 1;
    stats[1] += elems(t);
  }
  stats[2] = (int64_t)p->runs.size();
  for (const auto& t : p->tasks) {
    const int m = (t.mode == 1 || t.mode == 3) ? 3 : 5;
    stats[m] += 1;
    stats[m + 1] += elems(t);
  }
  stats[7] = p->total_tiles;
  return TK_OK;
}

int tk_permute(tk_ctx* ctx, const tk_plan* plan, const void* a, void* c, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || !plan || plan->kind != 0) return fail(ctx, TK_ERR_ARG, "not a permute plan");
  const tk::PermutePlan& pp = *plan->perm;
  if (!have(a, pp.in->numel) || !have(c, pp.out->numel)) return fail(ctx, TK_ERR_ARG, "null buffer");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  if (pp.out->numel == 0) return TK_OK;  // nothing to write: no launch
  if (pp.identity) {
    size_t bytes = (size_t)pp.in->numel * (pp.dtype == TK_C128 ? 16 : 8);
    if (a == c) return TK_OK;
    if (cudaMemcpyAsync(c, a, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
      return fail(ctx, TK_ERR_CUDA, "device copy failed");
    return TK_OK;
  }
  return tk::launch_permute(&ctx->c, pp, a, c, stream);
}

int tk_contract(tk_ctx* ctx, const tk_plan* plan, const void* a, const void* b, void* c,
                void* workspace, size_t workspace_bytes, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || !plan || plan->kind != 1) return fail(ctx, TK_ERR_ARG, "not a contraction plan");
  const tk::ContractPlan& cp = *plan->con;
  if (!operands_present(cp, a, b, c)) return fail(ctx, TK_ERR_ARG, "null buffer");
  const size_t need = tk::contract_ws_bytes(cp);
  if (workspace_bytes < need || (need > 0 && !workspace))
    return fail(ctx, TK_ERR_WORKSPACE, "workspace smaller than tk_plan_workspace_bytes()");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  if (cp.c->numel == 0) return TK_OK;  // nothing to write: no launch
  return tk::run_contract(&ctx->c, cp, a, b, c, workspace, stream);
}

int tk_contract_batch(tk_ctx* ctx, int n, const tk_plan* const* plans, const void* const* a,
                      const void* const* b, void* const* c, void* const* workspace,
                      const size_t* workspace_bytes, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || n < 0) return fail(ctx, TK_ERR_ARG, "bad batch");
  if (n == 0) return TK_OK;
  if (!plans || !a || !b || !c || !workspace || !workspace_bytes) return fail(ctx, TK_ERR_ARG, "null array");
  std::vector<const tk::ContractPlan*> cps((size_t)n);
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || plans[i]->kind != 1) return fail(ctx, TK_ERR_ARG, "not a contraction plan");
    const tk::ContractPlan& cp = *plans[i]->con;
    if (!operands_present(cp, a[i], b[i], c[i])) return fail(ctx, TK_ERR_ARG, "null buffer");
    if (workspace_bytes[i] < cp.ws_total || (cp.ws_total > 0 && !workspace[i]))
      return fail(ctx, TK_ERR_WORKSPACE, "workspace smaller than tk_plan_workspace_bytes()");
    if (cp.gemm_mode != plans[0]->con->gemm_mode || cp.dtype != plans[0]->con->dtype)
      return fail(ctx, TK_ERR_UNSUPPORTED, "a batch takes plans of one dtype and one gemm mode");
    if (cp.re) return fail(ctx, TK_ERR_UNSUPPORTED, "complex split-precision plans run one by one");
    cps[(size_t)i] = &cp;
  }
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  return tk::run_contract_batch(&ctx->c, n, cps.data(), a, b, c, workspace, stream);
}

static int autotune_contract(tk_ctx* ctx, tk::ContractPlan& cp, const void* a, const void* b, void* c,
                             void* workspace, size_t workspace_bytes, void* stream, int* choice) {
  int rc = TK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ctx, TK_ERR_CUDA, "stream synchronize failed");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "event creation failed");
  // time one configuration: median of three runs after one warm-up; infinite if it does not fit
  auto measure = [&](float* ms) -> int {
    *ms = 1e30f;
    int r = tk::finalize_device_tables(&ctx->c, cp);
    if (r != TK_OK) return r;
    if (cp.ws_total > workspace_bytes) return TK_OK;
    float t[3];
    if ((r = tk::run_contract(&ctx->c, cp, a, b, c, workspace, stream)) != TK_OK) return r;
    for (float& x : t) {
      cudaEventRecord(e0, s);
      if ((r = tk::run_contract(&ctx->c, cp, a, b, c, workspace, stream)) != TK_OK) return r;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return TK_ERR_CUDA;
      cudaEventElapsedTime(&x, e0, e1);
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return TK_OK;
  };
  struct Cand {
    int tile, split;
  };
  const Cand fp64c[] = {{0, 0}, {32, 1}, {64, 1}, {32, 2}, {64, 2}};
  const Cand ozc[] = {{0, 0}, {64, 1}, {128, 1}, {64, 2}, {128, 2}};
  int best_i = 0, best_j = 0, best_k = 0;
  float best = 1e30f, ms = 0;
  for (int i = 0; i < 5 && rc == TK_OK; ++i) {  // FP64 work list (heuristic split-precision choice)
    cp.tune_tile = fp64c[i].tile;
    cp.tune_split = fp64c[i].split;
    cp.tune_oz_bn = cp.tune_oz_split = 0;
    if ((rc = measure(&ms)) == TK_OK && ms < best) {
      best = ms;
      best_i = i;
    }
  }
  if (rc == TK_OK && cp.gemm_mode != TK_GEMM_FP64 && !cp.gemms_oz.empty()) {
    cp.tune_tile = fp64c[best_i].tile;
    cp.tune_split = fp64c[best_i].split;
    best = 1e30f;
    for (int j = 0; j < 5 && rc == TK_OK; ++j) {  // split-precision work list
      cp.tune_oz_bn = ozc[j].tile;
      cp.tune_oz_split = ozc[j].split;
      cp.tune_oz_img = 0;
      if ((rc = measure(&ms)) == TK_OK && ms < best) {
        best = ms;
        best_j = j;
      }
    }
    cp.tune_oz_bn = ozc[best_j].tile;
    cp.tune_oz_split = ozc[best_j].split;
    // the preparation without chunk images (where its heuristic uses them): only switching them
    // off is tried, since these back-to-back runs keep the operands in L2, which favours the
    // images more than a cold-cache run beside the double-float rows does
    for (int k = 1; k < 2 && rc == TK_OK; ++k) {
      cp.tune_oz_img = k;
      if ((rc = measure(&ms)) == TK_OK && ms < best) {
        best = ms;
        best_k = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cp.tune_tile = fp64c[best_i].tile;
  cp.tune_split = fp64c[best_i].split;
  cp.tune_oz_bn = ozc[best_j].tile;
  cp.tune_oz_split = ozc[best_j].split;
  cp.tune_oz_img = best_k;
  const int rc2 = tk::finalize_device_tables(&ctx->c, cp);
  if (rc != TK_OK) return fail(ctx, rc, "autotuning run failed");
  if (rc2 != TK_OK) return fail(ctx, rc2, "rebuilding the chosen work lists failed");
  if (choice) *choice = best_k * 64 + best_i * 8 + best_j;
  return TK_OK;
}

int tk_plan_set_choice(tk_ctx* ctx, tk_plan* plan, int choice) {
  if (!ctx || !plan || plan->kind != 1) return fail(ctx, TK_ERR_ARG, "not a contraction plan");
  const int i = (choice / 8) % 8, j = choice % 8, k = choice / 64;
  if (choice < 0 || i > 4 || j > 4 || k > 2) return fail(ctx, TK_ERR_ARG, "not an autotuner choice");
  static const int tile[] = {0, 32, 64, 32, 64}, split[] = {0, 1, 1, 2, 2};
  static const int oz_tile[] = {0, 64, 128, 64, 128};
  tk::ContractPlan& cp = plan->con->re ? *plan->con->re : *plan->con;
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  cp.tune_tile = tile[i];
  cp.tune_split = split[i];
  cp.tune_oz_bn = oz_tile[j];
  cp.tune_oz_split = split[j];
  cp.tune_oz_img = k;
  if ((rc = tk::finalize_device_tables(&ctx->c, cp)) != TK_OK) return fail(ctx, rc, "rebuilding the work lists failed");
  return TK_OK;
}

int tk_plan_autotune(tk_ctx* ctx, tk_plan* plan, const void* a, const void* b, void* c, void* workspace,
                     size_t workspace_bytes, void* stream, int* choice) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || !plan || plan->kind != 1) return fail(ctx, TK_ERR_ARG, "not a contraction plan");
  tk::ContractPlan& cp = *plan->con;
  if (!operands_present(cp, a, b, c) || !workspace) return fail(ctx, TK_ERR_ARG, "null buffer");
  if (cp.c->numel == 0) {  // nothing to time: keep the heuristic work lists
    if (choice) *choice = 0;
    return TK_OK;
  }
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  if (!cp.re) return autotune_contract(ctx, cp, a, b, c, workspace, workspace_bytes, stream, choice);
  // complex split precision: one full run leaves Re A and Re B in the workspace; the real plan
  // is tuned on them (its result buffer is the first real product's), then the total is resized
  if (workspace_bytes < tk::contract_ws_bytes(cp))
    return fail(ctx, TK_ERR_WORKSPACE, "workspace smaller than tk_plan_workspace_bytes()");
  if ((rc = tk::run_contract(&ctx->c, cp, a, b, c, workspace, stream)) != TK_OK) return fail(ctx, rc, "autotuning run failed");
  char* w = (char*)workspace;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const void* ar = w;
  const void* br = w + 2 * al((size_t)cp.cx_na * 8);
  void* t0 = w + 2 * al((size_t)cp.cx_na * 8) + 2 * al((size_t)cp.cx_nb * 8);
  rc = autotune_contract(ctx, *cp.re, ar, br, t0, w + cp.ws_cx, workspace_bytes - cp.ws_cx, stream, choice);
  return rc;
}

int tk_svd_plan(tk_ctx* ctx, const tk_tmap* a, int dtype, tk_plan** out) {
  if (!ctx || !a || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  return guarded(ctx, [&]() {
    if (ctx->c.device >= 0 && cudaSetDevice(ctx->c.device) != cudaSuccess)
      return fail(ctx, TK_ERR_CUDA, "cudaSetDevice failed");
    auto pl = new tk_plan();
    pl->kind = 2;
    try {
      pl->svd = tk::make_svd_plan(&ctx->c, a->st, dtype);
    } catch (...) {
      delete pl;
      throw;
    }
    *out = pl;
    return TK_OK;
  });
}

int tk_svd_outputs(tk_ctx* ctx, const tk_plan* plan, tk_tmap** u, tk_tmap** vh, int64_t* nvalues) {
  if (!plan || plan->kind != 2) return fail(ctx, TK_ERR_ARG, "not an SVD plan");
  if (u) {
    *u = new (std::nothrow) tk_tmap();
    if (!*u) return TK_ERR_OOM;
    (*u)->st = plan->svd->u;
  }
  if (vh) {
    *vh = new (std::nothrow) tk_tmap();
    if (!*vh) return TK_ERR_OOM;
    (*vh)->st = plan->svd->vh;
  }
  if (nvalues) *nvalues = plan->svd->nvalues;
  return TK_OK;
}

int64_t tk_svd_nblocks(const tk_plan* plan) { return plan && plan->kind == 2 ? (int64_t)plan->svd->blocks.size() : -1; }

int tk_svd_block(const tk_plan* plan, int64_t i, int32_t* sector, int64_t* rows, int64_t* cols, int64_t* values_offset) {
  if (!plan || plan->kind != 2 || i < 0 || i >= (int64_t)plan->svd->blocks.size()) return TK_ERR_ARG;
  const tk::SvdBlock& k = plan->svd->blocks[(size_t)i];
  if (sector) *sector = k.c;
  if (rows) *rows = k.m;
  if (cols) *cols = k.n;
  if (values_offset) *values_offset = k.s_off;
  return TK_OK;
}

int tk_svd(tk_ctx* ctx, const tk_plan* plan, const void* a, void* u, double* s, void* vh, void* workspace,
           size_t workspace_bytes, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || !plan || plan->kind != 2) return fail(ctx, TK_ERR_ARG, "not an SVD plan");
  const tk::SvdPlan& sp = *plan->svd;
  if (sp.blocks.empty()) return TK_OK;  // a map with no blocks: nothing to factor, no launch
  if (!a || !u || !s || !vh) return fail(ctx, TK_ERR_ARG, "null buffer");
  if (workspace_bytes < sp.ws_total || !workspace)
    return fail(ctx, TK_ERR_WORKSPACE, "workspace smaller than tk_plan_workspace_bytes()");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  rc = tk::run_svd(&ctx->c, sp, a, u, s, vh, workspace, stream);
  return rc == TK_OK ? TK_OK : fail(ctx, rc, ctx->c.last_error.empty() ? "block SVD failed" : ctx->c.last_error);
}

int tk_svd_truncate(tk_ctx* ctx, const tk_plan* plan, const int64_t* keep, const void* u, const double* s,
                    const void* vh, void* ut, double* st, void* vht, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || !plan || plan->kind != 2) return fail(ctx, TK_ERR_ARG, "not an SVD plan");
  const size_t nb = plan->svd->blocks.size();
  if (nb > 0 && !keep) return fail(ctx, TK_ERR_ARG, "null keep counts");
  int64_t kept = 0;
  for (size_t i = 0; i < nb; ++i) {
    if (keep[i] < 0 || keep[i] > plan->svd->blocks[i].r)
      return fail(ctx, TK_ERR_ARG, "keep count outside 0..min(rows, cols)");
    kept += keep[i];
  }
  if (kept == 0) return TK_OK;  // nothing kept: empty outputs, no copy
  if (!u || !s || !vh || !ut || !st || !vht) return fail(ctx, TK_ERR_ARG, "null buffer");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  rc = tk::run_svd_truncate(&ctx->c, *plan->svd, keep, u, s, vh, ut, st, vht, stream);
  return rc == TK_OK ? TK_OK : fail(ctx, rc, "truncation copy failed");
}

static int tmap_io_check(tk_ctx* ctx, const tk_tmap* t, int dtype, size_t bytes) {
  if (!t) return fail(ctx, TK_ERR_ARG, "null tensor map");
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  const size_t want = (size_t)t->st->numel * (dtype == TK_C128 ? 16 : 8);
  if (bytes != want)
    return fail(ctx, TK_ERR_ARG, "tensor map of " + std::to_string(t->st->numel) + " elements holds " +
                                     std::to_string(want) + " bytes, not " + std::to_string(bytes));
  return TK_OK;
}

int tk_tmap_upload(tk_ctx* ctx, const tk_tmap* t, int dtype, const void* host, size_t bytes, void* device,
                   void* stream) {
  if (!ctx) return TK_ERR_ARG;
  stream = use_stream(ctx, stream);
  int rc = tmap_io_check(ctx, t, dtype, bytes);
  if (rc != TK_OK) return rc;
  if (bytes && (!host || !device)) return fail(ctx, TK_ERR_ARG, "null buffer");
  if ((rc = set_device(ctx)) != TK_OK) return rc;
  if (bytes && cudaMemcpyAsync(device, host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "host to device copy failed");
  return TK_OK;
}

int tk_tmap_download(tk_ctx* ctx, const tk_tmap* t, int dtype, const void* device, void* host, size_t bytes,
                     void* stream) {
  if (!ctx) return TK_ERR_ARG;
  stream = use_stream(ctx, stream);
  int rc = tmap_io_check(ctx, t, dtype, bytes);
  if (rc != TK_OK) return rc;
  if (bytes && (!host || !device)) return fail(ctx, TK_ERR_ARG, "null buffer");
  if ((rc = set_device(ctx)) != TK_OK) return rc;
  if (bytes && cudaMemcpyAsync(host, device, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "device to host copy failed");
  return TK_OK;
}

int tk_tmap_alloc(tk_ctx* ctx, const tk_tmap* t, int dtype, void** out) {
  if (!ctx || !out) return fail(ctx, TK_ERR_ARG, "null argument");
  *out = nullptr;
  if (!t) return fail(ctx, TK_ERR_ARG, "null tensor map");
  if (dtype != TK_F64 && dtype != TK_C128) return fail(ctx, TK_ERR_ARG, "unknown dtype");
  return tk_ctx_alloc(ctx, (size_t)t->st->numel * (dtype == TK_C128 ? 16 : 8), out);
}

int tk_copy_h2d(tk_ctx* ctx, void* dst_device, const void* src_host, size_t bytes, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || (bytes && (!dst_device || !src_host))) return fail(ctx, TK_ERR_ARG, "null argument");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  if (cudaMemcpyAsync(dst_device, src_host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "host to device copy failed");
  return TK_OK;
}

int tk_copy_d2h(tk_ctx* ctx, void* dst_host, const void* src_device, size_t bytes, void* stream) {
  if (ctx) stream = use_stream(ctx, stream);
  if (!ctx || (bytes && (!dst_host || !src_device))) return fail(ctx, TK_ERR_ARG, "null argument");
  int rc = set_device(ctx);
  if (rc != TK_OK) return rc;
  if (cudaMemcpyAsync(dst_host, src_device, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return fail(ctx, TK_ERR_CUDA, "device to host copy failed");
  return TK_OK;
}

}  // extern "C"
