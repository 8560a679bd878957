// Device memory of libtk: every allocation the library makes goes through its context's
// DeviceMemory (the caller's allocator hooks, or cudaMalloc / cudaFree), counted against an
// optional budget.  A registry keyed by address lets a plan's tables be freed without the plan
// knowing which context allocated them; it keeps each DeviceMemory alive until its last
// allocation is freed.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "tk_internal.hpp"

namespace tk {

namespace {

struct Allocation {
  std::shared_ptr<DeviceMemory> mem;
  size_t bytes;
};

std::mutex g_registry_mu;
std::unordered_map<void*, Allocation>& registry() {
  static auto* r = new std::unordered_map<void*, Allocation>();  // never destroyed: frees may run at exit
  return *r;
}

}  // namespace

int dev_alloc(Ctx* ctx, void** dst, size_t bytes) {
  *dst = nullptr;
  if (bytes == 0) return TK_OK;
  DeviceMemory* m = ctx->mem.get();
  if (!m) return TK_ERR_OOM;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    if (m->budget && m->in_use + m->reserved + bytes > m->budget) return TK_ERR_BUDGET;
    m->in_use += bytes;
  }
  void* p = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) p = nullptr;
  else if (m->alloc) p = m->alloc(bytes, m->user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (!p) {
    std::lock_guard<std::mutex> lk(m->mu);
    m->in_use -= bytes;
    return TK_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(m->mu);
    m->allocations += 1;
  }
  std::lock_guard<std::mutex> lk(g_registry_mu);
  registry()[p] = Allocation{ctx->mem, bytes};
  *dst = p;
  return TK_OK;
}

int dev_upload(Ctx* ctx, void** dst, const void* src, size_t bytes) {
  int rc = dev_alloc(ctx, dst, bytes);
  if (rc != TK_OK || bytes == 0) return rc;
  cudaStream_t s = (cudaStream_t)ctx->stream;
  if (cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    dev_free(*dst);
    *dst = nullptr;
    return TK_ERR_CUDA;
  }
  return TK_OK;
}

void dev_free(void* p) {
  if (!p) return;
  Allocation a;
  {
    std::lock_guard<std::mutex> lk(g_registry_mu);
    auto it = registry().find(p);
    if (it == registry().end()) return;  // not the library's
    a = it->second;
    registry().erase(it);
  }
  DeviceMemory* m = a.mem.get();
  if (m->release) m->release(p, a.bytes, m->user);
  else cudaFree(p);
  std::lock_guard<std::mutex> lk(m->mu);
  m->in_use -= a.bytes;
  m->allocations -= 1;
}

bool dev_owns(void* p) {
  std::lock_guard<std::mutex> lk(g_registry_mu);
  return registry().count(p) != 0;
}

}  // namespace tk
