// tk_contract_noalloc: the contraction of tk_contract with its scratch memory taken from a
// fixed array compiled into this library, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted -- a host program
// whose device memory is entirely owned by another framework's allocator, a real-time or
// serving loop that must not take the implicit device synchronisation a cudaMalloc/cudaFree can
// cause, or a plug-in that is handed only its input and output buffers.  Those callers can still
// run a planned contraction: they pass A, B and C, and the permuted operands A~, B~ and the
// intermediate C~ live in the array below instead of in a caller-allocated workspace.
//
// The array is a file-scope __device__ object: every GPU that loads libtk holds
// kNoallocScratchBytes of it until the process exits.  In host code its name is only a host-side
// stand-in, so the device address is looked up once per device with cudaGetSymbolAddress (with
// that device current) and passed to the kernels.  Every call shares the array and it keeps the
// previous call's contents; each call writes every byte it reads before reading it, so nothing
// has to start at zero.  Two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "abi_handles.hpp"

namespace {

constexpr size_t kNoallocScratchBytes = TK_NOALLOC_SCRATCH_BYTES;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current); looked up once.
int scratch_address(int device, void** out, std::string& err) {
  if (device < 0 || device >= kMaxDevices) {
    err = "device index out of range for the built-in scratch table";
    return TK_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      err = std::string("cudaGetSymbolAddress of the built-in scratch array failed: ") + cudaGetErrorString(e);
      return TK_ERR_CUDA;
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return TK_OK;
}

}  // namespace

extern "C" size_t tk_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" int tk_contract_noalloc(tk_ctx* ctx, const tk_plan* plan, const void* a, const void* b, void* c,
                                   void* stream) {
  if (!ctx) return TK_ERR_ARG;
  if (!stream) stream = ctx->c.stream;
  if (!plan || plan->kind != 1) {
    ctx->c.last_error = "not a contraction plan";
    return TK_ERR_ARG;
  }
  const tk::ContractPlan& cp = *plan->con;
  // a buffer may be NULL only when its tensor map has no elements
  if ((!a && cp.pa->in->numel > 0) || (!b && cp.pb->in->numel > 0) || (!c && cp.c->numel > 0)) {
    ctx->c.last_error = "null buffer";
    return TK_ERR_ARG;
  }
  if (ctx->c.device < 0) {
    ctx->c.last_error = "execution call on a host-only context";
    return TK_ERR_NO_DEVICE;
  }
  if (tk::contract_ws_bytes(cp) > kNoallocScratchBytes) {
    ctx->c.last_error = "plan needs " + std::to_string(tk::contract_ws_bytes(cp)) +
                        " bytes of scratch; tk_contract_noalloc has " + std::to_string(kNoallocScratchBytes) +
                        " (use tk_contract with a caller-allocated workspace)";
    return TK_ERR_WORKSPACE;
  }
  if (cudaSetDevice(ctx->c.device) != cudaSuccess) {
    ctx->c.last_error = "cudaSetDevice failed";
    return TK_ERR_CUDA;
  }
  if (cp.c->numel == 0) return TK_OK;  // nothing to write: no launch
  void* scratch = nullptr;
  std::string err;
  int rc = scratch_address(ctx->c.device, &scratch, err);
  if (rc != TK_OK) {
    ctx->c.last_error = err;
    return rc;
  }
  return tk::run_contract(&ctx->c, cp, a, b, c, scratch, stream);
}
