// Split-precision grouped GEMM (K3): placeholder until the tcgen05 path lands.
#include <cuda_runtime.h>

#include "tk_internal.hpp"

namespace tk {

int upload_ozaki_tables(Ctx* ctx, ContractPlan& cp) {
  (void)ctx;
  (void)cp;
  return TK_ERR_UNSUPPORTED;
}

int launch_gemm_ozaki(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c,
                      void* slices_ws, void* stream) {
  (void)cp; (void)a; (void)b; (void)c; (void)slices_ws; (void)stream;
  ctx->last_error = "split-precision GEMM not available";
  return TK_ERR_UNSUPPORTED;
}

}  // namespace tk
