// Peak probe of the FP64 pipe (the roofline denominator of the FP64 sector GEMMs): every thread
// runs a 4 x 4 register outer product, acc[i][j] += a[i] b[j], the inner loop of a GEMM tile with
// its operands already in registers.  The 16 accumulators are independent chains and a, b are
// per-thread run-time values (never constant-bank operands), so nothing but the FP64 pipe's issue
// rate bounds the kernel.  Timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <string>

#include "abi_handles.hpp"

namespace {

constexpr int kUnroll = 32;

__global__ void __launch_bounds__(256) k_probe_dfma(int64_t iters, double* sink) {
  double a[4], b[4], acc[16];
  const double t = (double)threadIdx.x * 1e-9;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = 1.0 + 1e-3 * (double)i + t;
    b[i] = 1e-3 * (double)(i + 1) - t;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i * 4 + j] = fma(a[i], b[j], acc[i * 4 + j]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += acc[i];
  // the sum is positive and below iters * 32 * 16 * 0.005: never this value, so nothing is
  // written, but the compiler must keep every chain
  if (s == -1.0) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int tk_probe_fp64_peak(tk_ctx* ctx, double seconds, double* tflops, double* ms_out, void* stream) {
  if (!ctx || !tflops || seconds <= 0.0 || seconds > 30.0) return TK_ERR_ARG;
  if (ctx->c.device < 0) return TK_ERR_NO_DEVICE;
  if (!stream) stream = ctx->c.stream;
  if (cudaSetDevice(ctx->c.device) != cudaSuccess) return TK_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = ctx->c.num_sms * 4;  // 4 CTAs of 256 threads (56 registers each) per SM: one wave
  const int threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TK_ERR_CUDA;
  }
  auto run = [&](int64_t iters, float* ms) -> int {
    cudaEventRecord(e0, s);
    k_probe_dfma<<<blocks, threads, 0, s>>>(iters, nullptr);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) return TK_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return TK_OK;
  };
  float ms = 0.f;
  int rc = run(64, &ms);  // warm-up and calibration
  int64_t iters = 64;
  while (rc == TK_OK && ms < 20.f && iters < (int64_t)1 << 30) {
    iters *= 4;
    rc = run(iters, &ms);
  }
  if (rc == TK_OK) {
    iters = (int64_t)((double)iters * (seconds * 1e3) / (double)ms) + 1;
    rc = run(iters, &ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TK_OK) {
    ctx->c.last_error = "FP64 probe launch failed";
    return rc;
  }
  ctx->c.launches += 1;
  const double flops = 2.0 * (double)blocks * threads * (double)iters * kUnroll * 16;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return TK_OK;
}
