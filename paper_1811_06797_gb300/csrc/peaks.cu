// Instrumentation (no counterpart in the paper): the FMA issue rate of the
// CUDA cores, measured with CUDA events on the context stream, so that the
// roofline denominators of the FP64 and FP32 kernels come from this library
// and not from a constant.  Each thread runs FMA_CHAINS independent
// dependency chains of fma(a, b, c) for `iters` steps; the chains are folded
// into one store per thread so that nothing is optimised away.
#include <algorithm>

#include "iga_internal.cuh"

namespace iga {

constexpr int FMA_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, T b, T c, T* __restrict__ out) {
  T a[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static double fma_rate(iga_ctx* ctx) {
  // 8 CTAs of 256 threads per SM: enough resident warps to cover the FMA
  // latency; b < 1 keeps the chains finite
  const int blocks = ctx->nsm * 8, threads = 256, iters = 1 << 14;
  DevBuf<T> out((size_t)blocks * threads);
  cudaEvent_t e0, e1;
  IGA_CUDA(cudaEventCreate(&e0));
  IGA_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
    IGA_CUDA(cudaEventRecord(e0, ctx->stream));
    IGA_LAUNCH(ctx, fma_rate_kernel<T>, blocks, threads, 0, iters, (T)0.999, (T)1e-4, out.p);
    IGA_CUDA(cudaEventRecord(e1, ctx->stream));
    IGA_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    IGA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = 2.0 * FMA_CHAINS * (double)iters * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace iga

using namespace iga;

extern "C" iga_status iga_measure_fma(iga_ctx* ctx, iga_prec prec, double* tflops) {
  if (!ctx || !tflops) return IGA_EINVAL;
  try {
    AllocScope scope(ctx->stream);
    if (prec == IGA_FP64) *tflops = fma_rate<double>(ctx);
    else if (prec == IGA_FP32) *tflops = fma_rate<float>(ctx);
    else throw Error(IGA_EINVAL, "measure_fma: precision must be IGA_FP64 or IGA_FP32");
    return IGA_OK;
  } catch (const Error& e) {
    set_error(ctx, e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_error(ctx, e.what());
    return IGA_ECUDA;
  }
}

extern "C" iga_status iga_gemm_batched(iga_ctx* ctx, iga_prec prec, int tA, int tB, int M, int N,
                                       int K, double alpha, const void* A, int lda, long long sA,
                                       const void* B, int ldb, long long sB, double beta, void* C,
                                       int ldc, long long sC, int count) {
  if (!ctx) return IGA_EINVAL;
  try {
    IGA_REQUIRE(M >= 0 && N >= 0 && K >= 0 && count >= 0, "gemm_batched: negative size");
    if (M == 0 || N == 0 || count == 0) return IGA_OK;
    IGA_REQUIRE(A && B && C, "gemm_batched: null pointer");
    IGA_REQUIRE(lda >= (tA ? M : K) && ldb >= (tB ? K : N) && ldc >= N && lda > 0 && ldb > 0,
                "gemm_batched: leading dimension shorter than a row");
    AllocScope scope(ctx->stream);
    if (prec == IGA_FP64)
      gemm_rm_batched<double>(ctx, tA != 0, tB != 0, M, N, K, alpha, (const double*)A, lda, sA,
                              (const double*)B, ldb, sB, beta, (double*)C, ldc, sC, count);
    else if (prec == IGA_FP32)
      gemm_rm_batched<float>(ctx, tA != 0, tB != 0, M, N, K, (float)alpha, (const float*)A, lda,
                             sA, (const float*)B, ldb, sB, (float)beta, (float*)C, ldc, sC,
                             count);
    else if (prec == IGA_TF32) {
      tc_flag_reset(ctx);
      tc_gemm_tf32(ctx, tA != 0, tB != 0, false, M, N, K, (float)alpha, (const float*)A, lda, sA,
                   (const float*)B, ldb, sB, (float)beta, (float*)C, ldc, sC, count);
    } else
      throw Error(IGA_EINVAL, "gemm_batched: precision must be IGA_FP64, IGA_FP32 or IGA_TF32");
    if (prec == IGA_TF32) tc_flag_check(ctx, "gemm_batched");
    return IGA_OK;
  } catch (const Error& e) {
    set_error(ctx, e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_error(ctx, e.what());
    return IGA_ECUDA;
  }
}
