// Dense products of the solver's small and medium matrices (interface
// updates, frame projections, Gram matrices, TT expansions, the adjoint's
// fast-diagonalisation transforms, the TT-matrix apply's staged path) and
// the vector kernels of the local GMRES: written for this library instead of
// calling a BLAS.
//
// gemm: C_i (M x N) = alpha op(A_i) op(B_i) + beta C_i, row-major, a strided
// batch.  One CTA computes a BM x BN tile with 256 threads, each a TM x TN
// block of outputs in registers; the A and B panels of depth BK are staged
// in shared memory (transposed on the way in when an operand is transposed),
// so every shared-memory load feeds TM (or TN) FMAs.  FP64 uses 64 x 64,
// 64 x 16, 16 x 64 or 16 x 16 tiles (4 x 4 down to 1 x 1 per thread, the
// shape with the least padding: the FP64 pipe is the bound), FP32 128 x 128
// (8 x 8).
// A long reduction with few output tiles is split over the K dimension into
// partial products and summed by a second kernel in a fixed order, so that
// every result is deterministic.
#include <algorithm>
#include <cmath>

#include "iga_internal.cuh"

namespace iga {

template <typename T, int TM, int TN, int BK>
__global__ void __launch_bounds__(256)
gemm_tile_kernel(bool tA, bool tB, int M, int N, int K, T alpha, const T* __restrict__ A, int lda,
                 long long sA, const T* __restrict__ B, int ldb, long long sB, T beta,
                 T* __restrict__ C, int ldc, long long sC, int ksplit, int klen,
                 T* __restrict__ part) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int batch = blockIdx.z / ksplit, ks = blockIdx.z - batch * ksplit;
  const T* Ab = A + batch * sA;
  const T* Bb = B + batch * sB;
  const int kbeg = ks * klen, kend = min(K, kbeg + klen);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // op(A)(m, k) into As[k][m]: consecutive threads take consecutive k (A
    // row-major, contiguous in k) or consecutive m (A transposed)
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (tA) { mm = e % BM; kk = e / BM; }
      else { kk = e % BK; mm = e / BK; }
      const int m = m0 + mm, k = k0 + kk;
      T v = T(0);
      if (m < M && k < kend) v = tA ? Ab[(size_t)k * lda + m] : Ab[(size_t)m * lda + k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int nn, kk;
      if (tB) { kk = e % BK; nn = e / BK; }
      else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      T v = T(0);
      if (n < N && k < kend) v = tB ? Bb[(size_t)n * ldb + k] : Bb[(size_t)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      if (part) {
        part[((size_t)blockIdx.z * M + m) * N + n] = acc[i][j];
      } else {
        T* c = C + batch * sC + (size_t)m * ldc + n;
        *c = beta == T(0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
      }
    }
  }
}

// C_i = alpha sum_s part[i ksplit + s] + beta C_i, summed in split order
template <typename T>
__global__ void gemm_splitk_reduce_kernel(int M, int N, int ksplit, int count, T alpha,
                                          const T* __restrict__ part, T beta, T* __restrict__ C,
                                          int ldc, long long sC) {
  const size_t total = (size_t)count * M * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(idx % N);
    const size_t r = idx / N;
    const int m = (int)(r % M);
    const int b = (int)(r / M);
    T s = T(0);
    for (int k = 0; k < ksplit; ++k) s += part[(((size_t)b * ksplit + k) * M + m) * N + n];
    T* c = C + b * sC + (size_t)m * ldc + n;
    *c = beta == T(0) ? alpha * s : fma(alpha, s, beta * *c);
  }
}

// one tile shape: split the reduction when the output tiles cannot fill the
// GPU, then the tile kernel (and the ordered sum of the partial products)
template <typename T, int TM, int TN, int BK>
static void gemm_launch(iga_ctx* ctx, bool tA, bool tB, int M, int N, int K, T alpha, const T* A,
                        int lda, long long sA, const T* B, int ldb, long long sB, T beta, T* C,
                        int ldc, long long sC, int count) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const long long tiles = (long long)tm * tn * count;
  int ksplit = 1;
  if (K > 4 * BK && tiles < 2LL * ctx->nsm) {
    ksplit = (int)std::min<long long>((2LL * ctx->nsm + tiles - 1) / tiles, (K + 63) / 64);
    ksplit = std::max(1, std::min(ksplit, 256));
  }
  const int klen = ((K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
  ksplit = std::max(1, (K + klen - 1) / std::max(klen, 1));
  T* part = nullptr;
  if (ksplit > 1)
    part = scratch<T>(ctx, SLOT_GEMM_PART, (size_t)count * ksplit * M * N);
  // the grid's z extent is limited: long batches in chunks
  const int zmax = 65535 / ksplit;
  for (int b0 = 0; b0 < count; b0 += zmax) {
    const int nb = std::min(zmax, count - b0);
    dim3 grid(tn, tm, nb * ksplit);
    {
      // algorithmic: 2 M N K flop per product; the operands and the result
      // once
      prof_count(ctx, (double)nb * ((double)M * K + (double)K * N + (double)M * N) * sizeof(T),
                 2.0 * nb * (double)M * N * K);
    }
    IGA_LAUNCH(ctx, (gemm_tile_kernel<T, TM, TN, BK>), grid, 256, 0, tA, tB, M, N, K, alpha,
               A + b0 * sA, lda, sA, B + b0 * sB, ldb, sB, beta, C + b0 * sC, ldc, sC, ksplit,
               klen, part);
    if (ksplit > 1) {
      const size_t tot = (size_t)nb * M * N;
      IGA_LAUNCH(ctx, gemm_splitk_reduce_kernel<T>,
                 (unsigned)std::min<size_t>((tot + 255) / 256, 4096), 256, 0, M, N, ksplit, nb,
                 alpha, part, beta, C + b0 * sC, ldc, sC);
    }
  }
}

// FP64 tile shape: the FP64 pipe (two FMA per clock and SM) computes the
// padding of a partly filled tile at full cost, so the shape is the one with
// the fewest padded FMAs among 64 x 64, 64 x 16, 16 x 64 and 16 x 16 (the
// larger tile unless the smaller one saves a tenth: fewer blocks, more reuse
// of each staged element)
static int gemm_fp64_shape(int M, int N) {
  static const int bm[4] = {64, 64, 16, 16}, bn[4] = {64, 16, 64, 16};
  int best = 0;
  double cbest = 0.0;
  for (int v = 0; v < 4; ++v) {
    const double c = (double)((M + bm[v] - 1) / bm[v]) * bm[v] * ((N + bn[v] - 1) / bn[v]) * bn[v];
    if (v == 0 || c < 0.9 * cbest) { best = v; cbest = c; }
  }
  return best;
}

template <typename T>
void gemm_rm_batched(iga_ctx* ctx, bool tA, bool tB, int M, int N, int K, T alpha, const T* A,
                     int lda, long long sA, const T* B, int ldb, long long sB, T beta, T* C,
                     int ldc, long long sC, int count) {
  if (M <= 0 || N <= 0 || count <= 0) return;
  if constexpr (sizeof(T) == 8) {
    switch (gemm_fp64_shape(M, N)) {
      case 0:
        gemm_launch<T, 4, 4, 16>(ctx, tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, count);
        break;
      case 1:
        gemm_launch<T, 4, 1, 16>(ctx, tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, count);
        break;
      case 2:
        gemm_launch<T, 1, 4, 16>(ctx, tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, count);
        break;
      default:
        gemm_launch<T, 1, 1, 16>(ctx, tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, count);
    }
  } else {
    gemm_launch<T, 8, 8, 8>(ctx, tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                            sC, count);
  }
}

template void gemm_rm_batched<double>(iga_ctx*, bool, bool, int, int, int, double, const double*,
                                      int, long long, const double*, int, long long, double,
                                      double*, int, long long, int);
template void gemm_rm_batched<float>(iga_ctx*, bool, bool, int, int, int, float, const float*,
                                     int, long long, const float*, int, long long, float, float*,
                                     int, long long, int);

}  // namespace iga

namespace iga {

// y += A x for a column-major A (rows x cols, leading dimension rows): one
// thread per row, the columns in sequence (coalesced along each column)
template <typename T>
__global__ void gemv_cm_add_kernel(int rows, int cols, const T* __restrict__ A,
                                   const T* __restrict__ x, T* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    T s = T(0);
    for (int j = 0; j < cols; ++j) s = fma(A[(size_t)j * rows + i], x[j], s);
    y[i] += s;
  }
}

template <typename T>
__global__ void sub_kernel(size_t n, const T* __restrict__ a, const T* __restrict__ b,
                           T* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

__global__ void dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                   size_t n, double* __restrict__ part) {
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out) {
  // one warp, fixed order per lane, then a shuffle tree: deterministic
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
void gemv_cm_add(iga_ctx* ctx, int rows, int cols, const T* A, const T* x, T* y) {
  if (rows <= 0 || cols <= 0) return;
  IGA_LAUNCH(ctx, gemv_cm_add_kernel<T>, (unsigned)std::min(4 * ctx->nsm, (rows + 255) / 256),
             256, 0, rows, cols, A, x, y);
}
template void gemv_cm_add<double>(iga_ctx*, int, int, const double*, const double*, double*);
template void gemv_cm_add<float>(iga_ctx*, int, int, const float*, const float*, float*);

template <typename T>
void vec_sub(iga_ctx* ctx, size_t n, const T* a, const T* b, T* out) {
  if (n == 0) return;
  IGA_LAUNCH(ctx, sub_kernel<T>, (unsigned)std::min<size_t>((n + 255) / 256, 8 * ctx->nsm), 256,
             0, n, a, b, out);
}
template void vec_sub<double>(iga_ctx*, size_t, const double*, const double*, double*);
template void vec_sub<float>(iga_ctx*, size_t, const float*, const float*, float*);

double device_dot(iga_ctx* ctx, const double* a, const double* b, size_t n) {
  const int nbk = (int)std::min<size_t>((n + 255) / 256, 4 * ctx->nsm);
  if (nbk == 0) return 0.0;
  double* part = scratch<double>(ctx, SLOT_GEMM_DOT, nbk + 1);
  IGA_LAUNCH(ctx, dot_partial_kernel, nbk, 256, 0, a, b, n, part);
  IGA_LAUNCH(ctx, sum_partials_kernel, 1, 32, 0, part, nbk, part + nbk);
  double r = 0.0;
  IGA_CUDA(cudaMemcpyAsync(&r, part + nbk, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  return r;
}

}  // namespace iga
