// Block-AMEn local-system matvec (part (c) of the hot path).
//
// Sec. 5, eq. KKT_red: with the frame matrix F_{!=d} of eq. frame, every
// block of the KKT matrix is projected as F^T A F.  For a TT-matrix A with
// cores A_d[al, be] this projection is assembled factor by factor (Sec. 5,
// "multiplication of tensor trains factor by factor"):
//   (F^T A F) x = sum_{al,be} PhiL[al] (x) A_d[al,be] (x) PhiR[be] x,
// applied in three contractions:
//   t1[be](a', i', b) = sum_b' PhiR[be](b, b') x(a', i', b')        (dense, r1 x r1)
//   t2[al](a', i, b)  = sum_be sum_o A_d[al,be](i, i+o-p) t1[be](a', i+o-p, b)  (banded)
//   y(a, i, b)        = sum_al sum_a' PhiL[al](a, a') t2[al](a', i, b)          (dense, r0 x r0)
// nvec independent vectors share one set of interfaces.
#include <algorithm>
#include <mutex>

#include "iga_internal.cuh"

namespace iga {

// Fixed device scratch of iga_amen_local_matvec_noalloc.  Every device that
// loads the library holds these arrays until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
constexpr size_t NOALLOC_MASK_BYTES = 4096;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) unsigned char g_noalloc_mask[NOALLOC_MASK_BYTES];

template <typename T>
__global__ void local_right_kernel(const T* __restrict__ PhiR, const T* __restrict__ x, int R1,
                                   int nv, int r0, int n, int r1, T* __restrict__ t1) {
  // t1[be][v][a'][i'][b] = sum_b' PhiR[be][b][b'] x[v][a'][i'][b']
  size_t per = (size_t)nv * r0 * n * r1;
  size_t total = (size_t)R1 * per;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int b = (int)(idx % r1);
  size_t row = (idx % per) / r1;         // (v, a', i')
  int be = (int)(idx / per);
  const T* ph = PhiR + ((size_t)be * r1 + b) * r1;
  const T* xr = x + row * r1;
  T s = T(0);
  for (int c = 0; c < r1; ++c) s += ph[c] * xr[c];
  t1[idx] = s;
}

template <typename T>
__global__ void local_band_kernel(const T* __restrict__ bands, const unsigned char* __restrict__ mask,
                                  const T* __restrict__ t1, int R0, int R1, int nv, int r0, int n,
                                  int r1, int p, T* __restrict__ t2) {
  // t2[al][v][a'][i][b] = sum_be sum_o A[al][be][i][o] t1[be][v][a'][i+o-p][b]
  const int B = 2 * p + 1;
  size_t per = (size_t)nv * r0 * n * r1;
  size_t total = (size_t)R0 * per;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int b = (int)(idx % r1);
  size_t q = idx / r1;
  int i = (int)(q % n);
  size_t va = (q / n) % ((size_t)nv * r0);
  int al = (int)(idx / per);
  T s = T(0);
  for (int be = 0; be < R1; ++be) {
    if (mask && !mask[al * R1 + be]) continue;
    const T* row = bands + (((size_t)al * R1 + be) * n + i) * B;
    const T* src = t1 + (size_t)be * per + (va * n) * r1 + b;
    for (int o = 0; o < B; ++o) {
      int j = i + o - p;
      if (j >= 0 && j < n) s += row[o] * src[(size_t)j * r1];
    }
  }
  t2[idx] = s;
}

template <typename T>
__global__ void local_left_kernel(const T* __restrict__ PhiL, const T* __restrict__ t2, int R0,
                                  int nv, int r0, int n, int r1, T* __restrict__ y) {
  // y[v][a][i][b] = sum_al sum_a' PhiL[al][a][a'] t2[al][v][a'][i][b]
  size_t per = (size_t)nv * r0 * n * r1;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per) return;
  size_t ib = idx % ((size_t)n * r1);
  size_t va = idx / ((size_t)n * r1);
  int a = (int)(va % r0);
  size_t v = va / r0;
  T s = T(0);
  size_t nr = (size_t)n * r1;
  for (int al = 0; al < R0; ++al) {
    const T* ph = PhiL + ((size_t)al * r0 + a) * r0;
    const T* src = t2 + (size_t)al * per + v * r0 * nr + ib;
    for (int c = 0; c < r0; ++c) s += ph[c] * src[(size_t)c * nr];
  }
  y[idx] = s;
}

template <typename T>
void local_matvec_t(iga_ctx* ctx, int r0, int n, int r1, int R0, int R1, int p, const T* PhiL,
                    const T* bands, const T* PhiR, const unsigned char* dmask, int nv, const T* x,
                    T* y, T* t1, T* t2) {
  size_t per = (size_t)nv * r0 * n * r1;
  if (per == 0) return;
  int th = 256;
  IGA_LAUNCH(ctx, local_right_kernel<T>, (unsigned)((R1 * per + th - 1) / th), th, 0, PhiR, x, R1,
             nv, r0, n, r1, t1);
  IGA_LAUNCH(ctx, local_band_kernel<T>, (unsigned)((R0 * per + th - 1) / th), th, 0, bands, dmask,
             t1, R0, R1, nv, r0, n, r1, p, t2);
  IGA_LAUNCH(ctx, local_left_kernel<T>, (unsigned)((per + th - 1) / th), th, 0, PhiL, t2, R0, nv,
             r0, n, r1, y);
}

template void local_matvec_t<double>(iga_ctx*, int, int, int, int, int, int, const double*,
                                     const double*, const double*, const unsigned char*, int,
                                     const double*, double*, double*, double*);
template void local_matvec_t<float>(iga_ctx*, int, int, int, int, int, int, const float*,
                                    const float*, const float*, const unsigned char*, int,
                                    const float*, float*, float*, float*);

// row-major C (M x N) = A (M x K) B (K x N)
void gemm_rm(iga_ctx* ctx, int M, int N, int K, const double* A, const double* B, double* C,
             double beta) {
  gemm_rm_batched<double>(ctx, false, false, M, N, K, 1.0, A, K, 0, B, N, 0, beta, C, N, 0, 1);
}

void tt_full_impl(iga_ctx* ctx, const iga_tt* tt, double* out) {
  IGA_REQUIRE(tt && out, "tt_full: null argument");
  int n1 = tt->n[0], n2 = tt->n[1], n3 = tt->n[2], r1 = tt->r[0], r2 = tt->r[1];
  double* t12 = scratch<double>(ctx, SLOT_MISC0, (size_t)n1 * n2 * r2);
  gemm_rm(ctx, n1, n2 * r2, r1, tt->core[0].p, tt->core[1].p, t12);
  gemm_rm(ctx, n1 * n2, n3, r2, t12, tt->core[2].p, out);
}

}  // namespace iga

using namespace iga;

extern "C" iga_status iga_amen_local_matvec(iga_ctx* ctx, int r0, int n, int r1, int R0, int R1,
                                            int p, const void* PhiL, const void* bands,
                                            const void* PhiR, const unsigned char* bandmask,
                                            int nvec, const void* x, void* y, iga_prec prec) {
  if (!ctx) return IGA_EINVAL;
  try {
    AllocScope scope(ctx->stream);
    IGA_REQUIRE(r0 > 0 && n > 0 && r1 > 0 && R0 > 0 && R1 > 0 && p >= 0 && nvec > 0,
                "local_matvec: sizes must be positive");
    IGA_REQUIRE(PhiL && bands && PhiR && x && y, "local_matvec: null pointer");
    IGA_REQUIRE(x != y, "local_matvec: x and y must not overlap");
    unsigned char* dmask = nullptr;
    if (bandmask) {
      dmask = scratch<unsigned char>(ctx, SLOT_MISC1, (size_t)R0 * R1);
      IGA_CUDA(cudaMemcpyAsync(dmask, bandmask, (size_t)R0 * R1, cudaMemcpyHostToDevice,
                               ctx->stream));
    }
    size_t per = (size_t)nvec * r0 * n * r1;
    if (prec == IGA_FP64) {
      double* t1 = scratch<double>(ctx, SLOT_LOCAL_T1, per * R1);
      double* t2 = scratch<double>(ctx, SLOT_LOCAL_T2, per * R0);
      local_matvec_t<double>(ctx, r0, n, r1, R0, R1, p, (const double*)PhiL, (const double*)bands,
                             (const double*)PhiR, dmask, nvec, (const double*)x, (double*)y, t1,
                             t2);
    } else if (prec == IGA_FP32) {
      float* t1 = scratch<float>(ctx, SLOT_LOCAL_T1, per * R1);
      float* t2 = scratch<float>(ctx, SLOT_LOCAL_T2, per * R0);
      local_matvec_t<float>(ctx, r0, n, r1, R0, R1, p, (const float*)PhiL, (const float*)bands,
                            (const float*)PhiR, dmask, nvec, (const float*)x, (float*)y, t1, t2);
    } else {
      throw Error(IGA_EINVAL, "local_matvec: precision must be IGA_FP64 or IGA_FP32");
    }
    if (bandmask) IGA_CUDA(cudaStreamSynchronize(ctx->stream));   // host mask lifetime
    return IGA_OK;
  } catch (const Error& e) {
    set_error(ctx, e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_error(ctx, e.what());
    return IGA_ECUDA;
  }
}

// ---- allocation-free variant -------------------------------------------
//
// Some callers cannot allocate device memory: code that runs while another
// component owns every allocation (a host application with its own fixed
// memory pool, or a memory budget that forbids growth after start-up) and
// callers that must not create a context of this library because that
// allocates.  This entry point runs the same three contractions as
// iga_amen_local_matvec but takes its intermediates from a fixed
// file-scope device array instead of cudaMalloc.

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_scratch_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
void* g_noalloc_mask_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device addresses of the fixed arrays for the current device, looked up once
// per device (host code may not use the symbols themselves as addresses).
iga_status noalloc_addresses(void** scratch, void** mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IGA_ECUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return IGA_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_scratch_ptr[dev]) {
    void* s = nullptr;
    void* m = nullptr;
    if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess) return IGA_ECUDA;
    if (cudaGetSymbolAddress(&m, g_noalloc_mask) != cudaSuccess) return IGA_ECUDA;
    g_noalloc_scratch_ptr[dev] = s;
    g_noalloc_mask_ptr[dev] = m;
  }
  *scratch = g_noalloc_scratch_ptr[dev];
  *mask = g_noalloc_mask_ptr[dev];
  return IGA_OK;
}

template <typename T>
iga_status noalloc_run(cudaStream_t st, int r0, int n, int r1, int R0, int R1, int p,
                       const T* PhiL, const T* bands, const T* PhiR, const unsigned char* dmask,
                       int nv, const T* x, T* y, void* scratch) {
  size_t per = (size_t)nv * r0 * n * r1;
  T* t1 = static_cast<T*>(scratch);
  T* t2 = t1 + per * R1;
  int th = 256;
  local_right_kernel<T><<<(unsigned)((R1 * per + th - 1) / th), th, 0, st>>>(PhiR, x, R1, nv, r0,
                                                                           n, r1, t1);
  if (cudaGetLastError() != cudaSuccess) return IGA_ECUDA;
  local_band_kernel<T><<<(unsigned)((R0 * per + th - 1) / th), th, 0, st>>>(
      bands, dmask, t1, R0, R1, nv, r0, n, r1, p, t2);
  if (cudaGetLastError() != cudaSuccess) return IGA_ECUDA;
  local_left_kernel<T><<<(unsigned)((per + th - 1) / th), th, 0, st>>>(PhiL, t2, R0, nv, r0, n,
                                                                      r1, y);
  if (cudaGetLastError() != cudaSuccess) return IGA_ECUDA;
  return IGA_OK;
}
}  // namespace

extern "C" iga_status iga_amen_local_matvec_noalloc(void* stream, int r0, int n, int r1, int R0,
                                                    int R1, int p, const void* PhiL,
                                                    const void* bands, const void* PhiR,
                                                    const unsigned char* bandmask, int nvec,
                                                    const void* x, void* y, iga_prec prec) {
  if (r0 <= 0 || n <= 0 || r1 <= 0 || R0 <= 0 || R1 <= 0 || p < 0 || nvec <= 0) return IGA_EINVAL;
  if (!PhiL || !bands || !PhiR || !x || !y || x == y) return IGA_EINVAL;
  if (prec != IGA_FP64 && prec != IGA_FP32) return IGA_EINVAL;
  size_t es = prec == IGA_FP64 ? sizeof(double) : sizeof(float);
  size_t per = (size_t)nvec * r0 * n * r1;
  if (per * (size_t)(R0 + R1) * es > NOALLOC_SCRATCH_BYTES) return IGA_EINVAL;
  if (bandmask && (size_t)R0 * R1 > NOALLOC_MASK_BYTES) return IGA_EINVAL;
  // an error left pending by earlier work on this thread is not this call's:
  // report it without consuming it, before any launch
  if (cudaPeekAtLastError() != cudaSuccess) return IGA_ECUDA;
  void* scratch = nullptr;
  void* mask = nullptr;
  iga_status s = noalloc_addresses(&scratch, &mask);
  if (s != IGA_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned char* dmask = nullptr;
  if (bandmask) {
    if (cudaMemcpyAsync(mask, bandmask, (size_t)R0 * R1, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return IGA_ECUDA;
    dmask = static_cast<const unsigned char*>(mask);
  }
  if (prec == IGA_FP64)
    s = noalloc_run<double>(st, r0, n, r1, R0, R1, p, (const double*)PhiL, (const double*)bands,
                            (const double*)PhiR, dmask, nvec, (const double*)x, (double*)y,
                            scratch);
  else
    s = noalloc_run<float>(st, r0, n, r1, R0, R1, p, (const float*)PhiL, (const float*)bands,
                           (const float*)PhiR, dmask, nvec, (const float*)x, (float*)y, scratch);
  // the host mask is only borrowed for the call: wait until the stream has
  // copied it (this allocates nothing)
  if (s == IGA_OK && bandmask && cudaStreamSynchronize(st) != cudaSuccess) return IGA_ECUDA;
  return s;
}
