// Small dense FP64 linear algebra on the device and the TT-SVD (step a3).
//
// TT-SVD (Sec. 3 after eq. weightEquationSolve; format of eq. tt): the two
// unfoldings of a 3-way tensor are truncated one after the other at
// tol * ref / sqrt(D - 1).  Each truncated SVD is computed as
//   sketch  Y = A Omega (Gaussian Omega, k columns, k doubled until the
//           smallest sketched singular value is below the threshold),
//   Householder QR of Y,
//   B^T = A^T Q and the eigen-decomposition of B B^T by cyclic Jacobi,
//   taken twice (the second Gram matrix is nearly diagonal, which gives
//   the small singular values to relative accuracy),
// and the kept factor is recomputed exactly as U^T A.  Large products go to
// the library's tiled GEMM (gemm.cu); the QR, Jacobi and helper kernels are
// below.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>
#include <map>
#include <mutex>

#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in every thread; `red` holds >= 32 doubles
__device__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

__global__ void sumsq_kernel(const double* __restrict__ x, size_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = x[i];
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

double device_norm2(iga_ctx* ctx, const double* x, size_t n) {
  double* acc = scratch<double>(ctx, SLOT_TTSVD_NORM, 1);
  IGA_CUDA(cudaMemsetAsync(acc, 0, 8, ctx->stream));
  if (n > 0) {
    int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    IGA_LAUNCH(ctx, sumsq_kernel, blocks, 256, 0, x, n, acc);
  }
  double h = 0.0;
  IGA_CUDA(cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  return std::sqrt(h);
}

// sums of squares of `count` tensors of n elements each (x + t n), one launch
__global__ void sumsq_multi_kernel(const double* __restrict__ x, size_t n,
                                   double* __restrict__ out) {
  __shared__ double red[32];
  const double* xt = x + (size_t)blockIdx.y * n;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    acc = fma(xt[i], xt[i], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out + blockIdx.y, acc);
}

void device_norms(iga_ctx* ctx, const double* x, size_t n, int count, double* norms) {
  double* acc = scratch<double>(ctx, SLOT_TTSVD_NORM, (size_t)count);
  IGA_CUDA(cudaMemsetAsync(acc, 0, (size_t)count * 8, ctx->stream));
  if (n > 0) {
    int blocks = (int)std::min<size_t>((n + 255) / 256, (152 * 8 + count - 1) / count);
    IGA_LAUNCH(ctx, sumsq_multi_kernel, dim3(blocks, count), 256, 0, x, n, acc);
  }
  IGA_CUDA(cudaMemcpyAsync(norms, acc, (size_t)count * 8, cudaMemcpyDeviceToHost, ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int t = 0; t < count; ++t) norms[t] = std::sqrt(norms[t]);
}

// counter-based Gaussian numbers: splitmix64 hash -> two uniforms -> Box-Muller
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Gaussian test matrices for the randomized sketches (Box-Muller on two
// 24-bit uniforms from one splitmix64 hash).  The transform runs in FP32:
// the sketches need independent normal samples, not FP64 ones, and the FP64
// logarithm and cosine cost some 60 FP64 operations per sample on this GPU.
__global__ void gaussian_kernel(double* __restrict__ x, size_t n, uint64_t seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t h = splitmix64(seed ^ (0x9e3779b97f4a7c15ull * (i + 1)));
    const float u1 = (float)((h >> 40) + 1) * (1.0f / 16777216.0f);          // (0, 1]
    const float u2 = (float)((h >> 16) & 0xffffffull) * (1.0f / 16777216.0f);  // [0, 1)
    x[i] = (double)(sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2));
  }
}

void fill_gaussian(iga_ctx* ctx, double* x, size_t n, uint64_t seed) {
  if (n == 0) return;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  IGA_LAUNCH(ctx, gaussian_kernel, blocks, 256, 0, x, n, seed);
}

// B (cols x rows, col-major) = A^T for A (rows x cols, col-major)
__global__ void transpose_kernel(const double* __restrict__ A, int rows, int cols,
                                 double* __restrict__ B) {
  __shared__ double tile[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int r = bx + threadIdx.x, c = by + j;
    if (r < rows && c < cols) tile[j][threadIdx.x] = A[(size_t)c * rows + r];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int c = by + threadIdx.x, r = bx + j;
    if (r < rows && c < cols) B[(size_t)r * cols + c] = tile[threadIdx.x][j];
  }
}

void transpose_cm(iga_ctx* ctx, const double* A, int rows, int cols, double* B) {
  if (rows == 0 || cols == 0) return;
  dim3 grid((rows + 31) / 32, (cols + 31) / 32), block(32, 8);
  IGA_LAUNCH(ctx, transpose_kernel, grid, block, 0, A, rows, cols, B);
}

// --------------------------------------------------------- Householder QR

// Y (m x k, col-major) -> Q (m x k) with orthonormal columns spanning Y.
// One block; warps own columns for the reflector applications.
__global__ void householder_qr_kernel(double* __restrict__ Y, double* __restrict__ Q, int m,
                                      int k) {
  extern __shared__ double sm[];
  double* vtv = sm;            // k
  double* red = sm + k;        // 32
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    double* x = Y + (size_t)j * m;
    double s = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) s += x[i] * x[i];
    double nrm2 = block_sum(s, red);
    double x0 = x[j];
    double nrm = sqrt(nrm2);
    double alpha = (x0 >= 0.0) ? -nrm : nrm;
    double v0 = x0 - alpha;
    // v = x with v_j = x_j - alpha; v^T v = nrm2 - x0^2 + v0^2
    double vv = nrm2 - x0 * x0 + v0 * v0;
    __syncthreads();
    if (threadIdx.x == 0) {
      vtv[j] = (nrm > 0.0 && vv > 0.0) ? vv : 0.0;
      x[j] = v0;
    }
    __syncthreads();
    double tv = vtv[j];
    if (tv == 0.0) continue;
    for (int c = j + 1 + wid; c < k; c += nw) {
      double* y = Y + (size_t)c * m;
      double d = 0.0;
      for (int i = j + lane; i < m; i += 32) d += x[i] * y[i];
      d = warp_sum(d);
      double f = 2.0 * d / tv;
      for (int i = j + lane; i < m; i += 32) y[i] -= f * x[i];
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{k-1} [I; 0], applied from the last reflector
  for (size_t t = threadIdx.x; t < (size_t)m * k; t += blockDim.x) {
    int i = (int)(t % m), c = (int)(t / m);
    Q[t] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    double tv = vtv[j];
    if (tv == 0.0) continue;
    const double* x = Y + (size_t)j * m;
    for (int c = wid; c < k; c += nw) {
      double* q = Q + (size_t)c * m;
      double d = 0.0;
      for (int i = j + lane; i < m; i += 32) d += x[i] * q[i];
      d = warp_sum(d);
      double f = 2.0 * d / tv;
      for (int i = j + lane; i < m; i += 32) q[i] -= f * x[i];
    }
    __syncthreads();
  }
}

// Householder QR with the rows of Y split over the CTAs of one thread-block
// cluster: CTA c holds rows [c mc, (c + 1) mc) of Y and of Q in shared memory,
// and the column norms and the reflector dot products of every step are
// summed across the cluster through distributed shared memory.  The FP64
// work is spread over up to 16 SMs; every CTA takes the same decisions from
// the same sums, so all of them pass the same cluster barriers.
namespace cgx = cooperative_groups;

__device__ __forceinline__ double qr_block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

// out[t] = sum over the C CTAs of the cluster of buf[t] (distributed shared
// memory), t in [t0, t1): a power-of-two segment of S >= C lanes per column,
// one remote load per lane, then a segmented shuffle sum.  Every CTA runs the
// same reduction tree on the same values, so all get identical sums.  Ends
// with __syncthreads.
__device__ void cluster_colsum(cgx::cluster_group& cl, int C, double* buf, int t0, int t1,
                               double* out) {
  int S = 1;
  while (S < C) S <<= 1;                        // C <= 16, so S divides 32
  const int per_warp = 32 / S;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane / S, c = lane - (lane / S) * S;
  for (int base = t0 + w * per_warp; base < t1; base += nw * per_warp) {
    const int t = base + sub;
    double v = (c < C && t < t1) ? cl.map_shared_rank(buf, c)[t] : 0.0;
    for (int o = S >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (c == 0 && t < t1) out[t] = v;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) householder_qr_cluster_kernel(
    const double* __restrict__ Y, double* __restrict__ Q, int m, int k, int mc) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  extern __shared__ double sm[];
  double* A = sm;                               // mc x k, leading dimension mc
  double* Ql = A + (size_t)mc * k;              // mc x k
  double* pw = Ql + (size_t)mc * k;             // 2 x k partial dot products
  double* ps = pw + 2 * k;                      // [partial sum of squares, alpha]
  double* tau = ps + 2;                         // k
  double* wsum = tau + k;                       // k
  double* red = wsum + k;                       // 32
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r0 = me * mc;
  const int nloc = max(0, min(m, r0 + mc) - r0);
  for (int t = threadIdx.x; t < mc * k; t += blockDim.x) {
    int i = t % mc, c = t / mc;
    A[t] = i < nloc ? Y[(size_t)c * m + r0 + i] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    // local rows i >= j of this CTA: [lo, nloc)
    const int lo = min(nloc, max(0, j - r0));
    const int own = j / mc;                     // CTA holding row j
    double s = 0.0;
    for (int i = lo + threadIdx.x; i < nloc; i += blockDim.x)
      if (r0 + i > j) s += A[(size_t)j * mc + i] * A[(size_t)j * mc + i];
    s = qr_block_sum(s, red);
    if (threadIdx.x == 0) {
      ps[0] = s;
      ps[1] = (me == own) ? A[(size_t)j * mc + (j - r0)] : 0.0;
    }
    cl.sync();
    double sig2 = 0.0;
    for (int c = 0; c < C; ++c) sig2 += cl.map_shared_rank(ps, c)[0];
    const double alpha = cl.map_shared_rank(ps, own)[1];
    const double nrm = sqrt(alpha * alpha + sig2);
    double tj = 0.0, inv = 0.0;
    if (nrm > 0.0) {
      const double beta = alpha >= 0.0 ? -nrm : nrm;
      const double v0 = alpha - beta;
      tj = -v0 / beta;
      inv = 1.0 / v0;
    }
    if (threadIdx.x == 0) tau[j] = tj;
    if (tj != 0.0) {
      for (int i = lo + threadIdx.x; i < nloc; i += blockDim.x) {
        if (r0 + i > j) A[(size_t)j * mc + i] *= inv;
        else A[(size_t)j * mc + i] = 1.0;       // v_j = 1
      }
    }
    __syncthreads();
    // partial w_t = sum_i v_i A(i, t), t > j
    double* pb = pw + (j & 1) * k;
    for (int t = j + 1 + wid; t < k; t += nw) {
      double d = 0.0;
      if (tj != 0.0)
        for (int i = lo + lane; i < nloc; i += 32) d += A[(size_t)j * mc + i] * A[(size_t)t * mc + i];
      d = warp_sum(d);
      if (lane == 0) pb[t] = d;
    }
    cl.sync();
    cluster_colsum(cl, C, pb, j + 1, k, wsum);
    if (tj != 0.0) {
      const int w = k - j - 1;
      for (int e = threadIdx.x; e < w * (nloc - lo); e += blockDim.x) {
        int t = j + 1 + e / (nloc - lo), i = lo + e % (nloc - lo);
        A[(size_t)t * mc + i] -= tj * A[(size_t)j * mc + i] * wsum[t];
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{k-1} [I; 0], the last reflector first
  for (int t = threadIdx.x; t < mc * k; t += blockDim.x) {
    int i = t % mc, c = t / mc;
    Ql[t] = (r0 + i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  int it = 0;                                   // applied reflectors: buffer parity
  for (int j = k - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj == 0.0) continue;                    // the same in every CTA
    const int lo = min(nloc, max(0, j - r0));
    double* pb = pw + (it++ & 1) * k;
    for (int t = j + wid; t < k; t += nw) {
      double d = 0.0;
      for (int i = lo + lane; i < nloc; i += 32) d += A[(size_t)j * mc + i] * Ql[(size_t)t * mc + i];
      d = warp_sum(d);
      if (lane == 0) pb[t] = d;
    }
    cl.sync();
    cluster_colsum(cl, C, pb, j, k, wsum);
    const int w = k - j;
    for (int e = threadIdx.x; e < w * (nloc - lo); e += blockDim.x) {
      int t = j + e / (nloc - lo), i = lo + e % (nloc - lo);
      Ql[(size_t)t * mc + i] -= tj * A[(size_t)j * mc + i] * wsum[t];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < mc * k; t += blockDim.x) {
    int i = t % mc, c = t / mc;
    if (i < nloc) Q[(size_t)c * m + r0 + i] = Ql[t];
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

// ------------------------------------------- truncated QR with column pivoting
//
// The block core B (m x c3, B(i, a) = B[i si + a sa]) is truncated by
// Householder QR with column pivoting: each step takes the column with the
// largest norm below the current row, and pivoting stops at the first step
// whose remaining column norms sum to <= rel^2 * (sum of all), i.e. when the
// Frobenius error of projecting B on the chosen columns is within rel.  The
// columns of each field group (a / r, three groups) are first normalised to
// unit Frobenius norm, so y, u and lambda are truncated alike.  Then `kick`
// extra columns E (m x kick, col-major) are orthogonalised against the chosen
// ones by unpivoted Householder steps, and the nr = min(rk + kick, m)
// orthonormal columns Q are formed in place.  Working on B itself (not on
// B^T B) resolves column residuals down to the FP64 rounding of B.
//
// Rows are split over the CTAs of a cluster as in the QR above; the slice of
// each CTA lives in shared memory when it fits, else in a global workspace.
struct QrcpArgs {
  const double* B;
  const double* E;
  double* Q;
  double* gwork;     // nullptr: slices in shared memory
  int* rk;           // device: number of pivoted columns
  double rel;
  double w0;         // weight of the first field group
  int m, c3, si, sa, r, kick, jmax, mc;
};

__global__ void __launch_bounds__(256) qrcp_cluster_kernel(QrcpArgs a) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  extern __shared__ double sm[];
  const int ncol = a.c3 + a.kick;
  const int mc = a.mc;
  double* part = sm;                   // ncol: partial column norms
  double* rowj = part + ncol;          // ncol: row j, published by its owner
  double* pw = rowj + ncol;            // 2 ncol: partial dot products
  double* nrm = pw + 2 * ncol;         // ncol: column norms below row j
  double* tau = nrm + ncol;            // ncol
  double* gpart = tau + ncol;          // 4: partial group sums
  double* red = gpart + 4;             // 64
  int* ired = (int*)(red + 64);        // 32
  double* A = a.gwork ? a.gwork + (size_t)me * mc * ncol : (double*)(ired + 32);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = me * mc;
  const int nloc = max(0, min(a.m, r0 + mc) - r0);

  // load, with the sums of squares of the three field groups
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int t = tid; t < mc * ncol; t += blockDim.x) {
    const int i = t % mc, c = t / mc;
    double v = 0.0;
    if (i < nloc)
      v = c < a.c3 ? a.B[(size_t)(r0 + i) * a.si + (size_t)c * a.sa]
                   : a.E[(size_t)(c - a.c3) * a.m + r0 + i];
    A[t] = v;
    if (c < a.c3) {
      const int g = c / a.r;
      if (g == 0) g0 += v * v; else if (g == 1) g1 += v * v; else g2 += v * v;
    }
  }
  g0 = qr_block_sum(g0, red);
  g1 = qr_block_sum(g1, red);
  g2 = qr_block_sum(g2, red);
  if (tid == 0) { gpart[0] = g0; gpart[1] = g1; gpart[2] = g2; }
  cl.sync();
  double gsum[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < C; ++c) {
    const double* q = cl.map_shared_rank(gpart, c);
    gsum[0] += q[0]; gsum[1] += q[1]; gsum[2] += q[2];
  }
  double sc[3], tot = 0.0;
  for (int g = 0; g < 3; ++g) {
    sc[g] = gsum[g] > 0.0 ? (g == 0 ? a.w0 : 1.0) / sqrt(gsum[g]) : 0.0;
    tot += gsum[g] > 0.0 ? 1.0 : 0.0;
  }
  for (int t = tid; t < mc * a.c3; t += blockDim.x) A[t] *= sc[(t / mc) / a.r];
  __syncthreads();
  const double thr2 = a.rel * a.rel * tot;
  const int npiv = min(a.jmax, a.c3);
  int par = 0;                                   // parity of the partial-product buffer

  // one Householder step on column j (alpha = B(j, j), nrm2 = its squared
  // norm over rows >= j), updating columns (j, jend)
  // dst[t] = sum over this CTA's rows i >= lo of A(i, vc) A(i, t) (vc < 0:
  // A(i, t)^2), t in [t0, t1).  Short slices take one thread per column
  // (no shuffles on the critical path), tall ones a warp per column.
  auto partial_dots = [&](int lo, int vc, int t0, int t1, double* dst) {
    if (mc <= 96) {
      for (int t = t0 + tid; t < t1; t += blockDim.x) {
        const double* col = A + (size_t)t * mc;
        const double* v = vc >= 0 ? A + (size_t)vc * mc : col;
        double s0 = 0.0, s1 = 0.0;
        int i = lo;
        for (; i + 1 < nloc; i += 2) {
          s0 = fma(v[i], col[i], s0);
          s1 = fma(v[i + 1], col[i + 1], s1);
        }
        if (i < nloc) s0 = fma(v[i], col[i], s0);
        dst[t] = s0 + s1;
      }
    } else {
      for (int t = t0 + wid; t < t1; t += nw) {
        const double* col = A + (size_t)t * mc;
        const double* v = vc >= 0 ? A + (size_t)vc * mc : col;
        double d = 0.0;
        for (int i = lo + lane; i < nloc; i += 32) d = fma(v[i], col[i], d);
        d = warp_sum(d);
        if (lane == 0) dst[t] = d;
      }
    }
  };

  auto house = [&](int j, double alpha, double nrm2, int jend) {
    const int lo = min(nloc, max(0, j - r0));
    double tj = 0.0, inv = 0.0;
    const double nr_ = sqrt(fmax(nrm2, 0.0));
    if (nr_ > 0.0) {
      const double beta = alpha >= 0.0 ? -nr_ : nr_;
      const double v0 = alpha - beta;
      if (v0 != 0.0) {
        tj = -v0 / beta;
        inv = 1.0 / v0;
      }
    }
    if (tid == 0) tau[j] = tj;
    if (tj != 0.0)
      for (int i = lo + tid; i < nloc; i += blockDim.x)
        A[(size_t)j * mc + i] = (r0 + i > j) ? A[(size_t)j * mc + i] * inv : 1.0;
    __syncthreads();
    double* pb = pw + (par & 1) * ncol;
    if (tj != 0.0) partial_dots(lo, j, j + 1, jend, pb);
    cl.sync();
    ++par;
    if (tj != 0.0) {
      cluster_colsum(cl, C, pb, j + 1, jend, nrm);   // nrm reused for the products
      const int w = jend - j - 1, h = nloc - lo;
      for (int e = tid; e < w * h; e += blockDim.x) {
        const int t = j + 1 + e / h, i = lo + e % h;
        A[(size_t)t * mc + i] -= tj * A[(size_t)j * mc + i] * nrm[t];
      }
    }
    __syncthreads();
  };

  // pivoted steps
  int j = 0;
  for (; j < npiv; ++j) {
    const int lo = min(nloc, max(0, j - r0));
    const int own = j / mc;
    partial_dots(lo, -1, j, a.c3, part);
    if (me == own)
      for (int t = j + tid; t < ncol; t += blockDim.x) rowj[t] = A[(size_t)t * mc + (j - r0)];
    cl.sync();
    cluster_colsum(cl, C, part, j, a.c3, nrm);
    double sum = 0.0, mx = -1.0;
    int arg = j;
    for (int t = j + tid; t < a.c3; t += blockDim.x) {
      const double sq = nrm[t];
      sum += sq;
      if (sq > mx) { mx = sq; arg = t; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
      const double om = __shfl_xor_sync(0xffffffffu, mx, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (om > mx || (om == mx && oa < arg)) { mx = om; arg = oa; }
    }
    if (lane == 0) { red[wid] = sum; red[32 + wid] = mx; ired[wid] = arg; }
    __syncthreads();
    double rem = 0.0, bm = -1.0;
    int p = j;
    for (int w = 0; w < nw; ++w) {
      rem += red[w];
      if (red[32 + w] > bm || (red[32 + w] == bm && ired[w] < p)) { bm = red[32 + w]; p = ired[w]; }
    }
    const double alpha = cl.map_shared_rank(rowj, own)[p];
    const double nrm2 = nrm[p];
    __syncthreads();
    // the first column is always taken (a rank of at least one)
    if (j > 0 && (rem <= thr2 || !(bm > 0.0))) break;
    if (p != j)
      for (int i = tid; i < nloc; i += blockDim.x) {
        const double t0 = A[(size_t)j * mc + i];
        A[(size_t)j * mc + i] = A[(size_t)p * mc + i];
        A[(size_t)p * mc + i] = t0;
      }
    __syncthreads();
    house(j, alpha, nrm2, ncol);
  }
  const int rk = j;
  const int nr = min(rk + a.kick, a.m);
  // the extra columns move next to the chosen ones (no CTA may still read
  // this step's published norms when the next step writes them)
  cl.sync();
  for (int e = 0; e < nr - rk; ++e) {
    const int t1 = rk + e, t2 = a.c3 + e;
    if (t1 == t2) continue;
    for (int i = tid; i < nloc; i += blockDim.x) {
      const double t0 = A[(size_t)t1 * mc + i];
      A[(size_t)t1 * mc + i] = A[(size_t)t2 * mc + i];
      A[(size_t)t2 * mc + i] = t0;
    }
  }
  __syncthreads();
  // unpivoted steps on the extra columns
  for (j = rk; j < nr; ++j) {
    const int lo = min(nloc, max(0, j - r0));
    const int own = j / mc;
    double sq = 0.0;
    for (int i = lo + tid; i < nloc; i += blockDim.x) {
      const double v = A[(size_t)j * mc + i];
      sq += v * v;
    }
    sq = qr_block_sum(sq, red);
    if (tid == 0) part[0] = sq;
    if (me == own && tid == 0) rowj[0] = A[(size_t)j * mc + (j - r0)];
    cl.sync();
    double nrm2 = 0.0;
    for (int c = 0; c < C; ++c) nrm2 += cl.map_shared_rank(part, c)[0];
    const double alpha = cl.map_shared_rank(rowj, own)[0];
    house(j, alpha, nrm2, nr);
  }
  cl.sync();
  // Q in place: Q(:, j) = H_0 ... H_{nr-1} e_j, the last reflector first
  for (j = nr - 1; j >= 0; --j) {
    const double tj = tau[j];
    const int lo = min(nloc, max(0, j - r0));
    if (tj != 0.0 && j + 1 < nr) {
      double* pb = pw + (par & 1) * ncol;
      partial_dots(lo, j, j + 1, nr, pb);
      cl.sync();
      ++par;
      cluster_colsum(cl, C, pb, j + 1, nr, nrm);
      const int w = nr - j - 1, h = nloc - lo;
      for (int e = tid; e < w * h; e += blockDim.x) {
        const int t = j + 1 + e / h, i = lo + e % h;
        A[(size_t)t * mc + i] -= tj * A[(size_t)j * mc + i] * nrm[t];
      }
      __syncthreads();
    }
    for (int i = tid; i < nloc; i += blockDim.x) {
      const int g = r0 + i;
      double v;
      if (g < j) v = 0.0;
      else if (g == j) v = 1.0 - tj;
      else v = -tj * A[(size_t)j * mc + i];
      A[(size_t)j * mc + i] = v;
    }
    __syncthreads();
  }
  for (int t = tid; t < mc * nr; t += blockDim.x) {
    const int i = t % mc, c = t / mc;
    if (i < nloc) a.Q[(size_t)c * a.m + r0 + i] = A[t];
  }
  if (me == 0 && tid == 0) *a.rk = rk;
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

static int qr_cluster_max(iga_ctx* ctx);

void qrcp_truncate(iga_ctx* ctx, const double* B, int m, int c3, int si, int sa, int r,
                   const double* E, int kick, double rel, int jmax, double* Q, int* rk_dev,
                   double w0) {
  IGA_REQUIRE(m >= 1 && c3 >= 1 && r >= 1 && c3 <= 3 * r && kick >= 0, "qrcp: bad sizes");
  const size_t limit = 200 * 1024;
  const int cmax = qr_cluster_max(ctx);
  // at least 16 rows per CTA: one SM's FP64 rate (1/64 of FP32) makes even
  // 65-row slices worth spreading
  const int C = std::max(1, std::min(cmax, m / 16));
  const int mc = (m + C - 1) / C;
  const int ncol = c3 + kick;
  const size_t head = ((size_t)6 * ncol + 4 + 64) * sizeof(double) + 32 * sizeof(int);
  const size_t slice = (size_t)mc * ncol * sizeof(double);
  IGA_REQUIRE(head <= limit, "qrcp: too many columns");
  QrcpArgs a;
  a.B = B; a.E = E; a.Q = Q; a.rk = rk_dev; a.rel = rel; a.w0 = w0 > 1.0 ? w0 : 1.0;
  a.m = m; a.c3 = c3; a.si = si; a.sa = sa; a.r = r; a.kick = kick;
  a.jmax = std::max(1, std::min(jmax, m)); a.mc = mc;
  a.gwork = head + slice <= limit ? nullptr : scratch<double>(ctx, SLOT_QRCP_WORK, (size_t)C * mc * ncol);
  func_attr(qrcp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  func_attr(qrcp_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = a.gwork ? head : head + slice;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // algorithmic: pivoted Householder on m x c3 up to rank jmax plus the
  // extra columns, and forming Q: about 4 m c3 nr + 2 m nr^2 flop
  const double nr = std::min(a.jmax + kick, m);
  prof_count(ctx, 8.0 * m * (ncol + nr), 4.0 * m * c3 * nr + 2.0 * m * nr * nr);
  bool prof = prof_match(ctx, "qrcp_cluster_kernel");
  if (prof) prof_start(ctx);
  IGA_CUDA(cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel, a));
  if (prof) prof_stop(ctx);
  ctx->launches++;
  ctx->next_bytes = 0.0;
  ctx->next_flops = 0.0;
}

static size_t qr_cluster_smem(int mc, int k) {
  return ((size_t)2 * mc * k + 5 * (size_t)k + 2 + 32) * sizeof(double);
}

// largest cluster of 256-thread CTAs with 200 KB of shared memory each that
// the GPU can schedule (16 with the non-portable size, else 8, else 1)
static int qr_cluster_max(iga_ctx* ctx) {
  const size_t limit = 200 * 1024;
  func_attr(householder_qr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)limit);
  func_attr(householder_qr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  static std::mutex mu;
  static std::map<int, int> cmax_of;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cmax_of.find(ctx->device);
    if (it != cmax_of.end()) return it->second;
  }
  int best = 1;
  for (int c : {16, 8}) {
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(c);
    q.blockDim = dim3(256);
    q.dynamicSmemBytes = limit;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = c;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    q.attrs = a;
    q.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, householder_qr_cluster_kernel, &q) == cudaSuccess &&
        n >= 1) {
      best = c;
      break;
    }
    (void)cudaGetLastError();
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    cmax_of[ctx->device] = best;
  }
  return best;
}

void householder_qr(iga_ctx* ctx, double* Y, double* Q, int m, int k) {
  IGA_REQUIRE(k >= 1 && k <= 1024 && m >= k, "householder_qr: bad sizes");
  // algorithmic: Householder QR 2 m k^2 - 2 k^3 / 3, forming Q the same again
  const double by = 3.0 * 8.0 * m * k;
  const double fl = 2.0 * (2.0 * m * k * k - 2.0 * k * k * k / 3.0);
  // cluster of up to 16 CTAs with at least 64 rows each (one CTA for small
  // m) when a slice fits in shared memory, else the one-CTA global kernel
  const size_t limit = 200 * 1024;
  const int cmax = qr_cluster_max(ctx);
  int C = std::max(1, std::min(cmax, m / 64));
  int mc = (m + C - 1) / C;
  if (qr_cluster_smem(mc, k) <= limit) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = qr_cluster_smem(mc, k);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    prof_count(ctx, by, fl);
    bool prof = prof_match(ctx, "householder_qr_cluster_kernel");
    if (prof) prof_start(ctx);
    IGA_CUDA(cudaLaunchKernelEx(&cfg, householder_qr_cluster_kernel, (const double*)Y, Q, m, k,
                                mc));
    if (prof) prof_stop(ctx);
    ctx->launches++;
    ctx->next_bytes = 0.0;
    ctx->next_flops = 0.0;
    return;
  }
  size_t smem = (size_t)(k + 32) * sizeof(double);
  prof_count(ctx, by, fl);
  IGA_LAUNCH(ctx, householder_qr_kernel, 1, 1024, smem, Y, Q, m, k);
}

// ----------------------------------------------------------- Jacobi eigen

// Symmetric A (k x k, col-major) -> eigenvalues w (descending) and
// eigenvectors V (columns).  Cyclic Jacobi with round-robin parallel
// ordering: each round applies k/2 disjoint rotations (rows, then columns).
// At most 40 sweeps; stops when the off-diagonal norm is below 1e-14 (FP64)
// or 1e-4 (FP32) times the Frobenius norm.  Storage: mode 2 keeps A and V in
// shared memory, mode 1 keeps A in shared memory and V in global memory,
// mode 0 keeps both in global memory (A overwritten).  The FP32 variant
// (T = float) always runs in mode 2; input and output stay FP64.
struct JacobiProblem {
  double* A;
  double* Vwork;
  double* Vout;
  double* w;
  int k;
  int mode;
};
struct JacobiBatch {
  JacobiProblem p[4];
};

template <typename T>
struct JacobiTol;
template <>
struct JacobiTol<double> {
  static constexpr double off2 = 1e-28, skip = 1e-17, tiny = 1e-300;
  static constexpr int sweeps = 40;
};
template <>
struct JacobiTol<float> {
  // the FP32 eigenbases only feed a preconditioner: a relative off-diagonal
  // norm of 1e-4 is plenty (fewer sweeps cost more GMRES iterations)
  static constexpr float off2 = 1e-8f, skip = 1e-8f, tiny = 1e-30f;
  static constexpr int sweeps = 40;
};

template <typename T>
__host__ __device__ inline size_t jacobi_head_bytes(int k) {
  int kk = k + (k & 1);
  size_t b = (size_t)(kk / 2) * (2 * sizeof(T) + 2 * sizeof(int));
  b = (b + 7) / 8 * 8;
  return b + 32 * sizeof(double);
}

template <typename T>
__global__ void jacobi_eig_kernel(JacobiBatch batch) {
  extern __shared__ double sm[];
  const JacobiProblem& P = batch.p[blockIdx.x];
  double* __restrict__ Ag = P.A;
  double* __restrict__ Vout = P.Vout;
  double* __restrict__ w = P.w;
  const int k = P.k;
  const int mode = P.mode;
  int kk = k + (k & 1);
  int npair = kk / 2;
  T* cs = (T*)sm;                  // npair
  T* sn = cs + npair;              // npair
  int* pp = (int*)(sn + npair);
  int* qq = pp + npair;
  double* red = (double*)((char*)sm + (jacobi_head_bytes<T>(k) - 32 * sizeof(double)));
  T* A;
  T* V;
  if constexpr (sizeof(T) == sizeof(double)) {
    A = (T*)Ag;
    V = (T*)P.Vwork;
  }
  if (mode >= 1) {
    A = (T*)(red + 32);
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) A[t] = (T)Ag[t];
  }
  if (mode == 2) V = A + (size_t)k * k;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) V[t] = ((t % k) == (t / k)) ? T(1) : T(0);
  __syncthreads();
  double fro2 = 0.0;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) fro2 += (double)A[t] * (double)A[t];
  fro2 = block_sum(fro2, red);
  for (int sweep = 0; sweep < JacobiTol<T>::sweeps && k > 1; ++sweep) {
    double off2 = 0.0;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x)
      if ((t % k) != (t / k)) off2 += (double)A[t] * (double)A[t];
    off2 = block_sum(off2, red);
    if (off2 <= (double)JacobiTol<T>::off2 * fro2 || off2 == 0.0) break;
    for (int r = 0; r < kk - 1; ++r) {
      for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        int p, q;
        if (i == 0) { p = kk - 1; q = r; }
        else { p = (r + i) % (kk - 1); q = (r - i + kk - 1) % (kk - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        T c = T(1), s = T(0);
        if (q < k) {
          T apq = A[(size_t)q * k + p];
          T app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
          if (apq != T(0) &&
              fabs(apq) > JacobiTol<T>::tiny + JacobiTol<T>::skip * sqrt(fabs(app * aqq))) {
            T tau = (aqq - app) / (T(2) * apq);
            T t = (tau >= T(0)) ? T(1) / (tau + sqrt(T(1) + tau * tau))
                                : T(-1) / (-tau + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            s = t * c;
          }
        }
        cs[i] = c; sn[i] = s; pp[i] = p; qq[i] = q;
      }
      __syncthreads();
      // rows p, q of A:  a_p <- c a_p - s a_q,  a_q <- s a_p + c a_q
      for (int t = threadIdx.x; t < npair * k; t += blockDim.x) {
        int i = t / k, col = t % k;
        if (sn[i] == T(0)) continue;
        int p = pp[i], q = qq[i];
        T c = cs[i], s = sn[i];
        T ap = A[(size_t)col * k + p], aq = A[(size_t)col * k + q];
        A[(size_t)col * k + p] = c * ap - s * aq;
        A[(size_t)col * k + q] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and V
      for (int t = threadIdx.x; t < npair * k; t += blockDim.x) {
        int i = t / k, row = t % k;
        if (sn[i] == T(0)) continue;
        int p = pp[i], q = qq[i];
        T c = cs[i], s = sn[i];
        T ap = A[(size_t)p * k + row], aq = A[(size_t)q * k + row];
        A[(size_t)p * k + row] = c * ap - s * aq;
        A[(size_t)q * k + row] = s * ap + c * aq;
        T vp = V[(size_t)p * k + row], vq = V[(size_t)q * k + row];
        V[(size_t)p * k + row] = c * vp - s * vq;
        V[(size_t)q * k + row] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // sort descending: rank of each eigenvalue, then scatter columns
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    T wi = A[(size_t)i * k + i];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      T wj = A[(size_t)j * k + j];
      if (wj > wi || (wj == wi && j < i)) ++rank;
    }
    w[rank] = (double)wi;
    for (int row = 0; row < k; ++row) Vout[(size_t)rank * k + row] = (double)V[(size_t)i * k + row];
  }
  __syncthreads();
}

void jacobi_eig_batched(iga_ctx* ctx, double* const* A, double* const* V, double* const* w,
                        const int* k, int count, bool fp32) {
  IGA_REQUIRE(count >= 1 && count <= 4, "jacobi_eig: batch of 1..4 problems");
  const size_t limit = 220 * 1024;
  JacobiBatch batch{};
  size_t smem = 0;
  // modes from the largest problem so that one shared-memory size fits all
  int kmax = 0;
  for (int i = 0; i < count; ++i) kmax = std::max(kmax, k[i]);
  IGA_REQUIRE(kmax >= 1 && kmax <= 1024, "jacobi_eig: k out of range");
  // the FP32 variant needs A and V in shared memory; larger problems run in FP64
  size_t head32 = jacobi_head_bytes<float>(kmax);
  fp32 = fp32 && head32 + 2 * (size_t)kmax * kmax * sizeof(float) <= limit;
  size_t head = fp32 ? head32 : jacobi_head_bytes<double>(kmax);
  size_t one = (size_t)kmax * kmax * (fp32 ? sizeof(float) : sizeof(double));
  int mode = head + 2 * one <= limit ? 2 : (head + one <= limit ? 1 : 0);
  smem = head + (mode == 2 ? 2 * one : (mode == 1 ? one : 0));
  for (int i = 0; i < count; ++i) {
    IGA_REQUIRE(k[i] >= 1, "jacobi_eig: empty problem");
    batch.p[i].A = A[i];
    batch.p[i].Vout = V[i];
    batch.p[i].w = w[i];
    batch.p[i].k = k[i];
    batch.p[i].mode = mode;
    // with V outside shared memory the rotations accumulate in a global work
    // array and the sorted eigenvectors are scattered from there into V
    batch.p[i].Vwork = mode == 2 ? nullptr
                                 : scratch<double>(ctx, 220 + i, (size_t)k[i] * k[i]);
  }
  func_attr(jacobi_eig_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  func_attr(jacobi_eig_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  {
    // algorithmic: a symmetric eigen-decomposition with eigenvectors, 9 k^3 flop
    double fl = 0.0, by = 0.0;
    for (int i = 0; i < count; ++i) {
      fl += 9.0 * (double)k[i] * k[i] * k[i];
      by += 3.0 * 8.0 * (double)k[i] * k[i];
    }
    prof_count(ctx, by, fl);
  }
  // one thread per rotation element of a round (k/2 pairs x k), at most 1024
  int kkm2 = kmax + (kmax & 1);
  int threads = std::min(1024, std::max(64, ((kkm2 / 2) * kmax + 31) / 32 * 32));
  if (fp32)
    IGA_LAUNCH(ctx, jacobi_eig_kernel<float>, count, threads, smem, batch);
  else
    IGA_LAUNCH(ctx, jacobi_eig_kernel<double>, count, threads, smem, batch);
}

void jacobi_eig(iga_ctx* ctx, double* A, double* V, double* w, int k) {
  jacobi_eig_batched(ctx, &A, &V, &w, &k, 1);
}

// Generalised symmetric eigen-problem preparation in one block:
//   T = sym(sum_s PM[s]), S = sym(sum_s PK[s]), T <- sign(trace T) T,
//   T = L L^T (Cholesky), Linv = L^{-1}, C = Linv S Linv^T.
// If T is not positive definite the transform falls back to C = S, Linv = I.
// Work arrays in global memory (row-major k x k).
__global__ void gen_eig_prep_kernel(const double* __restrict__ PM, int SM,
                                    const double* __restrict__ PK, int SK, int k,
                                    double* __restrict__ T, double* __restrict__ S,
                                    double* __restrict__ X, double* __restrict__ C,
                                    double* __restrict__ Linv) {
  __shared__ double red[32];
  __shared__ int fail;
  const int kk = k * k;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    int i = t / k, j = t % k;
    double a = 0.0, b = 0.0;
    for (int s = 0; s < SM; ++s) a += PM[(size_t)s * kk + i * k + j] + PM[(size_t)s * kk + j * k + i];
    for (int s = 0; s < SK; ++s) b += PK[(size_t)s * kk + i * k + j] + PK[(size_t)s * kk + j * k + i];
    T[t] = 0.5 * a;
    S[t] = 0.5 * b;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  double tr = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) tr += T[i * k + i];
  tr = block_sum(tr, red);
  if (tr < 0.0)
    for (int t = threadIdx.x; t < kk; t += blockDim.x) T[t] = -T[t];
  __syncthreads();
  // right-looking Cholesky in place (lower triangle of T becomes L)
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = T[j * k + j];
      if (!(d > 0.0)) fail = 1;
      T[j * k + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    double ljj = T[j * k + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) T[i * k + j] /= ljj;
    __syncthreads();
    int m = k - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = j + 1 + t / m, l = j + 1 + t % m;
      if (l <= i) T[i * k + l] -= T[i * k + j] * T[l * k + j];
    }
    __syncthreads();
  }
  // Linv: column c solves L x = e_c by forward substitution
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int m = c; m < i; ++m) v -= T[i * k + m] * Linv[m * k + c];
      Linv[i * k + c] = i < c ? 0.0 : v / T[i * k + i];
    }
  }
  __syncthreads();
  if (fail) {
    for (int t = threadIdx.x; t < kk; t += blockDim.x) {
      Linv[t] = (t / k == t % k) ? 1.0 : 0.0;
      C[t] = S[t];
    }
    return;
  }
  // X = Linv S, C = X Linv^T
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    int i = t / k, j = t % k;
    double v = 0.0;
    for (int m = 0; m <= i; ++m) v += Linv[i * k + m] * S[m * k + j];
    X[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    int i = t / k, j = t % k;
    double v = 0.0;
    for (int m = 0; m <= j; ++m) v += X[i * k + m] * Linv[j * k + m];
    C[t] = v;
  }
}

void gen_eig_prep(iga_ctx* ctx, const double* PM, int SM, const double* PK, int SK, int k,
                  double* work, double* C, double* Linv) {
  double* T = work;
  double* S = work + (size_t)k * k;
  double* X = work + 2 * (size_t)k * k;
  IGA_LAUNCH(ctx, gen_eig_prep_kernel, 1, 256, 0, PM, SM, PK, SK, k, T, S, X, C, Linv);
}

// ----------------------------------------------------------------- TT-SVD

// column-major C (m x n, ldc) = op(A) op(B): the same storage as the
// row-major product C^T = op(B)^T op(A)^T
enum GemmOp { OP_N = 0, OP_T = 1 };
static void gemm(iga_ctx* ctx, GemmOp ta, GemmOp tb, int m, int n, int k, const double* A, int lda,
                 const double* B, int ldb, double* C, int ldc) {
  gemm_rm_batched<double>(ctx, tb == OP_T, ta == OP_T, n, m, k, 1.0, B, ldb, 0, A, lda, 0, 0.0, C,
                          ldc, 0, 1);
}

// ---- narrow products with a wide row-major A (ns x m, row length m >> ns)
//
// The randomized range finder multiplies the first unfolding (a few hundred
// rows of length n2 n3) by 8..16 columns.  Library GEMM tiles are 32 or 64
// columns wide and waste most of their FP64 work on such shapes; these
// kernels do only the k needed products per element.

constexpr int SKINNY_K = 16;        // widest block handled here
constexpr int SKINNY_R = 32;        // rows of A per CTA in the sketch
constexpr int SKINNY_T = 96;        // columns of A per shared-memory tile
constexpr int SKINNY_C = 2016;      // columns of A per CTA in the sketch (21 tiles)

// partial Y = A Om over this CTA's rows [i0, i0 + 32) and column chunk:
// P[chunk][i][c].  Thread (r, q), r = t / 8, q = t % 8, accumulates row i0 + r
// over the tile columns j = q, q + 8, ... in registers; A and Om tiles are
// staged in shared memory with coalesced loads, and the eight partial sums
// of a row (eight neighbouring lanes) meet by shuffles.
template <int KK>
__global__ void __launch_bounds__(256) skinny_sketch_kernel(
    const double* __restrict__ A, int ns, long long m, const double* __restrict__ Om, int k,
    long long clen, double* __restrict__ P) {
  __shared__ double As[SKINNY_R][SKINNY_T + 1];
  __shared__ double Os[SKINNY_T][KK];
  const int i0 = blockIdx.y * SKINNY_R;
  const long long c0 = (long long)blockIdx.x * clen;
  const long long cend = c0 + clen < m ? c0 + clen : m;
  const int r = threadIdx.x >> 3, q = threadIdx.x & 7;
  double acc[KK];
#pragma unroll
  for (int c = 0; c < KK; ++c) acc[c] = 0.0;
  for (long long j0 = c0; j0 < cend; j0 += SKINNY_T) {
    for (int t = threadIdx.x; t < SKINNY_R * SKINNY_T; t += blockDim.x) {
      const int rr = t / SKINNY_T, jj = t - rr * SKINNY_T;
      const long long j = j0 + jj;
      As[rr][jj] = (i0 + rr < ns && j < cend) ? A[(size_t)(i0 + rr) * m + j] : 0.0;
    }
    for (int t = threadIdx.x; t < SKINNY_T * KK; t += blockDim.x) {
      const int c = t / SKINNY_T, jj = t - c * SKINNY_T;
      const long long j = j0 + jj;
      Os[jj][c] = (c < k && j < cend) ? Om[(size_t)c * m + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = q; jj < SKINNY_T; jj += 8) {
      const double a = As[r][jj];
#pragma unroll
      for (int c = 0; c < KK; ++c)
        if (c < k) acc[c] = fma(a, Os[jj][c], acc[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < KK; ++c) {
    double v = acc[c];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    if (q == 0 && c < k && i0 + r < ns) P[((size_t)blockIdx.x * ns + i0 + r) * k + c] = v;
  }
}

// Y (ns x k col-major) = sum over CTAs of the partials
__global__ void skinny_reduce_kernel(const double* __restrict__ P, int nblk, int ns, int k,
                                     double* __restrict__ Y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * k) return;
  const int i = t / k, c = t - (t / k) * k;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += P[(size_t)b * ns * k + t];
  Y[(size_t)c * ns + i] = s;
}

// Bt (m x k col-major) = A^T Q, Q (ns x k col-major): one thread per column j of A
template <int KK>
__global__ void __launch_bounds__(256) skinny_at_kernel(
    const double* __restrict__ A, int ns, long long m, const double* __restrict__ Q, int k,
    double* __restrict__ Bt) {
  extern __shared__ double qs[];               // ns x k, row-major
  for (int t = threadIdx.x; t < ns * k; t += blockDim.x) {
    const int i = t / k, c = t - (t / k) * k;
    qs[t] = Q[(size_t)c * ns + i];
  }
  __syncthreads();
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double acc[KK];
#pragma unroll
  for (int c = 0; c < KK; ++c) acc[c] = 0.0;
  for (int i = 0; i < ns; ++i) {
    const double a = A[(size_t)i * m + j];
#pragma unroll
    for (int c = 0; c < KK; ++c)
      if (c < k) acc[c] = fma(a, qs[i * k + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KK; ++c)
    if (c < k) Bt[(size_t)c * m + j] = acc[c];
}

// partial Gram matrices of Bt (m x k col-major): P[blk] (k x k), rows split
// over the CTAs and threads; the reduce kernel above sums them
__global__ void __launch_bounds__(256) skinny_gram_kernel(const double* __restrict__ Bt,
                                                          long long m, int k,
                                                          double* __restrict__ P) {
  __shared__ double part[8][SKINNY_K * SKINNY_K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double g[SKINNY_K];
  // thread (w, lane) accumulates column c0 = lane % k of the Gram for rows in its stride
  for (int c0 = 0; c0 < k; ++c0) {
#pragma unroll
    for (int c = 0; c < SKINNY_K; ++c) g[c] = 0.0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
      const double b0 = Bt[(size_t)c0 * m + j];
#pragma unroll
      for (int c = 0; c < SKINNY_K; ++c)
        if (c < k) g[c] = fma(b0, Bt[(size_t)c * m + j], g[c]);
    }
#pragma unroll
    for (int c = 0; c < SKINNY_K; ++c) {
      if (c >= k) break;
      double v = g[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) part[w][c0 * k + c] = v;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += part[q][t];
    P[(size_t)blockIdx.x * k * k + t] = s;
  }
}

// T (kq x bt, col-major) = Q^T Y for Q (ns x kq), Y (ns x bt) col-major: one
// warp per entry
__global__ void qt_y_kernel(const double* __restrict__ Q, const double* __restrict__ Y, int ns,
                            int kq, int bt, double* __restrict__ T) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= kq * bt) return;
  const int a = e % kq, c = e / kq;
  double d = 0.0;
  for (int i = lane; i < ns; i += 32) d = fma(Q[(size_t)a * ns + i], Y[(size_t)c * ns + i], d);
  d = warp_sum(d);
  if (lane == 0) T[e] = d;
}

// Y -= Q T (Y ns x bt, Q ns x kq, T kq x bt; col-major): one thread per entry
__global__ void y_minus_qt_kernel(double* __restrict__ Y, const double* __restrict__ Q,
                                  const double* __restrict__ T, int ns, int kq, int bt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns * bt) return;
  const int i = e % ns, c = e / ns;
  double s = Y[e];
  for (int a = 0; a < kq; ++a) s = fma(-Q[(size_t)a * ns + i], T[(size_t)c * kq + a], s);
  Y[e] = s;
}

// C (m x r, col-major) = B (m x k, col-major) V(:, 0:r) with V (k x k col-major),
// k <= SKINNY_K: one thread per row of B
__global__ void rows_small_kernel(const double* __restrict__ B, long long m, int k,
                                  const double* __restrict__ V, int r, double* __restrict__ C) {
  __shared__ double vs[SKINNY_K * SKINNY_K];
  for (int t = threadIdx.x; t < k * r; t += blockDim.x) vs[t] = V[t];
  __syncthreads();
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double b[SKINNY_K];
#pragma unroll
  for (int a = 0; a < SKINNY_K; ++a) b[a] = a < k ? B[(size_t)a * m + j] : 0.0;
  for (int c = 0; c < r; ++c) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < SKINNY_K; ++a)
      if (a < k) s = fma(b[a], vs[c * k + a], s);
    C[(size_t)c * m + j] = s;
  }
}

// Y (ns x k) = A Om for A = X^T, X col-major (m x ns)
static void skinny_sketch(iga_ctx* ctx, const double* X, int ns, int m, const double* Om, int k,
                          double* Y) {
  // column chunks of at most SKINNY_C, and short enough (whole shared-memory
  // tiles) that the grid has about two CTAs per SM when A is small
  const int rb = (ns + SKINNY_R - 1) / SKINNY_R;
  const long long want = std::max<long long>(((long long)m + SKINNY_C - 1) / SKINNY_C,
                                             (2LL * ctx->nsm + rb - 1) / rb);
  long long clen = ((long long)m + want - 1) / want;
  clen = std::min<long long>(SKINNY_C, (clen + SKINNY_T - 1) / SKINNY_T * SKINNY_T);
  const int nb = (int)(((long long)m + clen - 1) / clen);
  double* P = scratch<double>(ctx, SLOT_TTSVD_PART, (size_t)nb * ns * k);
  // algorithmic: 2 ns m k flop, A read once
  prof_count(ctx, 8.0 * ns * (double)m, 2.0 * ns * (double)m * k);
  const dim3 grid(nb, rb);
  if (k <= 8)
    IGA_LAUNCH(ctx, skinny_sketch_kernel<8>, grid, 256, 0, X, ns, (long long)m, Om, k, clen, P);
  else
    IGA_LAUNCH(ctx, skinny_sketch_kernel<SKINNY_K>, grid, 256, 0, X, ns, (long long)m, Om, k,
               clen, P);
  IGA_LAUNCH(ctx, skinny_reduce_kernel, (ns * k + 255) / 256, 256, 0, P, nb, ns, k, Y);
}

// Bt (m x k) = A^T Q for A = X^T, X col-major (m x ns)
static void skinny_at(iga_ctx* ctx, const double* X, int ns, int m, const double* Q, int k,
                      double* Bt) {
  const size_t smem = (size_t)ns * k * sizeof(double);
  IGA_REQUIRE(smem <= 48 * 1024, "skinny_at: basis too large");
  prof_count(ctx, 8.0 * ns * (double)m, 2.0 * ns * (double)m * k);
  if (k <= 8)
    IGA_LAUNCH(ctx, skinny_at_kernel<8>, (unsigned)((m + 255) / 256), 256, smem, X, ns,
               (long long)m, Q, k, Bt);
  else
    IGA_LAUNCH(ctx, skinny_at_kernel<SKINNY_K>, (unsigned)((m + 255) / 256), 256, smem, X, ns,
               (long long)m, Q, k, Bt);
}

// G (k x k) = Bt^T Bt for Bt col-major (m x k)
static void skinny_gram(iga_ctx* ctx, const double* Bt, int m, int k, double* G) {
  const int nb = std::max(1, std::min(152 * 2, (m + 255) / 256));
  double* P = scratch<double>(ctx, SLOT_TTSVD_PART, (size_t)nb * k * k);
  IGA_LAUNCH(ctx, skinny_gram_kernel, nb, 256, 0, Bt, (long long)m, k, P);
  IGA_LAUNCH(ctx, skinny_reduce_kernel, (k * k + 255) / 256, 256, 0, P, nb, k, k, G);
}

// Truncated left singular factor of A (ns x m): A = X^T with X col-major
// (m x ns) when xT == false, A = Z with Z col-major (ns x m) when xT == true.
// Returns the rank r, U (ns x r) col-major in Uout, Ct = A^T U (m x r)
// col-major in Ctout.  Both outputs are (re)allocated here.
//
// Blocked adaptive randomized range finder: Gaussian blocks (8, 16, 32, ...
// columns) are applied to A, projected off the basis found so far (twice)
// and orthonormalised, until a fresh block's projected norm shows
// ||(I - Q Q^T) A||_F <= delta / 10 (for Gaussian columns w,
// E ||(I - QQ^T) A w||^2 = ||(I - QQ^T) A||_F^2).  Then Bt = A^T Q is formed
// once, its SVD comes from a two-pass Gram/Jacobi (the second Gram matrix is
// nearly diagonal, which gives relative accuracy to the small singular
// values), and the rank is the smallest r whose sketched tail plus the
// residual estimate is <= delta^2.  A is read once per block and once for Bt.
static int rsvd_left(iga_ctx* ctx, const double* X, bool xT, int ns, int m, double delta,
                     int rmax, DevBuf<double>& Uout, DevBuf<double>& Ctout, uint64_t seed) {
  const int kcap = std::min(ns, 256);
  double* Q = scratch<double>(ctx, SLOT_TTSVD_Q, (size_t)ns * kcap);    // (swapped with Yq)
  double* Om = scratch<double>(ctx, SLOT_TTSVD_OMEGA, (size_t)m * std::min(kcap, 128));
  double* Y = scratch<double>(ctx, SLOT_TTSVD_Y, (size_t)ns * std::min(kcap, 128));
  double* Yq = scratch<double>(ctx, SLOT_TTSVD_Y2, (size_t)ns * kcap);
  double* T = scratch<double>(ctx, SLOT_TTSVD_C, (size_t)kcap * std::min(kcap, 128));
  int kq = 0;
  int b = std::min(ns, 8);
  double est2 = 0.0;                           // squared residual estimate
  for (int blk = 0;; ++blk) {
    const int bt = std::min(b, kcap - kq);
    if (bt <= 0) { est2 = 0.0; break; }
    fill_gaussian(ctx, Om, (size_t)m * bt, seed + 7919u * (uint64_t)(blk + 1));
    if (!xT && bt <= SKINNY_K) skinny_sketch(ctx, X, ns, m, Om, bt, Y);
    else if (!xT) gemm(ctx, OP_T, OP_N, ns, bt, m, X, m, Om, m, Y, ns);
    else gemm(ctx, OP_N, OP_N, ns, bt, m, X, ns, Om, m, Y, ns);
    for (int pass = 0; pass < 2 && kq > 0; ++pass) {
      // Y -= Q (Q^T Y)
      IGA_LAUNCH(ctx, qt_y_kernel, (unsigned)((kq * bt + 7) / 8), 256, 0, Q, Y, ns, kq, bt, T);
      IGA_LAUNCH(ctx, y_minus_qt_kernel, (unsigned)((ns * bt + 255) / 256), 256, 0, Y, Q, T, ns,
                 kq, bt);
    }
    const double yn = device_norm2(ctx, Y, (size_t)ns * bt);
    est2 = yn * yn / bt;
    if (est2 <= 0.01 * delta * delta) break;
    // orthonormalise [Q, Y] as a whole: the kept columns come back up to
    // sign, and the new ones are orthogonal to them even when Y is
    // numerically rank deficient (Householder completes the basis)
    IGA_CUDA(cudaMemcpyAsync(Q + (size_t)kq * ns, Y, (size_t)ns * bt * sizeof(double),
                             cudaMemcpyDeviceToDevice, ctx->stream));
    householder_qr(ctx, Q, Yq, ns, kq + bt);
    std::swap(Q, Yq);
    kq += bt;
    if (kq >= kcap) { est2 = kq >= ns ? 0.0 : est2; break; }
    b = std::min(2 * b, 128);
  }
  const int k = std::max(kq, 1);
  if (kq == 0) {
    // A is below the threshold as a whole: one basis vector from a fresh sketch
    fill_gaussian(ctx, Om, (size_t)m, seed + 104729u);
    if (!xT) gemm(ctx, OP_T, OP_N, ns, 1, m, X, m, Om, m, Y, ns);
    else gemm(ctx, OP_N, OP_N, ns, 1, m, X, ns, Om, m, Y, ns);
    householder_qr(ctx, Y, Q, ns, 1);
  }
  double* Bt = scratch<double>(ctx, SLOT_TTSVD_BT, (size_t)m * k * 2);
  double* Bt2 = Bt + (size_t)m * k;
  double* G = scratch<double>(ctx, SLOT_TTSVD_G, (size_t)k * k * 2 + k);
  double* wv = G + (size_t)k * k * 2;
  double* V = scratch<double>(ctx, SLOT_TTSVD_V, (size_t)k * k * 3);
  double* V1 = V + (size_t)k * k;
  double* V2 = V1 + (size_t)k * k;
  const bool narrow = k <= SKINNY_K && (size_t)ns * k * sizeof(double) <= 48 * 1024;
  if (!xT && narrow) skinny_at(ctx, X, ns, m, Q, k, Bt);
  else if (!xT) gemm(ctx, OP_N, OP_N, m, k, ns, X, m, Q, ns, Bt, m);
  else gemm(ctx, OP_T, OP_N, m, k, ns, X, ns, Q, ns, Bt, m);
  // first Gram pass
  if (k <= SKINNY_K) skinny_gram(ctx, Bt, m, k, G);
  else gemm(ctx, OP_T, OP_N, k, k, m, Bt, m, Bt, m, G, k);
  jacobi_eig(ctx, G, V1, wv, k);
  // second pass on the rotated factor: nearly diagonal Gram matrix
  if (k <= SKINNY_K)
    IGA_LAUNCH(ctx, rows_small_kernel, (unsigned)((m + 255) / 256), 256, 0, Bt, (long long)m, k,
               V1, k, Bt2);
  else
    gemm(ctx, OP_N, OP_N, m, k, k, Bt, m, V1, k, Bt2, m);
  if (k <= SKINNY_K) skinny_gram(ctx, Bt2, m, k, G);
  else gemm(ctx, OP_T, OP_N, k, k, m, Bt2, m, Bt2, m, G, k);
  jacobi_eig(ctx, G, V2, wv, k);
  gemm(ctx, OP_N, OP_N, k, k, k, V1, k, V2, k, V, k);
  std::vector<double> lam(k);
  IGA_CUDA(cudaMemcpyAsync(lam.data(), wv, k * 8, cudaMemcpyDeviceToHost, ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  // smallest r with the sketched tail plus the residual estimate below delta
  std::vector<double> tail(k + 1, 0.0);
  tail[k] = est2;
  for (int i = k - 1; i >= 0; --i) tail[i] = tail[i + 1] + std::max(lam[i], 0.0);
  int r = k;
  for (int i = 1; i <= k; ++i)
    if (std::sqrt(tail[i]) <= delta) { r = i; break; }
  r = std::max(1, std::min(r, rmax));
  Uout.alloc((size_t)ns * r);
  gemm(ctx, OP_N, OP_N, ns, r, k, Q, ns, V, k, Uout.p, ns);
  // Ct = A^T U = Bt V_r
  Ctout.alloc((size_t)m * r);
  if (k <= SKINNY_K)
    IGA_LAUNCH(ctx, rows_small_kernel, (unsigned)((m + 255) / 256), 256, 0, Bt, (long long)m, k,
               V, r, Ctout.p);
  else
    gemm(ctx, OP_N, OP_N, m, r, k, Bt, m, V, k, Ctout.p, m);
  return r;
}

// ---- rank-1 cross test
//
// The cross approximation of Sec. 3 (TT-cross, named after eq.
// weightEquationSolve as an alternative to TT-SVD) at rank one: through the
// largest entry W(i0, j0, k0) = v take the three fibres a = W(:, j0, k0),
// b = W(i0, :, k0), c = W(i0, j0, :); the candidate is a (x) b (x) c / v^2.
// Its error is evaluated exactly over the whole tensor; when it is within the
// per-unfolding TT-SVD threshold tol * ref / sqrt(2) every unfolding has a
// rank-1 approximation that good, so TT-SVD would also stop at rank one, and
// the rank-1 TT is returned without any sketch.

__global__ void absmax_key_kernel(const double* __restrict__ x, size_t n,
                                  unsigned long long* __restrict__ key) {
  // key = (upper 32 bits of |x| as a double) << 32 | index: the upper bits of
  // a non-negative double order like its value, so the largest key marks an
  // entry within a factor 1 + 2^-20 of max |x| (any such entry is a good
  // pivot); one integer atomicMax per warp
  unsigned long long best = 0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long hi = (unsigned long long)__double_as_longlong(fabs(x[i])) >> 32;
    unsigned long long k = (hi << 32) | (unsigned long long)i;
    best = k > best ? k : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(key, best);
}

__global__ void fibres_kernel(const double* __restrict__ W, int n1, int n2, int n3,
                              const unsigned long long* __restrict__ idx, double* __restrict__ f) {
  // f = [a (n1) | b (n2) | c (n3) | v]; the pivot index is the low half of the key
  size_t id = (size_t)(*idx & 0xffffffffull);
  int k0 = (int)(id % n3);
  int j0 = (int)((id / n3) % n2);
  int i0 = (int)(id / ((size_t)n2 * n3));
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) f[t] = W[((size_t)t * n2 + j0) * n3 + k0];
  else if (t < n1 + n2) f[t] = W[((size_t)i0 * n2 + (t - n1)) * n3 + k0];
  else if (t < n1 + n2 + n3) f[t] = W[((size_t)i0 * n2 + j0) * n3 + (t - n1 - n2)];
  else if (t == n1 + n2 + n3) f[t] = W[id];
}

__global__ void rank1_residual_kernel(const double* __restrict__ W, int n1, int n2, int n3,
                                      const double* __restrict__ f, double* __restrict__ out) {
  // each block takes a contiguous range of (i, j) fibres, their factors
  // a_i b_j / v^2 staged in shared memory (one division per fibre), threads
  // along k: e = W - (a_i b_j / v^2) c_k
  constexpr int RB = 64;
  __shared__ double red[32];
  __shared__ double abs_[RB];
  const double* a = f;
  const double* b = f + n1;
  const double* c = f + n1 + n2;
  const double v = f[n1 + n2 + n3];
  const double iv2 = 1.0 / (v * v);
  const long long rows = (long long)n1 * n2;
  double acc0 = 0.0, acc1 = 0.0;
  for (long long r0 = (long long)blockIdx.x * RB; r0 < rows; r0 += (long long)gridDim.x * RB) {
    const int nr = (int)min((long long)RB, rows - r0);
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
      const long long rr = r0 + t;
      const int i = (int)(rr / n2), j = (int)(rr - (long long)i * n2);
      abs_[t] = a[i] * b[j] * iv2;
    }
    __syncthreads();
    const double* w = W + (size_t)r0 * n3;
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
      const double ck = c[k];
#pragma unroll 8
      for (int r = 0; r < nr; ++r) {
        const double e0 = fma(-abs_[r], ck, w[(size_t)r * n3 + k]);
        if (r & 1) acc1 = fma(e0, e0, acc1); else acc0 = fma(e0, e0, acc0);
      }
    }
  }
  double acc = block_sum(acc0 + acc1, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

__global__ void rank1_cores_kernel(const double* __restrict__ f, int n1, int n2, int n3,
                                   double* __restrict__ c1, double* __restrict__ c2,
                                   double* __restrict__ c3) {
  double v = f[n1 + n2 + n3];
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) c1[t] = f[t];
  else if (t < n1 + n2) c2[t - n1] = f[t] / v;
  else if (t < n1 + n2 + n3) c3[t - n1 - n2] = f[t] / v;
}

// returns a rank-1 TT when the cross candidate meets err <= limit, else nullptr
static iga_tt* rank1_cross(iga_ctx* ctx, const double* W, int n1, int n2, int n3, double limit) {
  size_t N = (size_t)n1 * n2 * n3;
  if (N >= (1ull << 32)) return nullptr;            // the pivot key holds a 32-bit index
  unsigned long long* keys = scratch<unsigned long long>(ctx, SLOT_TTSVD_C, 2);
  double* f = scratch<double>(ctx, SLOT_TTSVD_W, (size_t)n1 + n2 + n3 + 2);
  double* err = f + n1 + n2 + n3 + 1;
  IGA_CUDA(cudaMemsetAsync(keys, 0, 2 * sizeof(unsigned long long), ctx->stream));
  IGA_CUDA(cudaMemsetAsync(err, 0, sizeof(double), ctx->stream));
  int blocks = (int)std::min<size_t>((N + 255) / 256, 152 * 8);
  IGA_LAUNCH(ctx, absmax_key_kernel, blocks, 256, 0, W, N, keys);
  int nf = n1 + n2 + n3 + 1;
  IGA_LAUNCH(ctx, fibres_kernel, (nf + 255) / 256, 256, 0, W, n1, n2, n3, keys, f);
  prof_count(ctx, (double)N * 8.0, 4.0 * (double)N);
  int rblocks = (int)std::min<long long>(((long long)n1 * n2 + 63) / 64, 152 * 8);
  IGA_LAUNCH(ctx, rank1_residual_kernel, rblocks, 256, 0, W, n1, n2, n3, f, err);
  double h[2] = {0.0, 0.0};
  IGA_CUDA(cudaMemcpyAsync(h, f + n1 + n2 + n3, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  if (h[0] == 0.0 || !(std::sqrt(std::max(h[1], 0.0)) <= limit)) return nullptr;
  auto* tt = new iga_tt();
  try {
    tt->n[0] = n1; tt->n[1] = n2; tt->n[2] = n3;
    tt->r[0] = 1; tt->r[1] = 1;
    for (int d = 0; d < 3; ++d) tt->core[d].alloc(tt->n[d]);
    IGA_LAUNCH(ctx, rank1_cores_kernel, (nf + 255) / 256, 256, 0, f, n1, n2, n3, tt->core[0].p,
               tt->core[1].p, tt->core[2].p);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    delete tt;
    throw;
  }
  return tt;
}

void tt_svd3(iga_ctx* ctx, const double* W, int n1, int n2, int n3, double tol, double norm_ref,
             int rmax, iga_tt** out, double norm_w) {
  IGA_REQUIRE(W != nullptr && out != nullptr, "tt_svd: null pointer");
  IGA_REQUIRE(n1 > 0 && n2 > 0 && n3 > 0, "tt_svd: empty tensor");
  IGA_REQUIRE(tol >= 0.0, "tt_svd: negative tolerance");
  if (rmax <= 0) rmax = 1 << 30;
  *out = nullptr;
  size_t N = (size_t)n1 * n2 * n3;
  double nrm = norm_w >= 0.0 ? norm_w : device_norm2(ctx, W, N);
  double ref = norm_ref > 0.0 ? norm_ref : nrm;
  if (nrm == 0.0 || nrm <= tol * ref) return;            // rank 0
  double delta = tol * ref / std::sqrt(2.0);
  // rank-1 cross candidate within the per-unfolding threshold first
  if (iga_tt* r1 = rank1_cross(ctx, W, n1, n2, n3, delta)) {
    *out = r1;
    return;
  }
  // first unfolding (n1 x n2 n3): memory is X col-major (n2 n3 x n1)
  DevBuf<double> U1, C1, U2, C2;
  int m1 = n2 * n3;
  IGA_REQUIRE((size_t)n2 * n3 < (1u << 31), "tt_svd: unfolding too large");
  int r1 = rsvd_left(ctx, W, false, n1, m1, delta, rmax, U1, C1, 0x1811ull);
  // C1 col-major (m1 x r1) == row-major (r1, n2, n3): second unfolding
  // (r1 n2 x n3), memory Z col-major (n3 x r1 n2); right factor from A^T = Z
  int m2 = r1 * n2;
  int r2 = rsvd_left(ctx, C1.p, true, n3, m2, delta, rmax, U2, C2, 0x0797ull);
  auto* tt = new iga_tt();
  tt->n[0] = n1; tt->n[1] = n2; tt->n[2] = n3;
  tt->r[0] = r1; tt->r[1] = r2;
  try {
    tt->core[0].alloc((size_t)n1 * r1);
    transpose_cm(ctx, U1.p, n1, r1, tt->core[0].p);       // (n1 x r1) cm -> row-major (n1, r1)
    tt->core[1].alloc((size_t)m2 * r2);
    transpose_cm(ctx, C2.p, m2, r2, tt->core[1].p);       // (m2 x r2) cm -> row-major (r1,n2,r2)
    tt->core[2].alloc((size_t)r2 * n3);
    IGA_CUDA(cudaMemcpyAsync(tt->core[2].p, U2.p, (size_t)r2 * n3 * 8, cudaMemcpyDeviceToDevice,
                             ctx->stream));               // (n3 x r2) cm == row-major (r2, n3)
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    delete tt;
    throw;
  }
  *out = tt;
}

}  // namespace iga
