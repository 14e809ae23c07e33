// Adjoint state, reduced gradient and weight-factor gradient (step a9).
//
// Sec. 4 (Lagrangian and KKT conditions), stationary reading: for a control
// u the state solves K y = M u, the adjoint solves K^T lam = b - M y, and the
// reduced objective J(u) = 1/2 y^T M y - b^T y + beta/2 u^T M u has gradient
//   dJ/du = beta M u - M lam.
// With L = J + lam^T (K y - M u), the derivative of J with respect to any
// parameter of M or K is the partial derivative of L.  For a univariate weight
// factor w_d(e, q) of a rank-1 Kronecker term A = A_1 (x) A_2 (x) A_3 of M or K
// (Sec. 3, eqs. massMatrix1D / stiffnessFinal: A_d(i, j) = sum w_d(e,q)
// phi_i psi_j (x_eq)), the chain rule gives
//   d(a^T A c)/dw_d(e,q) = sum_{i,j} phi_i(x_eq) psi_j(x_eq) S_d(i, j),
//   S_d(i, j) = sum_{other indices} a(.., i, ..) [(x)_{e != d} A_e c](.., j, ..),
// the reverse of the univariate assembly.
//
// The SPD solves use conjugate gradients on the full FP64 vectors, with the
// fast-diagonalisation preconditioner P = sum_d c_d Kt_d (x) (x)_{e != d} Mt_e
// built from the generalised eigenvectors of (Kt_d, Mt_d) per direction
// (Mt_d: the mass factors of M, Kt_d: the derivative factor of the q_dd
// block of K, c_d: ratio of the other directions' factor traces).  For a
// rank-1 mass operator P_M = M exactly.
#include <algorithm>
#include <cmath>

#include "iga_internal.cuh"

namespace iga {

static inline unsigned nb(size_t n, int th = 256) { return (unsigned)((n + th - 1) / th); }

// row-major C (M x N) = op(A) op(B) (+ beta C)
static void rgemm(iga_ctx* ctx, bool tA, bool tB, int M, int N, int K, const double* A, int lda,
                  const double* B, int ldb, double* C, int ldc, double beta = 0.0) {
  gemm_rm_batched<double>(ctx, tA, tB, M, N, K, 1.0, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1);
}

static void rgemm_batched(iga_ctx* ctx, bool tA, bool tB, int M, int N, int K, const double* A,
                          int lda, long long sA, const double* B, int ldb, long long sB, double* C,
                          int ldc, long long sC, int batch) {
  gemm_rm_batched<double>(ctx, tA, tB, M, N, K, 1.0, A, lda, sA, B, ldb, sB, 0.0, C, ldc, sC,
                          batch);
}

__global__ void band_to_dense_kernel(const double* __restrict__ band, int n, int p, double sign,
                                     double* __restrict__ A) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int i = idx / n, j = idx % n;
  int o = j - i + p;
  A[idx] = (o >= 0 && o <= 2 * p) ? sign * band[(size_t)i * (2 * p + 1) + o] : 0.0;
}

__global__ void inv_sqrt_abs_vec_kernel(const double* __restrict__ w, int k,
                                        double* __restrict__ s) {
  double mx = 0.0;
  for (int j = 0; j < k; ++j) mx = fmax(mx, fabs(w[j]));
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double v = fmax(fabs(w[i]), 1e-15 * mx);
  s[i] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
}

__global__ void scale_cols_kernel(const double* __restrict__ U, const double* __restrict__ s,
                                  int k, double* __restrict__ B) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * k) return;
  B[idx] = U[idx] * s[idx / k];                // column idx/k of a col-major matrix
}

__global__ void fd_denom_kernel(const double* __restrict__ l1, const double* __restrict__ l2,
                                const double* __restrict__ l3, double c1, double c2, double c3,
                                int n1, int n2, int n3, double* __restrict__ den) {
  size_t N = (size_t)n1 * n2 * n3;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  int i3 = (int)(idx % n3);
  size_t r = idx / n3;
  int i2 = (int)(r % n2), i1 = (int)(r / n2);
  double v = c1 * l1[i1] + c2 * l2[i2] + c3 * l3[i3];
  den[idx] = v > 0.0 ? 1.0 / v : 0.0;
}

__global__ void mul_kernel(double* __restrict__ x, const double* __restrict__ s, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s[i];
}

__global__ void lincomb_kernel(double* __restrict__ y, double a, const double* __restrict__ x,
                               double b, size_t n) {
  // y = a x + b y
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

// y = A (along `mode`) x for one banded factor (runtime half-bandwidth p)
__global__ void mode_apply_kernel(const double* __restrict__ band, int p, int mode, int n1, int n2,
                                  int n3, const double* __restrict__ x, double* __restrict__ y) {
  size_t N = (size_t)n1 * n2 * n3;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  int i3 = (int)(idx % n3);
  size_t r = idx / n3;
  int i2 = (int)(r % n2), i1 = (int)(r / n2);
  int nm = mode == 0 ? n1 : (mode == 1 ? n2 : n3);
  int im = mode == 0 ? i1 : (mode == 1 ? i2 : i3);
  ptrdiff_t stride = mode == 0 ? (ptrdiff_t)n2 * n3 : (mode == 1 ? (ptrdiff_t)n3 : 1);
  const double* row = band + (size_t)im * (2 * p + 1);
  double s = 0.0;
  for (int o = 0; o <= 2 * p; ++o) {
    int j = im + o - p;
    if (j >= 0 && j < nm) s += row[o] * x[idx + (ptrdiff_t)(j - im) * stride];
  }
  y[idx] = s;
}

// S[i][o] += coef * sum_{other indices} a(.. i ..) z(.. i+o-p ..)  along `mode`
__global__ void band_gram_kernel(const double* __restrict__ a, const double* __restrict__ z,
                                 int mode, int n1, int n2, int n3, int p, double coef,
                                 double* __restrict__ S) {
  __shared__ double red[32];
  const int B = 2 * p + 1;
  int i = blockIdx.x / B, o = blockIdx.x % B;
  int nm = mode == 0 ? n1 : (mode == 1 ? n2 : n3);
  int j = i + o - p;
  if (j < 0 || j >= nm) return;                          // uniform for the block
  size_t rest = (size_t)n1 * n2 * n3 / nm;
  double acc = 0.0;
  for (size_t t = threadIdx.x; t < rest; t += blockDim.x) {
    size_t ia, iz;
    if (mode == 0) {
      ia = (size_t)i * rest + t;
      iz = (size_t)j * rest + t;
    } else if (mode == 1) {
      size_t i1 = t / n3, i3 = t % n3;
      ia = (i1 * n2 + i) * n3 + i3;
      iz = (i1 * n2 + j) * n3 + i3;
    } else {
      ia = t * n3 + i;
      iz = t * n3 + j;
    }
    acc += a[ia] * z[iz];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    S[(size_t)i * B + o] += coef * s;
  }
}

// out[e*q + k] += sum_{a,b} R_a(x_ek) C_b(x_ek) S(first_e + a - 1, b - a + p)
// over interior local functions (full indices 1..n-2)
__global__ void band_reverse_kernel(const double* __restrict__ S, const double* __restrict__ R,
                                    const double* __restrict__ C, const int* __restrict__ first,
                                    int n, int E, int q, int p, double* __restrict__ out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= E * q) return;
  int e = idx / q;
  const double* Rk = R + (size_t)idx * (p + 1);
  const double* Ck = C + (size_t)idx * (p + 1);
  int f = first[e];
  const int B = 2 * p + 1;
  double acc = 0.0;
  for (int a = 0; a <= p; ++a) {
    int i = f + a;
    if (i < 1 || i > n - 2) continue;
    for (int b = 0; b <= p; ++b) {
      int j = f + b;
      if (j < 1 || j > n - 2) continue;
      acc += Rk[a] * Ck[b] * S[(size_t)(i - 1) * B + (b - a + p)];
    }
  }
  out[idx] += acc;
}

// ------------------------------------------------------------------------

static const double* block_band(const iga_op* A, int k, int d, int idx = 0) {
  size_t len = (size_t)A->n[d] * (2 * A->p[d] + 1);
  return A->band64[d].p + (A->blocks[k].off[d] + idx) * len;
}

static double band_trace(iga_ctx* ctx, const double* band, int n, int p) {
  std::vector<double> h((size_t)n * (2 * p + 1));
  IGA_CUDA(cudaMemcpyAsync(h.data(), band, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += h[(size_t)i * (2 * p + 1) + p];
  return t;
}

// index of the K block carrying q_dd (derivative on both sides in direction d only)
static int qdd_block(const iga_op* K, int d) {
  for (size_t k = 0; k < K->blocks.size(); ++k) {
    const OpBlock& b = K->blocks[k];
    bool ok = true;
    for (int e = 0; e < 3; ++e) {
      int want = (e == d);
      ok = ok && b.deriv[e][0] == want && b.deriv[e][1] == want;
    }
    if (ok) return (int)k;
  }
  return -1;
}

struct FDPrecond {
  int n[3] = {0, 0, 0};
  DevBuf<double> V[3], lam[3], den;
  double c[3] = {1, 1, 1};

  void setup(iga_ctx* ctx, const iga_op* M, const iga_op* K) {
    for (int d = 0; d < 3; ++d) n[d] = M->n[d];
    double trM[3], trK[3][3];
    int kb[3];
    for (int d = 0; d < 3; ++d) {
      kb[d] = K ? qdd_block(K, d) : -1;
      trM[d] = band_trace(ctx, block_band(M, 0, d), n[d], M->p[d]);
    }
    for (int d = 0; d < 3; ++d)
      for (int e = 0; e < 3; ++e)
        trK[d][e] = kb[d] >= 0 ? band_trace(ctx, block_band(K, kb[d], e), n[e], K->p[e]) : trM[e];
    for (int d = 0; d < 3; ++d) {
      double cd = 1.0;
      for (int e = 0; e < 3; ++e)
        if (e != d) cd *= std::fabs(trK[d][e]) / std::max(std::fabs(trM[e]), 1e-300);
      c[d] = cd;
      int nn = n[d], p = M->p[d];
      size_t k2 = (size_t)nn * nn;
      double* Md = scratch<double>(ctx, SLOT_AMEN_BASE + 100, k2);
      double* Kd = scratch<double>(ctx, SLOT_AMEN_BASE + 101, k2);
      double* U = scratch<double>(ctx, SLOT_AMEN_BASE + 102, k2);
      double* w = scratch<double>(ctx, SLOT_AMEN_BASE + 103, nn);
      double* s = scratch<double>(ctx, SLOT_AMEN_BASE + 104, nn);
      double* B = scratch<double>(ctx, SLOT_AMEN_BASE + 105, k2);
      double* Tm = scratch<double>(ctx, SLOT_AMEN_BASE + 106, k2);
      double* Cm = scratch<double>(ctx, SLOT_AMEN_BASE + 107, k2);
      IGA_LAUNCH(ctx, band_to_dense_kernel, nb(k2), 256, 0, block_band(M, 0, d), nn, p,
                 trM[d] >= 0 ? 1.0 : -1.0, Md);
      const double* kband = kb[d] >= 0 ? block_band(K, kb[d], d) : block_band(M, 0, d);
      double tk = kb[d] >= 0 ? trK[d][d] : trM[d];
      IGA_LAUNCH(ctx, band_to_dense_kernel, nb(k2), 256, 0, kband, nn, p, tk >= 0 ? 1.0 : -1.0, Kd);
      // generalised eigenvectors: T^{-1/2} from eig(Mt), then eig(T^{-1/2} Kt T^{-1/2})
      jacobi_eig(ctx, Md, U, w, nn);
      IGA_LAUNCH(ctx, inv_sqrt_abs_vec_kernel, nb(nn), 256, 0, w, nn, s);
      IGA_LAUNCH(ctx, scale_cols_kernel, nb(k2), 256, 0, U, s, nn, B);
      rgemm(ctx, true, false, nn, nn, nn, U, nn, B, nn, Tm, nn);      // U diag(s) U^T
      rgemm(ctx, false, false, nn, nn, nn, Tm, nn, Kd, nn, B, nn);
      rgemm(ctx, false, false, nn, nn, nn, B, nn, Tm, nn, Cm, nn);
      jacobi_eig(ctx, Cm, U, w, nn);
      V[d].ensure(k2);
      lam[d].ensure(nn);
      // V = Tm W (col-major): row-major V^T = W^T Tm
      rgemm(ctx, false, false, nn, nn, nn, U, nn, Tm, nn, V[d].p, nn);
      IGA_CUDA(cudaMemcpyAsync(lam[d].p, w, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    size_t N = (size_t)n[0] * n[1] * n[2];
    den.ensure(N);
    IGA_LAUNCH(ctx, fd_denom_kernel, nb(N), 256, 0, lam[0].p, lam[1].p, lam[2].p, c[0], c[1], c[2],
               n[0], n[1], n[2], den.p);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  }

  // t = (V1^T (x) V2^T (x) V3^T) r   (transpose = true)  or  (V1 (x) V2 (x) V3) r
  void transform(iga_ctx* ctx, const double* r, double* out, bool transpose) {
    int n1 = n[0], n2 = n[1], n3 = n[2];
    size_t N = (size_t)n1 * n2 * n3;
    double* t1 = scratch<double>(ctx, SLOT_AMEN_BASE + 110, N);
    double* t2 = scratch<double>(ctx, SLOT_AMEN_BASE + 111, N);
    // V col-major == V^T row-major
    rgemm(ctx, false, transpose, n1 * n2, n3, n3, r, n3, V[2].p, n3, t1, n3);
    rgemm_batched(ctx, !transpose, false, n2, n3, n2, V[1].p, n2, 0, t1, n3, (long long)n2 * n3, t2,
                  n3, (long long)n2 * n3, n1);
    rgemm(ctx, !transpose, false, n1, n2 * n3, n1, V[0].p, n1, t2, n2 * n3, out, n2 * n3);
  }

  // z = P^{-1} r; stiffness: scale by 1 / (c1 l1 + c2 l2 + c3 l3); mass: no scaling
  void apply(iga_ctx* ctx, const double* r, double* z, bool stiffness) {
    size_t N = (size_t)n[0] * n[1] * n[2];
    double* t = scratch<double>(ctx, SLOT_AMEN_BASE + 112, N);
    transform(ctx, r, t, true);
    if (stiffness) IGA_LAUNCH(ctx, mul_kernel, nb(N), 256, 0, t, den.p, N);
    transform(ctx, t, z, false);
  }
};

static double dot(iga_ctx* ctx, const double* a, const double* b, size_t n) {
  return device_dot(ctx, a, b, n);
}

// preconditioned CG for A x = b (A = M or K, SPD); x holds the initial guess
static int pcg(iga_ctx* ctx, const iga_op* A, FDPrecond& P, bool stiffness, const double* b,
               double* x, double tol, int maxit, double* relres) {
  size_t N = (size_t)A->n[0] * A->n[1] * A->n[2];
  double* r = scratch<double>(ctx, SLOT_AMEN_BASE + 120, N);
  double* z = scratch<double>(ctx, SLOT_AMEN_BASE + 121, N);
  double* pv = scratch<double>(ctx, SLOT_AMEN_BASE + 122, N);
  double* q = scratch<double>(ctx, SLOT_AMEN_BASE + 123, N);
  double bn = std::sqrt(dot(ctx, b, b, N));
  if (bn == 0.0) {
    IGA_CUDA(cudaMemsetAsync(x, 0, N * 8, ctx->stream));
    if (relres) *relres = 0.0;
    return 0;
  }
  kron_apply_impl(ctx, A, 1.0, x, 0.0, q, IGA_FP64);
  IGA_LAUNCH(ctx, lincomb_kernel, nb(N), 256, 0, q, 1.0, b, -1.0, N);     // q = b - A x
  IGA_CUDA(cudaMemcpyAsync(r, q, N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  P.apply(ctx, r, z, stiffness);
  IGA_CUDA(cudaMemcpyAsync(pv, z, N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  double rz = dot(ctx, r, z, N);
  double rn = std::sqrt(dot(ctx, r, r, N));
  int it = 0;
  while (rn > tol * bn && it < maxit) {
    kron_apply_impl(ctx, A, 1.0, pv, 0.0, q, IGA_FP64);
    double pq = dot(ctx, pv, q, N);
    if (!(pq > 0.0)) throw Error(IGA_ENONFINITE, "pcg: operator not positive definite");
    double al = rz / pq;
    IGA_LAUNCH(ctx, lincomb_kernel, nb(N), 256, 0, x, al, pv, 1.0, N);     // x += al p
    IGA_LAUNCH(ctx, lincomb_kernel, nb(N), 256, 0, r, -al, q, 1.0, N);     // r -= al q
    rn = std::sqrt(dot(ctx, r, r, N));
    ++it;
    if (!std::isfinite(rn)) throw Error(IGA_ENONFINITE, "pcg: non-finite residual");
    if (rn <= tol * bn) break;
    P.apply(ctx, r, z, stiffness);
    double rz2 = dot(ctx, r, z, N);
    IGA_LAUNCH(ctx, lincomb_kernel, nb(N), 256, 0, pv, 1.0, z, rz2 / rz, N);   // p = z + b p
    rz = rz2;
  }
  if (relres) *relres = rn / bn;
  return it;
}

}  // namespace iga

using namespace iga;

#define IGA_TRY2(ctx, ...)                                                        \
  try {                                                                           \
    ::iga::AllocScope scope__((ctx)->stream);                                     \
    __VA_ARGS__;                                                                  \
    return IGA_OK;                                                                \
  } catch (const ::iga::Error& e) {                                               \
    set_error(ctx, e.what());                                                     \
    return e.status;                                                              \
  } catch (const std::exception& e) {                                             \
    set_error(ctx, e.what());                                                     \
    return IGA_ECUDA;                                                             \
  }

extern "C" {

iga_status iga_spd_solve(iga_ctx* ctx, const iga_op* A, const iga_op* M, const iga_op* K,
                         const double* b, double* x, double tol, int maxit, int* iters,
                         double* relres) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY2(ctx, {
    IGA_REQUIRE(A && M && b && x && (A == M || A == K), "spd_solve: A must be M or K");
    IGA_REQUIRE(tol > 0.0 && maxit > 0, "spd_solve: bad tolerance or iteration limit");
    FDPrecond P;
    P.setup(ctx, M, K);
    double rr = 0.0;
    int it = pcg(ctx, A, P, A != M, b, x, tol, maxit, &rr);
    if (iters) *iters = it;
    if (relres) *relres = rr;
    if (rr > tol) throw Error(IGA_ENOCONV, "spd_solve: tolerance not reached");
  })
}

iga_status iga_reduced_gradient(iga_ctx* ctx, const iga_op* M, const iga_op* K,
                                const iga_tt* load, double beta, int nbatch, const double* u,
                                double tol, double* grad, double* y, double* lam, double* J) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY2(ctx, {
    IGA_REQUIRE(M && K && u && grad && y && lam && J && nbatch > 0,
                "reduced_gradient: null argument");
    IGA_REQUIRE(tol > 0.0, "reduced_gradient: tolerance must be positive");
    for (int d = 0; d < 3; ++d) IGA_REQUIRE(M->n[d] == K->n[d], "reduced_gradient: M, K mismatch");
    size_t N = (size_t)M->n[0] * M->n[1] * M->n[2];
    double* bvec = scratch<double>(ctx, SLOT_AMEN_BASE + 130, N);
    double* Mu = scratch<double>(ctx, SLOT_AMEN_BASE + 131, N);
    double* My = scratch<double>(ctx, SLOT_AMEN_BASE + 132, N);
    double* rhs = scratch<double>(ctx, SLOT_AMEN_BASE + 133, N);
    if (load) tt_full_impl(ctx, load, bvec);
    else IGA_CUDA(cudaMemsetAsync(bvec, 0, N * 8, ctx->stream));
    FDPrecond P;
    P.setup(ctx, M, K);
    for (int s = 0; s < nbatch; ++s) {
      const double* us = u + s * N;
      double* ys = y + s * N;
      double* ls = lam + s * N;
      double* gs = grad + s * N;
      double rr = 0.0;
      // state: K y = M u
      kron_apply_impl(ctx, M, 1.0, us, 0.0, Mu, IGA_FP64);
      IGA_CUDA(cudaMemsetAsync(ys, 0, N * 8, ctx->stream));
      pcg(ctx, K, P, true, Mu, ys, tol, 5000, &rr);
      if (rr > tol) throw Error(IGA_ENOCONV, "reduced_gradient: state solve did not converge");
      // adjoint: K^T lam = b - M y   (K symmetric)
      kron_apply_impl(ctx, M, 1.0, ys, 0.0, My, IGA_FP64);
      IGA_CUDA(cudaMemcpyAsync(rhs, bvec, N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
      IGA_LAUNCH(ctx, lincomb_kernel, nb(N), 256, 0, rhs, -1.0, My, 1.0, N);   // rhs = b - M y
      IGA_CUDA(cudaMemsetAsync(ls, 0, N * 8, ctx->stream));
      pcg(ctx, K, P, true, rhs, ls, tol, 5000, &rr);
      if (rr > tol) throw Error(IGA_ENOCONV, "reduced_gradient: adjoint solve did not converge");
      // gradient: beta M u - M lam
      kron_apply_impl(ctx, M, beta, us, 0.0, gs, IGA_FP64);
      kron_apply_impl(ctx, M, -1.0, ls, 1.0, gs, IGA_FP64);
      // J = 1/2 y^T M y - b^T y + beta/2 u^T M u (the constant 1/2 int yhat^2 omitted)
      J[s] = 0.5 * dot(ctx, ys, My, N) - dot(ctx, bvec, ys, N) + 0.5 * beta * dot(ctx, us, Mu, N);
    }
  })
}

iga_status iga_weight_gradient(iga_ctx* ctx, const iga_space* space, const iga_op* M,
                               const iga_op* K, double beta, const double* y, const double* u,
                               const double* lam, double* grad_w) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY2(ctx, {
    IGA_REQUIRE(space && M && K && y && u && lam && grad_w, "weight_gradient: null argument");
    SpaceTables st;
    build_space_tables(ctx, space, st);
    int Q[3];
    size_t tot = 0;
    for (int d = 0; d < 3; ++d) {
      Q[d] = st.dir[d].E * st.dir[d].q;
      tot += Q[d];
      IGA_REQUIRE(M->n[d] == st.dir[d].n - 2, "weight_gradient: space does not match M");
    }
    for (auto& b : M->blocks) IGA_REQUIRE(b.R1 == 1 && b.R2 == 1, "weight_gradient: rank-1 M only");
    for (auto& b : K->blocks) IGA_REQUIRE(b.R1 == 1 && b.R2 == 1, "weight_gradient: rank-1 K only");
    IGA_CUDA(cudaMemsetAsync(grad_w, 0, 7 * tot * 8, ctx->stream));
    int n[3] = {M->n[0], M->n[1], M->n[2]};
    size_t N = (size_t)n[0] * n[1] * n[2];
    double* z1 = scratch<double>(ctx, SLOT_AMEN_BASE + 140, N);
    double* z2 = scratch<double>(ctx, SLOT_AMEN_BASE + 141, N);
    const int qidx[3][3] = {{1, 2, 3}, {2, 4, 5}, {3, 5, 6}};
    auto process = [&](const iga_op* A, int k, int widx, const double* const* as,
                       const double* const* cs, const double* coefs, int nforms) {
      const OpBlock& blk = A->blocks[k];
      for (int d = 0; d < 3; ++d) {
        int p = A->p[d], B = 2 * p + 1;
        double* S = scratch<double>(ctx, SLOT_AMEN_BASE + 142, (size_t)n[d] * B);
        IGA_CUDA(cudaMemsetAsync(S, 0, (size_t)n[d] * B * 8, ctx->stream));
        int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
        for (int f = 0; f < nforms; ++f) {
          // z = (x)_{e != d} A_e c
          IGA_LAUNCH(ctx, mode_apply_kernel, nb(N), 256, 0, block_band(A, k, e1), A->p[e1], e1,
                     n[0], n[1], n[2], cs[f], z1);
          IGA_LAUNCH(ctx, mode_apply_kernel, nb(N), 256, 0, block_band(A, k, e2), A->p[e2], e2,
                     n[0], n[1], n[2], z1, z2);
          IGA_LAUNCH(ctx, band_gram_kernel, (unsigned)(n[d] * B), 256, 0, as[f], z2, d, n[0], n[1],
                     n[2], p, coefs[f], S);
        }
        const DirTables& T = st.dir[d];
        double* out = grad_w + (size_t)widx * tot + (d == 0 ? 0 : (d == 1 ? Q[0] : Q[0] + Q[1]));
        IGA_LAUNCH(ctx, band_reverse_kernel, nb((size_t)T.E * T.q), 256, 0, S,
                   blk.deriv[d][0] ? T.dD.p : T.dV.p, blk.deriv[d][1] ? T.dD.p : T.dV.p,
                   T.dfirst.p, T.n, T.E, T.q, T.p, out);
      }
    };
    // M: 1/2 y^T M y + beta/2 u^T M u - lam^T M u
    {
      const double* as[3] = {y, u, lam};
      const double* cs[3] = {y, u, u};
      const double coefs[3] = {0.5, 0.5 * beta, -1.0};
      process(M, 0, 0, as, cs, coefs, 3);
    }
    // K: + lam^T K_kl y for every (k, l) block, accumulated on the weight of q_kl
    for (size_t k = 0; k < K->blocks.size(); ++k) {
      const OpBlock& b = K->blocks[k];
      int kk = -1, ll = -1;
      for (int d = 0; d < 3; ++d) {
        if (b.deriv[d][0]) ll = d;
        if (b.deriv[d][1]) kk = d;
      }
      IGA_REQUIRE(kk >= 0 && ll >= 0, "weight_gradient: unexpected K block");
      const double* as[1] = {lam};
      const double* cs[1] = {y};
      const double coefs[1] = {1.0};
      process(K, (int)k, qidx[kk][ll], as, cs, coefs, 1);
    }
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

}  // extern "C"
