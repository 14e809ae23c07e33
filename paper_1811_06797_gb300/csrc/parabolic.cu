// Space-time operators and the FP64 residual of the parabolic KKT system
// (Sec. 4, eqs. timeDiscrete and KKTSystem; Sec. 5, eqs. M_kron and K_kron).
//
// With N_t implicit Euler steps of size tau the KKT blocks are built from
//   MM = I (x) M                (every block of the y-row, u-row, ...)
//   KK = I (x) tau K + C (x) M  (C: ones on the diagonal, minus ones below)
// The block-AMEn solver takes the time index as a fourth TT dimension in
// front of the three spatial ones (time the slowest index, as in
// y = [y_1; ...; y_{N_t}]).  Scaling the whole system by one factor does
// not change its solution, so the solver sees the stationary block layout
//   [ A_M  0        KK^T ]      A_M = tau MM
//   [ 0    beta A_M -A_M ]
//   [ KK  -A_M      0    ]
// with the time band of A_M equal to tau I and those of KK equal to tau I
// (the K blocks) and C (the M blocks).
#include "iga_internal.cuh"

#include <memory>

namespace iga {

namespace {

// time bands (count, nt, 3): band[k][0] = A(k, k-1), [1] = A(k, k), [2] = A(k, k+1);
// kind 0 = s I, kind 1 = C
__global__ void time_band_kernel(double* __restrict__ band, float* __restrict__ band32, int nt,
                                 int kind, double s) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  double lo = 0.0, di = s, up = 0.0;
  if (kind == 1) {
    di = 1.0;
    lo = k > 0 ? -1.0 : 0.0;
  }
  band[3 * k + 0] = lo;
  band[3 * k + 1] = di;
  band[3 * k + 2] = up;
  band32[3 * k + 0] = (float)lo;
  band32[3 * k + 1] = (float)di;
  band32[3 * k + 2] = (float)up;
}

// zt (nt, 3, N) from z (3, nt, N)
__global__ void field_time_swap_kernel(const double* __restrict__ z, int nt, size_t N,
                                       double* __restrict__ zt) {
  const size_t total = (size_t)3 * nt * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % N;
    const size_t q = idx / N;
    const int f = (int)(q % 3);
    const int k = (int)(q / 3);
    zt[idx] = z[((size_t)f * nt + k) * N + i];
  }
}

// res (3, nt, N) = F - tau S - coupling, with S (nt, 3, N) the stationary
// KKT rows per step and the time differences of C (x) M:
//   y-row:   M lam_k - M lam_{k+1}  (lam_{nt} = 0)
//   lam-row: M y_k - M y_{k-1}      (y_{-1} = 0)
__global__ void parabolic_combine_kernel(const double* __restrict__ F,
                                         const double* __restrict__ S,
                                         const double* __restrict__ My,
                                         const double* __restrict__ Ml, int nt, size_t N,
                                         double tau, double* __restrict__ res) {
  const size_t total = (size_t)3 * nt * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % N;
    const size_t q = idx / N;
    const int k = (int)(q % nt);
    const int f = (int)(q / nt);
    double a = tau * S[((size_t)k * 3 + f) * N + i];
    if (f == 0) {
      a += Ml[(size_t)k * N + i];
      if (k + 1 < nt) a -= Ml[(size_t)(k + 1) * N + i];
    } else if (f == 2) {
      a += My[(size_t)k * N + i];
      if (k > 0) a -= My[(size_t)(k - 1) * N + i];
    }
    res[idx] = F[idx] - a;
  }
}

// inputs of the fused step rows, each (nt, N), from z (3, nt, N):
//   a_k = tau y_k + lam_k - lam_{k+1},  d_k = tau (beta u_k - lam_k),
//   f_k = y_k - y_{k-1} - tau u_k       (lam_{nt} = 0, y_{-1} = 0)
__global__ void parabolic_inputs_kernel(const double* __restrict__ z, int nt, size_t N,
                                        double tau, double beta, double* __restrict__ a,
                                        double* __restrict__ dd, double* __restrict__ f) {
  const size_t NT = (size_t)nt * N;
  const double* y = z;
  const double* u = z + NT;
  const double* l = z + 2 * NT;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NT;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / N);
    const double lnext = k + 1 < nt ? l[idx + N] : 0.0;
    const double yprev = k > 0 ? y[idx - N] : 0.0;
    a[idx] = tau * y[idx] + l[idx] - lnext;
    dd[idx] = tau * (beta * u[idx] - l[idx]);
    f[idx] = y[idx] - yprev - tau * u[idx];
  }
}

unsigned grid_for(size_t n, int nsm) {
  return (unsigned)std::min<size_t>((n + 255) / 256, (size_t)8 * nsm);
}

void copy_bands(iga_ctx* ctx, iga_op* dst, int dd, const iga_op* a, int da, const iga_op* b,
                int db) {
  const size_t na = a->band64[da].n, nb = b ? b->band64[db].n : 0;
  const size_t len = (size_t)a->n[da] * (2 * a->p[da] + 1);
  dst->band64[dd].alloc(std::max<size_t>(1, na + nb));
  dst->band32[dd].alloc(std::max<size_t>(1, na + nb));
  dst->nbands[dd] = a->nbands[da] + (b ? b->nbands[db] : 0);
  IGA_CUDA(cudaMemcpyAsync(dst->band64[dd].p, a->band64[da].p, a->nbands[da] * len * 8,
                           cudaMemcpyDeviceToDevice, ctx->stream));
  IGA_CUDA(cudaMemcpyAsync(dst->band32[dd].p, a->band32[da].p, a->nbands[da] * len * 4,
                           cudaMemcpyDeviceToDevice, ctx->stream));
  if (b) {
    IGA_CUDA(cudaMemcpyAsync(dst->band64[dd].p + a->nbands[da] * len, b->band64[db].p,
                             b->nbands[db] * len * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    IGA_CUDA(cudaMemcpyAsync(dst->band32[dd].p + a->nbands[da] * len, b->band32[db].p,
                             b->nbands[db] * len * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  }
}

}  // namespace

void space_time_ops(iga_ctx* ctx, const iga_op* M, const iga_op* K, int nt, double tau,
                    std::unique_ptr<iga_op>& AM, std::unique_ptr<iga_op>& AK) {
  AM.reset(new iga_op());
  AK.reset(new iga_op());
  for (iga_op* A : {AM.get(), AK.get()}) {
    A->dims = 4;
    A->n[0] = nt;
    A->p[0] = 1;
    for (int d = 0; d < 3; ++d) {
      A->n[d + 1] = M->n[d];
      A->p[d + 1] = M->p[d];
    }
    A->rank1 = false;
  }
  const unsigned g = (unsigned)((nt + 127) / 128);
  // A_M = tau I (x) M: one time band, M's spatial bands
  AM->nbands[0] = 1;
  AM->band64[0].alloc((size_t)3 * nt);
  AM->band32[0].alloc((size_t)3 * nt);
  IGA_LAUNCH(ctx, time_band_kernel, g, 128, 0, AM->band64[0].p, AM->band32[0].p, nt, 0, tau);
  for (int d = 0; d < 3; ++d) copy_bands(ctx, AM.get(), d + 1, M, d, nullptr, 0);
  for (const OpBlock& b : M->blocks) {
    OpBlock nb = b;
    nb.off[0] = 0;
    for (int d = 0; d < 3; ++d) nb.off[d + 1] = b.off[d];
    AM->blocks.push_back(nb);
  }
  // KK = tau I (x) K + C (x) M: time bands [tau I, C], spatial bands K's then M's
  AK->nbands[0] = 2;
  AK->band64[0].alloc((size_t)6 * nt);
  AK->band32[0].alloc((size_t)6 * nt);
  IGA_LAUNCH(ctx, time_band_kernel, g, 128, 0, AK->band64[0].p, AK->band32[0].p, nt, 0, tau);
  IGA_LAUNCH(ctx, time_band_kernel, g, 128, 0, AK->band64[0].p + 3 * nt,
             AK->band32[0].p + 3 * nt, nt, 1, 1.0);
  for (int d = 0; d < 3; ++d) copy_bands(ctx, AK.get(), d + 1, K, d, M, d);
  for (const OpBlock& b : K->blocks) {
    OpBlock nb = b;
    nb.off[0] = 0;
    for (int d = 0; d < 3; ++d) nb.off[d + 1] = b.off[d];
    AK->blocks.push_back(nb);
  }
  for (const OpBlock& b : M->blocks) {
    OpBlock nb = b;
    nb.off[0] = 1;
    for (int d = 0; d < 3; ++d) nb.off[d + 1] = K->nbands[d] + b.off[d];
    AK->blocks.push_back(nb);
  }
}

double parabolic_residual(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta, int nt,
                          double tau, const double* F, const double* z, double* res, size_t N) {
  const size_t tot = (size_t)3 * nt * N;
  const size_t NT = (size_t)nt * N;
  if (M->rank1 && K->rank1) {
    // rank-one operators: res = F, then the three rows of every step in one
    // fused launch (five products per step, as in the stationary KKT apply)
    double* in3 = scratch<double>(ctx, SLOT_PARA_S, tot);
    IGA_CUDA(cudaMemcpyAsync(res, F, tot * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    IGA_LAUNCH(ctx, parabolic_inputs_kernel, grid_for(NT, ctx->nsm), 256, 0, z, nt, N, tau, beta,
               in3, in3 + NT, in3 + 2 * NT);
    bool fused = true;
    for (int k = 0; k < nt && fused; ++k) {
      const size_t o = (size_t)k * N;
      const double* in[5] = {in3 + o, in3 + NT + o, in3 + 2 * NT + o, z + o, z + 2 * NT + o};
      double* out[3] = {res + o, res + NT + o, res + 2 * NT + o};
      fused = parabolic_rows_fused(ctx, M, K, tau, in, out);
      IGA_REQUIRE(fused || k == 0, "parabolic residual: fused rows not applicable");
    }
    if (fused) return device_norm2(ctx, res, tot);
  }
  double* zt = scratch<double>(ctx, SLOT_PARA_ZT, tot);
  double* S = scratch<double>(ctx, SLOT_PARA_S, tot);
  double* MyMl = scratch<double>(ctx, SLOT_PARA_MV, (size_t)2 * nt * N);
  double* My = MyMl;
  double* Ml = MyMl + (size_t)nt * N;
  IGA_LAUNCH(ctx, field_time_swap_kernel, grid_for(tot, ctx->nsm), 256, 0, z, nt, N, zt);
  for (int k = 0; k < nt; ++k) {
    // the stationary rows [M y + K lam, beta M u - M lam, K y - M u] of step k
    kkt_apply_internal(ctx, M, K, beta, zt + (size_t)k * 3 * N, S + (size_t)k * 3 * N,
                       IGA_FP64);
    kron_apply_impl(ctx, M, 1.0, z + (size_t)k * N, 0.0, My + (size_t)k * N, IGA_FP64);
    kron_apply_impl(ctx, M, 1.0, z + ((size_t)2 * nt + k) * N, 0.0, Ml + (size_t)k * N,
                    IGA_FP64);
  }
  IGA_LAUNCH(ctx, parabolic_combine_kernel, grid_for(tot, ctx->nsm), 256, 0, F, S, My, Ml, nt, N,
             tau, res);
  return device_norm2(ctx, res, tot);
}

}  // namespace iga
