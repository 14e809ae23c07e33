// Batched univariate Gauss-quadrature assembly (step a4).
//
// Sec. 3, eq. massMatrix1D: M^(d)(w) = int B (x) B w dx, and the univariate
// stiffness factors K_kl^(d)(q) = int (delta(l,d) B) (x) (delta(k,d) B) q dx
// that build eq. stiffnessFinal.  The weight of every TT term is known at the
// Gauss points (sampled there, Gauss weights folded in), so each entry is
//   A_t(i, j) = sum_{e in supp i cap supp j} sum_q w_t(e, q) phi_i(x_eq) psi_j(x_eq).
// One thread owns one band entry (t, i, o); the (p+1) x q products of an
// entry are summed in registers.  Consecutive threads differ in o, then i, so
// band writes are coalesced and the weight rows of a term are shared through
// L1 by the threads of that term.
#include "iga_internal.cuh"

namespace iga {

__global__ void assemble_bands_kernel(const double* __restrict__ w, int T, int E, int q, int p,
                                      int n, int interior, const int* __restrict__ first,
                                      const int* __restrict__ elo, const int* __restrict__ ehi,
                                      const double* __restrict__ R, const double* __restrict__ C,
                                      double* __restrict__ band) {
  const int b = 2 * p + 1;
  const int nrow = n - 2 * interior;
  size_t total = (size_t)T * nrow * b;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int o = (int)(idx % b);
  size_t ti = idx / b;
  int i = (int)(ti % nrow) + interior;
  int t = (int)(ti / nrow);
  int j = i + o - p;
  double acc = 0.0;
  if (j >= interior && j < n - interior) {
    int e0 = max(elo[i], elo[j]);
    int e1 = min(ehi[i], ehi[j]);
    const double* wt = w + (size_t)t * E * q;
    for (int e = e0; e <= e1; ++e) {
      int ai = i - first[e], aj = j - first[e];
      const double* Re = R + (size_t)e * q * (p + 1);
      const double* Ce = C + (size_t)e * q * (p + 1);
      for (int k = 0; k < q; ++k)
        acc += wt[e * q + k] * Re[k * (p + 1) + ai] * Ce[k * (p + 1) + aj];
    }
  }
  band[idx] = acc;
}

void launch_assemble_bands(iga_ctx* ctx, const DirTables& t, const double* w, int T, int drow,
                           int dcol, int interior, double* band) {
  IGA_REQUIRE(T >= 0, "negative term count");
  if (T == 0) return;
  int nrow = t.n - 2 * interior;
  size_t total = (size_t)T * nrow * (2 * t.p + 1);
  int threads = 256;
  IGA_LAUNCH(ctx, assemble_bands_kernel, (unsigned)((total + threads - 1) / threads), threads, 0,
             w, T, t.E, t.q, t.p, t.n, interior, t.dfirst.p, t.delo.p, t.dehi.p,
             drow ? t.dD.p : t.dV.p, dcol ? t.dD.p : t.dV.p, band);
}

// Univariate load vectors: out[t][i] = sum_{e,q} w_t(e,q) phi_i(x_eq).
__global__ void load_vectors_kernel(const double* __restrict__ w, int T, int E, int q, int p,
                                    int n, int interior, const int* __restrict__ first,
                                    const int* __restrict__ elo, const int* __restrict__ ehi,
                                    const double* __restrict__ V, double* __restrict__ out) {
  const int nrow = n - 2 * interior;
  size_t total = (size_t)T * nrow;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int i = (int)(idx % nrow) + interior;
  int t = (int)(idx / nrow);
  const double* wt = w + (size_t)t * E * q;
  double acc = 0.0;
  for (int e = elo[i]; e <= ehi[i]; ++e) {
    int ai = i - first[e];
    for (int k = 0; k < q; ++k) acc += wt[e * q + k] * V[((size_t)e * q + k) * (p + 1) + ai];
  }
  out[idx] = acc;
}

void launch_load_vectors(iga_ctx* ctx, const DirTables& t, const double* w, int T, int interior,
                         double* out) {
  if (T == 0) return;
  size_t total = (size_t)T * (t.n - 2 * interior);
  int threads = 256;
  IGA_LAUNCH(ctx, load_vectors_kernel, (unsigned)((total + threads - 1) / threads), threads, 0, w,
             T, t.E, t.q, t.p, t.n, interior, t.dfirst.p, t.delo.p, t.dehi.p, t.dV.p, out);
}

}  // namespace iga
