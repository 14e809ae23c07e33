// The weights interpolated in a spline space S~ (Sec. 3, eqs.
// weightEquationSystem and weightEquationSolve) instead of sampled on the
// Gauss grid.
//
// S~ has degree pt (default 2p + 1, the degree of the paper's experiments)
// on the break points of the discretisation.  The eight weights (omega, the
// six entries of Q, the load density) are sampled at the tensor grid of the
// Greville abscissae xi of S~ -- (E + pt)^3 points instead of (E q)^3 --
// and compressed by TT-SVD.  The collocation system
// (Bt_1 (x) Bt_2 (x) Bt_3) W = w(xi) separates: one solve with the banded
// Bt_d per direction and core.  The assembly then needs the interpolant at
// the Gauss points, so every core goes through the Q_d x n_d map
// L_d = diag(g_d) E_d Bt_d^{-1} (E_d[g, j] = Bt_j(x_g), g_d the Gauss
// weights), a product with a small dense matrix per core on the device.  The
// result is a TT of the same kind as the sampled route (weights times Gauss
// weights at the Gauss points) and feeds the same univariate assembly.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "iga_internal.cuh"

namespace iga {

namespace {

// all B-splines of degree p on `knots` at x (row of length n = #knots - p - 1):
// span search, then the triangular Cox-de Boor table of the p + 1 nonzero
// values; at x = 1 the last nonempty span is taken as closed
void bspline_row(const std::vector<double>& t, int p, double x, std::vector<double>& row) {
  const int n = (int)t.size() - p - 1;
  row.assign(n, 0.0);
  int mu = p;
  while (mu < n - 1 && !(x < t[mu + 1])) ++mu;
  std::vector<double> N(p + 1, 0.0), left(p + 1), right(p + 1);
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - t[mu + 1 - j];
    right[j] = t[mu + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      const double den = right[r + 1] + left[j - r];
      const double tmp = den != 0.0 ? N[r] / den : 0.0;
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
  }
  for (int r = 0; r <= p; ++r) row[mu - p + r] = N[r];
}

// dense LU with partial pivoting of the n x n matrix A (row-major, in place)
void lu_factor(std::vector<double>& A, int n, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int pr = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)pr * n + k])) pr = i;
    piv[k] = pr;
    if (pr != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)pr * n + j]);
    const double d = A[(size_t)k * n + k];
    IGA_REQUIRE(d != 0.0, "interpolation: singular collocation matrix");
    for (int i = k + 1; i < n; ++i) {
      const double f = (A[(size_t)i * n + k] /= d);
      if (f != 0.0)
        for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
    }
  }
}

// x^T A = b^T for the factorised A (solve with A^T): A^T = U^T L^T P
void lu_solve_transposed(const std::vector<double>& LU, const std::vector<int>& piv, int n,
                         std::vector<double>& b) {
  for (int i = 0; i < n; ++i) {          // U^T z = b
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= LU[(size_t)k * n + i] * b[k];
    b[i] = s / LU[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {     // L^T w = z (unit diagonal)
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= LU[(size_t)k * n + i] * b[k];
    b[i] = s;
  }
  for (int k = n - 1; k >= 0; --k)       // x = P^T w
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
}

}  // namespace

// open knot vector of degree pt on the break points of a discretisation
// direction, its Greville abscissae and the map L (Qd x n) from node values
// to the interpolant times the Gauss weight at the Gauss points (row-major)
void interp_direction(const DirTables& T, int pt, std::vector<double>& xi,
                      std::vector<double>& L) {
  std::vector<double> br;
  for (double k : T.knots)
    if (br.empty() || k > br.back()) br.push_back(k);
  std::vector<double> kt(pt, br.front());
  kt.insert(kt.end(), br.begin(), br.end());
  kt.insert(kt.end(), pt, br.back());
  const int n = (int)kt.size() - pt - 1;
  xi.resize(n);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 1; j <= pt; ++j) s += kt[i + j];
    xi[i] = s / pt;
  }
  std::vector<double> Bt((size_t)n * n), row;
  for (int i = 0; i < n; ++i) {
    bspline_row(kt, pt, xi[i], row);
    std::copy(row.begin(), row.end(), Bt.begin() + (size_t)i * n);
  }
  std::vector<int> piv;
  lu_factor(Bt, n, piv);
  const int Qd = (int)T.xq.size();
  L.assign((size_t)Qd * n, 0.0);
  for (int g = 0; g < Qd; ++g) {
    // row g of E Bt^{-1}: solve Bt^T l = E_g^T
    bspline_row(kt, pt, T.xq[g], row);
    lu_solve_transposed(Bt, piv, n, row);
    for (int j = 0; j < n; ++j) L[(size_t)g * n + j] = T.gq[g] * row[j];
  }
}

// core (r0, n, r1) -> (r0, Qd, r1) with the map L (Qd x n)
static iga_tt* map_to_gauss(iga_ctx* ctx, const iga_tt* src, const DevBuf<double> dL[3],
                            const int Qd[3]) {
  if (!src) return nullptr;
  std::unique_ptr<iga_tt> out(new iga_tt());
  const int rl[4] = {1, src->r[0], src->r[1], 1};
  out->r[0] = src->r[0];
  out->r[1] = src->r[1];
  for (int d = 0; d < 3; ++d) {
    const int n = src->n[d], r0 = rl[d], r1 = rl[d + 1];
    out->n[d] = Qd[d];
    out->core[d].alloc((size_t)r0 * Qd[d] * r1);
    // C_out[a] (Qd x r1) = L (Qd x n) C_in[a] (n x r1), a batch over r0
    gemm_rm_batched<double>(ctx, false, false, Qd[d], r1, n, 1.0, dL[d].p, n, 0,
                            src->core[d].p, r1, (long long)n * r1, 0.0, out->core[d].p, r1,
                            (long long)Qd[d] * r1, r0);
  }
  return out.release();
}

void weight_tts_interp_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                            const iga_target* target, double tol, int pt, iga_tt* tts[8]) {
  IGA_REQUIRE(pt >= 1 && pt <= 15, "interpolation: degree must be 1..15");
  std::vector<double> xi[3], L[3];
  DevBuf<double> dL[3];
  int nn[3], Qd[3];
  for (int d = 0; d < 3; ++d) {
    interp_direction(st.dir[d], pt, xi[d], L[d]);
    nn[d] = (int)xi[d].size();
    Qd[d] = (int)st.dir[d].xq.size();
    dL[d].alloc(L[d].size());
    IGA_CUDA(cudaMemcpyAsync(dL[d].p, L[d].data(), L[d].size() * 8, cudaMemcpyHostToDevice,
                             ctx->stream));
  }
  const size_t S = (size_t)nn[0] * nn[1] * nn[2];
  DevBuf<double> samples(8 * S);
  sample_weights_points(ctx, geo, xi, target, samples.p);
  double nrm[8];
  device_norms(ctx, samples.p, S, 8, nrm);
  double qn2 = 0.0;
  for (int c = 1; c <= 6; ++c)
    qn2 += (c == 2 || c == 3 || c == 5) ? 2 * nrm[c] * nrm[c] : nrm[c] * nrm[c];
  const double qnorm = std::sqrt(qn2);
  iga_tt* node[8] = {nullptr};
  try {
    const int last = (target && target->kind != IGA_TARGET_ZERO) ? 7 : 6;
    for (int c = 0; c <= last; ++c) {
      tt_svd3(ctx, samples.p + c * S, nn[0], nn[1], nn[2], tol,
              (c >= 1 && c <= 6) ? qnorm : 0.0, 0, &node[c], nrm[c]);
      tts[c] = map_to_gauss(ctx, node[c], dL, Qd);
      delete node[c];
      node[c] = nullptr;
    }
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    for (int c = 0; c < 8; ++c) {
      delete node[c];
      delete tts[c];
      tts[c] = nullptr;
    }
    throw;
  }
}

}  // namespace iga
