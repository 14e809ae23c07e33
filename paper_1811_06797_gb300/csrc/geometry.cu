// Geometry sampling (steps a1, a2): Gauss rule, B-spline tables, and the
// per-point NURBS Jacobian, omega = |det J| and Q = (J^T J)^{-1} omega.
//
// Sec. 2 (knot vectors, Cox-de Boor recursion, NURBS map G = C : B),
// Sec. 2 after eq. stiffness (omega and Q), Sec. 3 eq. weightEquationSystem
// (the weights are sampled on a tensor point grid).
#include <algorithm>
#include <cmath>

#include "iga_internal.cuh"

namespace iga {

constexpr int MAXP = 8;

void check_knots(const double* k, int nk, int p, const char* what) {
  IGA_REQUIRE(k != nullptr, std::string(what) + ": null knot vector");
  IGA_REQUIRE(p >= 0 && p <= MAXP, std::string(what) + ": degree must be in 0..8");
  int n = nk - p - 1;
  IGA_REQUIRE(n >= p + 1, std::string(what) + ": too few knots for the degree");
  for (int i = 0; i + 1 < nk; ++i)
    IGA_REQUIRE(k[i] <= k[i + 1], std::string(what) + ": knots must be nondecreasing");
  for (int i = 0; i <= p; ++i)
    IGA_REQUIRE(k[i] == 0.0 && k[nk - 1 - i] == 1.0,
                std::string(what) + ": end knots must be 0 and 1 with multiplicity p+1");
  int run = 1;
  for (int i = p + 1; i < n; ++i) {
    run = (k[i] == k[i - 1]) ? run + 1 : 1;
    IGA_REQUIRE(k[i] > 0.0 && k[i] < 1.0, std::string(what) + ": interior knot outside (0,1)");
    IGA_REQUIRE(run <= p, std::string(what) + ": interior knot multiplicity exceeds degree");
  }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_q.
static void gauss_rule(int q, std::vector<double>& t, std::vector<double>& w) {
  t.resize(q);
  w.resize(q);
  for (int k = 0; k < q; ++k) {
    double x = std::cos(M_PI * (k + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= q; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = x; p0 = 1.0; }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= q; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = x; p0 = 1.0; }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
    }
    t[q - 1 - k] = x;          // ascending order
    w[q - 1 - k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// span index mu with k[mu] <= x < k[mu+1] (the last nonempty span for x = 1)
__device__ __forceinline__ int find_span(const double* k, int nk, int p, double x) {
  int n = nk - p - 1;
  if (x >= k[n]) {
    int mu = n - 1;
    while (mu > p && k[mu] == k[mu + 1]) --mu;
    return mu;
  }
  int lo = p, hi = n;           // k[lo] <= x < k[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (x < k[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// The p+1 B-splines beta_{mu-p..mu} of degree p that are nonzero at x, and
// their first derivatives, by the Cox-de Boor recursion restricted to the
// nonzero functions (beta_{i,0} = 1 on span mu; degree j from degree j-1).
__device__ void local_basis(const double* k, int mu, int p, double x, double* N, double* dN) {
  double B[MAXP + 2], Bp[MAXP + 2];
  B[0] = 1.0;                       // degree 0: only beta_mu
  for (int a = 0; a <= p; ++a) Bp[a] = 0.0;
  if (p == 0) Bp[0] = 0.0;
  for (int j = 1; j <= p; ++j) {
    if (j == p)
      for (int a = 0; a < j; ++a) Bp[a] = B[a];   // degree p-1 values, i = mu-p+1+a
    double nb[MAXP + 2];
    for (int a = 0; a <= j; ++a) {
      int i = mu - j + a;
      double v = 0.0;
      if (a - 1 >= 0) {               // beta_{i, j-1} (old index a-1)
        double d1 = k[i + j] - k[i];
        if (d1 > 0.0) v += (x - k[i]) / d1 * B[a - 1];
      }
      if (a <= j - 1) {               // beta_{i+1, j-1} (old index a)
        double d2 = k[i + j + 1] - k[i + 1];
        if (d2 > 0.0) v += (k[i + j + 1] - x) / d2 * B[a];
      }
      nb[a] = v;
    }
    for (int a = 0; a <= j; ++a) B[a] = nb[a];
  }
  for (int a = 0; a <= p; ++a) N[a] = B[a];
  if (p == 0) { dN[0] = 0.0; return; }
  // beta'_{i,p} = p [beta_{i,p-1} / (k_{i+p} - k_i) - beta_{i+1,p-1} / (k_{i+p+1} - k_{i+1})]
  for (int a = 0; a <= p; ++a) {
    int i = mu - p + a;
    double v = 0.0;
    if (a - 1 >= 0) {
      double d1 = k[i + p] - k[i];
      if (d1 > 0.0) v += Bp[a - 1] / d1;
    }
    if (a <= p - 1) {
      double d2 = k[i + p + 1] - k[i + 1];
      if (d2 > 0.0) v -= Bp[a] / d2;
    }
    dN[a] = p * v;
  }
}

// Basis tables at a list of points: span[pt], V[pt][a], D[pt][a], a = 0..p.
__global__ void basis_table_kernel(const double* __restrict__ knots, int nk, int p,
                                   const double* __restrict__ x, int npts, int* __restrict__ span,
                                   double* __restrict__ V, double* __restrict__ D) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npts) return;
  double xx = x[t];
  int mu = find_span(knots, nk, p, xx);
  double N[MAXP + 1], dN[MAXP + 1];
  local_basis(knots, mu, p, xx, N, dN);
  if (span) span[t] = mu;
  for (int a = 0; a <= p; ++a) {
    V[t * (p + 1) + a] = N[a];
    D[t * (p + 1) + a] = dN[a];
  }
}

static void basis_tables(iga_ctx* ctx, const std::vector<double>& knots, int p,
                         const double* dx, int npts, int* dspan, double* dV, double* dD) {
  DevBuf<double> dk(knots.size());
  IGA_CUDA(cudaMemcpyAsync(dk.p, knots.data(), knots.size() * 8, cudaMemcpyHostToDevice,
                           ctx->stream));
  int threads = 128;
  IGA_LAUNCH(ctx, basis_table_kernel, (npts + threads - 1) / threads, threads, 0, dk.p,
             (int)knots.size(), p, dx, npts, dspan, dV, dD);
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));   // dk is released on return
}

void build_space_tables(iga_ctx* ctx, const iga_space* sp, SpaceTables& st) {
  IGA_REQUIRE(sp != nullptr, "null space");
  IGA_REQUIRE(sp->nquad >= 1 && sp->nquad <= 16, "nquad must be in 1..16");
  st.nquad = sp->nquad;
  std::vector<double> t, w;
  gauss_rule(sp->nquad, t, w);
  for (int d = 0; d < 3; ++d) {
    DirTables& T = st.dir[d];
    int p = sp->degree[d];
    check_knots(sp->knots[d], sp->nknots[d], p, "space");
    T.p = p;
    T.q = sp->nquad;
    T.knots.assign(sp->knots[d], sp->knots[d] + sp->nknots[d]);
    T.n = sp->nknots[d] - p - 1;
    IGA_REQUIRE(T.n >= 3, "space needs at least 3 basis functions per direction");
    // elements = nonempty spans; first nonzero basis function on each
    std::vector<double> u;
    for (double v : T.knots) if (u.empty() || v > u.back()) u.push_back(v);
    T.E = (int)u.size() - 1;
    T.first.resize(T.E);
    T.xq.resize((size_t)T.E * T.q);
    T.gq.resize((size_t)T.E * T.q);
    for (int e = 0; e < T.E; ++e) {
      double a = u[e], b = u[e + 1];
      int mu = (int)(std::upper_bound(T.knots.begin(), T.knots.end(), a) - T.knots.begin()) - 1;
      T.first[e] = mu - p;
      for (int j = 0; j < T.q; ++j) {
        T.xq[(size_t)e * T.q + j] = 0.5 * (a + b) + 0.5 * (b - a) * t[j];
        T.gq[(size_t)e * T.q + j] = 0.5 * (b - a) * w[j];
      }
    }
    T.elo.assign(T.n, T.E);
    T.ehi.assign(T.n, -1);
    for (int e = 0; e < T.E; ++e)
      for (int a = 0; a <= p; ++a) {
        int i = T.first[e] + a;
        T.elo[i] = std::min(T.elo[i], e);
        T.ehi[i] = std::max(T.ehi[i], e);
      }
    int npts = T.E * T.q;
    T.dx.alloc(npts);
    T.dV.alloc((size_t)npts * (p + 1));
    T.dD.alloc((size_t)npts * (p + 1));
    T.dfirst.alloc(T.E);
    T.delo.alloc(T.n);
    T.dehi.alloc(T.n);
    IGA_CUDA(cudaMemcpyAsync(T.dx.p, T.xq.data(), npts * 8, cudaMemcpyHostToDevice, ctx->stream));
    IGA_CUDA(cudaMemcpyAsync(T.dfirst.p, T.first.data(), T.E * 4, cudaMemcpyHostToDevice,
                             ctx->stream));
    IGA_CUDA(cudaMemcpyAsync(T.delo.p, T.elo.data(), T.n * 4, cudaMemcpyHostToDevice,
                             ctx->stream));
    IGA_CUDA(cudaMemcpyAsync(T.dehi.p, T.ehi.data(), T.n * 4, cudaMemcpyHostToDevice,
                             ctx->stream));
    basis_tables(ctx, T.knots, p, T.dx.p, npts, nullptr, T.dV.p, T.dD.p);
  }
}

struct GeoDev {
  const double* V[3];
  const double* D[3];
  const int* span[3];
  const double* g[3];
  int pg[3];
  int nc[3];
  int Q[3];
  const double* ctrl;
  const double* H2;       // sum-factorised partial sums (stage 2 output)
  int comp;               // -1: write all eight tensors; c >= 0: only tensor c
  double* qn2;            // optional: accumulates ||Q g||_F^2 over all nine entries
  int kind;
  double twist;
  int tkind;
  double tp[4];
};

// Sum factorisation of the homogeneous map and its parametric derivatives
// (Sec. 2, eq. geometryMapping: G = C : B with B the tensor-product basis):
//   stage 3: H3[A][B][i3][m][v]   = sum_c (B3 | B3')(x3) C[A][B][c][m]
//   stage 2: H2[A][i2][i3][m][w]  = sum_b (B2 | B2')(x2) H3[A][b][i3][m][.]
//            w = (B2 B3, B2' B3, B2 B3')
//   point:   A_m, dA_m/dxhat_k    = sum_a (B1 | B1')(x1) H2[a][i2][i3][m][.]
__global__ void geo_stage3_kernel(GeoDev G, double* __restrict__ H3) {
  size_t total = (size_t)G.nc[0] * G.nc[1] * G.Q[2];
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int i3 = (int)(t % G.Q[2]);
  size_t ab = t / G.Q[2];
  const int p3 = G.pg[2];
  int s3 = G.span[2][i3] - p3;
  const double* V3 = G.V[2] + (size_t)i3 * (p3 + 1);
  const double* D3 = G.D[2] + (size_t)i3 * (p3 + 1);
  const double* C = G.ctrl + (ab * G.nc[2] + s3) * 4;
  double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c <= p3; ++c)
    for (int m = 0; m < 4; ++m) {
      double cm = __ldg(C + c * 4 + m);
      h[2 * m] += V3[c] * cm;
      h[2 * m + 1] += D3[c] * cm;
    }
  double* o = H3 + t * 8;
  for (int k = 0; k < 8; ++k) o[k] = h[k];
}

__global__ void geo_stage2_kernel(GeoDev G, const double* __restrict__ H3, double* __restrict__ H2) {
  size_t total = (size_t)G.nc[0] * G.Q[1] * G.Q[2];
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int i3 = (int)(t % G.Q[2]);
  size_t r = t / G.Q[2];
  int i2 = (int)(r % G.Q[1]);
  int A = (int)(r / G.Q[1]);
  const int p2 = G.pg[1];
  int s2 = G.span[1][i2] - p2;
  const double* V2 = G.V[1] + (size_t)i2 * (p2 + 1);
  const double* D2 = G.D[1] + (size_t)i2 * (p2 + 1);
  double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b <= p2; ++b) {
    const double* h = H3 + (((size_t)A * G.nc[1] + s2 + b) * G.Q[2] + i3) * 8;
    for (int m = 0; m < 4; ++m) {
      double hv = h[2 * m], hd = h[2 * m + 1];
      acc[3 * m + 0] += V2[b] * hv;
      acc[3 * m + 1] += D2[b] * hv;
      acc[3 * m + 2] += V2[b] * hd;
    }
  }
  double* o = H2 + t * 12;
  for (int k = 0; k < 12; ++k) o[k] = acc[k];
}

// The eight weights of one tensor Gauss point (i1, i2, i3): homogeneous map
// and derivatives from the partial sums, quotient rule for the rational map,
// optional twist, then omega, Q and the load density, all times g1 g2 g3.
// Returns the orientation code of the point: 1 det < 0, 2 det > 0, 4 det zero
// or not finite.
__device__ __forceinline__ int point_weights(const GeoDev& G, int i1, int i2, int i3,
                                             double v[8]) {
  const size_t rem = (size_t)i2 * G.Q[2] + i3;
  const size_t Q12 = (size_t)G.Q[1] * G.Q[2];
  const int p1 = G.pg[0];
  const double* V1 = G.V[0] + (size_t)i1 * (p1 + 1);
  const double* D1 = G.D[0] + (size_t)i1 * (p1 + 1);
  int s1 = G.span[0][i1] - p1;
  double A[4] = {0, 0, 0, 0}, dA[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int a = 0; a <= p1; ++a) {
    const double* h = G.H2 + ((size_t)(s1 + a) * Q12 + rem) * 12;
    double v1 = V1[a], d1 = D1[a];
    for (int m = 0; m < 4; ++m) {
      double h0 = h[3 * m], h1 = h[3 * m + 1], h2 = h[3 * m + 2];
      A[m] += v1 * h0;
      dA[0][m] += d1 * h0;
      dA[1][m] += v1 * h1;
      dA[2][m] += v1 * h2;
    }
  }
  double iw = 1.0 / A[3];
  double X[3] = {A[0] * iw, A[1] * iw, A[2] * iw};
  double J[3][3];                                    // J[a][k] = dG_a / dxhat_k
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) J[a][k] = (dA[k][a] - X[a] * dA[k][3]) * iw;
  if (G.kind == IGA_GEO_NURBS_TWIST) {
    double th = G.twist * X[2];
    double s, c;
    sincos(th, &s, &c);
    double x = X[0], y = X[1];
    double J0[3], J1[3];
    for (int k = 0; k < 3; ++k) {
      J0[k] = c * J[0][k] - s * J[1][k] + G.twist * (-s * x - c * y) * J[2][k];
      J1[k] = s * J[0][k] + c * J[1][k] + G.twist * (c * x - s * y) * J[2][k];
    }
    for (int k = 0; k < 3; ++k) { J[0][k] = J0[k]; J[1][k] = J1[k]; }
    X[0] = c * x - s * y;
    X[1] = s * x + c * y;
  }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  const int code = (!(det != 0.0) || !isfinite(det)) ? 4 : (det > 0.0 ? 2 : 1);
  double adet = fabs(det);
  // metric m = J^T J; Q = adj(m) / det(m) * |det J| = adj(m) / |det J|
  // symmetric metric m = J^T J (six entries)
  double m00 = J[0][0] * J[0][0] + J[1][0] * J[1][0] + J[2][0] * J[2][0];
  double m01 = J[0][0] * J[0][1] + J[1][0] * J[1][1] + J[2][0] * J[2][1];
  double m02 = J[0][0] * J[0][2] + J[1][0] * J[1][2] + J[2][0] * J[2][2];
  double m11 = J[0][1] * J[0][1] + J[1][1] * J[1][1] + J[2][1] * J[2][1];
  double m12 = J[0][1] * J[0][2] + J[1][1] * J[1][2] + J[2][1] * J[2][2];
  double m22 = J[0][2] * J[0][2] + J[1][2] * J[1][2] + J[2][2] * J[2][2];
  double g = G.g[0][i1] * G.g[1][i2] * G.g[2][i3];
  // the Gauss weight folded into the scale of the adjugate
  double inv = g / adet;
  v[1] = (m11 * m22 - m12 * m12) * inv;
  v[2] = (m02 * m12 - m01 * m22) * inv;
  v[3] = (m01 * m12 - m02 * m11) * inv;
  v[4] = (m00 * m22 - m02 * m02) * inv;
  v[5] = (m02 * m01 - m00 * m12) * inv;
  v[6] = (m00 * m11 - m01 * m01) * inv;
  double yh = 0.0;
  if (G.tkind == IGA_TARGET_SINPROD) {
    yh = sin(M_PI * X[0]) * sin(M_PI * X[1]) * sin(M_PI * X[2]);
  } else if (G.tkind == IGA_TARGET_GAUSS) {
    double dx = X[0] - G.tp[0], dy = X[1] - G.tp[1], dz = X[2] - G.tp[2];
    yh = exp(-(dx * dx + dy * dy + dz * dz) / G.tp[3]);
  }
  const double wg = adet * g;
  v[0] = wg;
  v[7] = yh * wg;
  return code;
}

// one OR of the orientation codes per warp, an atomic only when it adds a bit
__device__ __forceinline__ void record_orientation(int code, int* flag) {
  const int wcode = __reduce_or_sync(0xffffffffu, code);
  if ((threadIdx.x & 31) == 0 && wcode != 0 && (wcode & ~*(volatile int*)flag) != 0)
    atomicOr(flag, wcode);
}

// One thread per tensor Gauss point of the whole grid.
__global__ void sample_weights_kernel(GeoDev G, double* __restrict__ out, int* __restrict__ flag) {
  size_t Q12 = (size_t)G.Q[1] * G.Q[2];
  size_t total = (size_t)G.Q[0] * Q12;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // lanes past the end evaluate point 0 and write nothing, so every warp stays
  // converged for the reductions below
  const bool valid = t < total;
  if (!valid) t = 0;
  int i1 = (int)(t / Q12);
  size_t rem = t - (size_t)i1 * Q12;
  int i2 = (int)(rem / G.Q[2]);
  int i3 = (int)(rem - (size_t)i2 * G.Q[2]);
  double v[8];
  const int code = point_weights(G, i1, i2, i3, v);
  record_orientation(valid ? code : 0, flag);
  if (valid) {
    if (G.comp < 0) {
      for (int c = 0; c < 8; ++c) out[c * total + t] = v[c];
    } else {
      out[t] = v[G.comp];
    }
  }
  if (G.qn2) {
    double q2 = valid ? (v[1] * v[1] + v[4] * v[4] + v[6] * v[6] +
                         2.0 * (v[2] * v[2] + v[3] * v[3] + v[5] * v[5]))
                      : 0.0;
    for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(G.qn2, q2);
  }
}

// The weights at P listed points (i1, i2, i3) = idx[3p .. 3p+2]: all eight
// channels, out[c P + p] (the fibres and test points of the TT-cross).
__global__ void sample_points_kernel(GeoDev G, const int* __restrict__ idx, int P,
                                     double* __restrict__ out, int* __restrict__ flag) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < P;
  const int q = valid ? p : 0;
  double v[8];
  const int code = point_weights(G, idx[3 * q], idx[3 * q + 1], idx[3 * q + 2], v);
  record_orientation(valid ? code : 0, flag);
  if (valid)
    for (int c = 0; c < 8; ++c) out[(size_t)c * P + p] = v[c];
}

struct GeoSampler {
  GeoDev G{};
  DevBuf<double> gV[3], gD[3], gw[3], ctrl, H2;
  DevBuf<int> gspan[3];
  size_t total = 0;

  void prepare(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
               const iga_target* target) {
    const double* pts[3];
    const double* wts[3];
    int np[3];
    for (int d = 0; d < 3; ++d) {
      pts[d] = st.dir[d].dx.p;
      wts[d] = st.dir[d].gq.data();
      np[d] = st.dir[d].E * st.dir[d].q;
    }
    prepare_grid(ctx, geo, pts, wts, np, target);
  }

  // the tensor grid of arbitrary 1-D point sets (device arrays) with the given
  // host weights per point (folded into every sample as on the Gauss grid)
  DevBuf<double> own_pts[3];
  void prepare_points(iga_ctx* ctx, const iga_geometry* geo, const std::vector<double> hp[3],
                      const iga_target* target) {
    const double* pts[3];
    std::vector<double> ones[3];
    const double* wts[3];
    int np[3];
    for (int d = 0; d < 3; ++d) {
      own_pts[d].alloc(hp[d].size());
      IGA_CUDA(cudaMemcpyAsync(own_pts[d].p, hp[d].data(), hp[d].size() * 8,
                               cudaMemcpyHostToDevice, ctx->stream));
      pts[d] = own_pts[d].p;
      ones[d].assign(hp[d].size(), 1.0);
      wts[d] = ones[d].data();
      np[d] = (int)hp[d].size();
    }
    prepare_grid(ctx, geo, pts, wts, np, target);
  }

  void prepare_grid(iga_ctx* ctx, const iga_geometry* geo, const double* const dpts[3],
                    const double* const hwts[3], const int npts_d[3], const iga_target* target) {
    IGA_REQUIRE(geo != nullptr, "null geometry");
    IGA_REQUIRE(geo->kind == IGA_GEO_NURBS || geo->kind == IGA_GEO_NURBS_TWIST,
                "unknown geometry kind");
    IGA_REQUIRE(geo->ctrl_hw != nullptr, "null control net");
    size_t nctrl = 1;
    for (int d = 0; d < 3; ++d) {
      check_knots(geo->knots[d], geo->nknots[d], geo->degree[d], "geometry");
      IGA_REQUIRE(geo->nctrl[d] == geo->nknots[d] - geo->degree[d] - 1,
                  "geometry: nctrl must equal nknots - degree - 1");
      nctrl *= geo->nctrl[d];
      const int npts = npts_d[d];
      std::vector<double> k(geo->knots[d], geo->knots[d] + geo->nknots[d]);
      gV[d].alloc((size_t)npts * (geo->degree[d] + 1));
      gD[d].alloc((size_t)npts * (geo->degree[d] + 1));
      gspan[d].alloc(npts);
      gw[d].alloc(npts);
      IGA_CUDA(cudaMemcpyAsync(gw[d].p, hwts[d], npts * 8, cudaMemcpyHostToDevice, ctx->stream));
      basis_tables(ctx, k, geo->degree[d], dpts[d], npts, gspan[d].p, gV[d].p, gD[d].p);
      G.V[d] = gV[d].p;
      G.D[d] = gD[d].p;
      G.span[d] = gspan[d].p;
      G.g[d] = gw[d].p;
      G.pg[d] = geo->degree[d];
      G.nc[d] = geo->nctrl[d];
      G.Q[d] = npts;
    }
    ctrl.alloc(nctrl * 4);
    IGA_CUDA(cudaMemcpyAsync(ctrl.p, geo->ctrl_hw, nctrl * 4 * 8, cudaMemcpyHostToDevice,
                             ctx->stream));
    G.ctrl = ctrl.p;
    G.kind = geo->kind;
    G.twist = geo->twist;
    G.tkind = target ? target->kind : IGA_TARGET_ZERO;
    IGA_REQUIRE(G.tkind >= 0 && G.tkind <= 2, "unknown target kind");
    for (int i = 0; i < 4; ++i) G.tp[i] = target ? target->params[i] : 0.0;
    if (G.tkind == IGA_TARGET_GAUSS) IGA_REQUIRE(G.tp[3] > 0.0, "target width must be > 0");
    int threads = 256;
    size_t n3 = (size_t)G.nc[0] * G.nc[1] * G.Q[2];
    size_t n2 = (size_t)G.nc[0] * G.Q[1] * G.Q[2];
    DevBuf<double> H3(n3 * 8);
    H2.alloc(n2 * 12);
    G.H2 = H2.p;
    IGA_LAUNCH(ctx, geo_stage3_kernel, (unsigned)((n3 + threads - 1) / threads), threads, 0, G,
               H3.p);
    IGA_LAUNCH(ctx, geo_stage2_kernel, (unsigned)((n2 + threads - 1) / threads), threads, 0, G,
               H3.p, H2.p);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));    // H3 is released on return
    total = (size_t)G.Q[0] * G.Q[1] * G.Q[2];
  }

  // comp = -1: all eight tensors into out (8 x total); comp >= 0: tensor comp
  void run(iga_ctx* ctx, double* out, int comp, double* qn2) {
    G.comp = comp;
    G.qn2 = qn2;
    IGA_CUDA(cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->stream));
    int threads = 256;
    // algorithmic per point: 16 (p1 + 1) FMA for the map and its derivatives,
    // about 128 flop for the quotient rule (30), det (14), the symmetric
    // metric (30), the adjugate with the Gauss weight (26), the target (about
    // 24 with exp) and the products; one (comp >= 0) or eight FP64 outputs
    prof_count(ctx, (double)total * 8.0 * (comp < 0 ? 8 : 1),
               (double)total * (32.0 * (G.pg[0] + 1) + 128.0));
    IGA_LAUNCH(ctx, sample_weights_kernel, (unsigned)((total + threads - 1) / threads), threads, 0,
               G, out, ctx->dflag);
    IGA_CUDA(cudaMemcpyAsync(ctx->hflag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                             ctx->stream));
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    // omega = |det J| admits a map of either orientation, but not a vanishing
    // determinant or one that changes sign (a map that folds over itself)
    IGA_REQUIRE((*ctx->hflag & 4) == 0, "geometry: zero or non-finite Jacobian determinant");
    IGA_REQUIRE((*ctx->hflag & 3) != 3,
                "geometry: the Jacobian determinant changes sign (the map folds over itself)");
  }
};

void sample_weights_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                         const iga_target* target, double* out) {
  IGA_REQUIRE(out != nullptr, "null output");
  GeoSampler S;
  S.prepare(ctx, geo, st, target);
  S.run(ctx, out, -1, nullptr);
}

// The eight weights on the tensor grid of the 1-D point sets hp (no
// quadrature weights): out holds 8 consecutive tensors (n1, n2, n3).
void sample_weights_points(iga_ctx* ctx, const iga_geometry* geo, const std::vector<double> hp[3],
                           const iga_target* target, double* out) {
  IGA_REQUIRE(out != nullptr, "null output");
  GeoSampler S;
  S.prepare_points(ctx, geo, hp, target);
  S.run(ctx, out, -1, nullptr);
}

// The weights one tensor at a time (for grids whose eight sample tensors do not
// fit next to each other): calls back with each tensor in `buf`.
void sample_weights_each(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                         const iga_target* target, double* buf, double* qnorm2,
                         void (*cb)(void*, int, const double*), void* user) {
  GeoSampler S;
  S.prepare(ctx, geo, st, target);
  IGA_CUDA(cudaMemsetAsync(qnorm2, 0, sizeof(double), ctx->stream));
  int last = (target && target->kind != IGA_TARGET_ZERO) ? 7 : 6;
  for (int c = 0; c <= last; ++c) {
    S.run(ctx, buf, c, c == 0 ? qnorm2 : nullptr);
    cb(user, c, buf);
  }
}

}  // namespace iga
