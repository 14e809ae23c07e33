// Rows of the KKT residual for a solution held as TTs (Sec. 4, eq.
// KKTSystem with one time step): for every listed interior index i the three
// equations' residuals
//   r_1(i) = b_i - (M y)_i - (K lambda)_i
//   r_2(i) = -(beta (M u)_i - (M lambda)_i)
//   r_3(i) = -((K y)_i - (M u)_i)
// with M and K the assembled TT-matrix operators and b the load TT.  Every
// entry A_ij of an operator is formed from its univariate bands
// (sum over blocks and TT-matrix ranks of A1(i1,j1) A2(i2,j2) A3(i3,j3)) and
// every solution value z_j from the TT cores, over the (2p+1)^3 stencil of
// row i; nothing of full size is formed.  Uniformly sampled rows give an
// unbiased estimate of the squared residual norm, (N / S) sum of the squares
// over S rows, at any grid size.
#include <vector>

#include "iga_internal.cuh"

namespace iga {

namespace {

struct RowOp {
  const double* band[3];   // (nbands, n, 2p+1) per direction
  const int* R1;           // block ranks
  const int* R2;
  const long long* off;    // (nblocks, 3) band offsets
  int nblocks;
};

struct RowTT {
  const double* core[3];
  int r1, r2;
};

struct RowArgs {
  RowOp op[2];             // M, K
  RowTT f[3];              // y, u, lambda
  RowTT load;
  int has_load;
  int n[3], p[3];
  double beta;
  const int* rows;         // (S, 3)
  int S;
  double* out;             // (S, 3)
};

__device__ double tt_value(const RowTT& t, const int n[3], int j1, int j2, int j3) {
  double s = 0.0;
  for (int a = 0; a < t.r1; ++a) {
    const double x1 = t.core[0][(size_t)j1 * t.r1 + a];
    if (x1 == 0.0) continue;
    double u = 0.0;
    const double* x2 = t.core[1] + ((size_t)a * n[1] + j2) * t.r2;
    for (int b = 0; b < t.r2; ++b) u = fma(x2[b], t.core[2][(size_t)b * n[2] + j3], u);
    s = fma(x1, u, s);
  }
  return s;
}

// entry (i, j) of an operator, j = i + o - p per direction
__device__ double op_entry(const RowOp& A, const int n[3], const int p[3], const int i[3],
                           const int o[3]) {
  double s = 0.0;
  for (int k = 0; k < A.nblocks; ++k) {
    const int R1 = A.R1[k], R2 = A.R2[k];
    const long long* off = A.off + 3 * k;
    for (int al = 0; al < R1; ++al) {
      const double a1 =
          A.band[0][((size_t)(off[0] + al) * n[0] + i[0]) * (2 * p[0] + 1) + o[0]];
      if (a1 == 0.0) continue;
      double t = 0.0;
      for (int be = 0; be < R2; ++be) {
        const double a2 = A.band[1][((size_t)(off[1] + (long long)al * R2 + be) * n[1] + i[1]) *
                                        (2 * p[1] + 1) + o[1]];
        const double a3 =
            A.band[2][((size_t)(off[2] + be) * n[2] + i[2]) * (2 * p[2] + 1) + o[2]];
        t = fma(a2, a3, t);
      }
      s = fma(a1, t, s);
    }
  }
  return s;
}

__global__ void __launch_bounds__(128) kkt_rows_kernel(RowArgs A) {
  const int s = blockIdx.x;
  int i[3];
  for (int d = 0; d < 3; ++d) i[d] = A.rows[3 * s + d];
  const int w0 = 2 * A.p[0] + 1, w1 = 2 * A.p[1] + 1, w2 = 2 * A.p[2] + 1;
  const int T = w0 * w1 * w2;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // M y, M u, M lam, K y, K lam
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    int o[3] = {t / (w1 * w2), (t / w2) % w1, t % w2};
    int j[3];
    bool in = true;
    for (int d = 0; d < 3; ++d) {
      j[d] = i[d] + o[d] - A.p[d];
      in = in && j[d] >= 0 && j[d] < A.n[d];
    }
    if (!in) continue;
    const double m = op_entry(A.op[0], A.n, A.p, i, o);
    const double k = op_entry(A.op[1], A.n, A.p, i, o);
    const double zy = tt_value(A.f[0], A.n, j[0], j[1], j[2]);
    const double zu = tt_value(A.f[1], A.n, j[0], j[1], j[2]);
    const double zl = tt_value(A.f[2], A.n, j[0], j[1], j[2]);
    acc[0] = fma(m, zy, acc[0]);
    acc[1] = fma(m, zu, acc[1]);
    acc[2] = fma(m, zl, acc[2]);
    acc[3] = fma(k, zy, acc[3]);
    acc[4] = fma(k, zl, acc[4]);
  }
  __shared__ double red[5][4];
  for (int c = 0; c < 5; ++c) {
    double v = acc[c];
    for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v[5];
    for (int c = 0; c < 5; ++c) v[c] = red[c][0] + red[c][1] + red[c][2] + red[c][3];
    const double b = A.has_load ? tt_value(A.load, A.n, i[0], i[1], i[2]) : 0.0;
    A.out[3 * s + 0] = b - v[0] - v[4];
    A.out[3 * s + 1] = -(A.beta * v[1] - v[2]);
    A.out[3 * s + 2] = -(v[3] - v[1]);
  }
}

struct OpMeta {
  DevBuf<int> R1, R2;
  DevBuf<long long> off;
};

void fill_op(iga_ctx* ctx, const iga_op* op, RowOp& r, OpMeta& m) {
  const int nb = (int)op->blocks.size();
  std::vector<int> R1(nb), R2(nb);
  std::vector<long long> off(3 * nb);
  for (int k = 0; k < nb; ++k) {
    R1[k] = op->blocks[k].R1;
    R2[k] = op->blocks[k].R2;
    for (int d = 0; d < 3; ++d) off[3 * k + d] = (long long)op->blocks[k].off[d];
  }
  m.R1.alloc(nb);
  m.R2.alloc(nb);
  m.off.alloc(3 * nb);
  IGA_CUDA(cudaMemcpyAsync(m.R1.p, R1.data(), nb * sizeof(int), cudaMemcpyHostToDevice,
                           ctx->stream));
  IGA_CUDA(cudaMemcpyAsync(m.R2.p, R2.data(), nb * sizeof(int), cudaMemcpyHostToDevice,
                           ctx->stream));
  IGA_CUDA(cudaMemcpyAsync(m.off.p, off.data(), 3 * nb * sizeof(long long),
                           cudaMemcpyHostToDevice, ctx->stream));
  for (int d = 0; d < 3; ++d) r.band[d] = op->band64[d].p;
  r.R1 = m.R1.p;
  r.R2 = m.R2.p;
  r.off = m.off.p;
  r.nblocks = nb;
}

RowTT tt_args(const iga_tt* t, const iga_op* M, const char* what) {
  IGA_REQUIRE(t != nullptr, std::string("kkt_residual_rows: null ") + what);
  for (int d = 0; d < 3; ++d)
    IGA_REQUIRE(t->n[d] == M->n[d], std::string("kkt_residual_rows: size of ") + what);
  RowTT r;
  for (int d = 0; d < 3; ++d) r.core[d] = t->core[d].p;
  r.r1 = t->r[0];
  r.r2 = t->r[1];
  return r;
}

}  // namespace

}  // namespace iga

using namespace iga;

extern "C" iga_status iga_kkt_residual_rows(iga_ctx* ctx, const iga_op* M, const iga_op* K,
                                            double beta, const iga_tt* load, const iga_tt* y,
                                            const iga_tt* u, const iga_tt* lam, int nrows,
                                            const int* rows, double* res) {
  if (!ctx) return IGA_EINVAL;
  try {
    IGA_REQUIRE(M && K, "kkt_residual_rows: null operator");
    IGA_REQUIRE(nrows >= 0, "kkt_residual_rows: negative row count");
    if (nrows == 0) return IGA_OK;
    IGA_REQUIRE(rows && res, "kkt_residual_rows: null rows or result");
    for (int d = 0; d < 3; ++d) {
      IGA_REQUIRE(M->n[d] == K->n[d] && M->p[d] == K->p[d], "kkt_residual_rows: M, K mismatch");
      IGA_REQUIRE(M->p[d] <= 4, "kkt_residual_rows: degree above 4");
    }
    for (int s = 0; s < nrows; ++s)
      for (int d = 0; d < 3; ++d)
        IGA_REQUIRE(rows[3 * s + d] >= 0 && rows[3 * s + d] < M->n[d],
                    "kkt_residual_rows: row index outside the interior grid");
    AllocScope scope(ctx->stream);
    RowArgs a{};
    OpMeta meta[2];
    fill_op(ctx, M, a.op[0], meta[0]);
    fill_op(ctx, K, a.op[1], meta[1]);
    a.f[0] = tt_args(y, M, "y");
    a.f[1] = tt_args(u, M, "u");
    a.f[2] = tt_args(lam, M, "lambda");
    a.has_load = load != nullptr;
    if (load) a.load = tt_args(load, M, "load");
    for (int d = 0; d < 3; ++d) {
      a.n[d] = M->n[d];
      a.p[d] = M->p[d];
    }
    a.beta = beta;
    DevBuf<int> drows(3 * (size_t)nrows);
    DevBuf<double> dout(3 * (size_t)nrows);
    IGA_CUDA(cudaMemcpyAsync(drows.p, rows, 3 * (size_t)nrows * sizeof(int),
                             cudaMemcpyHostToDevice, ctx->stream));
    a.rows = drows.p;
    a.S = nrows;
    a.out = dout.p;
    IGA_LAUNCH(ctx, kkt_rows_kernel, nrows, 128, 0, a);
    IGA_CUDA(cudaMemcpyAsync(res, dout.p, 3 * (size_t)nrows * sizeof(double),
                             cudaMemcpyDeviceToHost, ctx->stream));
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    return IGA_OK;
  } catch (const Error& e) {
    set_error(ctx, e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_error(ctx, e.what());
    return IGA_ECUDA;
  }
}
