// Internal declarations shared by the libiga translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/iga.h"

namespace iga {

// Error carried from the internals to the C ABI boundary (never crosses it).
struct Error : public std::runtime_error {
  iga_status status;
  Error(iga_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define IGA_REQUIRE(cond, msg)                                                   \
  do {                                                                           \
    if (!(cond)) throw ::iga::Error(IGA_EINVAL, std::string(msg));               \
  } while (0)

#define IGA_CUDA(call)                                                           \
  do {                                                                           \
    cudaError_t e__ = (call);                                                    \
    if (e__ != cudaSuccess) {                                                    \
      if (e__ == cudaErrorMemoryAllocation)                                      \
        throw ::iga::Error(IGA_ENOMEM, std::string(#call) + ": " +               \
                                           cudaGetErrorString(e__));             \
      throw ::iga::Error(IGA_ECUDA, std::string(#call) + ": " +                  \
                                        cudaGetErrorString(e__));                \
    }                                                                            \
  } while (0)

// Launch on the context stream, count it, and surface launch errors.  When
// the context profiles a kernel whose name contains ctx->prof_name, the launch
// is bracketed by CUDA events on the same stream.
#define IGA_LAUNCH(ctx, kernel, grid, block, smem, ...)                          \
  do {                                                                           \
    bool prof__ = ::iga::prof_match((ctx), #kernel);                             \
    if (prof__) ::iga::prof_start(ctx);                                          \
    kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);             \
    if (prof__) ::iga::prof_stop(ctx);                                           \
    (ctx)->launches++;                                                           \
    (ctx)->next_bytes = 0.0;                                                     \
    (ctx)->next_flops = 0.0;                                                     \
    IGA_CUDA(cudaGetLastError());                                                \
  } while (0)

// Device memory of the library.  While a C-ABI entry runs (an AllocScope on
// its context stream is active on the calling thread), buffers come from a
// per-device stream-ordered pool: allocation and release are queued on that
// stream, so freeing a temporary does not wait for the device to drain (a
// plain cudaFree synchronises the whole device).  Every use of such a buffer
// is on the same stream, and an entry that returns a handle synchronises its
// stream first.  Outside an entry (a handle destroyed by the caller) a pooled
// buffer is freed after a device synchronisation.
struct AllocScope {
  explicit AllocScope(cudaStream_t s);
  ~AllocScope();
  AllocScope(const AllocScope&) = delete;
  AllocScope& operator=(const AllocScope&) = delete;
  cudaStream_t prev_stream;
  bool prev_active;
};
void* dev_alloc(size_t bytes, bool* pooled);
void dev_free(void* p, bool pooled) noexcept;

// Device buffer owned by RAII (library-internal allocations only).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  bool pooled = false;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), pooled(o.pooled) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; pooled = o.pooled;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    p = static_cast<T*>(dev_alloc(count * sizeof(T), &pooled));
    n = count;
  }
  void ensure(size_t count) { if (count > n) alloc(count); }
  void release() noexcept {
    if (p) dev_free(p, pooled);
    p = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
};

// Per-direction quadrature and basis tables of a tensor B-spline space.
struct DirTables {
  int p = 0, n = 0, E = 0, q = 0;
  std::vector<double> knots;          // host copy
  std::vector<double> xq, gq;         // host: Gauss points / weights, E*q
  std::vector<int> first;             // host: first nonzero basis index per element
  std::vector<int> elo, ehi;          // host: element range of each basis function
  DevBuf<double> dx;                  // device E*q points
  DevBuf<double> dV, dD;              // device (E, q, p+1) values / derivatives
  DevBuf<int> dfirst, delo, dehi;     // device copies
};

struct SpaceTables {
  DirTables dir[3];
  int nquad = 0;
};

// Device-resident Kronecker / TT-matrix operator (Dirichlet-reduced).
// Operators of the library are 3-D; the parabolic solve builds 4-D
// space-time operators internally (direction 0 = time), which never cross
// the C ABI.
struct OpBlock {
  int R1 = 1, R2 = 1;
  size_t off[4] = {0, 0, 0, 0};       // offsets (in bands) into the per-direction arrays
  int deriv[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
};

}  // namespace iga

struct iga_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 1;                              // SMs of the device
  std::string err;
  uint64_t launches = 0;
  std::vector<iga::DevBuf<char>> scratch;   // reusable scratch slots
  int* dflag = nullptr;                     // device status flags (zeroed per use)
  int* hflag = nullptr;                     // pinned host mirror
  // kernel timing (instrumentation): events around launches of one kernel
  std::string prof_name;
  std::vector<cudaEvent_t> prof_ev;         // pairs (start, stop)
  size_t prof_used = 0;
  double prof_bytes = 0.0, prof_flops = 0.0;
  double next_bytes = 0.0, next_flops = 0.0;   // algorithmic counts of the next launch
  size_t scratch_bytes() const {
    size_t s = 0;
    for (auto& b : scratch) s += b.n;
    return s;
  }
};

struct iga_op {
  int dims = 3;                       // 3; 4 for the internal space-time operators
  int n[4] = {0, 0, 0, 0};            // interior sizes
  int p[4] = {0, 0, 0, 0};
  std::vector<iga::OpBlock> blocks;
  size_t nbands[4] = {0, 0, 0, 0};
  iga::DevBuf<double> band64[4];      // (nbands[d], n[d], 2p+1)
  iga::DevBuf<float> band32[4];
  bool rank1 = true;
  size_t bytes() const {
    size_t s = 0;
    for (int d = 0; d < dims; ++d) s += band64[d].n * 8 + band32[d].n * 4;
    return s;
  }
};

struct iga_tt {
  int n[3] = {0, 0, 0};
  int r[2] = {1, 1};
  iga::DevBuf<double> core[3];        // (r_{d-1}, n_d, r_d), C order
};

namespace iga {

inline bool prof_match(const iga_ctx* ctx, const char* name) {
  return !ctx->prof_name.empty() && std::string(name).find(ctx->prof_name) != std::string::npos;
}
void prof_start(iga_ctx* ctx);
void prof_stop(iga_ctx* ctx);
// algorithmic bytes / flops of the next launch (used only while profiling)
inline void prof_count(iga_ctx* ctx, double bytes, double flops) {
  ctx->next_bytes = bytes;
  ctx->next_flops = flops;
}

// scratch slot helper: returns a device pointer with at least `bytes` bytes
template <typename T>
T* scratch(iga_ctx* ctx, int slot, size_t count) {
  if ((int)ctx->scratch.size() <= slot) ctx->scratch.resize(slot + 1);
  auto& b = ctx->scratch[slot];
  size_t bytes = count * sizeof(T);
  if (bytes > b.n) {
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    b.alloc(bytes + (bytes >> 3) + 256);
  }
  return reinterpret_cast<T*>(b.p);
}

// scratch slot numbers (kept apart so nested helpers do not collide)
enum {
  SLOT_TTSVD_OMEGA = 0, SLOT_TTSVD_Y, SLOT_TTSVD_Q, SLOT_TTSVD_BT, SLOT_TTSVD_G, SLOT_TTSVD_V,
  SLOT_TTSVD_W, SLOT_TTSVD_C, SLOT_TTSVD_NORM, SLOT_QRCP_WORK, SLOT_ASM_W, SLOT_ASM_SAMPLES, SLOT_KRON_Z,
  SLOT_KRON_Z2, SLOT_LOCAL_T1, SLOT_LOCAL_T2, SLOT_KKT_TMP, SLOT_MISC0, SLOT_MISC1,
  SLOT_TTM_W, SLOT_QNORM, SLOT_TTSVD_Y2, SLOT_TTSVD_PART, SLOT_GEMM_PART, SLOT_GEMM_DOT,
  SLOT_PARA_ZT, SLOT_PARA_S, SLOT_PARA_MV,
  SLOT_AMEN_BASE = 32
};

// geometry.cu
void build_space_tables(iga_ctx* ctx, const iga_space* sp, SpaceTables& t);
void check_knots(const double* k, int nk, int p, const char* what);

void sample_weights_points(iga_ctx* ctx, const iga_geometry* geo, const std::vector<double> hp[3],
                           const iga_target* target, double* out);
void sample_weights_each(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                         const iga_target* target, double* buf, double* qnorm2,
                         void (*cb)(void*, int, const double*), void* user);

// assembly.cu
void launch_assemble_bands(iga_ctx* ctx, const DirTables& t, const double* w, int T, int drow,
                           int dcol, int interior, double* band);
void launch_load_vectors(iga_ctx* ctx, const DirTables& t, const double* w, int T, int interior,
                         double* out);

// linalg.cu
void tt_svd3(iga_ctx* ctx, const double* W, int n1, int n2, int n3, double tol, double norm_ref,
             int rmax, iga_tt** out, double norm_w = -1.0);   // norm_w >= 0: ||W||_F known
double device_norm2(iga_ctx* ctx, const double* x, size_t n);   // synchronises
// Frobenius norms of `count` consecutive tensors of n elements (host array)
void device_norms(iga_ctx* ctx, const double* x, size_t n, int count, double* norms);
void jacobi_eig(iga_ctx* ctx, double* A, double* V, double* w, int k);  // device, col-major
// fp32: run the rotations in FP32 (shared memory; falls back to FP64 when the
// problem does not fit), for eigenbases that only feed a preconditioner
void jacobi_eig_batched(iga_ctx* ctx, double* const* A, double* const* V, double* const* w,
                        const int* k, int count, bool fp32 = false);
void gen_eig_prep(iga_ctx* ctx, const double* PM, int SM, const double* PK, int SK, int k,
                  double* work, double* C, double* Linv);
void householder_qr(iga_ctx* ctx, double* Y, double* Q, int m, int k);  // Y overwritten
// truncated QR with column pivoting of B (m x c3, B(i, a) = B[i si + a sa],
// field groups of r columns normalised, the first one weighted by w0), then
// kick extra columns E (m x kick
// col-major) orthogonalised; Q (m x min(rk + kick, m), col-major) and *rk_dev
// (device) receive the basis and the number of pivoted columns
void qrcp_truncate(iga_ctx* ctx, const double* B, int m, int c3, int si, int sa, int r,
                   const double* E, int kick, double rel, int jmax, double* Q, int* rk_dev,
                   double w0 = 1.0);
void fill_gaussian(iga_ctx* ctx, double* x, size_t n, uint64_t seed);
void transpose_cm(iga_ctx* ctx, const double* A, int rows, int cols, double* B);

// local.cu
void tt_full_impl(iga_ctx* ctx, const iga_tt* tt, double* out);
void gemm_rm(iga_ctx* ctx, int M, int N, int K, const double* A, const double* B, double* C,
             double beta = 0.0);
template <typename T>
void local_matvec_t(iga_ctx* ctx, int r0, int n, int r1, int R0, int R1, int p, const T* PhiL,
                    const T* bands, const T* PhiR, const unsigned char* dmask, int nv, const T* x,
                    T* y, T* t1, T* t2);

// api.cu
void weight_tts_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                     const iga_target* target, double tol, iga_tt* tts[8]);
// interp.cu: the eight weight TTs at the Gauss points from the interpolant
// of degree pt (Sec. 3, weightEquationSystem / weightEquationSolve)
void weight_tts_interp_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                            const iga_target* target, double tol, int pt, iga_tt* tts[8]);
void ops_from_weights_impl(iga_ctx* ctx, const SpaceTables& st, const iga_tt* const w[7],
                           iga_op** M, iga_op** K);
void kkt_apply_internal(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta, const void* z,
                        void* out, iga_prec prec);

// kron.cu
// the KKT operator on (y, u, lambda) in one fused launch when M and K are
// rank-1 Kronecker sums (false: not applicable, nothing launched)
bool kkt_apply_fused(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta, const void* z,
                     void* out, iga_prec prec);
void kron_apply_impl(iga_ctx* ctx, const iga_op* A, double alpha, const void* x, double beta,
                     void* y, iga_prec prec);
// the parabolic KKT rows of one time step in one FP64 launch when M and K
// are rank-1 Kronecker sums: out_y -= M a + tau K lam_k, out_u -= M d,
// out_lam -= tau K y_k + M f for in = {a, d, f, y_k, lam_k} (false: not
// applicable, nothing launched)
bool parabolic_rows_fused(iga_ctx* ctx, const iga_op* M, const iga_op* K, double tau,
                          const double* const in[5], double* const out[3]);
// the same with A^T (every band transposed)
void kron_apply_transposed(iga_ctx* ctx, const iga_op* A, double alpha, const void* x, double beta,
                           void* y, iga_prec prec);

// ttm_tc.cu: one TT-matrix block y += alpha (A1 (x) A2 (x) A3) x in FP32
// storage with the rank contraction on the tensor cores (TF32 or BF16
// operands, FP32 accumulation); false when the shape has no tile plan
// (nothing launched).
// A bounded wait that gives up sets ctx->dflag[1] to IGA_ETIMEOUT.
bool ttm_tc_block(iga_ctx* ctx, const float* A1, const float* A2, const float* A3, int R1, int R2,
                  const int* n, int P, float alpha, const float* x, float* y, bool bf16);
bool ttm_tc_supported(int n1, int n3, int R1, int R2, int P, int nsm);
// zero / check the tensor-core timeout flag around a TF32 entry (the check
// synchronises the context stream)
void tc_flag_reset(iga_ctx* ctx);
void tc_flag_check(iga_ctx* ctx, const char* what);

void set_error(iga_ctx* ctx, const std::string& m);

// parabolic.cu: the space-time operators of N_t implicit Euler steps,
// A_M = tau I (x) M and KK = I (x) tau K + C (x) M, as internal 4-D operators
// (direction 0 = time), and the FP64 residual res = F - A z of the parabolic
// KKT system for z, F, res laid out (3, nt, N); returns ||res||_2
// (synchronises)
void space_time_ops(iga_ctx* ctx, const iga_op* M, const iga_op* K, int nt, double tau,
                    std::unique_ptr<iga_op>& AM, std::unique_ptr<iga_op>& AK);
double parabolic_residual(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta, int nt,
                          double tau, const double* F, const double* z, double* res, size_t N);

// gemm.cu: row-major strided batch C_i = alpha op(A_i) op(B_i) + beta C_i
// (op(A) is M x K: A[m lda + k], or A[k lda + m] when tA), the local GMRES's
// vector kernels and a deterministic FP64 dot product (synchronises)
template <typename T>
void gemm_rm_batched(iga_ctx* ctx, bool tA, bool tB, int M, int N, int K, T alpha, const T* A,
                     int lda, long long sA, const T* B, int ldb, long long sB, T beta, T* C,
                     int ldc, long long sC, int count);
template <typename T>
void gemv_cm_add(iga_ctx* ctx, int rows, int cols, const T* A, const T* x, T* y);
template <typename T>
void vec_sub(iga_ctx* ctx, size_t n, const T* a, const T* b, T* out);
double device_dot(iga_ctx* ctx, const double* a, const double* b, size_t n);
// tc_gemm.cu: the same product in FP32 storage on the tensor cores (TF32
// operands, FP32 accumulation); tC stores C transposed (C[n ldc + m])
void tc_gemm_tf32(iga_ctx* ctx, bool tA, bool tB, bool tC, int M, int N, int K, float alpha,
                  const float* A, int lda, long long sA, const float* B, int ldb, long long sB,
                  float beta, float* C, int ldc, long long sC, int count);

// cudaFuncSetAttribute(fn, attr, value) per (function, attribute, device),
// raising the value monotonically (a smaller later request keeps the larger
// value already set): a function attribute belongs to the device that was
// current when it was set, so a second device needs its own call.  Thread
// safe.
void func_attr(const void* fn, cudaFuncAttribute attr, int value);
template <typename F>
inline void func_attr(F* fn, cudaFuncAttribute attr, int value) {
  func_attr(reinterpret_cast<const void*>(fn), attr, value);
}

}  // namespace iga
