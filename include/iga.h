/*
 * libiga -- low-rank isogeometric assembly, Kronecker/TT operator apply and
 * block-AMEn KKT solve on one GB300 (sm_103a).
 *
 * Method: Buenger, Dolgov, Stoll, "A low-rank tensor method for
 * PDE-constrained optimization with isogeometric analysis".
 *
 * Conventions shared by every entry point
 *   - All calls are asynchronous on the stream given to iga_create() unless
 *     stated otherwise; calls that return host values synchronise that stream.
 *   - "device" pointers are CUDA global-memory addresses owned by the caller
 *     and only borrowed for the duration of the call; "host" pointers are
 *     plain host memory, also borrowed.
 *   - Handles (iga_ctx, iga_op, iga_tt) are owned by the library and freed
 *     by the matching destroy call.
 *   - Errors are returned as iga_status; iga_last_error() gives a text.
 *     No call aborts the process or traps on the GPU.
 *   - Tensors over the tensor-product index (i1, i2, i3) are stored in C
 *     order (i3 fastest).  Operators act on the Dirichlet-reduced space:
 *     the first and last basis function of every direction are omitted
 *     (Sec. 4, discrete quadratic problem).
 *   - Banded univariate matrices are stored row-major as band[i][o] with
 *     A(i, i + o - p), o = 0..2p, entries outside the matrix are zero.
 *   - Device memory the library needs during a call comes from a per-device
 *     stream-ordered pool on the context stream, which keeps up to 4 GB of
 *     released memory cached for later calls (so free memory reported by
 *     the driver can stay lower after a call).  Calls that return handles
 *     synchronise their stream first, so a handle is usable on any stream;
 *     destroying a handle synchronises the device.
 */
#ifndef IGA_H
#define IGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IGA_OK = 0,
  IGA_EINVAL = 1,      /* invalid argument (sizes, knots, null pointers) */
  IGA_ENOMEM = 2,      /* device or host allocation failed */
  IGA_ECUDA = 3,       /* CUDA runtime error */
  IGA_ENOCONV = 4,     /* iteration limit reached before the tolerance */
  IGA_ENONFINITE = 5,  /* NaN or Inf detected in a reduction */
  IGA_ETIMEOUT = 6     /* a bounded device wait gave up */
} iga_status;

/* Arithmetic of an operator apply or a solve.  IGA_FP64 and IGA_FP32: CUDA
 * cores in that precision on double / float vectors.  IGA_TF32 and IGA_BF16:
 * float vectors; the dense rank contraction of TT-matrix blocks runs on the
 * tensor cores with TF32 or BF16 operands and FP32 accumulation (rank-1
 * blocks, which have no dense contraction, run in FP32). */
typedef enum { IGA_FP64 = 0, IGA_FP32 = 1, IGA_TF32 = 2, IGA_BF16 = 3 } iga_prec;

enum { IGA_GEO_NURBS = 0, IGA_GEO_NURBS_TWIST = 1 };
enum { IGA_TARGET_ZERO = 0, IGA_TARGET_SINPROD = 1, IGA_TARGET_GAUSS = 2 };

typedef struct iga_ctx iga_ctx;
typedef struct iga_op iga_op;
typedef struct iga_tt iga_tt;

/* Geometry map G = C : B(xhat) (Sec. 2, eq. geometryMapping), rational when
 * the weights differ (NURBS curve definition of Sec. 2).  kind
 * IGA_GEO_NURBS_TWIST composes G with a rotation by twist * z about e_z. */
typedef struct {
  int kind;
  int degree[3];
  int nknots[3];
  const double* knots[3];   /* host; open knot vectors (eq. knotVector) */
  int nctrl[3];             /* nctrl[d] = nknots[d] - degree[d] - 1 */
  const double* ctrl_hw;    /* host; [i1][i2][i3][4] = (w x, w y, w z, w) */
  double twist;             /* radians per unit z */
} iga_geometry;

/* Trial/test B-spline space (Sec. 2, tensor-product spline space) and the
 * Gauss rule used for every integral: nquad points per element and
 * direction. */
typedef struct {
  int degree[3];
  int nknots[3];
  const double* knots[3];   /* host; open knot vectors */
  int nquad;                /* 1..16 */
} iga_space;

/* Desired state yhat of the control problem (Sec. 1 / Sec. 4):
 * SINPROD: prod_k sin(pi x_k);  GAUSS: exp(-|x - c|^2 / params[3]),
 * c = params[0..2]. */
typedef struct {
  int kind;
  double params[4];
} iga_target;

/* ---- context --------------------------------------------------------- */

/* Create a context bound to the CUDA stream `stream` (a cudaStream_t, may
 * be NULL for the legacy default stream) on the current device. */
iga_status iga_create(iga_ctx** ctx, void* stream);
void iga_destroy(iga_ctx* ctx);
const char* iga_last_error(const iga_ctx* ctx);
/* Number of kernels this context has launched so far (all entry points). */
uint64_t iga_launch_count(const iga_ctx* ctx);
/* Device bytes currently held by the context's scratch pool. */
size_t iga_scratch_bytes(const iga_ctx* ctx);

/* Instrumentation (no counterpart in the paper): from iga_profile_begin until
 * iga_profile_end, every launch of a library kernel whose name contains
 * `kernel` is bracketed by CUDA events on the context stream.
 * iga_profile_end synchronises the stream and returns the number of such
 * launches, their summed device time in milliseconds and the summed
 * algorithmic bytes and flops the launch sites declared for them (0 where a
 * kernel declares none). */
iga_status iga_profile_begin(iga_ctx* ctx, const char* kernel);
iga_status iga_profile_end(iga_ctx* ctx, uint64_t* launches, double* ms, double* bytes,
                           double* flops);
/* Instrumentation (no counterpart in the paper): the FMA rate of the CUDA
 * cores in TFLOP/s (2 flop per FMA) for prec IGA_FP64 or IGA_FP32, measured
 * by a kernel of independent FMA chains over every SM, timed with CUDA
 * events on the context stream (best of three launches after one warm-up).
 * Synchronises. */
iga_status iga_measure_fma(iga_ctx* ctx, iga_prec prec, double* tflops);
/* Utility (no counterpart in the paper): the library's own dense product,
 * the one its contractions use, for count row-major matrices
 *   C_i = alpha op(A_i) op(B_i) + beta C_i,   i < count,
 * op(A_i) M x K, op(B_i) K x N, A_i = A + i sA (elements; likewise B, C),
 * op = transpose when tA / tB is nonzero (A_i then K x M with leading
 * dimension lda).  Device pointers in FP64 (prec IGA_FP64) or FP32
 * (IGA_FP32 on the CUDA cores; IGA_TF32 on the tcgen05 tensor cores with
 * TF32 operands and FP32 accumulation, which synchronises and returns
 * IGA_ETIMEOUT if a bounded wait of its pipeline gives up); the caller owns
 * them.  Deterministic: a reduction split over K is summed in a fixed order.
 * Queued on the context stream (no synchronisation) except for IGA_TF32.  IGA_EINVAL for a null pointer, a negative size or a
 * leading dimension shorter than a row. */
iga_status iga_gemm_batched(iga_ctx* ctx, iga_prec prec, int tA, int tB, int M, int N, int K,
                            double alpha, const void* A, int lda, long long sA, const void* B,
                            int ldb, long long sB, double beta, void* C, int ldc, long long sC,
                            int count);

/* ---- (a1, a2) geometry sampling ------------------------------------- */

/* Sample the geometry weights on the tensor Gauss grid of `space`
 * (Sec. 2: omega = |det grad G|, Q = (J^T J)^{-1} omega, J = dG/dxhat;
 * Sec. 3 eq. weightEquationSystem samples omega on a point grid).
 * Every sample is multiplied by the tensor Gauss weight g1 g2 g3.
 * out: device, 8 consecutive tensors of shape (Q1, Q2, Q3), Q_d = E_d * nquad:
 *   [0] omega g, [1] q11 g, [2] q12 g, [3] q13 g, [4] q22 g, [5] q23 g,
 *   [6] q33 g, [7] yhat(G) omega g.
 * Fails with IGA_EINVAL on invalid knots, a Jacobian determinant that is
 * zero or not finite at a Gauss point, or one that changes sign between
 * Gauss points (a map folding over itself); a map of constant negative
 * orientation is accepted (omega = |det J|).  Detected on the device and
 * reported after the call (the call synchronises). */
iga_status iga_sample_weights(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                              const iga_target* target, double* out);

/* ---- (a3) TT-SVD ------------------------------------------------------ */

/* TT decomposition of a device tensor W of shape (n1, n2, n3) (Sec. 3,
 * eq. tt and the TT-SVD named after eq. weightEquationSolve): truncation of
 * each unfolding at tol * ref / sqrt(2), ref = norm_ref if > 0 else ||W||_F;
 * ranks are capped at rmax.  A tensor with ||W||_F <= tol * ref gives a
 * rank-0 TT (*out = NULL, IGA_OK).  FP64 throughout.  Synchronises. */
iga_status iga_tt_svd(iga_ctx* ctx, const double* W, int n1, int n2, int n3, double tol,
                      double norm_ref, int rmax, iga_tt** out);
/* n[3] and ranks r[2] of a TT; core d copied to host buffer `core`
 * (shape (r_{d-1}, n_d, r_d), C order).  Synchronises. */
iga_status iga_tt_info(const iga_tt* tt, int n[3], int r[2]);
iga_status iga_tt_core(iga_ctx* ctx, const iga_tt* tt, int d, double* core);
/* Expand to a full device tensor (n1, n2, n3), FP64. */
iga_status iga_tt_full(iga_ctx* ctx, const iga_tt* tt, double* out);
void iga_tt_destroy(iga_tt* tt);
/* Save a TT to a host file / load it back (no counterpart in the paper;
 * it stores the TT of eq. tt).  Format: the 8 bytes "IGATT" 1 0 0, int32
 * n1 n2 n3 r1 r2, then the three cores (r_{d-1}, n_d, r_d) in C order as
 * float64, little-endian.  iga_tt_load checks the magic, the sizes and the
 * file length (IGA_EINVAL on a mismatch or an unreadable file) and returns a
 * library-owned TT.  Both synchronise the context stream. */
iga_status iga_tt_save(iga_ctx* ctx, const iga_tt* tt, const char* path);
iga_status iga_tt_load(iga_ctx* ctx, const char* path, iga_tt** out);

/* ---- (a4) batched univariate assembly ------------------------------- */

/* Univariate weighted Gauss-quadrature matrices of one direction d
 * (Sec. 3, eqs. massMatrix1D and the stiffness factors K_kl^(d)):
 *   band[t][i][o] = sum_{e,q} w[t][e*nquad+q] phi_i(x_eq) psi_j(x_eq),
 *   j = i + o - p, phi = B or B' (deriv_row), psi = B or B' (deriv_col).
 * w: device (T, E*nquad); band: device (T, nrow, 2p+1) with nrow = n
 * (interior = 0) or n - 2 (interior = 1: Dirichlet rows and columns
 * omitted). */
iga_status iga_assemble_bands(iga_ctx* ctx, const iga_space* space, int d, const double* w,
                              int T, int deriv_row, int deriv_col, int interior, double* band);

/* ---- composite assembly (a1..a4) ------------------------------------ */

/* Low-rank assembly of the Dirichlet-reduced mass and stiffness operators
 * and of the load vector b_i = int yhat(G) beta_i omega (Sec. 3 eqs.
 * massFinal / stiffnessFinal with the TT cores of eq. TTranks as the
 * Kronecker terms).  Q entries are truncated relative to the norm of all of
 * Q.  Outputs are library-owned; *load is NULL for a zero target. */
iga_status iga_lowrank_assemble(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                                const iga_target* target, double tol, iga_op** M, iga_op** K,
                                iga_tt** load);

/* The same assembly with the paper's weight interpolation (Sec. 3, eqs.
 * weightEquationSystem and weightEquationSolve) in place of sampling on the
 * Gauss grid: each weight is interpolated in the tensor spline space of
 * degree `degree` (0: 2p + 1, p the largest degree of `space`) on the break
 * points of `space`, from its values at the Greville abscissae of that space
 * ((E + degree)^3 points instead of (E nquad)^3); the node values are
 * compressed by TT-SVD at tol, every core is mapped by the per-direction
 * collocation solve and the evaluation of the interpolant at the Gauss points
 * (times the Gauss weights), and the univariate assembly proceeds as above.
 * The operators then carry the interpolation error of the weights (of order
 * h^(degree+1) for a smooth map) besides the truncation. */
iga_status iga_lowrank_assemble_interp(iga_ctx* ctx, const iga_geometry* geo,
                                       const iga_space* space, const iga_target* target,
                                       double tol, int degree, iga_op** M, iga_op** K,
                                       iga_tt** load);
/* The eight weight TTs of that route at the Gauss points (the layout of
 * iga_weight_tts). */
iga_status iga_weight_tts_interp(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                                 const iga_target* target, double tol, int degree,
                                 iga_tt* out[8]);

/* The eight sampled weights of the composite assembly as TT tensors on the
 * Gauss grid (Sec. 3: omega g, q11 g, q12 g, q13 g, q22 g, q23 g, q33 g and
 * the load density yhat(G) omega g), truncated as in iga_lowrank_assemble.
 * out[c] is NULL for a rank-0 (zero) tensor.  Library-owned. */
iga_status iga_weight_tts(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                          const iga_target* target, double tol, iga_tt* out[8]);
/* TT from device cores (copied): core d has shape (r_{d-1}, n_d, r_d),
 * r_0 = r_3 = 1. */
iga_status iga_tt_from_cores(iga_ctx* ctx, const int n[3], const int r[2],
                             const double* const cores[3], iga_tt** out);
/* Dirichlet-reduced M and K from weight TTs on the Gauss grid of `space`
 * (weights[0] = omega g, weights[1..6] = q11, q12, q13, q22, q23, q33 times
 * g, NULL = zero weight): the univariate assembly step alone (Sec. 3, eqs.
 * massFinal and stiffnessFinal, with q_lk = q_kl). */
iga_status iga_ops_from_weights(iga_ctx* ctx, const iga_space* space,
                                const iga_tt* const weights[7], iga_op** M, iga_op** K);
/* Load vector TT from the TT of the load density (sampled yhat(G) omega g):
 * b_i = sum_{e,q} f(e, q) beta_i(x_eq) per direction, Dirichlet-reduced. */
iga_status iga_load_from_density(iga_ctx* ctx, const iga_space* space, const iga_tt* density,
                                 iga_tt** load);

/* A Kronecker / TT-matrix operator from its banded univariate factors
 * (Sec. 5, eqs. M_kron / K_kron):
 *   A = sum_k sum_{a,b} A1_k[a] (x) A2_k[a,b] (x) A3_k[b],
 * acting on C-ordered tensors of size n[0] x n[1] x n[2] with half-bandwidth
 * p[d] in direction d (the apply needs p[0] = p[1] = p[2] in 1..4).  Block k
 * has ranks (R[2k], R[2k+1]); bands[3k + d] is a device FP64 array of block
 * k, direction d: d=0 (R1, n1, 2p+1), d=1 (R1, R2, n2, 2p+1), d=2
 * (R2, n3, 2p+1), band[i][o] = A(i, i + o - p); entries outside the matrix
 * are ignored.  The bands are copied (an FP32 copy is made for the FP32 and
 * tensor-core applies); *out is library-owned.  Synchronises. */
iga_status iga_op_from_bands(iga_ctx* ctx, const int n[3], const int p[3], int nblocks,
                             const int* R, const double* const* bands, iga_op** out);

/* Operator structure: interior sizes n[3], degrees p[3], number of blocks
 * (one per TT weight term group), summed TT-matrix ranks R[2] and device
 * bytes of its factors. */
iga_status iga_op_info(const iga_op* op, int n[3], int p[3], int* nblocks, int R[2],
                       size_t* bytes);
/* Ranks (R1, R2) of block k. */
iga_status iga_op_block(const iga_op* op, int k, int R[2]);
/* Copy the bands of direction d of block k to host: d=0: (R1, n1, 2p+1),
 * d=1: (R1, R2, n2, 2p+1), d=2: (R2, n3, 2p+1).  Synchronises. */
iga_status iga_op_bands(iga_ctx* ctx, const iga_op* op, int k, int d, double* host);
void iga_op_destroy(iga_op* op);

/* ---- (a5) Kronecker-sum apply --------------------------------------- */

/* y = alpha * op(A) x + beta * y with A = sum_blocks sum_{r1,r2}
 * A1[r1] (x) A2[r1,r2] (x) A3[r2] (Sec. 5, eqs. M_kron / K_kron; kron
 * ordering kron(A1, kron(A2, A3)) on C-ordered x), op(A) = A (transpose = 0)
 * or A^T = sum A1^T (x) A2^T (x) A3^T (transpose != 0, the bands transposed
 * into a temporary on the context stream).  x, y: device, length n1 n2 n3,
 * double (IGA_FP64) or float (IGA_FP32, IGA_TF32, IGA_BF16); x and y must
 * not overlap (IGA_EINVAL).  Rank-1 blocks run as one fused launch of banded
 * mode products.  TT-matrix blocks (ranks above one): IGA_TF32 / IGA_BF16
 * run the rank contraction as tcgen05 tensor-core MMAs (TF32 or BF16
 * operands, FP32 accumulation) in one fused launch per block; IGA_FP64 /
 * IGA_FP32 use staged mode products and a batched GEMM per i2.  With
 * IGA_TF32 / IGA_BF16 the call synchronises the stream and returns
 * IGA_ETIMEOUT if a bounded wait of the tensor-core pipeline gave up. */
iga_status iga_kron_apply(iga_ctx* ctx, const iga_op* A, int transpose, double alpha,
                          const void* x, double beta, void* y, iga_prec prec);

/* out = KKT z for the stationary KKT matrix (Sec. 4 eq. KKTSystem with one
 * time step and tau = 1):  [[M, 0, K^T], [0, beta M, -M], [K, -M, 0]].
 * z, out: device, 3N (y, u, lambda stacked), precision as above; z and out
 * must not overlap (IGA_EINVAL).  When M and K are rank-1 Kronecker sums the
 * five operator products run as one fused launch. */
iga_status iga_kkt_apply(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                         const void* z, void* out, iga_prec prec);

/* ---- (c) block-AMEn local-system matvec ----------------------------- */

/* Projected operator apply at one TT core (Sec. 5, eq. KKT_red, assembled
 * factor by factor):
 *   y(a,i,b) = sum_{al,be} PhiL[al](a,a') A[al][be](i,i') PhiR[be](b,b') x(a',i',b')
 * PhiL: device (R0, r0, r0); bands: device (R0, R1, n, 2p+1) banded A;
 * PhiR: device (R1, r1, r1); x, y: device (nvec, r0, n, r1) for nvec
 * independent vectors.  Precision: IGA_FP64 (double in/out) or IGA_FP32
 * (float in/out, FP32 arithmetic).  bandmask (host, R0*R1 bytes, may be
 * NULL) marks which (al, be) bands are nonzero. */
iga_status iga_amen_local_matvec(iga_ctx* ctx, int r0, int n, int r1, int R0, int R1, int p,
                                 const void* PhiL, const void* bands, const void* PhiR,
                                 const unsigned char* bandmask, int nvec, const void* x, void* y,
                                 iga_prec prec);

/* Allocation-free variant of iga_amen_local_matvec for callers that cannot
 * allocate device memory (the paper has no counterpart; it exists for host
 * applications whose device memory is owned by a fixed pool or budget, and
 * which therefore can call neither cudaMalloc nor iga_create, which
 * allocates).  Same arguments and results as iga_amen_local_matvec, except:
 *   - `stream` is the cudaStream_t to launch on (NULL: legacy default
 *     stream); the calling thread's current device must be the device of
 *     that stream and of every pointer; no iga_ctx is used and no error
 *     text is kept;
 *   - a CUDA error already pending on the calling thread is reported as
 *     IGA_ECUDA before any launch and left pending for its owner;
 *   - with a bandmask the call waits for the stream to reach it before
 *     returning (the mask is host memory borrowed for the call); without
 *     one it returns as soon as the work is queued;
 *   - the intermediates live in a fixed 16 MiB file-scope device array, so
 *     (R0 + R1) * nvec * r0 * n * r1 * sizeof(element) must not exceed
 *     16 MiB and R0 * R1 must not exceed 4096 when a bandmask is given;
 *     larger sizes are rejected with IGA_EINVAL before any GPU work;
 *   - nothing is allocated or freed: no cudaMalloc, cudaFree or allocating
 *     library routine is called;
 *   - the first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture;
 *   - every call on a device shares the one array, which keeps the previous
 *     call's contents (each call overwrites what it reads), so calls that
 *     overlap on the GPU (on different streams, or from several threads
 *     without ordering) race and give wrong results. */
iga_status iga_amen_local_matvec_noalloc(void* stream, int r0, int n, int r1, int R0, int R1,
                                         int p, const void* PhiL, const void* bands,
                                         const void* PhiR, const unsigned char* bandmask,
                                         int nvec, const void* x, void* y, iga_prec prec);

/* ---- adjoint / gradient (a9) ----------------------------------------- */

/* Solve A x = b for A = M or A = K (both symmetric positive definite after
 * the Dirichlet reduction) by preconditioned conjugate gradients in FP64.
 * The preconditioner is the fast-diagonalisation inverse of
 * sum_d c_d Kt_d (x) Mt_e (x) Mt_f built from the mass factors of M and the
 * derivative factors of the q_dd blocks of K (K may be NULL when A == M).
 * x holds the initial guess on entry.  b, x: device, length N.  Returns
 * IGA_ENOCONV when ||b - A x|| > tol ||b|| after maxit iterations. */
iga_status iga_spd_solve(iga_ctx* ctx, const iga_op* A, const iga_op* M, const iga_op* K,
                         const double* b, double* x, double tol, int maxit, int* iters,
                         double* relres);

/* Reduced objective and gradient for nbatch controls (Sec. 4, Lagrangian
 * and KKT conditions, stationary reading): for each control u_s
 *   K y = M u,  K^T lam = b - M y,  grad = beta M u - M lam,
 *   J = 1/2 y^T M y - b^T y + beta/2 u^T M u (without the constant
 *   1/2 int yhat^2 omega).
 * u, grad, y, lam: device (nbatch, N); J: host (nbatch).  The state and
 * adjoint solves run to relative residual tol. */
iga_status iga_reduced_gradient(iga_ctx* ctx, const iga_op* M, const iga_op* K,
                                const iga_tt* load, double beta, int nbatch, const double* u,
                                double tol, double* grad, double* y, double* lam, double* J);

/* Derivative of the reduced objective with respect to the univariate weight
 * factors (the reverse of the univariate assembly, Sec. 3 eq. massMatrix1D):
 * for the TT of every weight c (omega, q11, q12, q13, q22, q23, q33) with
 * ranks (1, 1) and every direction d, grad_w[c][d][e*nquad + q] =
 * dJ/dw_{c,d}(e, q) at the state y, control u and adjoint lam returned by
 * iga_reduced_gradient (the load vector is held fixed).  grad_w: device,
 * 7 * (Q1 + Q2 + Q3) doubles, Q_d = E_d nquad; weights absent from M and K
 * get zeros.  Every block of M and K must have TT ranks (1, 1). */
iga_status iga_weight_gradient(iga_ctx* ctx, const iga_space* space, const iga_op* M,
                               const iga_op* K, double beta, const double* y, const double* u,
                               const double* lam, double* grad_w);

/* ---- KKT solve (a6..a8) ---------------------------------------------- */

/* Truncation of the block core when the block index moves to the next core
 * (Sec. 5, eqs. svd1 and svd2).  IGA_TRUNC_SVD is the paper's truncated SVD,
 * computed from the Gram matrix of the reshaped block core by a Jacobi
 * eigen-decomposition.  IGA_TRUNC_PIVOTED (default) runs Householder QR with
 * column pivoting on the reshaped block core itself and stops at the first
 * rank whose remaining column norms meet trunc_tol, so the Frobenius error of
 * each field obeys the same bound as the SVD's; the rank can be a little
 * larger, and the work is one pass of pivoted QR instead of an
 * eigen-decomposition of the Gram matrix. */
typedef enum { IGA_TRUNC_PIVOTED = 0, IGA_TRUNC_SVD = 1 } iga_trunc;

/* How the solve measures its residual.  IGA_RESID_FULL (default): after
 * every local solve the exact FP64 residual of the full KKT system is formed
 * with the Kronecker apply; it drives the enrichment, the stopping test and
 * an outer iterative refinement z <- z + delta.  Its cost grows with the
 * operators' TT-matrix ranks (a KKT apply is about 2 (2p+1) N sum_blocks
 * (R1 + R1 R2 + R2) flop per operator application).
 * IGA_RESID_LOCAL: the method of the paper's Sec. 5 without any full-size
 * operator apply.  The stopping test is the local residual: before each
 * local solve, ||F_{!=d}^T (rhs - KKT z)||_2, the projection of the residual
 * onto the current frame, computed with the FP64 interfaces; the solve stops
 * after the sweep whose largest such value is <= tol ||rhs||_2.  The
 * enrichment takes the residual sketched by Khatri-Rao products of Gaussian
 * vectors (a rank-one test tensor per sketch column) through interfaces of
 * the same kind as the local operator's.  There is no outer refinement; the
 * full solution is expanded once at the end.  info->residual then reports
 * the largest projected residual of the last sweep (each measured before its
 * local solve, and each a lower bound of the true residual of the iterate
 * at that moment). */
typedef enum { IGA_RESID_FULL = 0, IGA_RESID_LOCAL = 1 } iga_residual;

typedef struct {
  double tol;          /* stop when ||rhs - KKT z||_2 / ||rhs||_2 <= tol (the
                          projected residual with IGA_RESID_LOCAL) */
  double inner_tol;    /* tolerance of each AMEn correction (0: tol itself) */
  int max_sweeps;      /* AMEn sweeps per correction */
  int kick_rank;       /* AMEn enrichment rank */
  int rmax;            /* TT rank cap */
  int local_maxit;     /* Krylov iterations per local system */
  int refine_max;      /* outer FP64 refinement steps */
  int precision;       /* arithmetic of the AMEn local systems: IGA_FP64,
                          IGA_FP32, or IGA_TF32 (FP32 with the large
                          interface products on the tensor cores, TF32
                          operands and FP32 accumulation) */
  int verbose;         /* print one line per sweep to stderr */
  double trunc_tol;    /* relative truncation of each field in the block core
                          when the block index moves (0: tol / 1000; with
                          IGA_RESID_FULL lowered 100-fold down to tol * 1e-5
                          whenever a sweep reduces the residual by less than a
                          factor 4, with IGA_RESID_LOCAL kept fixed) */
  int truncation;      /* how the block index moves: IGA_TRUNC_PIVOTED or
                          IGA_TRUNC_SVD (see iga_trunc) */
  int residual;        /* IGA_RESID_FULL or IGA_RESID_LOCAL (see iga_residual) */
  double state_weight; /* weight of the state y in the truncation of the block
                          core: y is kept to a relative error of about
                          trunc_tol / state_weight, u and lambda to trunc_tol
                          (the stiffness operator amplifies the error of y in
                          the state equation's residual); <= 1: no weight */
} iga_solve_opts;

typedef struct {
  int sweeps;          /* AMEn sweeps over all corrections */
  int refinements;     /* FP64 refinement steps taken */
  int max_rank;        /* largest TT rank of the solution components */
  int local_iters;     /* Krylov iterations over all local solves */
  double residual;     /* final ||rhs - KKT z|| / ||rhs|| in FP64 */
  double seconds;      /* wall time of the solve */
  double t_local;      /* device seconds: local systems (preconditioner + GMRES) */
  double t_residual;   /* device seconds: full correction and FP64 residual after
                          each local solve */
  double t_move;       /* device seconds: truncation, orthogonalisation,
                          enrichment and interface updates */
  double t_refine;     /* device seconds: outer refinement residuals */
} iga_solve_info;

/* Fill opts with defaults. */
void iga_solve_opts_default(iga_solve_opts* opts);

/* Solve the stationary KKT system with rhs = [b; 0; 0], b the load vector
 * (TT), by block AMEn (Sec. 5: block TT eq. btt, SVD moves eqs. svd1/svd2,
 * reduced KKT eq. KKT_red) inside FP64 iterative refinement of the full
 * residual.  y, u, lam: device FP64 vectors of length N (full format).
 * Returns IGA_ENOCONV (with the best iterate written) when the tolerance
 * is not reached. */
iga_status iga_kkt_solve_amen(iga_ctx* ctx, const iga_op* M, const iga_op* K, const iga_tt* load,
                              double beta, const iga_solve_opts* opts, double* y, double* u,
                              double* lam, iga_solve_info* info);

/* Rows of the KKT residual (Sec. 4, eq. KKTSystem, one time step) for a
 * solution held as TTs, without forming anything of full size: for each of
 * the nrows interior multi-indices rows[3s .. 3s+2] (0-based, i_d < n_d;
 * host int32) res[3s + e] (host) receives equation e's residual,
 *   e = 0: b_i - (M y)_i - (K lambda)_i,
 *   e = 1: -(beta (M u)_i - (M lambda)_i),
 *   e = 2: -((K y)_i - (M u)_i),
 * with every operator entry formed from the univariate bands over the row's
 * (2p+1)^3 stencil and every solution value from the TT cores (FP64).  load
 * may be NULL (b = 0).  Uniformly sampled rows estimate ||rhs - KKT z||_2^2
 * without bias as (N / S) sum_s sum_e res[3s+e]^2.  IGA_EINVAL for a row
 * outside the interior grid, mismatched sizes or a degree above 4.
 * Synchronises. */
iga_status iga_kkt_residual_rows(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                                 const iga_tt* load, const iga_tt* y, const iga_tt* u,
                                 const iga_tt* lam, int nrows, const int* rows, double* res);

/* The same solve with the solution returned as TT tensors (Sec. 5: the
 * block-AMEn solution is the block TT of eq. btt; here one TT per field).
 * The solve runs into full device vectors owned by the call, each field is
 * compressed by TT-SVD to a relative Frobenius error of opts->tol / 10, and
 * *y, *u, *lam receive library-owned TTs (NULL for a field that is exactly
 * zero); iga_tt_full expands them.  With opts->residual IGA_RESID_LOCAL no
 * full vector is formed: the fields are the solve's own block TT split by
 * field (the frame cores shared, the block core's slice per field; a zero
 * right-hand side gives rank-one zero TTs).  Returns what the solve returns
 * (IGA_ENOCONV with the best iterate). */
iga_status iga_kkt_solve_amen_tt(iga_ctx* ctx, const iga_op* M, const iga_op* K,
                                 const iga_tt* load, double beta, const iga_solve_opts* opts,
                                 iga_tt** y, iga_tt** u, iga_tt** lam, iga_solve_info* info);

/* Solve the parabolic KKT system of Sec. 4 (eq. timeDiscrete discretised by
 * nt implicit Euler steps of size tau, eq. KKTSystem):
 *   [ tau MM   0            KK^T    ] [y  ]   [b]
 *   [ 0        tau beta MM  -tau MM ] [u  ] = [0]
 *   [ KK       -tau MM      0       ] [lam]   [0]
 * with MM = I_nt (x) M, KK = I_nt (x) tau K + C (x) M and C the lower
 * bidiagonal time difference (ones on the diagonal, minus ones below), by
 * block AMEn on the space-time TT (the time index as a fourth TT core in
 * front of the spatial ones; Sec. 5 eqs. M_kron, K_kron, KKT_red) inside
 * FP64 iterative refinement of the full residual.  M, K: the spatial
 * operators (same sizes and degrees).  load: device FP64 (nt, N), the y-row
 * right-hand side b = [b_1; ...; b_nt] (b_k = tau M yhat_k for a desired
 * state yhat), or NULL for zero.  y, u, lam: device FP64 (nt, N) each, time
 * the slow index; load must not overlap y, u or lam.  opts->residual must be
 * IGA_RESID_FULL.  Synchronises the context stream.  IGA_EINVAL for
 * nt < 1, tau <= 0, beta <= 0, nt N of 2^31 or more or mismatched operators; IGA_ENOCONV (best
 * iterate written) when the tolerance is not reached. */
iga_status iga_kkt_solve_parabolic(iga_ctx* ctx, const iga_op* M, const iga_op* K, int nt,
                                   double tau, const double* load, double beta,
                                   const iga_solve_opts* opts, double* y, double* u, double* lam,
                                   iga_solve_info* info);

#ifdef __cplusplus
}
#endif
#endif /* IGA_H */
