// C ABI of libiga: context, handles and the composite low-rank assembly.
//
// iga_lowrank_assemble follows Sec. 3: sample omega, Q (and the load
// density) on the tensor Gauss grid, TT-SVD each sample tensor (eq. tt), and
// assemble one banded univariate matrix per TT core slice (eqs.
// massMatrix1D, stiffnessFinal), so that M = sum (x)_d M_d and
// K = sum_{k,l} sum (x)_d K_kl^(d) with the core slices of eq. TTranks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>

#include "iga_internal.cuh"

namespace iga {

void set_error(iga_ctx* ctx, const std::string& m) {
  if (ctx) ctx->err = m;
}

void tc_flag_reset(iga_ctx* ctx) {
  IGA_CUDA(cudaMemsetAsync(ctx->dflag + 1, 0, sizeof(int), ctx->stream));
}

void tc_flag_check(iga_ctx* ctx, const char* what) {
  IGA_CUDA(cudaMemcpyAsync(ctx->hflag + 1, ctx->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost,
                           ctx->stream));
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->hflag[1] != 0)
    throw Error(IGA_ETIMEOUT, std::string(what) + ": a bounded wait of the tensor-core pipeline "
                                                  "gave up");
}

void func_attr(const void* fn, cudaFuncAttribute attr, int value) {
  // one value per (function, attribute, device), raised monotonically: a
  // launch needs at least the value it asks for, so a later request for a
  // smaller value keeps the larger one that is already set
  struct Key {
    const void* fn;
    int attr, dev;
    bool operator<(const Key& o) const {
      if (fn != o.fn) return fn < o.fn;
      if (attr != o.attr) return attr < o.attr;
      return dev < o.dev;
    }
  };
  static std::mutex mu;
  static std::map<Key, int> cur;
  int dev = 0;
  IGA_CUDA(cudaGetDevice(&dev));
  Key k{fn, (int)attr, dev};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cur.find(k);
  if (it != cur.end() && it->second >= value) return;
  IGA_CUDA(cudaFuncSetAttribute(fn, attr, value));
  cur[k] = value;
}

void prof_start(iga_ctx* ctx) {
  if (ctx->prof_used + 2 > ctx->prof_ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      IGA_CUDA(cudaEventCreate(&e));
      ctx->prof_ev.push_back(e);
    }
  }
  IGA_CUDA(cudaEventRecord(ctx->prof_ev[ctx->prof_used], ctx->stream));
  ctx->prof_bytes += ctx->next_bytes;
  ctx->prof_flops += ctx->next_flops;
}

void prof_stop(iga_ctx* ctx) {
  IGA_CUDA(cudaEventRecord(ctx->prof_ev[ctx->prof_used + 1], ctx->stream));
  ctx->prof_used += 2;
}

void sample_weights_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                         const iga_target* target, double* out);

// (r0, Q, r1) core -> (r0 * r1, Q) slices
__global__ void core_to_slices_kernel(const double* __restrict__ c, int r0, int Q, int r1,
                                      double* __restrict__ s) {
  size_t total = (size_t)r0 * Q * r1;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int b = (int)(i % r1);
  size_t t = i / r1;
  int q = (int)(t % Q);
  int a = (int)(t / Q);
  s[((size_t)a * r1 + b) * Q + q] = c[i];
}

// (r0 * r1, n) slices -> (r0, n, r1) core
__global__ void slices_to_core_kernel(const double* __restrict__ s, int r0, int n, int r1,
                                      double* __restrict__ c) {
  size_t total = (size_t)r0 * n * r1;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int b = (int)(i % r1);
  size_t t = i / r1;
  int j = (int)(t % n);
  int a = (int)(t / n);
  c[i] = s[((size_t)a * r1 + b) * n + j];
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

static void core_slices(iga_ctx* ctx, const double* core, int r0, int Q, int r1, double* out) {
  size_t total = (size_t)r0 * Q * r1;
  IGA_LAUNCH(ctx, core_to_slices_kernel, (unsigned)((total + 255) / 256), 256, 0, core, r0, Q, r1,
             out);
}

// Append one block (the operator term of a TT weight with given derivative
// pattern) to the band lists of an operator under construction.
struct OpBuilder {
  std::vector<OpBlock> blocks;
  std::vector<std::vector<double>> host;    // unused: bands stay on the device
  std::vector<DevBuf<double>> parts[3];
  size_t count[3] = {0, 0, 0};
};

static void add_block(iga_ctx* ctx, const SpaceTables& st, const iga_tt* tt, const int deriv[3][2],
                      OpBuilder& B) {
  OpBlock blk;
  blk.R1 = tt->r[0];
  blk.R2 = tt->r[1];
  int rl[4] = {1, tt->r[0], tt->r[1], 1};
  for (int d = 0; d < 3; ++d) {
    const DirTables& T = st.dir[d];
    int Q = T.E * T.q;
    int nT = rl[d] * rl[d + 1];
    double* sl = scratch<double>(ctx, SLOT_ASM_W, (size_t)nT * Q);
    core_slices(ctx, tt->core[d].p, rl[d], Q, rl[d + 1], sl);
    DevBuf<double> band((size_t)nT * (T.n - 2) * (2 * T.p + 1));
    launch_assemble_bands(ctx, T, sl, nT, deriv[d][0], deriv[d][1], 1, band.p);
    blk.off[d] = B.count[d];
    blk.deriv[d][0] = deriv[d][0];
    blk.deriv[d][1] = deriv[d][1];
    B.count[d] += nT;
    B.parts[d].push_back(std::move(band));
    // the slice buffer is reused by the next launch on the same stream: no sync needed
  }
  B.blocks.push_back(blk);
}

static iga_op* finish_op(iga_ctx* ctx, const int* n_int, const int* p_deg, OpBuilder& B) {
  auto* op = new iga_op();
  try {
    for (int d = 0; d < 3; ++d) {
      op->n[d] = n_int[d];
      op->p[d] = p_deg[d];
      size_t len = (size_t)op->n[d] * (2 * op->p[d] + 1);
      op->nbands[d] = B.count[d];
      op->band64[d].alloc(std::max<size_t>(1, B.count[d] * len));
      op->band32[d].alloc(std::max<size_t>(1, B.count[d] * len));
      size_t off = 0;
      for (auto& part : B.parts[d]) {
        IGA_CUDA(cudaMemcpyAsync(op->band64[d].p + off, part.p, part.n * 8,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
        off += part.n;
      }
      size_t n = B.count[d] * len;
      if (n)
        IGA_LAUNCH(ctx, to_float_kernel, (unsigned)((n + 255) / 256), 256, 0, op->band64[d].p,
                   op->band32[d].p, n);
    }
    op->blocks = B.blocks;
    op->rank1 = true;
    for (auto& b : op->blocks) op->rank1 = op->rank1 && b.R1 == 1 && b.R2 == 1;
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    delete op;
    throw;
  }
  return op;
}

static iga_tt* load_tt(iga_ctx* ctx, const SpaceTables& st, const iga_tt* f) {
  auto* tt = new iga_tt();
  try {
    int rl[4] = {1, f->r[0], f->r[1], 1};
    tt->r[0] = f->r[0];
    tt->r[1] = f->r[1];
    for (int d = 0; d < 3; ++d) {
      const DirTables& T = st.dir[d];
      int Q = T.E * T.q;
      int nT = rl[d] * rl[d + 1];
      int ni = T.n - 2;
      tt->n[d] = ni;
      double* sl = scratch<double>(ctx, SLOT_ASM_W, (size_t)nT * Q);
      core_slices(ctx, f->core[d].p, rl[d], Q, rl[d + 1], sl);
      double* vec = scratch<double>(ctx, SLOT_MISC0, (size_t)nT * ni);
      launch_load_vectors(ctx, T, sl, nT, 1, vec);
      tt->core[d].alloc((size_t)nT * ni);
      size_t total = (size_t)nT * ni;
      IGA_LAUNCH(ctx, slices_to_core_kernel, (unsigned)((total + 255) / 256), 256, 0, vec, rl[d],
                 ni, rl[d + 1], tt->core[d].p);
    }
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    delete tt;
    throw;
  }
  return tt;
}

static void kkt_apply_impl(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                           const void* z, void* out, iga_prec prec) {
  IGA_REQUIRE(M && K && z && out, "kkt_apply: null argument");
  for (int d = 0; d < 3; ++d) IGA_REQUIRE(M->n[d] == K->n[d], "kkt_apply: M and K sizes differ");
  size_t N = (size_t)M->n[0] * M->n[1] * M->n[2];
  size_t es = prec == IGA_FP64 ? 8 : 4;
  const char* zc = static_cast<const char*>(z);
  char* oc = static_cast<char*>(out);
  const void* y = zc;
  const void* u = zc + N * es;
  const void* l = zc + 2 * N * es;
  void* o1 = oc;
  void* o2 = oc + N * es;
  void* o3 = oc + 2 * N * es;
  // K is symmetric by construction (the (k,l) and (l,k) blocks share the
  // weight q_kl = q_lk and have transposed factors), so K^T = K.
  {
    const char* ze = zc + 3 * N * es;
    const char* oe = oc + 3 * N * es;
    IGA_REQUIRE(ze <= oc || oe <= zc, "kkt_apply: z and out must not overlap");
  }
  if (kkt_apply_fused(ctx, M, K, beta, z, out, prec)) return;
  kron_apply_impl(ctx, M, 1.0, y, 0.0, o1, prec);
  kron_apply_impl(ctx, K, 1.0, l, 1.0, o1, prec);
  kron_apply_impl(ctx, M, beta, u, 0.0, o2, prec);
  kron_apply_impl(ctx, M, -1.0, l, 1.0, o2, prec);
  kron_apply_impl(ctx, K, 1.0, y, 0.0, o3, prec);
  kron_apply_impl(ctx, M, -1.0, u, 1.0, o3, prec);
}

void kkt_apply_internal(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                        const void* z, void* out, iga_prec prec) {
  kkt_apply_impl(ctx, M, K, beta, z, out, prec);
}

// Sample the eight weight tensors and TT-compress them (Sec. 3): omega g,
// the six entries of Q g (truncated relative to ||Q||_F over all nine
// entries), and the load density yhat(G) omega g.  Rank-0 tensors stay NULL.
struct EachCtx {
  iga_ctx* ctx;
  int Q[3];
  double tol;
  double* qn2dev;
  double qnorm;
  iga_tt** tts;
};

static void weight_tt_cb(void* user, int c, const double* buf) {
  EachCtx* e = static_cast<EachCtx*>(user);
  if (c == 1) {
    IGA_CUDA(cudaMemcpyAsync(&e->qnorm, e->qn2dev, 8, cudaMemcpyDeviceToHost, e->ctx->stream));
    IGA_CUDA(cudaStreamSynchronize(e->ctx->stream));
    e->qnorm = std::sqrt(e->qnorm);
  }
  double ref = (c >= 1 && c <= 6) ? e->qnorm : 0.0;
  tt_svd3(e->ctx, buf, e->Q[0], e->Q[1], e->Q[2], e->tol, ref, 0, &e->tts[c]);
}

void weight_tts_impl(iga_ctx* ctx, const iga_geometry* geo, const SpaceTables& st,
                     const iga_target* target, double tol, iga_tt* tts[8]) {
  int Q[3];
  for (int d = 0; d < 3; ++d) Q[d] = st.dir[d].E * st.dir[d].q;
  size_t S = (size_t)Q[0] * Q[1] * Q[2];
  size_t free_b = 0, tot_b = 0;
  IGA_CUDA(cudaMemGetInfo(&free_b, &tot_b));
  if (8 * S * sizeof(double) > free_b / 3) {
    // large grids: one sample tensor at a time, each compressed before the next
    double* buf = scratch<double>(ctx, SLOT_ASM_SAMPLES, S);
    double* qn2 = scratch<double>(ctx, SLOT_QNORM, 1);
    EachCtx e{ctx, {Q[0], Q[1], Q[2]}, tol, qn2, 0.0, tts};
    try {
      sample_weights_each(ctx, geo, st, target, buf, qn2, weight_tt_cb, &e);
    } catch (...) {
      for (int c = 0; c < 8; ++c) { delete tts[c]; tts[c] = nullptr; }
      throw;
    }
    return;
  }
  double* samples = scratch<double>(ctx, SLOT_ASM_SAMPLES, 8 * S);
  sample_weights_impl(ctx, geo, st, target, samples);
  // the eight Frobenius norms in one pass
  double nrm[8];
  device_norms(ctx, samples, S, 8, nrm);
  double qn2 = 0.0;
  for (int c = 1; c <= 6; ++c)
    qn2 += (c == 2 || c == 3 || c == 5) ? 2 * nrm[c] * nrm[c] : nrm[c] * nrm[c];
  double qnorm = std::sqrt(qn2);
  try {
    tt_svd3(ctx, samples, Q[0], Q[1], Q[2], tol, 0.0, 0, &tts[0], nrm[0]);
    for (int c = 1; c <= 6; ++c)
      tt_svd3(ctx, samples + c * S, Q[0], Q[1], Q[2], tol, qnorm, 0, &tts[c], nrm[c]);
    if (target && target->kind != IGA_TARGET_ZERO)
      tt_svd3(ctx, samples + 7 * S, Q[0], Q[1], Q[2], tol, 0.0, 0, &tts[7], nrm[7]);
  } catch (...) {
    for (int c = 0; c < 8; ++c) { delete tts[c]; tts[c] = nullptr; }
    throw;
  }
}

// M from the TT of omega g; K from the TTs of q_kl g with the derivative
// pattern delta(l,d) on the row and delta(k,d) on the column factor
// (Sec. 3, eqs. massFinal and stiffnessFinal); q_lk shares the TT of q_kl.
void ops_from_weights_impl(iga_ctx* ctx, const SpaceTables& st, const iga_tt* const w[7],
                           iga_op** M, iga_op** K) {
  IGA_REQUIRE(w[0] != nullptr, "operators: omega weight missing");
  OpBuilder bm, bk;
  int dm[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  add_block(ctx, st, w[0], dm, bm);
  const int qidx[3][3] = {{1, 2, 3}, {2, 4, 5}, {3, 5, 6}};
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      const iga_tt* t = w[qidx[k][l]];
      if (!t) continue;
      int dk[3][2];
      for (int d = 0; d < 3; ++d) {
        dk[d][0] = (l == d);
        dk[d][1] = (k == d);
      }
      add_block(ctx, st, t, dk, bk);
    }
  int ni[3], pd[3];
  for (int d = 0; d < 3; ++d) {
    ni[d] = st.dir[d].n - 2;
    pd[d] = st.dir[d].p;
  }
  iga_op* m = finish_op(ctx, ni, pd, bm);
  iga_op* kk = nullptr;
  try {
    kk = finish_op(ctx, ni, pd, bk);
  } catch (...) {
    delete m;
    throw;
  }
  *M = m;
  *K = kk;
}

// copy of a band array with the entries outside the matrix set to zero
__global__ void band_clean_kernel(const double* __restrict__ in, double* __restrict__ out,
                                  size_t total, int n, int P) {
  const int B = 2 * P + 1;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx % B);
    const int i = (int)((idx / B) % n);
    const int j = i + o - P;
    out[idx] = (j >= 0 && j < n) ? in[idx] : 0.0;
  }
}

iga_op* op_from_bands_impl(iga_ctx* ctx, const int n[3], const int p[3], int nblocks,
                           const int* R, const double* const* bands) {
  IGA_REQUIRE(nblocks >= 1 && R && bands, "op_from_bands: no blocks");
  for (int d = 0; d < 3; ++d)
    IGA_REQUIRE(n[d] >= 1 && p[d] >= 0 && p[d] <= 8, "op_from_bands: invalid size or degree");
  OpBuilder b;
  for (int k = 0; k < nblocks; ++k) {
    const int R1 = R[2 * k], R2 = R[2 * k + 1];
    IGA_REQUIRE(R1 >= 1 && R2 >= 1, "op_from_bands: ranks must be positive");
    OpBlock blk;
    blk.R1 = R1;
    blk.R2 = R2;
    const size_t cnt[3] = {(size_t)R1, (size_t)R1 * R2, (size_t)R2};
    for (int d = 0; d < 3; ++d) {
      const double* src = bands[3 * k + d];
      IGA_REQUIRE(src != nullptr, "op_from_bands: null band array");
      const size_t total = cnt[d] * n[d] * (2 * p[d] + 1);
      DevBuf<double> band(total);
      IGA_LAUNCH(ctx, band_clean_kernel, (unsigned)std::min<size_t>((total + 255) / 256, 4096),
                 256, 0, src, band.p, total, n[d], p[d]);
      blk.off[d] = b.count[d];
      b.count[d] += cnt[d];
      b.parts[d].push_back(std::move(band));
    }
    b.blocks.push_back(blk);
  }
  return finish_op(ctx, n, p, b);
}

}  // namespace iga

namespace iga {

namespace {
thread_local cudaStream_t t_alloc_stream = nullptr;
thread_local bool t_alloc_active = false;

// one stream-ordered pool per device, keeping up to 4 GB of released memory
// cached across synchronisations; nullptr on a device without memory pools
// (allocations then go through cudaMalloc)
cudaMemPool_t device_pool() {
  int dev = 0;
  IGA_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  int supported = 0;
  IGA_CUDA(cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev));
  if (!supported) {
    pools[dev] = nullptr;
    return nullptr;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  IGA_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = 4ull << 30;
  IGA_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}
}  // namespace

AllocScope::AllocScope(cudaStream_t s) : prev_stream(t_alloc_stream), prev_active(t_alloc_active) {
  t_alloc_stream = s;
  t_alloc_active = true;
}

AllocScope::~AllocScope() {
  t_alloc_stream = prev_stream;
  t_alloc_active = prev_active;
}

void* dev_alloc(size_t bytes, bool* pooled) {
  void* p = nullptr;
  cudaMemPool_t pool = t_alloc_active ? device_pool() : nullptr;
  cudaError_t e;
  if (pool) {
    e = cudaMallocFromPoolAsync(&p, bytes, pool, t_alloc_stream);
    *pooled = true;
  } else {
    e = cudaMalloc(&p, bytes);
    *pooled = false;
  }
  if (e != cudaSuccess) {
    // a refused allocation is not a sticky error: clear the thread's last
    // error so that the next launch check does not report it again
    (void)cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA,
                std::string("device allocation of ") + std::to_string(bytes) +
                    " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void dev_free(void* p, bool pooled) noexcept {
  if (!p) return;
  if (!pooled) {
    cudaFree(p);
  } else if (t_alloc_active) {
    cudaFreeAsync(p, t_alloc_stream);
  } else {
    // released outside any entry: the stream that used it is unknown
    cudaDeviceSynchronize();
    cudaFree(p);
  }
}

}  // namespace iga

using namespace iga;

#define IGA_TRY(ctx, ...)                                                         \
  try {                                                                           \
    ::iga::AllocScope scope__((ctx)->stream);                                     \
    __VA_ARGS__;                                                                  \
    return IGA_OK;                                                                \
  } catch (const ::iga::Error& e) {                                               \
    set_error(ctx, e.what());                                                     \
    return e.status;                                                              \
  } catch (const std::bad_alloc&) {                                               \
    set_error(ctx, "host allocation failed");                                     \
    return IGA_ENOMEM;                                                            \
  } catch (const std::exception& e) {                                             \
    set_error(ctx, e.what());                                                     \
    return IGA_ECUDA;                                                             \
  }

extern "C" {

iga_status iga_create(iga_ctx** out, void* stream) {
  if (!out) return IGA_EINVAL;
  *out = nullptr;
  iga_ctx* ctx = nullptr;
  try {
    ctx = new iga_ctx();
    ctx->stream = static_cast<cudaStream_t>(stream);
    IGA_CUDA(cudaGetDevice(&ctx->device));
    IGA_CUDA(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    IGA_CUDA(cudaMalloc((void**)&ctx->dflag, 64 * sizeof(int)));
    IGA_CUDA(cudaMallocHost((void**)&ctx->hflag, 64 * sizeof(int)));
    IGA_CUDA(cudaMemset(ctx->dflag, 0, 64 * sizeof(int)));
    *out = ctx;
    return IGA_OK;
  } catch (const ::iga::Error& e) {
    if (ctx) iga_destroy(ctx);
    return e.status;
  } catch (...) {
    if (ctx) iga_destroy(ctx);
    return IGA_ENOMEM;
  }
}

void iga_destroy(iga_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  ctx->scratch.clear();
  if (ctx->dflag) cudaFree(ctx->dflag);
  if (ctx->hflag) cudaFreeHost(ctx->hflag);
  delete ctx;
}

iga_status iga_profile_begin(iga_ctx* ctx, const char* kernel) {
  if (!ctx) return IGA_EINVAL;
  ctx->prof_name = kernel ? kernel : "";
  ctx->prof_used = 0;
  ctx->prof_bytes = 0.0;
  ctx->prof_flops = 0.0;
  return IGA_OK;
}

iga_status iga_profile_end(iga_ctx* ctx, uint64_t* launches, double* ms, double* bytes,
                           double* flops) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < ctx->prof_used; i += 2) {
      float t = 0.f;
      IGA_CUDA(cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
      tot += t;
    }
    if (launches) *launches = ctx->prof_used / 2;
    if (ms) *ms = tot;
    if (bytes) *bytes = ctx->prof_bytes;
    if (flops) *flops = ctx->prof_flops;
    ctx->prof_name.clear();
    ctx->prof_used = 0;
  })
}

const char* iga_last_error(const iga_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t iga_launch_count(const iga_ctx* ctx) { return ctx ? ctx->launches : 0; }

size_t iga_scratch_bytes(const iga_ctx* ctx) { return ctx ? ctx->scratch_bytes() : 0; }

iga_status iga_sample_weights(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                              const iga_target* target, double* out) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    SpaceTables st;
    build_space_tables(ctx, space, st);
    sample_weights_impl(ctx, geo, st, target, out);
  })
}

iga_status iga_tt_svd(iga_ctx* ctx, const double* W, int n1, int n2, int n3, double tol,
                      double norm_ref, int rmax, iga_tt** out) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    tt_svd3(ctx, W, n1, n2, n3, tol, norm_ref, rmax, out);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));   // the handle is usable on any stream
  })
}

iga_status iga_tt_info(const iga_tt* tt, int n[3], int r[2]) {
  if (!tt) return IGA_EINVAL;
  for (int d = 0; d < 3; ++d) if (n) n[d] = tt->n[d];
  if (r) { r[0] = tt->r[0]; r[1] = tt->r[1]; }
  return IGA_OK;
}

iga_status iga_tt_core(iga_ctx* ctx, const iga_tt* tt, int d, double* core) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(tt && core && d >= 0 && d < 3, "tt_core: bad argument");
    IGA_CUDA(cudaMemcpyAsync(core, tt->core[d].p, tt->core[d].n * 8, cudaMemcpyDeviceToHost,
                             ctx->stream));
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

iga_status iga_tt_full(iga_ctx* ctx, const iga_tt* tt, double* out) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, tt_full_impl(ctx, tt, out))
}

void iga_tt_destroy(iga_tt* tt) { delete tt; }

// File format of a TT tensor: the 8 bytes "IGATT" 0x01 0x00 0x00, the int32
// sizes n1 n2 n3 and ranks r1 r2, then the cores (r_{d-1}, n_d, r_d) in C
// order as float64, all little-endian (the byte order of every host this
// library builds for).
static const unsigned char TT_MAGIC[8] = {'I', 'G', 'A', 'T', 'T', 1, 0, 0};

iga_status iga_tt_save(iga_ctx* ctx, const iga_tt* tt, const char* path) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(tt && path, "tt_save: null argument");
    std::vector<double> host[3];
    for (int d = 0; d < 3; ++d) {
      host[d].resize(tt->core[d].n);
      if (!host[d].empty())
        IGA_CUDA(cudaMemcpyAsync(host[d].data(), tt->core[d].p, host[d].size() * 8,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    }
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    FILE* f = std::fopen(path, "wb");
    IGA_REQUIRE(f != nullptr, std::string("tt_save: cannot open ") + path);
    int32_t hdr[5] = {tt->n[0], tt->n[1], tt->n[2], tt->r[0], tt->r[1]};
    bool ok = std::fwrite(TT_MAGIC, 1, 8, f) == 8 && std::fwrite(hdr, 4, 5, f) == 5;
    for (int d = 0; d < 3 && ok; ++d)
      ok = std::fwrite(host[d].data(), 8, host[d].size(), f) == host[d].size();
    ok = (std::fclose(f) == 0) && ok;
    IGA_REQUIRE(ok, std::string("tt_save: write failed for ") + path);
  })
}

iga_status iga_tt_load(iga_ctx* ctx, const char* path, iga_tt** out) {
  if (!ctx || !out) return IGA_EINVAL;
  *out = nullptr;
  IGA_TRY(ctx, {
    IGA_REQUIRE(path != nullptr, "tt_load: null path");
    FILE* f = std::fopen(path, "rb");
    IGA_REQUIRE(f != nullptr, std::string("tt_load: cannot open ") + path);
    unsigned char magic[8];
    int32_t hdr[5];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, TT_MAGIC, 8) == 0 &&
              std::fread(hdr, 4, 5, f) == 5;
    for (int k = 0; k < 5 && ok; ++k) ok = hdr[k] >= 1 && hdr[k] <= (1 << 24);
    std::vector<double> host[3];
    if (ok) {
      const int rl[4] = {1, hdr[3], hdr[4], 1};
      for (int d = 0; d < 3 && ok; ++d) {
        const size_t cnt = (size_t)rl[d] * hdr[d] * rl[d + 1];
        ok = cnt <= ((size_t)1 << 34);
        if (ok) {
          host[d].resize(cnt);
          ok = std::fread(host[d].data(), 8, cnt, f) == cnt;
        }
      }
      ok = ok && std::fgetc(f) == EOF;     // nothing after the cores
    }
    std::fclose(f);
    IGA_REQUIRE(ok, std::string("tt_load: not a TT file of this library: ") + path);
    std::unique_ptr<iga_tt> tt(new iga_tt());
    for (int d = 0; d < 3; ++d) tt->n[d] = hdr[d];
    tt->r[0] = hdr[3];
    tt->r[1] = hdr[4];
    for (int d = 0; d < 3; ++d) {
      tt->core[d].alloc(host[d].size());
      IGA_CUDA(cudaMemcpyAsync(tt->core[d].p, host[d].data(), host[d].size() * 8,
                               cudaMemcpyHostToDevice, ctx->stream));
    }
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = tt.release();
  })
}

iga_status iga_assemble_bands(iga_ctx* ctx, const iga_space* space, int d, const double* w, int T,
                              int deriv_row, int deriv_col, int interior, double* band) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(d >= 0 && d < 3 && w && band && T >= 0, "assemble_bands: bad argument");
    IGA_REQUIRE(interior == 0 || interior == 1, "assemble_bands: interior must be 0 or 1");
    SpaceTables st;
    build_space_tables(ctx, space, st);
    launch_assemble_bands(ctx, st.dir[d], w, T, deriv_row != 0, deriv_col != 0, interior, band);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

iga_status iga_weight_tts(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                          const iga_target* target, double tol, iga_tt* out[8]) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(out != nullptr, "weight_tts: null output");
    IGA_REQUIRE(tol >= 0.0, "weight_tts: negative tolerance");
    for (int c = 0; c < 8; ++c) out[c] = nullptr;
    SpaceTables st;
    build_space_tables(ctx, space, st);
    weight_tts_impl(ctx, geo, st, target, tol, out);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

iga_status iga_tt_from_cores(iga_ctx* ctx, const int n[3], const int r[2],
                             const double* const cores[3], iga_tt** out) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(n && r && cores && out, "tt_from_cores: null argument");
    IGA_REQUIRE(n[0] > 0 && n[1] > 0 && n[2] > 0 && r[0] > 0 && r[1] > 0,
                "tt_from_cores: sizes must be positive");
    *out = nullptr;
    auto* tt = new iga_tt();
    try {
      int rl[4] = {1, r[0], r[1], 1};
      for (int d = 0; d < 3; ++d) {
        IGA_REQUIRE(cores[d] != nullptr, "tt_from_cores: null core");
        tt->n[d] = n[d];
        size_t cnt = (size_t)rl[d] * n[d] * rl[d + 1];
        tt->core[d].alloc(cnt);
        IGA_CUDA(cudaMemcpyAsync(tt->core[d].p, cores[d], cnt * 8, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
      }
      tt->r[0] = r[0];
      tt->r[1] = r[1];
      IGA_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
      delete tt;
      throw;
    }
    *out = tt;
  })
}

iga_status iga_ops_from_weights(iga_ctx* ctx, const iga_space* space,
                                const iga_tt* const weights[7], iga_op** M, iga_op** K) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(weights && M && K, "ops_from_weights: null argument");
    *M = nullptr;
    *K = nullptr;
    SpaceTables st;
    build_space_tables(ctx, space, st);
    for (int c = 0; c < 7; ++c)
      if (weights[c])
        for (int d = 0; d < 3; ++d)
          IGA_REQUIRE(weights[c]->n[d] == st.dir[d].E * st.dir[d].q,
                      "ops_from_weights: weight TT is not on the Gauss grid of the space");
    ops_from_weights_impl(ctx, st, weights, M, K);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

iga_status iga_load_from_density(iga_ctx* ctx, const iga_space* space, const iga_tt* density,
                                 iga_tt** load) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(density && load, "load_from_density: null argument");
    SpaceTables st;
    build_space_tables(ctx, space, st);
    *load = load_tt(ctx, st, density);
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

// the composite assembly with the weights sampled on the Gauss grid (pt = 0)
// or interpolated in the spline space of degree pt (pt > 0)
static void lowrank_assemble_impl(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                                  const iga_target* target, double tol, int pt, iga_op** M,
                                  iga_op** K, iga_tt** load) {
  IGA_REQUIRE(M && K, "lowrank_assemble: null output");
  IGA_REQUIRE(tol >= 0.0, "lowrank_assemble: negative tolerance");
  *M = nullptr;
  *K = nullptr;
  if (load) *load = nullptr;
  SpaceTables st;
  build_space_tables(ctx, space, st);
  iga_tt* tts[8] = {nullptr};
  struct Guard {
    iga_tt** t;
    ~Guard() { for (int i = 0; i < 8; ++i) delete t[i]; }
  } guard{tts};
  if (pt > 0) weight_tts_interp_impl(ctx, geo, st, target, tol, pt, tts);
  else weight_tts_impl(ctx, geo, st, target, tol, tts);
  IGA_REQUIRE(tts[0] != nullptr, "lowrank_assemble: omega is zero");
  const iga_tt* w[7] = {tts[0], tts[1], tts[2], tts[3], tts[4], tts[5], tts[6]};
  ops_from_weights_impl(ctx, st, w, M, K);
  if (load && tts[7]) {
    try {
      *load = load_tt(ctx, st, tts[7]);
    } catch (...) {
      delete *M;
      delete *K;
      *M = nullptr;
      *K = nullptr;
      throw;
    }
  }
  IGA_CUDA(cudaStreamSynchronize(ctx->stream));   // the handles are usable on any stream
}

static int interp_degree(const iga_space* space, int degree) {
  IGA_REQUIRE(space != nullptr, "null space");
  int p = std::max({space->degree[0], space->degree[1], space->degree[2]});
  return degree > 0 ? degree : 2 * p + 1;
}

iga_status iga_lowrank_assemble(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                                const iga_target* target, double tol, iga_op** M, iga_op** K,
                                iga_tt** load) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, lowrank_assemble_impl(ctx, geo, space, target, tol, 0, M, K, load))
}

iga_status iga_lowrank_assemble_interp(iga_ctx* ctx, const iga_geometry* geo,
                                       const iga_space* space, const iga_target* target,
                                       double tol, int degree, iga_op** M, iga_op** K,
                                       iga_tt** load) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, lowrank_assemble_impl(ctx, geo, space, target, tol, interp_degree(space, degree),
                                     M, K, load))
}

iga_status iga_weight_tts_interp(iga_ctx* ctx, const iga_geometry* geo, const iga_space* space,
                                 const iga_target* target, double tol, int degree,
                                 iga_tt* out[8]) {
  if (!ctx || !out) return IGA_EINVAL;
  for (int c = 0; c < 8; ++c) out[c] = nullptr;
  IGA_TRY(ctx, {
    SpaceTables st;
    build_space_tables(ctx, space, st);
    weight_tts_interp_impl(ctx, geo, st, target, tol, interp_degree(space, degree), out);
  })
}

iga_status iga_op_info(const iga_op* op, int n[3], int p[3], int* nblocks, int R[2],
                       size_t* bytes) {
  if (!op) return IGA_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (n) n[d] = op->n[d];
    if (p) p[d] = op->p[d];
  }
  if (nblocks) *nblocks = (int)op->blocks.size();
  if (R) {
    R[0] = 0;
    R[1] = 0;
    for (auto& b : op->blocks) { R[0] += b.R1; R[1] += b.R2; }
  }
  if (bytes) *bytes = op->bytes();
  return IGA_OK;
}

iga_status iga_op_block(const iga_op* op, int k, int R[2]) {
  if (!op || k < 0 || k >= (int)op->blocks.size() || !R) return IGA_EINVAL;
  R[0] = op->blocks[k].R1;
  R[1] = op->blocks[k].R2;
  return IGA_OK;
}

iga_status iga_op_bands(iga_ctx* ctx, const iga_op* op, int k, int d, double* host) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    IGA_REQUIRE(op && host && d >= 0 && d < 3 && k >= 0 && k < (int)op->blocks.size(),
                "op_bands: bad argument");
    const OpBlock& b = op->blocks[k];
    size_t cnt = d == 0 ? b.R1 : (d == 1 ? (size_t)b.R1 * b.R2 : b.R2);
    size_t len = (size_t)op->n[d] * (2 * op->p[d] + 1);
    IGA_CUDA(cudaMemcpyAsync(host, op->band64[d].p + b.off[d] * len, cnt * len * 8,
                             cudaMemcpyDeviceToHost, ctx->stream));
    IGA_CUDA(cudaStreamSynchronize(ctx->stream));
  })
}

void iga_op_destroy(iga_op* op) { delete op; }

iga_status iga_op_from_bands(iga_ctx* ctx, const int n[3], const int p[3], int nblocks,
                             const int* R, const double* const* bands, iga_op** out) {
  if (!ctx || !out || !n || !p) return IGA_EINVAL;
  *out = nullptr;
  IGA_TRY(ctx, *out = op_from_bands_impl(ctx, n, p, nblocks, R, bands))
}

iga_status iga_kron_apply(iga_ctx* ctx, const iga_op* A, int transpose, double alpha,
                          const void* x, double beta, void* y, iga_prec prec) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    if (prec == IGA_TF32 || prec == IGA_BF16) tc_flag_reset(ctx);
    if (transpose) kron_apply_transposed(ctx, A, alpha, x, beta, y, prec);
    else kron_apply_impl(ctx, A, alpha, x, beta, y, prec);
    if (prec == IGA_TF32 || prec == IGA_BF16) tc_flag_check(ctx, "kron_apply");
  })
}

iga_status iga_kkt_apply(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                         const void* z, void* out, iga_prec prec) {
  if (!ctx) return IGA_EINVAL;
  IGA_TRY(ctx, {
    if (prec == IGA_TF32 || prec == IGA_BF16) tc_flag_reset(ctx);
    kkt_apply_impl(ctx, M, K, beta, z, out, prec);
    if (prec == IGA_TF32 || prec == IGA_BF16) tc_flag_check(ctx, "kkt_apply");
  })
}

}  // extern "C"
