// Dense products on the 5th-generation tensor cores in TF32 with FP32
// accumulation, for the large interface contractions of the local systems of
// block AMEn (Sec. 5, eq. KKT_red: the local operator applied factor by
// factor as Phi_R, the banded core, then Phi_L) when the solve runs with
// IGA_TF32:
//
//   C_i = alpha op(A_i) op(B_i) + beta C_i,   op(A) M x K, op(B) K x N,
//
// FP32 storage, row-major (A[m lda + k], or A[k lda + m] when transposed;
// B[k ldb + n], or B[n ldb + k]; C[m ldc + n], or C[n ldc + m] when tC).
// One CTA owns 128 rows of C (one tensor-memory lane per row) and NT <= 256
// columns (the D matrix of the MMA, FP32 in tensor memory); K is consumed in
// chunks of 32: the four warps stage op(A) (128 x 32) and op(B) (NT x 32) in
// shared memory in the canonical K-major layout (8-row x 16-byte core
// matrices, one warp writes one core matrix per step, conflict-free), one
// thread issues four tcgen05.mma of K = 8, and the next chunk is staged into
// the other buffer while they run.  The epilogue reads the accumulator with
// tcgen05.ld.  Bounded mbarrier waits: a wait that gives up sets the
// context's error flag and the CTA skips its remaining work.
#include <algorithm>

#include "iga_internal.cuh"

namespace iga {

namespace {

__device__ __forceinline__ uint32_t g_su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t g_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ bool g_wait(uint32_t addr, uint32_t parity) {
  for (unsigned long long i = 0; i < (1ull << 22); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i > 16) __nanosleep(64);
  }
  return false;
}

}  // namespace

constexpr int TCG_KC = 32;          // K per stage
constexpr int TCG_THREADS = 128;

struct TcGemmArgs {
  int M, N, K;
  float alpha, beta;
  const float* A;
  int lda;
  long long sA;
  const float* B;
  int ldb;
  long long sB;
  float* C;
  int ldc;
  long long sC;
  int tA, tB, tC;
  int vecA, vecB;        // 16-byte loads (aligned base, stride and batch stride)
  int NT;                // columns per CTA (multiple of 16, <= 256)
  int tcols;             // tensor-memory columns allocated
  int* err;
};

__global__ void __launch_bounds__(TCG_THREADS) tc_gemm_tf32_kernel(const TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int NT = g.NT;
  const uint32_t AST = 128u * TCG_KC * 4, BST = (uint32_t)NT * TCG_KC * 4;
  const uint32_t SBO = (TCG_KC / 4) * 128u;            // 8-row group stride
  unsigned char* sA = smem_raw;                        // 2 stages
  unsigned char* sB = sA + 2 * AST;                    // 2 stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * BST);   // done[2], fin
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  volatile int* bad = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
  const int bz = blockIdx.z;
  const float* A = g.A + bz * g.sA;
  const float* B = g.B + bz * g.sB;
  float* C = g.C + bz * g.sC;
  const uint32_t done0 = g_su32(bars), done1 = done0 + 8, fin = done0 + 16;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fin) : "memory");
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_su32(tslot)),
                 "r"(g.tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const uint32_t idesc =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const int nchunk = (g.K + TCG_KC - 1) / TCG_KC;
  // lane -> position inside one core matrix (8 rows x 4 elements): for a
  // K-contiguous operand the lanes walk k fastest, for a transposed one the
  // rows fastest; either way the 32 lanes write one 128-byte core matrix
  for (int c = 0; c < nchunk; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      if (!g_wait(s ? done1 : done0, (uint32_t)((c >> 1) - 1) & 1)) {
        *bad = 1;
        atomicExch(g.err, (int)IGA_ETIMEOUT);
      }
    }
    __syncthreads();
    if (*bad) break;
    const int k0 = c * TCG_KC;
    unsigned char* a_st = sA + s * AST;
    unsigned char* b_st = sB + s * BST;
    // op(A): 16 row groups x 8 k-quads = 128 core matrices
    if (g.vecA) {
      // 16-byte loads of four elements contiguous in memory (k for a
      // row-major A, m for a transposed one): a warp covers four core matrices
      for (int cm0 = warp * 4; cm0 < 128; cm0 += 16) {
        const int cm = cm0 + (lane >> 3), rg = cm >> 3, kq = cm & 7, t = lane & 7;
        if (!g.tA) {
          const int m = m0 + rg * 8 + t, k = k0 + kq * 4;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (m < g.M && k + 3 < g.K)
            v = *reinterpret_cast<const float4*>(A + (size_t)m * g.lda + k);
          else if (m < g.M)
            for (int u = 0; u < 4; ++u)
              if (k + u < g.K) (&v.x)[u] = A[(size_t)m * g.lda + k + u];
          *reinterpret_cast<float4*>(a_st + rg * SBO + kq * 128 + t * 16) = v;
        } else {
          const int kk = t & 3, mq = t >> 2;
          const int m = m0 + rg * 8 + mq * 4, k = k0 + kq * 4 + kk;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (k < g.K && m + 3 < g.M)
            v = *reinterpret_cast<const float4*>(A + (size_t)k * g.lda + m);
          else if (k < g.K)
            for (int u = 0; u < 4; ++u)
              if (m + u < g.M) (&v.x)[u] = A[(size_t)k * g.lda + m + u];
          unsigned char* base = a_st + rg * SBO + kq * 128 + (mq * 4) * 16 + kk * 4;
          for (int u = 0; u < 4; ++u) *reinterpret_cast<float*>(base + u * 16) = (&v.x)[u];
        }
      }
    } else {
      for (int cm = warp; cm < 128; cm += 4) {
        const int rg = cm >> 3, kq = cm & 7;
        int r, kk;
        if (g.tA) { r = lane & 7; kk = lane >> 3; }
        else { r = lane >> 2; kk = lane & 3; }
        const int m = m0 + rg * 8 + r, k = k0 + kq * 4 + kk;
        float v = 0.f;
        if (m < g.M && k < g.K) v = g.tA ? A[(size_t)k * g.lda + m] : A[(size_t)m * g.lda + k];
        *reinterpret_cast<float*>(a_st + rg * SBO + kq * 128 + r * 16 + kk * 4) = v;
      }
    }
    // op(B)^T: NT/8 row groups (rows n) x 8 k-quads
    if (g.vecB) {
      for (int cm0 = warp * 4; cm0 < (NT / 8) * 8; cm0 += 16) {
        const int cm = cm0 + (lane >> 3), rg = cm >> 3, kq = cm & 7, t = lane & 7;
        if (cm >= (NT / 8) * 8) continue;
        if (g.tB) {
          const int n = n0 + rg * 8 + t, k = k0 + kq * 4;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (n < g.N && k + 3 < g.K)
            v = *reinterpret_cast<const float4*>(B + (size_t)n * g.ldb + k);
          else if (n < g.N)
            for (int u = 0; u < 4; ++u)
              if (k + u < g.K) (&v.x)[u] = B[(size_t)n * g.ldb + k + u];
          *reinterpret_cast<float4*>(b_st + rg * SBO + kq * 128 + t * 16) = v;
        } else {
          const int kk = t & 3, nq = t >> 2;
          const int n = n0 + rg * 8 + nq * 4, k = k0 + kq * 4 + kk;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (k < g.K && n + 3 < g.N)
            v = *reinterpret_cast<const float4*>(B + (size_t)k * g.ldb + n);
          else if (k < g.K)
            for (int u = 0; u < 4; ++u)
              if (n + u < g.N) (&v.x)[u] = B[(size_t)k * g.ldb + n + u];
          unsigned char* base = b_st + rg * SBO + kq * 128 + (nq * 4) * 16 + kk * 4;
          for (int u = 0; u < 4; ++u) *reinterpret_cast<float*>(base + u * 16) = (&v.x)[u];
        }
      }
    } else {
      for (int cm = warp; cm < (NT / 8) * 8; cm += 4) {
        const int rg = cm >> 3, kq = cm & 7;
        int r, kk;
        if (g.tB) { r = lane >> 2; kk = lane & 3; }
        else { r = lane & 7; kk = lane >> 3; }
        const int n = n0 + rg * 8 + r, k = k0 + kq * 4 + kk;
        float v = 0.f;
        if (n < g.N && k < g.K) v = g.tB ? B[(size_t)n * g.ldb + k] : B[(size_t)k * g.ldb + n];
        *reinterpret_cast<float*>(b_st + rg * SBO + kq * 128 + r * 16 + kk * 4) = v;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int ks = 0; ks < TCG_KC / 8; ++ks) {
        const uint64_t ad = g_desc(g_su32(a_st) + ks * 256, 128, SBO);
        const uint64_t bd = g_desc(g_su32(b_st) + ks * 256, 128, SBO);
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tbase),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s ? done1 : done0)
                   : "memory");
    }
  }
  // all MMAs issued must have finished before the accumulator is read and
  // the tensor memory released
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(fin)
                 : "memory");
  }
  bool ok = g_wait(fin, 0);
  if (!ok) atomicExch(g.err, (int)IGA_ETIMEOUT);
  ok = __all_sync(0xffffffffu, ok) && !*bad;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int m = m0 + warp * 32 + lane;
    const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < g.N) {
            float* cp = g.tC ? C + (size_t)n * g.ldc + m : C + (size_t)m * g.ldc + n;
            const float v = g.alpha * __uint_as_float(r[j]);
            *cp = g.beta == 0.f ? v : fmaf(g.beta, *cp, v);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tcols)
                 : "memory");
  }
}

void tc_gemm_tf32(iga_ctx* ctx, bool tA, bool tB, bool tC, int M, int N, int K, float alpha,
                  const float* A, int lda, long long sA, const float* B, int ldb, long long sB,
                  float beta, float* C, int ldc, long long sC, int count) {
  if (M <= 0 || N <= 0 || count <= 0) return;
  TcGemmArgs a{};
  a.M = M; a.N = N; a.K = K; a.alpha = alpha; a.beta = beta;
  a.A = A; a.lda = lda; a.sA = sA; a.B = B; a.ldb = ldb; a.sB = sB;
  a.C = C; a.ldc = ldc; a.sC = sC;
  a.tA = tA; a.tB = tB; a.tC = tC;
  // 16-byte operand loads when every row (or column) starts 16-byte aligned
  auto al16 = [](const float* p, int ld, long long st) {
    return ((uintptr_t)p % 16 == 0) && ld % 4 == 0 && st % 4 == 0;
  };
  a.vecA = al16(A, lda, sA);
  a.vecB = al16(B, ldb, sB);
  a.NT = std::min(256, (N + 15) / 16 * 16);
  a.tcols = 32;
  while (a.tcols < a.NT) a.tcols *= 2;
  a.err = ctx->dflag + 1;
  const size_t smem = 2 * (128 + (size_t)a.NT) * TCG_KC * 4 + 64;
  func_attr(tc_gemm_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int b0 = 0; b0 < count; b0 += 65535) {
    const int nb = std::min(65535, count - b0);
    TcGemmArgs ab = a;
    ab.A = A + b0 * sA;
    ab.B = B + b0 * sB;
    ab.C = C + b0 * sC;
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + a.NT - 1) / a.NT), (unsigned)nb);
    prof_count(ctx, (double)nb * ((double)M * K + (double)K * N + (double)M * N) * 4.0,
               2.0 * nb * (double)M * N * K);
    IGA_LAUNCH(ctx, tc_gemm_tf32_kernel, grid, TCG_THREADS, smem, ab);
  }
}

}  // namespace iga
