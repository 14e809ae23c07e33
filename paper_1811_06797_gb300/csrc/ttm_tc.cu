// TT-matrix Kronecker apply on the 5th-generation tensor cores (step a5,
// blocks with TT ranks above one):
//
//   y += alpha sum_{a,b} (A1[a] (x) A2[a,b] (x) A3[b]) x        (Sec. 5, eq. K_kron)
//
// with banded univariate factors of half-bandwidth P.  Written as three
// contractions,
//   Z[j2][b](j1, i3)  = sum_o3 A3[b](i3, o3) x(j1, j2, i3 + o3 - P)       mode 3
//   C[i2][a](j1, i3)  = sum_{j2, b} A2[a,b](i2, j2 - i2 + P) Z[j2][b](j1, i3)
//   y(i1, i2, i3)    += alpha sum_{a, o1} A1[a](i1, o1) C[i2][a](i1 + o1 - P, i3)
// the middle one is the dense rank contraction and runs as tcgen05.mma
// (TF32 operands, FP32 accumulation in tensor memory); modes 1 and 3 run on
// the CUDA cores in FP32.
//
// One CTA owns a tile of PTS = 128 H points (j1, i3): T3 consecutive i3 and
// T1 + 2P consecutive j1 (the mode-1 halo), T1 outputs along i1.  Each point
// is one tensor-memory lane.  The CTA streams over j2 = 0 .. n2-1:
//   * producer warps (one thread per point) form the slab Z[j2] in shared
//     memory in the canonical K-major layout of the MMA (rows = points,
//     K = b), and one of them starts a bulk copy (TMA, cp.async.bulk) of
//     column j2 of the A2 bands, pre-packed in global memory as the B operand
//     (rows (t, a), K = b, t = target offset) of the MMA;
//   * one thread issues the MMAs: slab j2 contributes to the 2P+1 outputs
//     i2 = j2 - P + t, whose FP32 accumulators form a ring of 2P+1 tensor-
//     memory column blocks (per half of the tile); contiguous targets are
//     one MMA with N = (targets) x R1p columns, and the first MMA into a
//     target (its first slab, first K step) overwrites the accumulator;
//   * epilogue warps drain an accumulator as soon as its last slab is in
//     (tcgen05.ld), apply the banded mode-1 product across the lanes
//     through shared memory and add the result into y.
// Z and the A2 column are double buffered, so the mode-3 product and the copy
// of slab j2+1 overlap the MMAs of slab j2, and the epilogue of i2 overlaps
// them too.  Every wait on an mbarrier is bounded: a wait that gives up sets
// the context's error flag, the CTA stops issuing work, waits (bounded) for
// its outstanding copies and MMAs, frees its tensor memory and exits; the
// host reports IGA_ETIMEOUT.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "iga_internal.cuh"

namespace iga {

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte distance of neighbouring core matrices along
// K, sbo = along M/N (8-row groups)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
  return d;
}

// instruction descriptor of kind::tf32 (fmt 2) or kind::f16 with BF16
// operands (fmt 1): D FP32, A and B K-major
__device__ __forceinline__ uint32_t idesc_mma(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

constexpr unsigned long long WAIT_POLLS = 1ull << 22;   // about a second with the back-off

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of the given parity; false after WAIT_POLLS
// polls or once another role has aborted
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort) {
  for (unsigned long long i = 0; i < WAIT_POLLS; ++i) {
    if (mbar_try(addr, parity)) return true;
    if (*abort) return false;
    if (i > 16) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(addr)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(addr),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
// tcgen05.ld without the wait: the registers are valid only after
// tc_wait_ld16 on the same array (which names them as read-write operands, so
// that no use is moved above the wait)
__device__ __forceinline__ void tc_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
// named barrier over the epilogue warps with an OR of `pred` handed to all
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred q, p;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, %2, %3, q;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}

}  // namespace

}  // namespace iga

namespace iga {

struct TtmTcArgs {
  const float* x;
  float* y;
  float alpha;
  const float* A1;     // (R1, n1, 2P+1) bands of direction 1
  const float* A3;     // (R2, n3, 2P+1) bands of direction 3
  const void* V;       // packed A2 columns: (n2, 2P+1, R1p x R2p MMA image), TF32 or BF16
  int n1, n2, n3;
  int R1, R2, R1p, R2p;
  int T1, T3, nt3;
  int NV;              // stages of the A2-column ring (2..4)
  int tcols;           // tensor-memory columns allocated (power of two >= 32)
  int* err;            // set to IGA_ETIMEOUT when a bounded wait gives up
};

// Row strides (floats) of the A1 and A3 tiles in shared memory: threads of a
// warp read rows of different i1 (A1) or i3 (A3) at once, so each stride is
// an odd multiple of four floats (16 bytes) modulo 128 bytes and the rows
// fall into distinct 16-byte bank groups.
__host__ __device__ inline int ttm_tc_s1(int R1p) { return R1p + ((R1p / 4) % 2 == 0 ? 4 : 0); }
__host__ __device__ inline int ttm_tc_s3(int P, int R2p) {
  const int w = (2 * P + 1) * R2p;
  return w + ((w / 4) % 2 == 0 ? 4 : 0);
}

// shared-memory footprint of one CTA in bytes (es = operand element size)
__host__ __device__ inline size_t ttm_tc_smem(int P, int H, int es, int NV, int R1p, int R2p,
                                              int T1, int T3) {
  const size_t B = 2 * P + 1, PTS = 128 * (size_t)H;
  size_t z = 2 * (size_t)H * 128 * R2p * es;             // Z slabs, two stages
  size_t v = (size_t)NV * B * (size_t)R1p * R2p * es;    // A2-column ring
  size_t a1 = (size_t)T1 * B * ttm_tc_s1(R1p) * 4, a3 = (size_t)T3 * ttm_tc_s3(P, R2p) * 4;
  size_t part = 2 * PTS * B * 4;
  return z + v + a1 + a3 + part + 256 + 16;
}

template <bool BF>
__device__ __forceinline__ void store_z_chunk(unsigned char* dst, const float* acc);
template <>
__device__ __forceinline__ void store_z_chunk<false>(unsigned char* dst, const float* acc) {
  *reinterpret_cast<float4*>(dst) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}
template <>
__device__ __forceinline__ void store_z_chunk<true>(unsigned char* dst, const float* acc) {
  __nv_bfloat162 h[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) h[u] = __floats2bfloat162_rn(acc[2 * u], acc[2 * u + 1]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

}  // namespace iga

namespace iga {

// Warp roles: [0, 4H) producers (one thread per point), [4H, 8H) epilogue
// (warp w reads tensor-memory lanes 32 (w % 4) ..), 8H the MMA issuer, 8H+1
// the loader of the A2-column ring.
template <int P, int H, bool BF>
__global__ void __launch_bounds__((8 * H + 2) * 32, 1) ttm_tc_kernel(const TtmTcArgs g) {
  constexpr int B = 2 * P + 1;
  constexpr int PTS = 128 * H;
  constexpr int NPW = 4 * H;             // producer warps = epilogue warps
  constexpr int MMA_WARP = 8 * H, LOAD_WARP = 8 * H + 1;
  constexpr int ES = BF ? 2 : 4;         // operand element size
  constexpr int EPC = 16 / ES;           // elements per 16-byte core-matrix row
  constexpr int KSTEP = 32 / ES;         // K of one MMA (two core matrices)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw;
  const int R1p = g.R1p, R2p = g.R2p, T1 = g.T1, T3 = g.T3, NV = g.NV;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const uint32_t ZH = 128u * R2p * ES, VT = (uint32_t)R1p * R2p * ES;
  const uint32_t SBO = (uint32_t)(R2p / EPC) * 128u;   // 8-row group stride of both operands
  const int S1 = ttm_tc_s1(R1p), S3 = ttm_tc_s3(P, R2p);
  unsigned char* zbuf = sm;
  unsigned char* vbuf = zbuf + 2 * H * ZH;
  float* a1s = reinterpret_cast<float*>(vbuf + (size_t)NV * B * VT);   // [(ii B + o) S1 + a]
  float* a3s = a1s + T1 * B * S1;                                       // [k S3 + o R2p + b]
  float* part = a3s + T3 * S3;
  uint64_t* bars = reinterpret_cast<uint64_t*>(part + 2 * PTS * B);
  constexpr int NA = B;                  // accumulator ring: the 2P+1 planes in use
  const uint32_t z_full = su32(bars), z_free = z_full + 16, v_full = z_full + 32,
                 v_free = v_full + 32, acc_full = v_free + 32, acc_empty = acc_full + 8 * NA,
                 mma_done = acc_empty + 8 * NA;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 32);
  volatile int* abort_ = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t3 = blockIdx.x % g.nt3, t1 = blockIdx.x / g.nt3;
  const int I1 = t1 * T1, I3 = t3 * T3;
  auto fail = [&]() {
    *abort_ = 1;
    atomicExch(g.err, (int)IGA_ETIMEOUT);
  };

  // ---- prologue: factor tiles, barriers, tensor memory
  for (int idx = threadIdx.x; idx < T1 * B * R1p; idx += blockDim.x) {
    const int a = idx % R1p, r = idx / R1p, o = r % B, i1 = I1 + r / B;
    a1s[r * S1 + a] = (a < g.R1 && i1 < n1) ? g.A1[((size_t)a * n1 + i1) * B + o] : 0.f;
  }
  for (int idx = threadIdx.x; idx < T3 * B * R2p; idx += blockDim.x) {
    const int b = idx % R2p, r = idx / R2p, o = r % B, k = r / B, i3 = I3 + k;
    a3s[k * S3 + o * R2p + b] = (b < g.R2 && i3 < n3) ? g.A3[((size_t)b * n3 + i3) * B + o] : 0.f;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(z_full + 8 * s, NPW);
      mbar_init(z_free + 8 * s, 1);
    }
    for (int s = 0; s < NV; ++s) {
      mbar_init(v_full + 8 * s, 1);
      mbar_init(v_free + 8 * s, 1);
    }
    for (int c = 0; c < NA; ++c) {
      mbar_init(acc_full + 8 * c, 1);
      mbar_init(acc_empty + 8 * c, NPW);
    }
    mbar_init(mma_done, 1);
    *abort_ = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(g.tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  // (no zeroing of the accumulators: the first MMA into a target overwrites)

  if (warp < NPW) {
    // ---- producers: mode-3 slabs
    const int pt = threadIdx.x;
    const int jj = pt / T3, k = pt - jj * T3, h = pt >> 7, m = pt & 127;
    const int j1 = I1 - P + jj, i3 = I3 + k;
    const bool valid = j1 >= 0 && j1 < n1 && i3 < n3;
    unsigned char* zrow = zbuf + h * ZH + (m >> 3) * SBO + (m & 7) * 16;
    const float4* a3r = reinterpret_cast<const float4*>(a3s + k * S3);
    const int R2q = R2p >> 2;
    // x of the next slab is loaded one iteration ahead (its latency hides
    // behind the wait and the arithmetic of the current slab)
    float xn[B];
    auto load_x = [&](int j2, float* xv) {
#pragma unroll
      for (int o = 0; o < B; ++o) {
        const int j3 = i3 + o - P;
        xv[o] = (valid && j3 >= 0 && j3 < n3) ? __ldg(g.x + ((size_t)j1 * n2 + j2) * n3 + j3)
                                              : 0.f;
      }
    };
    load_x(0, xn);
    for (int j2 = 0; j2 < n2; ++j2) {
      const int s = j2 & 1;
      float xw[B];
#pragma unroll
      for (int o = 0; o < B; ++o) xw[o] = xn[o];
      if (j2 + 1 < n2) load_x(j2 + 1, xn);
      if (j2 >= 2) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait(z_free + 8 * s, (uint32_t)((j2 >> 1) - 1) & 1, abort_);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) fail();
          break;
        }
      }
      unsigned char* zr = zrow + s * H * ZH;
      // two 16-byte chunks per pass (R2p / EPC is even): 2 EPC independent
      // accumulation chains of length B
      for (int c = 0; c < R2p / EPC; c += 2) {
        float acc[2 * EPC];
#pragma unroll
        for (int u = 0; u < 2 * EPC; ++u) acc[u] = 0.f;
#pragma unroll
        for (int o = 0; o < B; ++o) {
#pragma unroll
          for (int u4 = 0; u4 < EPC / 2; ++u4) {
            const float4 a = a3r[o * R2q + c * (EPC / 4) + u4];
            acc[4 * u4 + 0] = fmaf(a.x, xw[o], acc[4 * u4 + 0]);
            acc[4 * u4 + 1] = fmaf(a.y, xw[o], acc[4 * u4 + 1]);
            acc[4 * u4 + 2] = fmaf(a.z, xw[o], acc[4 * u4 + 2]);
            acc[4 * u4 + 3] = fmaf(a.w, xw[o], acc[4 * u4 + 3]);
          }
        }
        store_z_chunk<BF>(zr + c * 128, acc);
        store_z_chunk<BF>(zr + (c + 1) * 128, acc + EPC);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(z_full + 8 * s);
    }
  } else if (warp < 2 * NPW) {
    // ---- epilogue: drain accumulators, mode-1 product, y update
    const int e = warp - NPW, h = e >> 2, q = e & 3;
    const int pt = h * 128 + q * 32 + lane;
    const int jj = pt / T3, k = pt - jj * T3;
    const uint32_t la = tbase + ((uint32_t)(q * 32) << 16);
    // this thread's output column (i1, ., i3), if any; y of the next i2 is
    // loaded one iteration ahead
    const int oi1 = I1 + jj - P, oi3 = I3 + k;
    const bool outp = jj >= P && jj < P + T1 && oi1 < n1 && oi3 < n3;
    float* ycol = outp ? g.y + (size_t)oi1 * n2 * n3 + oi3 : nullptr;
    float ynext = outp ? ycol[0] : 0.f;
    for (int i2 = 0; i2 < n2; ++i2) {
      const int acc = i2 % NA;
      const float ycur = ynext;
      if (outp && i2 + 1 < n2) ynext = ycol[(size_t)(i2 + 1) * n3];
      bool ok = true;
      if (lane == 0) ok = mbar_wait(acc_full + 8 * acc, (uint32_t)(i2 / NA) & 1, abort_);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      // four partial sums per band offset o (independent FMA chains), added
      // at the end
      float c[B], cp[B][4];
#pragma unroll
      for (int o = 0; o < B; ++o)
#pragma unroll
        for (int u = 0; u < 4; ++u) cp[o][u] = 0.f;
      if (ok) {
        tc_fence_after();
        const uint32_t col0 = (uint32_t)((h * NA + acc) * R1p);
        // chunks of 16 columns (loading the next chunk while the current one
        // is used was measured slower)
        for (int ch = 0; ch < R1p; ch += 16) {
          uint32_t rn[16];
          tc_ld16_async(la + col0 + ch, rn);
          tc_wait_ld16(rn);
          float d[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) d[j] = __uint_as_float(rn[j]);
#pragma unroll
          for (int o = 0; o < B; ++o) {
            const int ii = jj - o;
            if (ii >= 0 && ii < T1) {
              const float4* ar = reinterpret_cast<const float4*>(a1s + (ii * B + o) * S1 + ch);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 av = ar[u];
                cp[o][0] = fmaf(av.x, d[4 * u], cp[o][0]);
                cp[o][1] = fmaf(av.y, d[4 * u + 1], cp[o][1]);
                cp[o][2] = fmaf(av.z, d[4 * u + 2], cp[o][2]);
                cp[o][3] = fmaf(av.w, d[4 * u + 3], cp[o][3]);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty + 8 * acc);
      }
#pragma unroll
      for (int o = 0; o < B; ++o) c[o] = (cp[o][0] + cp[o][1]) + (cp[o][2] + cp[o][3]);
      float* pb = part + (i2 & 1) * PTS * B;
#pragma unroll
      for (int o = 0; o < B; ++o) pb[pt * B + o] = c[o];
      const bool bad = bar_or(1, NPW * 32, !ok || *abort_ != 0);
      if (bad) {
        if (!ok && lane == 0) fail();
        break;
      }
      if (outp) {
        const int ii = jj - P;
        float v = 0.f;
#pragma unroll
        for (int o = 0; o < B; ++o) v += pb[((ii + o) * T3 + k) * B + o];
        ycol[(size_t)i2 * n3] = fmaf(g.alpha, v, ycur);
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      // ---- MMA issuer
      const int maxrun = 256 / R1p;
      // `first`: these targets start with this slab, so the MMA of the first
      // K step overwrites the accumulator (no zeroing pass in the epilogue)
      auto issue = [&](int j2, int s, int sv, int ta, int tb, bool first) {
        int t = ta;
        while (t <= tb) {
          const int c0 = (j2 - P + t) % NA;
          const int len = min(min(tb - t + 1, NA - c0), maxrun);
          const uint32_t idesc = idesc_mma(BF ? 1 : 2, 128, len * R1p);
          for (int kb = 0; kb < R2p / KSTEP; ++kb) {
            const uint64_t bd =
                umma_desc(su32(vbuf + ((size_t)sv * B + t) * VT) + kb * 256, 128, SBO);
#pragma unroll
            for (int h = 0; h < H; ++h) {
              const uint64_t ad = umma_desc(su32(zbuf + (s * H + h) * ZH) + kb * 256, 128, SBO);
              const uint32_t acc = (first && kb == 0) ? 0u : 1u;
              if (BF) tc_mma_bf16(tbase + (uint32_t)((h * NA + c0) * R1p), ad, bd, idesc, acc);
              else tc_mma_tf32(tbase + (uint32_t)((h * NA + c0) * R1p), ad, bd, idesc, acc);
            }
          }
          t += len;
        }
      };
      for (int j2 = 0; j2 < n2; ++j2) {
        const int s = j2 & 1, sv = j2 % NV;
        if (!mbar_wait(z_full + 8 * s, (uint32_t)(j2 >> 1) & 1, abort_) ||
            !mbar_wait(v_full + 8 * sv, (uint32_t)(j2 / NV) & 1, abort_)) {
          fail();
          break;
        }
        tc_fence_after();
        const int tlo = max(0, P - j2), thi = min(B - 1, n2 - 1 - j2 + P);
        if (j2 == 0) {
          // every target of the first slab starts here
          issue(j2, s, sv, tlo, thi, true);
        } else {
          // target i2 = j2 + P starts with this slab (the others continue)
          const bool newt = j2 + P < n2;
          issue(j2, s, sv, tlo, newt ? B - 2 : thi, false);
          // accumulator i2 = j2 - P is complete with these MMAs: hand it to
          // the epilogue before waiting for the slot of the new target, so
          // that the epilogue of i2 runs under the MMAs of the next slab
          if (j2 - P >= 0) tc_commit(acc_full + 8 * ((j2 - P) % NA));
          if (newt) {
            const int i2n = j2 + P;
            if (i2n >= NA &&
                !mbar_wait(acc_empty + 8 * (i2n % NA), (uint32_t)(i2n / NA - 1) & 1, abort_)) {
              fail();
              break;
            }
            tc_fence_after();
            issue(j2, s, sv, B - 1, B - 1, true);
          }
        }
        tc_commit(z_free + 8 * s);
        tc_commit(v_free + 8 * sv);
        if (j2 == n2 - 1)
          for (int i2 = max(0, j2 - P + 1); i2 < n2; ++i2) tc_commit(acc_full + 8 * (i2 % NA));
      }
      // every MMA issued must finish before the tensor memory is released
      tc_commit(mma_done);
      volatile int never = 0;
      if (!mbar_wait(mma_done, 0, &never)) fail();
    }
  } else if (warp == LOAD_WARP && lane == 0) {
    // ---- loader: bulk copies of the A2 columns into the NV-stage ring
    int last[4] = {-1, -1, -1, -1};
    const unsigned char* V = static_cast<const unsigned char*>(g.V);
    for (int j2 = 0; j2 < n2; ++j2) {
      const int sv = j2 % NV;
      if (j2 >= NV && !mbar_wait(v_free + 8 * sv, (uint32_t)(j2 / NV - 1) & 1, abort_)) {
        fail();
        break;
      }
      mbar_expect_tx(v_full + 8 * sv, (uint32_t)B * VT);
      bulk_g2s(su32(vbuf + (size_t)sv * B * VT), V + (size_t)j2 * B * VT, (uint32_t)B * VT,
               v_full + 8 * sv);
      last[sv] = j2;
    }
    // copies still in flight must land before the CTA exits
    for (int sv = 0; sv < NV; ++sv)
      if (last[sv] >= 0) {
        volatile int never = 0;
        if (!mbar_wait(v_full + 8 * sv, (uint32_t)(last[sv] / NV) & 1, &never)) fail();
      }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tcols)
                 : "memory");
  }
}

}  // namespace iga

namespace iga {

// Column j2 of the A2 bands of one block as the B operand of the MMAs of slab
// j2: V[j2][t] is an R1p x R2p K-major image (core matrices of 8 rows x 16
// bytes) of A2[a][b](i2, 2P - t), i2 = j2 - P + t, zero outside the ranks
// and the matrix; TF32 keeps the FP32 bits, BF16 rounds to nearest.
template <typename E>
__global__ void ttm_tc_pack_kernel(const float* __restrict__ A2, int R1, int R2, int n2, int P,
                                   int R1p, int R2p, E* __restrict__ V) {
  constexpr int EPC = 16 / (int)sizeof(E);
  const int B = 2 * P + 1;
  const size_t img = (size_t)R1p * R2p;
  const size_t total = (size_t)n2 * B * img;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t jt = idx / img;
    const int e = (int)(idx - jt * img);
    const int t = (int)(jt % B), j2 = (int)(jt / B);
    // e = (a/8) 8 R2p + (b/EPC) 8 EPC + (a%8) EPC + b%EPC
    const int g8 = e / (8 * R2p), r8 = e - g8 * 8 * R2p;
    const int c = r8 / (8 * EPC), r = r8 - c * 8 * EPC;
    const int a = g8 * 8 + r / EPC, b = c * EPC + r % EPC;
    const int i2 = j2 - P + t;
    float v = 0.f;
    if (a < R1 && b < R2 && i2 >= 0 && i2 < n2)
      v = A2[(((size_t)a * R2 + b) * n2 + i2) * B + (2 * P - t)];
    if constexpr (sizeof(E) == 2) V[idx] = __float2bfloat16_rn(v);
    else V[idx] = v;
  }
}

struct TtmTcPlan {
  bool ok = false;
  int H = 1, T1 = 0, T3 = 0, R1p = 0, R2p = 0, NV = 2, tcols = 0;
  size_t smem = 0;
};

static constexpr size_t TTM_TC_SMEM_MAX = 227 * 1024;

// Tile plan.  Per slab a CTA spends about H * 128 * B * R1p * R2p / rate
// cycles in MMAs (rate: TF32 ~1500, BF16 ~3000 multiply-adds per SM and
// cycle) plus about 1500 H cycles of CUDA-core work (the mode-3 and mode-1
// products of 128 H points), and waits up to ~2500 cycles for one A2-column
// copy, which an NV-stage ring spreads over NV - 1 slabs; the plan with the
// least (waves of CTAs) x (cycles per slab) that fits tensor memory
// (H B R1p <= 512 columns) and shared memory wins.  The accumulator ring
// holds the 2P+1 planes in use at once: deeper rings (up to 9 slots at
// H = 1) were measured slower (4.58 against 4.38 ms at 320^3, and they
// exclude H = 2, which the 512^3 shape needs: 16.8 against 9.9 ms).
static TtmTcPlan ttm_tc_plan(int n1, int n3, int R1, int R2, int P, bool bf16, int nsm) {
  TtmTcPlan best;
  const int B = 2 * P + 1, es = bf16 ? 2 : 4, kstep = bf16 ? 16 : 8;
  const int R1p = (R1 + 15) / 16 * 16, R2p = (R2 + kstep - 1) / kstep * kstep;
  if (R1p > 256 || R2p > 256 || P < 1 || P > 3) return best;
  const double rate = bf16 ? 3000.0 : 1500.0, vlat = 2500.0;
  double bestc = 1e300;
  for (int H = 2; H >= 1; --H) {
    if (H * B * R1p > 512) continue;
    for (int NV = 4; NV >= 2; --NV)
      for (int T3 : {16, 8, 4}) {
        const int T1 = 128 * H / T3 - 2 * P;
        if (T1 < 1) continue;
        const size_t smem = ttm_tc_smem(P, H, es, NV, R1p, R2p, T1, T3) + 1024;
        if (smem > TTM_TC_SMEM_MAX) continue;
        const long nt = (long)((n1 + T1 - 1) / T1) * ((n3 + T3 - 1) / T3);
        // per-slab cost: a fixed part (barrier hand-offs, the copy latency
        // spread over NV - 1 slabs) and a part proportional to the points
        const double slab = vlat / (NV - 1) + H * (128.0 * B * R1p * R2p / rate + 1500.0);
        const double c = std::ceil((double)nt / nsm) * slab;
        if (c < bestc * (1 - 1e-9)) {
          bestc = c;
          best.ok = true;
          best.H = H; best.T1 = T1; best.T3 = T3; best.R1p = R1p; best.R2p = R2p; best.NV = NV;
          best.smem = smem;
          int tc = 32;
          while (tc < H * B * R1p) tc *= 2;
          best.tcols = tc;
        }
      }
  }
  return best;
}

bool ttm_tc_supported(int n1, int n3, int R1, int R2, int P, int nsm) {
  return ttm_tc_plan(n1, n3, R1, R2, P, false, nsm).ok;
}

template <int P, int H, bool BF>
static void ttm_tc_launch(iga_ctx* ctx, const TtmTcArgs& a, const TtmTcPlan& pl, unsigned grid) {
  func_attr(ttm_tc_kernel<P, H, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  IGA_LAUNCH(ctx, (ttm_tc_kernel<P, H, BF>), grid, (8 * H + 2) * 32, pl.smem, a);
}

template <bool BF>
static bool ttm_tc_dispatch(iga_ctx* ctx, const TtmTcArgs& a, const TtmTcPlan& pl, int P,
                            unsigned grid) {
  switch (P * 2 + (pl.H - 1)) {
    case 2: ttm_tc_launch<1, 1, BF>(ctx, a, pl, grid); return true;
    case 3: ttm_tc_launch<1, 2, BF>(ctx, a, pl, grid); return true;
    case 4: ttm_tc_launch<2, 1, BF>(ctx, a, pl, grid); return true;
    case 5: ttm_tc_launch<2, 2, BF>(ctx, a, pl, grid); return true;
    case 6: ttm_tc_launch<3, 1, BF>(ctx, a, pl, grid); return true;
    case 7: ttm_tc_launch<3, 2, BF>(ctx, a, pl, grid); return true;
    default: return false;
  }
}

// y += alpha (sum_{a,b} A1[a] (x) A2[a,b] (x) A3[b]) x for one TT-matrix block
// in FP32 storage with the rank contraction on the tensor cores (TF32, or
// BF16 operands when bf16), FP32 accumulation.  Returns false (and launches
// nothing) when the block's shape has no plan.
bool ttm_tc_block(iga_ctx* ctx, const float* A1, const float* A2, const float* A3, int R1, int R2,
                  const int* n, int P, float alpha, const float* x, float* y, bool bf16) {
  const TtmTcPlan pl = ttm_tc_plan(n[0], n[2], R1, R2, P, bf16, ctx->nsm);
  if (!pl.ok) return false;
  const int B = 2 * P + 1;
  const size_t vcount = (size_t)n[1] * B * pl.R1p * pl.R2p;
  void* V = scratch<char>(ctx, SLOT_TTM_W, vcount * (bf16 ? 2 : 4));
  const unsigned pg = (unsigned)std::min<size_t>((vcount + 255) / 256, 4096);
  if (bf16)
    IGA_LAUNCH(ctx, ttm_tc_pack_kernel<__nv_bfloat16>, pg, 256, 0, A2, R1, R2, n[1], P, pl.R1p,
               pl.R2p, static_cast<__nv_bfloat16*>(V));
  else
    IGA_LAUNCH(ctx, ttm_tc_pack_kernel<float>, pg, 256, 0, A2, R1, R2, n[1], P, pl.R1p, pl.R2p,
               static_cast<float*>(V));
  TtmTcArgs a{};
  a.x = x; a.y = y; a.alpha = alpha;
  a.A1 = A1; a.A3 = A3; a.V = V;
  a.n1 = n[0]; a.n2 = n[1]; a.n3 = n[2];
  a.R1 = R1; a.R2 = R2; a.R1p = pl.R1p; a.R2p = pl.R2p;
  a.T1 = pl.T1; a.T3 = pl.T3; a.nt3 = (n[2] + pl.T3 - 1) / pl.T3;
  a.NV = pl.NV;
  a.tcols = pl.tcols;
  a.err = ctx->dflag + 1;
  const unsigned grid = (unsigned)(((n[0] + pl.T1 - 1) / pl.T1) * a.nt3);
  {
    // algorithmic: mode 3 and mode 1 banded products and the rank
    // contraction; x read once, y read and written once
    const double N = (double)n[0] * n[1] * n[2];
    prof_count(ctx, N * 4.0 * 3.0, 2.0 * B * N * (R2 + (double)R1 * R2 + R1));
  }
  return bf16 ? ttm_tc_dispatch<true>(ctx, a, pl, P, grid)
              : ttm_tc_dispatch<false>(ctx, a, pl, P, grid);
}

}  // namespace iga
