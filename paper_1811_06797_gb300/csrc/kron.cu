// Kronecker-sum operator apply (step a5):
//   y = alpha * sum_blocks sum_{r1,r2} (A1[r1] (x) A2[r1,r2] (x) A3[r2]) x + beta * y
// (Sec. 5 eqs. M_kron / K_kron; the univariate factors are banded with
// half-bandwidth p).
//
// Rank-1 blocks (every block of the configurations with exact-rank
// geometry) go through one fused kernel: a CTA owns an output tile
// T1 x T2 x T3, computes the mode-3 product on the tile plus its halo in
// directions 1 and 2 (reading x through L1), then the mode-2 and mode-1
// products in shared memory, for every term in turn, and writes y once.
// x is read from HBM once per tile (halo re-reads hit L1/L2) and y written
// once.  TT-matrix blocks (ranks > 1) in TF32 / BF16 go through the fused
// tcgen05 kernel of ttm_tc.cu; in FP64 and plain FP32 they use staged
// single-mode products with full-size intermediates and the library's batched
// GEMM (gemm.cu) for the rank contraction.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "iga_internal.cuh"

namespace iga {

constexpr int KRON_MAXTERMS = 32;
constexpr int KRON_THREADS = 256;
constexpr int KRON_MO = 8;         // outputs per thread and output field held in registers

// One launch of the fused rank-1 apply.  Term t reads input x[xin[t]], forms
// its three banded mode products on the tile and adds coef[t][o] times the
// result to output o (o < NY); finally y[o] = acc_o + beta[o] y[o].  One
// operator is NY = 1 with one input; the KKT operator is NY = 3 with the
// three fields as inputs, so that each product feeds every block row that
// uses it (M u enters rows two and three).
template <typename T>
struct KronJob {
  const T* b[3][KRON_MAXTERMS];
  T coef[KRON_MAXTERMS][3];
  unsigned char cmask[KRON_MAXTERMS];   // bit o set when coef[t][o] != 0
  unsigned char xin[KRON_MAXTERMS];
  int nterms;
  const T* x[5];
  T* y[3];
  T beta[3];
};

struct KronTile {
  int n1, n2, n3;
  int T1, T2, T3;
  int nt1, nt2, nt3;     // tiles along 1, 2 and 3
};

template <typename T, int P, int NY>
__global__ void __launch_bounds__(KRON_THREADS)
kron_rank1_kernel(const __grid_constant__ KronJob<T> job, KronTile g) {
  constexpr int B = 2 * P + 1;
  extern __shared__ unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int T1 = g.T1, T2 = g.T2, T3 = g.T3;
  const int H1 = T1 + 2 * P, H2 = T2 + 2 * P;
  T* z3 = sm;                                   // H1 * H2 * T3
  T* z2 = z3 + (size_t)H1 * H2 * T3;            // H1 * T2 * T3
  T* a1 = z2 + (size_t)H1 * T2 * T3;            // T1 * B
  T* a2 = a1 + T1 * B;                          // T2 * B
  T* a3 = a2 + T2 * B;                          // T3 * B
  const int T3h = T3 + 2 * P;
  T* xs = a3 + T3 * B;                          // H1 * H2 * T3h: the x slab of the tile
  int bid = blockIdx.x;
  int t3 = bid % g.nt3;
  int t2 = (bid / g.nt3) % g.nt2;
  int t1 = bid / (g.nt3 * g.nt2);
  const int I1 = t1 * T1, I2 = t2 * T2, I3 = t3 * T3;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int nout = T1 * T2 * T3;
  T acc[NY][KRON_MO];
#pragma unroll
  for (int o = 0; o < NY; ++o)
#pragma unroll
    for (int k = 0; k < KRON_MO; ++k) acc[o][k] = T(0);

  int staged = -1;
  for (int t = 0; t < job.nterms; ++t) {
    const T* A1 = job.b[0][t];
    const T* A2 = job.b[1][t];
    const T* A3 = job.b[2][t];
    const int xi = job.xin[t];
    for (int idx = threadIdx.x; idx < (T1 + T2 + T3) * B; idx += blockDim.x) {
      int r = idx / B, o = idx - r * B;
      T v = T(0);
      if (r < T1) { int i = I1 + r; if (i < n1) v = A1[(size_t)i * B + o]; a1[r * B + o] = v; }
      else if (r < T1 + T2) { int i = I2 + r - T1; if (i < n2) v = A2[(size_t)i * B + o]; a2[(r - T1) * B + o] = v; }
      else { int i = I3 + r - T1 - T2; if (i < n3) v = A3[(size_t)i * B + o]; a3[(r - T1 - T2) * B + o] = v; }
    }
    if (xi != staged) {
      // the (H1 x H2 x T3+2P) slab of this term's input, zero outside the
      // domain, read once per input (the terms are grouped by input)
      const T* __restrict__ x =
          xi == 0 ? job.x[0]
                  : (xi == 1 ? job.x[1] : (xi == 2 ? job.x[2] : (xi == 3 ? job.x[3] : job.x[4])));
      for (int idx = threadIdx.x; idx < H1 * H2 * T3h; idx += blockDim.x) {
        const int kk = idx % T3h;
        const int ac = idx / T3h;
        const int c = ac % H2, a = ac / H2;
        const int j1 = I1 + a - P, j2 = I2 + c - P, j3 = I3 + kk - P;
        T v = T(0);
        if (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < n2 && j3 >= 0 && j3 < n3)
          v = __ldg(x + ((size_t)j1 * n2 + j2) * n3 + j3);
        xs[idx] = v;
      }
      staged = xi;
    }
    __syncthreads();
    // mode 3 on the (H1 x H2) halo slab of the i3 tile, from shared memory
    for (int idx = threadIdx.x; idx < H1 * H2 * T3; idx += blockDim.x) {
      int k = idx % T3;
      int ac = idx / T3;
      int c = ac % H2, a = ac / H2;
      int j1 = I1 + a - P, j2 = I2 + c - P, i3 = I3 + k;
      T s = T(0);
      if (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < n2 && i3 < n3) {
        const T* xr = xs + (size_t)ac * T3h + k;
#pragma unroll
        for (int o = 0; o < B; ++o) s += a3[k * B + o] * xr[o];
      }
      z3[idx] = s;
    }
    __syncthreads();
    // mode 2: z2[a][c][k] = sum_o A2(I2+c, I2+c+o-P) z3[a][c+o][k]; rows a
    // outside the domain and columns past n2 stay zero without arithmetic
    for (int idx = threadIdx.x; idx < H1 * T2 * T3; idx += blockDim.x) {
      int k = idx % T3;
      int ac = idx / T3;
      int c = ac % T2, a = ac / T2;
      int j1 = I1 + a - P;
      T s = T(0);
      if (j1 >= 0 && j1 < n1 && I2 + c < n2) {
#pragma unroll
        for (int o = 0; o < B; ++o) s += a2[c * B + o] * z3[((size_t)a * H2 + c + o) * T3 + k];
      }
      z2[idx] = s;
    }
    __syncthreads();
    // mode 1 into the register accumulators of every output the term feeds
    // (which outputs from an integer mask: an FP64 comparison per output and
    // point would occupy the narrow FP64 pipe)
    T cf[NY];
#pragma unroll
    for (int o = 0; o < NY; ++o) cf[o] = job.coef[t][o];
    const unsigned cm = job.cmask[t];
#pragma unroll
    for (int m = 0; m < KRON_MO; ++m) {
      int idx = threadIdx.x + m * KRON_THREADS;
      if (idx < nout) {
        int k = idx % T3;
        int ac = idx / T3;
        int c = ac % T2, a = ac / T2;
        T s = T(0);
#pragma unroll
        for (int o = 0; o < B; ++o) s += a1[a * B + o] * z2[((size_t)(a + o) * T2 + c) * T3 + k];
#pragma unroll
        for (int o = 0; o < NY; ++o)
          if (cm & (1u << o)) acc[o][m] = fma(cf[o], s, acc[o][m]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < KRON_MO; ++m) {
    int idx = threadIdx.x + m * KRON_THREADS;
    if (idx < nout) {
      int k = idx % T3;
      int ac = idx / T3;
      int c = ac % T2, a = ac / T2;
      int i1 = I1 + a, i2 = I2 + c, i3 = I3 + k;
      if (i1 < n1 && i2 < n2 && i3 < n3) {
        size_t off = ((size_t)i1 * n2 + i2) * n3 + i3;
#pragma unroll
        for (int o = 0; o < NY; ++o) {
          T v = acc[o][m];
          if (job.beta[o] != T(0)) v += job.beta[o] * job.y[o][off];
          job.y[o][off] = v;
        }
      }
    }
  }
}

template <typename T>
__global__ void scale_kernel(T* __restrict__ y, size_t n, T a) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] *= a;
}

// single-mode banded product:  y (+)= A (along `mode`) x,  A band (n_mode, 2P+1)
template <typename T, int P>
__global__ void mode_product_kernel(const T* __restrict__ A, int mode, int n1, int n2, int n3,
                                    const T* __restrict__ x, T* __restrict__ y, T alpha,
                                    int accumulate) {
  constexpr int B = 2 * P + 1;
  size_t N = (size_t)n1 * n2 * n3;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  int i3 = (int)(idx % n3);
  size_t r = idx / n3;
  int i2 = (int)(r % n2), i1 = (int)(r / n2);
  int nm = mode == 0 ? n1 : (mode == 1 ? n2 : n3);
  int im = mode == 0 ? i1 : (mode == 1 ? i2 : i3);
  size_t stride = mode == 0 ? (size_t)n2 * n3 : (mode == 1 ? (size_t)n3 : 1);
  const T* row = A + (size_t)im * B;
  T s = T(0);
#pragma unroll
  for (int o = 0; o < B; ++o) {
    int j = im + o - P;
    if (j >= 0 && j < nm) s += row[o] * x[idx + (ptrdiff_t)(j - im) * (ptrdiff_t)stride];
  }
  y[idx] = accumulate ? y[idx] + alpha * s : alpha * s;
}

// Tile of the fused apply: edges T1, T2 in 8..40 and T3 >= 1 with at most
// KRON_MO x KRON_THREADS outputs, minimising the busiest SM's work, i.e.
// ceil(CTAs / SMs) times the mode-product points of an interior tile.  Halo
// rows outside the domain cost nothing (the kernel skips them), so a
// direction covered by one or two tiles pays little halo.  Ties go to the
// thicker i3 slab, which re-reads less of the x halo.
static KronTile choose_tile(int n1, int n2, int n3, int P, int nsm, int es) {
  struct Key { int n1, n2, n3, P, nsm, es; };
  static std::mutex mu;
  static std::vector<std::pair<Key, KronTile>> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : cache)
      if (e.first.n1 == n1 && e.first.n2 == n2 && e.first.n3 == n3 && e.first.P == P &&
          e.first.nsm == nsm && e.first.es == es)
        return e.second;
  }
  auto span = [](int n, int T, int P) {
    // rows of the halo slab [I - P, I + T + P) inside [0, n) for the most
    // expensive tile (an interior one when there are three or more)
    int nt = (n + T - 1) / T;
    if (nt == 1) return std::min(n, T);
    if (nt == 2) return std::min(n, T + P);
    return T + 2 * P;
  };
  KronTile best{};
  double bestc = 1e300;
  for (int t1 = std::min(n1, 8); t1 <= std::min(n1, 40); ++t1)
    for (int t2 = std::min(n2, 8); t2 <= std::min(n2, 40); ++t2) {
      int h1 = span(n1, t1, P), h2 = span(n2, t2, P);
      int nt12 = ((n1 + t1 - 1) / t1) * ((n2 + t2 - 1) / t2);
      int max3 = std::min(n3, KRON_MO * KRON_THREADS / (t1 * t2));
      for (int t3 = 1; t3 <= max3; ++t3) {
        int nt3 = (n3 + t3 - 1) / t3;
        if (nt3 > 1 && (n3 + nt3 - 1) / nt3 != t3) continue;    // balanced slabs only
        // shared memory (mode-3 and mode-2 results, bands, the x slab) small
        // enough for two CTAs per SM
        const size_t h1f = t1 + 2 * P, h2f = t2 + 2 * P;
        const size_t sm = (h1f * h2f * t3 + h1f * t2 * t3 + (size_t)(t1 + t2 + t3) * (2 * P + 1) +
                           h1f * h2f * (t3 + 2 * P)) * es;
        if (sm > 113 * 1024) continue;
        double w = (double)t3 * ((double)h1 * h2 + (double)h1 * t2 + (double)t1 * t2);
        double waves = std::ceil((double)nt12 * nt3 / nsm);
        double c = waves * w;
        if (c < bestc * (1.0 - 1e-9) || (c <= bestc * (1.0 + 1e-9) && t3 > best.T3)) {
          bestc = c;
          best.T1 = t1; best.T2 = t2; best.T3 = t3;
        }
      }
    }
  best.n1 = n1; best.n2 = n2; best.n3 = n3;
  best.nt1 = (n1 + best.T1 - 1) / best.T1;
  best.nt2 = (n2 + best.T2 - 1) / best.T2;
  best.nt3 = (n3 + best.T3 - 1) / best.T3;
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() > 64) cache.clear();
  cache.push_back({Key{n1, n2, n3, P, nsm, es}, best});
  return best;
}

// ---- marching apply for large grids (HBM-bound FP32 applies)
//
// One CTA owns a KM_T2 x KM_T3 column of (i2, i3) points and a chunk
// [I1a, I1b) of i1.  It streams the input planes j1 = I1a - P .. I1b + P - 1
// through shared memory (cp.async, KM_STAGES planes of one input in
// flight), applies modes 3 and 2 of every term to the plane (a 2-D halo of P
// rows and columns only), and scatters mode 1 into a register ring of 2P+1
// output planes: plane j1 adds A1(i1, j1) w(j1) to every i1 in
// [j1 - P, j1 + P], so plane j1 - P is complete after plane j1 and is
// written once.  Every x element comes from DRAM about once (the halos of
// neighbouring columns from L2), y is written once, and the index
// arithmetic uses compile-time tile sizes.
constexpr int KM_T2 = 16, KM_T3 = 32, KM_THREADS = 256, KM_STAGES = 4;

struct KronRuns {
  int nrun;
  int xin[5];
  int t0[6];          // terms of run k: [t0[k], t0[k + 1])
};

template <typename T>
__device__ __forceinline__ void km_cp_async(T* smem, const T* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}

// stage plane j1 of run k's input into buffer `stage` of the marching
// apply (nothing for a plane outside the grid or past the last unit), then
// commit.  off[m] / okmask bit m: the in-plane offset and validity of the
// thread's m-th staged element, the same for every plane (zero fill outside
// the grid).
template <typename T, int P>
__device__ __forceinline__ void km_issue(T* xs, const KronJob<T>& job, const KronRuns& runs,
                                         bool live, int j1, int k, int stage, int n1,
                                         size_t plane_len, const int* off, unsigned okmask,
                                         int tid) {
  constexpr int H2 = KM_T2 + 2 * P, W3 = KM_T3 + 2 * P;
  constexpr int NE = (H2 * W3 + KM_THREADS - 1) / KM_THREADS;
  if (live && j1 >= 0 && j1 < n1) {
    const int xi = runs.xin[k];
    const T* __restrict__ x =
        xi == 0 ? job.x[0]
                : (xi == 1 ? job.x[1] : (xi == 2 ? job.x[2] : (xi == 3 ? job.x[3] : job.x[4])));
    T* dst = xs + stage * (H2 * W3);
    const T* plane = x + (size_t)j1 * plane_len;
#pragma unroll
    for (int m = 0; m < NE; ++m) {
      const int e = tid + m * KM_THREADS;
      if (e < H2 * W3) {
        const bool ok = (okmask >> m) & 1u;
        km_cp_async(dst + e, ok ? plane + off[m] : x, ok);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

template <typename T, int P, int NY>
__global__ void __launch_bounds__(KM_THREADS)
kron_march_kernel(const __grid_constant__ KronJob<T> job, const __grid_constant__ KronRuns runs,
                  int n1, int n2, int n3, int L1, int nb3, int nb2) {
  constexpr int B = 2 * P + 1;
  constexpr int W = 2 * P + 1;                 // ring of output planes
  constexpr int H2 = KM_T2 + 2 * P, W3 = KM_T3 + 2 * P;
  constexpr int NE = (H2 * W3 + KM_THREADS - 1) / KM_THREADS;
  extern __shared__ unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);                      // KM_STAGES x H2 x W3
  T* v = xs + KM_STAGES * H2 * W3;                          // 2 x H2 x KM_T3
  T* a3s = v + 2 * H2 * KM_T3;                              // nterms x KM_T3 x B
  T* a2s = a3s + job.nterms * KM_T3 * B;                    // nterms x KM_T2 x B
  const int tid = threadIdx.x, c = tid & 31, ty = tid >> 5;
  int bid = blockIdx.x;
  const int b3 = bid % nb3;
  bid /= nb3;
  const int b2 = bid % nb2;
  const int ch = bid / nb2;
  const int I3 = b3 * KM_T3, I2 = b2 * KM_T2;
  const int I1a = ch * L1, I1b = min(n1, I1a + L1);
  // the bands of modes 3 and 2 for this column, zero outside the matrix
  for (int e = tid; e < job.nterms * KM_T3 * B; e += KM_THREADS) {
    const int t = e / (KM_T3 * B), r = e - t * (KM_T3 * B), cc = r / B, o = r - cc * B;
    const int i = I3 + cc, j = i + o - P;
    a3s[e] = (i < n3 && j >= 0 && j < n3) ? job.b[2][t][(size_t)i * B + o] : T(0);
  }
  for (int e = tid; e < job.nterms * KM_T2 * B; e += KM_THREADS) {
    const int t = e / (KM_T2 * B), r = e - t * (KM_T2 * B), rr = r / B, o = r - rr * B;
    const int i = I2 + rr, j = i + o - P;
    a2s[e] = (i < n2 && j >= 0 && j < n2) ? job.b[1][t][(size_t)i * B + o] : T(0);
  }
  int off[NE];
  unsigned okmask = 0u;
#pragma unroll
  for (int m = 0; m < NE; ++m) {
    const int e = tid + m * KM_THREADS;
    const int r = e / W3, cc = e - r * W3;
    const int i2 = I2 - P + r, i3 = I3 - P + cc;
    const bool ok = e < H2 * W3 && i2 >= 0 && i2 < n2 && i3 >= 0 && i3 < n3;
    off[m] = ok ? i2 * n3 + i3 : 0;
    okmask |= ok ? (1u << m) : 0u;
  }
  const size_t plane_len = (size_t)n2 * n3;
  const int jbeg = I1a - P, jend = I1b + P;
  const int nrun = runs.nrun;
  const int nunits = (jend - jbeg) * nrun;
  // acc[z] collects output plane j1 - P + z while plane j1 is processed
  T acc[W][2][NY];
#pragma unroll
  for (int z = 0; z < W; ++z)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int o = 0; o < NY; ++o) acc[z][p][o] = T(0);
  // the next unit to stage: plane ij of run ik, unit number iu
  int ij = jbeg, ik = 0, iu = 0;
  auto stage_next = [&]() {
    km_issue<T, P>(xs, job, runs, iu < nunits, ij, ik, iu % KM_STAGES, n1, plane_len, off,
                   okmask, tid);
    ++iu;
    if (++ik == nrun) {
      ik = 0;
      ++ij;
    }
  };
#pragma unroll
  for (int q = 0; q < KM_STAGES - 1; ++q) stage_next();
  int u = 0, par = 0;
  const int rp0 = ty, rp1 = ty + 8;
  // output offsets of the thread's two points within a plane
  const size_t yo0 = (size_t)(I2 + rp0) * n3 + I3 + c, yo1 = (size_t)(I2 + rp1) * n3 + I3 + c;
  for (int j1 = jbeg; j1 < jend; ++j1) {
    // planes whose whole band lies inside the grid need no row checks
    const bool inner = j1 >= P && j1 + P < n1;
    for (int k = 0; k < nrun; ++k, ++u) {
      stage_next();
      asm volatile("cp.async.wait_group %0;\n" ::"n"(KM_STAGES - 1));
      __syncthreads();
      if (j1 >= 0 && j1 < n1) {
        const T* xb = xs + (u % KM_STAGES) * (H2 * W3);
        for (int t = runs.t0[k]; t < runs.t0[k + 1]; ++t, par ^= 1) {
          // mode 3 on the H2 halo rows of the column (v double-buffered by
          // term, so one barrier per term suffices)
          T* vb = v + par * (H2 * KM_T3);
          const T* a3 = a3s + (t * KM_T3 + c) * B;
          T c3[B];
#pragma unroll
          for (int o = 0; o < B; ++o) c3[o] = a3[o];
#pragma unroll
          for (int rr = 0; rr < (H2 + 7) / 8; ++rr) {
            const int r = ty + 8 * rr;
            if (r < H2) {
              const T* xr = xb + r * W3 + c;
              T sv = T(0);
#pragma unroll
              for (int o = 0; o < B; ++o) sv = fma(c3[o], xr[o], sv);
              vb[r * KM_T3 + c] = sv;
            }
          }
          __syncthreads();
          // mode 2 for the thread's two rows
          T w0 = T(0), w1 = T(0);
          {
            const T* a20 = a2s + (t * KM_T2 + rp0) * B;
            const T* a21 = a2s + (t * KM_T2 + rp1) * B;
#pragma unroll
            for (int o = 0; o < B; ++o) {
              w0 = fma(a20[o], vb[(rp0 + o) * KM_T3 + c], w0);
              w1 = fma(a21[o], vb[(rp1 + o) * KM_T3 + c], w1);
            }
          }
          // mode 1 scattered into the ring: i1 = j1 + q (slot q + P),
          // A1(i1, j1) at band[i1][P - q] = A1r[q (B - 1)]
          const T* A1r = job.b[0][t] + (ptrdiff_t)j1 * B + P;
          T cf[NY];
#pragma unroll
          for (int o = 0; o < NY; ++o) cf[o] = job.coef[t][o];
          const unsigned cm = job.cmask[t];
#pragma unroll
          for (int q = -P; q <= P; ++q) {
            if (inner || (unsigned)(j1 + q) < (unsigned)n1) {
              const T a1 = __ldg(A1r + q * (B - 1));
              const T p0 = a1 * w0, p1 = a1 * w1;
#pragma unroll
              for (int o = 0; o < NY; ++o)
                if (cm & (1u << o)) {
                  acc[q + P][0][o] = fma(cf[o], p0, acc[q + P][0][o]);
                  acc[q + P][1][o] = fma(cf[o], p1, acc[q + P][1][o]);
                }
            }
          }
        }
      }
    }
    // plane j1 - P is complete: write slot 0, then shift the ring
    const int i1 = j1 - P;
    if (i1 >= I1a && i1 < I1b) {
      const int i3 = I3 + c;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int i2 = I2 + (p ? rp1 : rp0);
        if (i2 < n2 && i3 < n3) {
          const size_t o2 = (size_t)i1 * plane_len + (p ? yo1 : yo0);
#pragma unroll
          for (int o = 0; o < NY; ++o) {
            T val = acc[0][p][o];
            if (job.beta[o] != T(0)) val += job.beta[o] * job.y[o][o2];
            job.y[o][o2] = val;
          }
        }
      }
    }
#pragma unroll
    for (int z = 0; z + 1 < W; ++z)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int o = 0; o < NY; ++o) acc[z][p][o] = acc[z + 1][p][o];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int o = 0; o < NY; ++o) acc[W - 1][p][o] = T(0);
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// The marching kernel takes the FP32 applies of large grids, which are
// bound by HBM (one term) or by the FP32 units (the KKT operator); the FP64
// applies keep the tiled kernel, whose halo work is hidden behind the
// FP64 pipe.
static bool use_march(const KronTile& g, int es) {
  return es == 4 && (double)g.n1 * g.n2 * g.n3 >= 4194304.0 && g.n2 >= KM_T2 && g.n3 >= KM_T3;
}

template <typename T, int P, int NY>
static void launch_march(iga_ctx* ctx, const KronJob<T>& jm, int n1, int n2, int n3) {
  constexpr int B = 2 * P + 1;
  constexpr int H2 = KM_T2 + 2 * P, W3 = KM_T3 + 2 * P;
  KronRuns runs{};
  runs.nrun = 0;
  for (int t = 0; t < jm.nterms; ++t)
    if (t == 0 || jm.xin[t] != jm.xin[t - 1]) {
      IGA_REQUIRE(runs.nrun < 5, "kron_apply: too many input runs");
      runs.xin[runs.nrun] = jm.xin[t];
      runs.t0[runs.nrun] = t;
      ++runs.nrun;
    }
  runs.t0[runs.nrun] = jm.nterms;
  const size_t smem = ((size_t)KM_STAGES * H2 * W3 + (size_t)2 * H2 * KM_T3 +
                       (size_t)jm.nterms * (KM_T3 + KM_T2) * B) * sizeof(T);
  IGA_REQUIRE(smem <= 227 * 1024, "kron_apply: marching tile does not fit in shared memory");
  func_attr(kron_march_kernel<T, P, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)smem);
  int occ = 1;
  IGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kron_march_kernel<T, P, NY>,
                                                         KM_THREADS, smem));
  occ = std::max(1, occ);
  const int nb3 = (n3 + KM_T3 - 1) / KM_T3, nb2 = (n2 + KM_T2 - 1) / KM_T2;
  // chunks of i1 so that the columns fill the resident CTAs once; a chunk
  // of at least 4 (2P+1) planes keeps the recomputed halo planes below a
  // quarter
  const int cols = nb3 * nb2;
  int nch = std::max(1, (ctx->nsm * occ + cols - 1) / cols);
  const int L1min = 4 * B;
  nch = std::max(1, std::min(nch, (n1 + L1min - 1) / L1min));
  const int L1 = (n1 + nch - 1) / nch;
  nch = (n1 + L1 - 1) / L1;
  IGA_LAUNCH(ctx, (kron_march_kernel<T, P, NY>), (unsigned)(cols * nch), KM_THREADS, smem, jm,
             runs, n1, n2, n3, L1, nb3, nb2);
}

template <typename T, int P, int NY>
static void launch_kron_job(iga_ctx* ctx, const KronJob<T>& job, const KronTile& g) {
  constexpr int B = 2 * P + 1;
  size_t H1 = g.T1 + 2 * P, H2 = g.T2 + 2 * P;
  size_t smem = (H1 * H2 * g.T3 + H1 * g.T2 * g.T3 + (size_t)(g.T1 + g.T2 + g.T3) * B +
                 H1 * H2 * (g.T3 + 2 * P)) * sizeof(T);
  IGA_REQUIRE(smem <= 227 * 1024, "kron_apply: tile does not fit in shared memory");
  func_attr(kron_rank1_kernel<T, P, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  {
    // algorithmic: read every input, write every output (and read it when
    // accumulating); 3 banded mode products of 2(2P+1) flop per point and term
    double N = (double)g.n1 * g.n2 * g.n3;
    int nin = 0;
    for (int i = 0; i < 5; ++i) {
      bool used = false;
      for (int t = 0; t < job.nterms; ++t) used |= job.xin[t] == i;
      nin += used;
    }
    double outs = 0.0;
    for (int o = 0; o < NY; ++o) outs += job.beta[o] != T(0) ? 2.0 : 1.0;
    prof_count(ctx, N * sizeof(T) * (nin + outs), 6.0 * B * N * job.nterms);
  }
  KronJob<T> jm = job;
  for (int t = 0; t < jm.nterms; ++t) {
    jm.cmask[t] = 0;
    for (int o = 0; o < NY; ++o)
      if (jm.coef[t][o] != T(0)) jm.cmask[t] |= (unsigned char)(1u << o);
  }
  if (use_march(g, (int)sizeof(T))) {
    launch_march<T, P, NY>(ctx, jm, g.n1, g.n2, g.n3);
    return;
  }
  IGA_LAUNCH(ctx, (kron_rank1_kernel<T, P, NY>), (unsigned)(g.nt1 * g.nt2 * g.nt3), KRON_THREADS,
             smem, jm, g);
}

template <typename T>
static const T* band_ptr(const iga_op* A, int d, size_t k) {
  size_t len = (size_t)A->n[d] * (2 * A->p[d] + 1);
  if constexpr (sizeof(T) == 8) return A->band64[d].p + k * len;
  else return A->band32[d].p + k * len;
}

template <typename T, int P>
static void kron_rank1(iga_ctx* ctx, const iga_op* A, T alpha, const T* x, T beta, T* y) {
  KronTile g = choose_tile(A->n[0], A->n[1], A->n[2], P, ctx->nsm, (int)sizeof(T));
  // terms in chunks of KRON_MAXTERMS (beta applies to the first chunk only)
  size_t nterm = A->blocks.size();
  for (size_t c0 = 0; c0 < nterm || c0 == 0; c0 += KRON_MAXTERMS) {
    KronJob<T> job{};
    int cnt = 0;
    for (size_t t = c0; t < std::min(nterm, c0 + KRON_MAXTERMS); ++t, ++cnt) {
      for (int d = 0; d < 3; ++d) job.b[d][cnt] = band_ptr<T>(A, d, A->blocks[t].off[d]);
      job.coef[cnt][0] = alpha;
      job.xin[cnt] = 0;
    }
    job.nterms = cnt;
    job.x[0] = job.x[1] = job.x[2] = x;
    job.y[0] = job.y[1] = job.y[2] = y;
    job.beta[0] = (c0 == 0) ? beta : T(1);
    launch_kron_job<T, P, 1>(ctx, job, g);
    if (nterm == 0) break;
  }
}

// The KKT operator [[M, 0, K^T], [0, beta M, -M], [K, -M, 0]] on z = (y, u,
// lambda) in one launch when M and K are rank-1 Kronecker sums: the products
// M y, M u, M lambda, K y and K lambda (K^T = K) are each formed once and
// added to the block rows that use them.
template <typename T, int P>
static void kkt_rank1(iga_ctx* ctx, const iga_op* M, const iga_op* K, T beta, const T* z,
                      T* out) {
  KronTile g = choose_tile(M->n[0], M->n[1], M->n[2], P, ctx->nsm, (int)sizeof(T));
  size_t N = (size_t)M->n[0] * M->n[1] * M->n[2];
  KronJob<T> job{};
  int cnt = 0;
  auto add = [&](const iga_op* A, int xin, T c0, T c1, T c2) {
    for (const OpBlock& blk : A->blocks) {
      for (int d = 0; d < 3; ++d) job.b[d][cnt] = band_ptr<T>(A, d, blk.off[d]);
      job.xin[cnt] = (unsigned char)xin;
      job.coef[cnt][0] = c0;
      job.coef[cnt][1] = c1;
      job.coef[cnt][2] = c2;
      ++cnt;
    }
  };
  // terms grouped by input so that the x halo of one input stays in L1
  add(M, 0, T(1), T(0), T(0));       // M y      -> row 1
  add(K, 0, T(0), T(0), T(1));       // K y      -> row 3
  add(M, 1, T(0), beta, T(-1));      // M u      -> rows 2 and 3
  add(M, 2, T(0), T(-1), T(0));      // M lambda -> row 2
  add(K, 2, T(1), T(0), T(0));       // K lambda -> row 1
  job.nterms = cnt;
  for (int i = 0; i < 3; ++i) {
    job.x[i] = z + i * N;
    job.y[i] = out + i * N;
    job.beta[i] = T(0);
  }
  launch_kron_job<T, P, 3>(ctx, job, g);
}

// The parabolic KKT rows of one time step (Sec. 4, eq. KKTSystem) in one
// launch, accumulated into out[] (which holds the right-hand side):
//   out_y -= M a + tau K lam_k,  out_u -= M d,  out_lam -= tau K y_k + M f
// with in = {a, d, f, y_k, lam_k} formed by the caller (the time differences
// and scalings folded into a, d and f), so that every product is formed
// once: three with M and two with K, as in the stationary KKT apply.
template <typename T, int P>
static void parabolic_rank1(iga_ctx* ctx, const iga_op* M, const iga_op* K, T tau,
                            const T* const in[5], T* const out[3]) {
  KronTile g = choose_tile(M->n[0], M->n[1], M->n[2], P, ctx->nsm, (int)sizeof(T));
  KronJob<T> job{};
  int cnt = 0;
  auto add = [&](const iga_op* A, int xin, T c0, T c1, T c2) {
    for (const OpBlock& blk : A->blocks) {
      for (int d = 0; d < 3; ++d) job.b[d][cnt] = band_ptr<T>(A, d, blk.off[d]);
      job.xin[cnt] = (unsigned char)xin;
      job.coef[cnt][0] = c0;
      job.coef[cnt][1] = c1;
      job.coef[cnt][2] = c2;
      ++cnt;
    }
  };
  // terms grouped by input so that each input slab is staged once
  add(M, 0, T(-1), T(0), T(0));      // M a      -> y-row
  add(M, 1, T(0), T(-1), T(0));      // M d      -> u-row
  add(M, 2, T(0), T(0), T(-1));      // M f      -> lambda-row
  add(K, 3, T(0), T(0), -tau);       // K y_k    -> lambda-row
  add(K, 4, -tau, T(0), T(0));       // K lam_k  -> y-row
  job.nterms = cnt;
  for (int i = 0; i < 5; ++i) job.x[i] = in[i];
  for (int o = 0; o < 3; ++o) {
    job.y[o] = out[o];
    job.beta[o] = T(1);
  }
  launch_kron_job<T, P, 3>(ctx, job, g);
}

bool parabolic_rows_fused(iga_ctx* ctx, const iga_op* M, const iga_op* K, double tau,
                          const double* const in[5], double* const out[3]) {
  int P = M->p[0];
  for (int d = 0; d < 3; ++d)
    if (M->p[d] != P || K->p[d] != P || M->n[d] != K->n[d]) return false;
  if (!M->rank1 || !K->rank1 || M->blocks.empty() || K->blocks.empty() ||
      3 * M->blocks.size() + 2 * K->blocks.size() > (size_t)KRON_MAXTERMS)
    return false;
  switch (P) {
    case 1: parabolic_rank1<double, 1>(ctx, M, K, tau, in, out); return true;
    case 2: parabolic_rank1<double, 2>(ctx, M, K, tau, in, out); return true;
    case 3: parabolic_rank1<double, 3>(ctx, M, K, tau, in, out); return true;
    case 4: parabolic_rank1<double, 4>(ctx, M, K, tau, in, out); return true;
    default: return false;
  }
}

template <typename T, int P>
static void mode_product(iga_ctx* ctx, const T* band, int mode, const int* n, const T* x, T* y,
                         T alpha, int accumulate) {
  size_t N = (size_t)n[0] * n[1] * n[2];
  int threads = 256;
  IGA_LAUNCH(ctx, (mode_product_kernel<T, P>), (unsigned)((N + threads - 1) / threads), threads, 0,
             band, mode, n[0], n[1], n[2], x, y, alpha, accumulate);
}

// ---- TT-matrix blocks (R1 R2 > 1): rank contraction as a batched GEMM
//
// For a block sum_{a,b} A1[a] (x) A2[a][b] (x) A3[b]:
//   z3[j2][b][i1][i3] = (A3[b] x)(i1, j2, i3)          mode-3 products, j2 padded by P
//   C[i2][a][(i1,i3)] = sum_{o,b} A2[a][b](i2, o) z3[i2+o][b][(i1,i3)]
//                     = (W_{i2} Z_{i2})[a][(i1,i3)]   one GEMM per i2: M = R1, K = (2P+1) R2,
//                                                      N = n1 n3 (Z_{i2} is a contiguous block)
//   y += alpha sum_a (A1[a] (x) I (x) I) C[.][a]       mode-1 products, summed over a

template <typename T, int P>
__global__ void ttm_mode3_kernel(const T* __restrict__ bands3, int R2, int n1, int n2, int n3,
                                 const T* __restrict__ x, T* __restrict__ z3) {
  // grid.x = (padded j2, b) pair, grid.y * blockDim.x covers (i1, i3)
  constexpr int B = 2 * P + 1;
  const size_t N13 = (size_t)n1 * n3;
  const int jj = blockIdx.x / R2, b = blockIdx.x - (blockIdx.x / R2) * R2;
  const int j2 = jj - P;
  T* out = z3 + (size_t)blockIdx.x * N13;
  const T* band = bands3 + (size_t)b * n3 * B;
  for (size_t t = (size_t)blockIdx.y * blockDim.x + threadIdx.x; t < N13;
       t += (size_t)gridDim.y * blockDim.x) {
    int i1 = (int)(t / n3), i3 = (int)(t - (size_t)i1 * n3);
    T s = T(0);
    if (j2 >= 0 && j2 < n2) {
      const T* row = band + (size_t)i3 * B;
      const T* xr = x + ((size_t)i1 * n2 + j2) * n3;
#pragma unroll
      for (int o = 0; o < B; ++o) {
        int j3 = i3 + o - P;
        if (j3 >= 0 && j3 < n3) s += row[o] * xr[j3];
      }
    }
    out[t] = s;
  }
}

template <typename T>
__global__ void ttm_wpack_kernel(const T* __restrict__ bands2, int R1, int R2, int n2, int B,
                                 T* __restrict__ W) {
  // W[i2][a][o R2 + b] = A2[a][b](i2, o)
  size_t total = (size_t)n2 * R1 * B * R2;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int b = (int)(idx % R2);
  size_t r = idx / R2;
  int o = (int)(r % B);
  r /= B;
  int a = (int)(r % R1);
  int i2 = (int)(r / R1);
  W[idx] = bands2[(((size_t)a * R2 + b) * n2 + i2) * B + o];
}

template <typename T, int P>
__global__ void ttm_mode1_kernel(const T* __restrict__ bands1, int R1, int n1, int n2, int n3,
                                 const T* __restrict__ C, T alpha, T* __restrict__ y) {
  // grid.x = (i2, i1), threads over i3
  constexpr int B = 2 * P + 1;
  const size_t N13 = (size_t)n1 * n3;
  const int i2 = blockIdx.x / n1, i1 = blockIdx.x - (blockIdx.x / n1) * n1;
  for (int i3 = threadIdx.x; i3 < n3; i3 += blockDim.x) {
    T s = T(0);
    for (int a = 0; a < R1; ++a) {
      const T* row = bands1 + ((size_t)a * n1 + i1) * B;
      const T* c = C + ((size_t)i2 * R1 + a) * N13 + i3;
#pragma unroll
      for (int o = 0; o < B; ++o) {
        int j1 = i1 + o - P;
        if (j1 >= 0 && j1 < n1) s += row[o] * c[(size_t)j1 * n3];
      }
    }
    y[((size_t)i1 * n2 + i2) * n3 + i3] += alpha * s;
  }
}

// tensor-core mode of an FP32 apply
enum { TC_NONE = 0, TC_TF32 = 1, TC_BF16 = 2 };

template <typename T, int P>
static void ttm_block_gemm(iga_ctx* ctx, const iga_op* A, const OpBlock& blk, T alpha, const T* x,
                           T* y, int tc) {
  if constexpr (sizeof(T) == 4) {
    // TF32 / BF16: the fused tcgen05 kernel (one launch per block, O(tile) scratch)
    if (tc != TC_NONE && ttm_tc_block(ctx, band_ptr<float>(A, 0, blk.off[0]),
                                      band_ptr<float>(A, 1, blk.off[1]),
                                      band_ptr<float>(A, 2, blk.off[2]), blk.R1, blk.R2, A->n, P,
                                      (float)alpha, x, y, tc == TC_BF16))
      return;
  }
  const bool tf32 = tc != TC_NONE;
  const int n1 = A->n[0], n2 = A->n[1], n3 = A->n[2];
  constexpr int B = 2 * P + 1;
  const int R1 = blk.R1, R2 = blk.R2, Kd = B * R2;
  const size_t N13 = (size_t)n1 * n3, N = (size_t)n1 * n2 * n3;
  T* z3 = scratch<T>(ctx, SLOT_KRON_Z, (size_t)(n2 + 2 * P) * R2 * N13);
  T* C = scratch<T>(ctx, SLOT_KRON_Z2, (size_t)n2 * R1 * N13);
  T* W = scratch<T>(ctx, SLOT_TTM_W, (size_t)n2 * R1 * Kd);
  size_t t3 = (size_t)(n2 + 2 * P) * R2 * N13;
  {
    // algorithmic: mode 3 and mode 1 banded products plus the rank contraction
    double fl = 2.0 * B * N * (R2 + (double)R1 * R2 + R1);
    prof_count(ctx, (double)N * sizeof(T) * 3.0, fl);
  }
  {
    dim3 grid((unsigned)((n2 + 2 * P) * R2), (unsigned)std::min<size_t>((N13 + 255) / 256, 64));
    IGA_LAUNCH(ctx, (ttm_mode3_kernel<T, P>), grid, 256, 0, band_ptr<T>(A, 2, blk.off[2]), R2, n1,
               n2, n3, x, z3);
  }
  (void)t3;
  size_t tw = (size_t)n2 * R1 * Kd;
  IGA_LAUNCH(ctx, ttm_wpack_kernel<T>, (unsigned)((tw + 255) / 256), 256, 0,
             band_ptr<T>(A, 1, blk.off[1]), R1, R2, n2, B, W);
  // C_{i2} (R1 x n1 n3) = W_{i2} (R1 x (2P+1) R2) Z_{i2}, Z_{i2} = the window of
  // z3 starting at slab i2 (stride R2 n1 n3 between consecutive i2)
  (void)tf32;
  gemm_rm_batched<T>(ctx, false, false, R1, (int)N13, Kd, T(1), W, Kd, (long long)R1 * Kd, z3,
                     (int)N13, (long long)R2 * N13, T(0), C, (int)N13, (long long)R1 * N13, n2);
  {
    int th = std::min(256, ((n3 + 31) / 32) * 32);
    dim3 grid((unsigned)((size_t)n2 * n1), 1);
    IGA_LAUNCH(ctx, (ttm_mode1_kernel<T, P>), grid, th, 0, band_ptr<T>(A, 0, blk.off[0]), R1, n1,
               n2, n3, C, alpha, y);
  }
}

template <typename T, int P>
static void kron_general(iga_ctx* ctx, const iga_op* A, T alpha, const T* x, T beta, T* y,
                         int tc) {
  const int* n = A->n;
  size_t N = (size_t)n[0] * n[1] * n[2];
  // y <- beta y first, then accumulate every block
  if (beta == T(0)) IGA_CUDA(cudaMemsetAsync(y, 0, N * sizeof(T), ctx->stream));
  else if (beta != T(1))
    IGA_LAUNCH(ctx, scale_kernel<T>, (unsigned)((N + 255) / 256), 256, 0, y, N, beta);
  for (const OpBlock& blk : A->blocks) {
    if (blk.R1 == 1 && blk.R2 == 1) {
      T* z3 = scratch<T>(ctx, SLOT_KRON_Z, N);
      T* z2 = scratch<T>(ctx, SLOT_KRON_Z2, N);
      mode_product<T, P>(ctx, band_ptr<T>(A, 2, blk.off[2]), 2, n, x, z3, T(1), 0);
      mode_product<T, P>(ctx, band_ptr<T>(A, 1, blk.off[1]), 1, n, z3, z2, T(1), 0);
      mode_product<T, P>(ctx, band_ptr<T>(A, 0, blk.off[0]), 0, n, z2, y, alpha, 1);
      continue;
    }
    ttm_block_gemm<T, P>(ctx, A, blk, alpha, x, y, tc);
  }
}

template <typename T>
static void kron_dispatch(iga_ctx* ctx, const iga_op* A, double alpha, const void* x, double beta,
                          void* y, int tc = TC_NONE) {
  int P = A->p[0];
  IGA_REQUIRE(A->p[1] == P && A->p[2] == P, "kron_apply: equal degrees per direction required");
  const T* xx = static_cast<const T*>(x);
  T* yy = static_cast<T*>(y);
  bool fused = A->rank1 && A->blocks.size() <= 64;
  switch (P) {
#define IGA_KRON_CASE(PP)                                                                   \
  case PP:                                                                                  \
    if (fused) kron_rank1<T, PP>(ctx, A, (T)alpha, xx, (T)beta, yy);                        \
    else kron_general<T, PP>(ctx, A, (T)alpha, xx, (T)beta, yy, tc);                        \
    break;
    IGA_KRON_CASE(1)
    IGA_KRON_CASE(2)
    IGA_KRON_CASE(3)
    IGA_KRON_CASE(4)
#undef IGA_KRON_CASE
    default:
      throw Error(IGA_EINVAL, "kron_apply: degree must be 1..4");
  }
}

template <typename T>
static bool kkt_dispatch(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta,
                         const void* z, void* out) {
  int P = M->p[0];
  for (int d = 0; d < 3; ++d)
    if (M->p[d] != P || K->p[d] != P || M->n[d] != K->n[d]) return false;
  if (!M->rank1 || !K->rank1 || M->blocks.empty() || K->blocks.empty() ||
      3 * M->blocks.size() + 2 * K->blocks.size() > (size_t)KRON_MAXTERMS)
    return false;
  const T* zz = static_cast<const T*>(z);
  T* oo = static_cast<T*>(out);
  switch (P) {
    case 1: kkt_rank1<T, 1>(ctx, M, K, (T)beta, zz, oo); return true;
    case 2: kkt_rank1<T, 2>(ctx, M, K, (T)beta, zz, oo); return true;
    case 3: kkt_rank1<T, 3>(ctx, M, K, (T)beta, zz, oo); return true;
    case 4: kkt_rank1<T, 4>(ctx, M, K, (T)beta, zz, oo); return true;
    default: return false;
  }
}

bool kkt_apply_fused(iga_ctx* ctx, const iga_op* M, const iga_op* K, double beta, const void* z,
                     void* out, iga_prec prec) {
  if (prec == IGA_FP64) return kkt_dispatch<double>(ctx, M, K, beta, z, out);
  if (prec == IGA_FP32) return kkt_dispatch<float>(ctx, M, K, beta, z, out);
  return false;
}

// band of the transposed univariate matrix: A^T(i, i + o - p) = A(i + o - p, i)
template <typename T>
__global__ void band_transpose_kernel(const T* __restrict__ in, T* __restrict__ out, size_t nb,
                                      int n, int P) {
  const int B = 2 * P + 1;
  const size_t total = nb * n * B;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx % B);
    const size_t r = idx / B;
    const int i = (int)(r % n);
    const size_t k = r / n;
    const int j = i + o - P;
    out[idx] = (j >= 0 && j < n) ? in[(k * n + j) * B + (2 * P - o)] : T(0);
  }
}

void kron_apply_transposed(iga_ctx* ctx, const iga_op* A, double alpha, const void* x, double beta,
                           void* y, iga_prec prec) {
  // (sum A1 (x) A2 (x) A3)^T = sum A1^T (x) A2^T (x) A3^T: the same blocks with
  // every band transposed, in a temporary operator on the context stream
  IGA_REQUIRE(A != nullptr, "kron_apply: null operator");
  iga_op At;
  for (int d = 0; d < 3; ++d) {
    At.n[d] = A->n[d];
    At.p[d] = A->p[d];
    At.nbands[d] = A->nbands[d];
  }
  At.blocks = A->blocks;
  At.rank1 = A->rank1;
  for (int d = 0; d < 3; ++d) {
    const size_t len = A->band64[d].n;
    if (len == 0) continue;
    const unsigned g = (unsigned)std::min<size_t>((len + 255) / 256, 4096);
    At.band64[d].alloc(len);
    IGA_LAUNCH(ctx, band_transpose_kernel<double>, g, 256, 0, A->band64[d].p, At.band64[d].p,
               A->nbands[d], A->n[d], A->p[d]);
    At.band32[d].alloc(A->band32[d].n);
    IGA_LAUNCH(ctx, band_transpose_kernel<float>, g, 256, 0, A->band32[d].p, At.band32[d].p,
               A->nbands[d], A->n[d], A->p[d]);
  }
  kron_apply_impl(ctx, &At, alpha, x, beta, y, prec);
}

void kron_apply_impl(iga_ctx* ctx, const iga_op* A, double alpha, const void* x, double beta,
                     void* y, iga_prec prec) {
  IGA_REQUIRE(A != nullptr && x != nullptr && y != nullptr, "kron_apply: null argument");
  IGA_REQUIRE(x != y, "kron_apply: x and y must not overlap");
  if (prec == IGA_FP64) kron_dispatch<double>(ctx, A, alpha, x, beta, y);
  else if (prec == IGA_FP32) kron_dispatch<float>(ctx, A, alpha, x, beta, y);
  else if (prec == IGA_TF32) kron_dispatch<float>(ctx, A, alpha, x, beta, y, TC_TF32);
  else if (prec == IGA_BF16) kron_dispatch<float>(ctx, A, alpha, x, beta, y, TC_BF16);
  else throw Error(IGA_EINVAL, "kron_apply: unknown precision");
}

}  // namespace iga
