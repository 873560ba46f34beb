// Learned support proposer: an MLP m -> h1 -> h2 -> K (GELU hidden layers) that
// scores atoms for a signal, trained on (signal, OMP support) pairs with binary
// cross-entropy, and used to restrict OMP to its top candidates with full OMP as
// the fallback.  This is an extension beyond the paper (its Sec. 1 OMP stage is
// the thing being accelerated).
//
// All products are BF16 x BF16 -> FP32 on the tensor cores (tcgen05.mma with the
// accumulator tile in tensor memory); the master weights, the Adam moments and
// the loss are FP32.  One generic kernel computes C = A B^T for A [M][Kd] and
// B [N][Kd] (both K contiguous, BF16) with fused epilogues.
#include <cuda_bf16.h>
#include <math.h>

#include <string>
#include <vector>

#include "omp_common.cuh"
#include "sdl_internal.cuh"
#include "tc_ptx.cuh"

namespace sdl {
namespace prop {

using bf16 = __nv_bfloat16;

enum EpMode { kStore = 0, kAtomic = 1, kBiasGelu = 2, kBias = 3, kDGelu = 4 };

struct GemmArgs {
  const bf16 *A; int lda;    // [M][Kd]
  const bf16 *B; int ldb;    // [N][Kd]
  int M, N, Kd;
  int kchunks_per_split;     // split-K: blockIdx.z covers chunks [z c, (z+1) c)
  int mode;
  float *C; int ldc;         // FP32 output
  const float *bias;         // [N]
  const float *pre; int ldp; // pre-activation for kDGelu
  bf16 *H; int ldh;          // BF16 [M][N] output (may be null)
  bf16 *HT; int ldt;         // BF16 [N][M] output (may be null)
  int32_t *err;
  int staged;                // epilogue through shared memory (large grids) or straight from registers
};

constexpr int kGemmThreads = 128;
constexpr int kKc = 64;      // K chunk per MMA batch (4 MMAs of K=16)
constexpr int kNT = 128;     // N tile (TMEM columns)

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143267794f;
}

// Load a [rows][kKc] BF16 tile (rows r0.., columns k0..) into the canonical image.
__device__ __forceinline__ void load_tile(unsigned char *img, const bf16 *src, int ld, int nrows_total, int r0,
                                          int rows, int k0, int Kd, int tid) {
  for (int q = tid; q < rows * (kKc / 8); q += kGemmThreads) {
    const int r = q >> 3, c8 = q & 7;
    const int gr = r0 + r, gk = k0 + c8 * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < nrows_total && gk < Kd) v = *reinterpret_cast<const uint4 *>(src + (size_t)gr * ld + gk);
    *reinterpret_cast<uint4 *>(img + tc::image_offset(r, c8 * 8, kKc)) = v;
  }
}

__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *Aim = smem;                         // 128 x 64 BF16
  unsigned char *Bim = smem + 128 * kKc * 2;         // kNT x 64 BF16
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (128 + kNT) * kKc * 2);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * kNT;
  const int nch = (g.Kd + kKc - 1) / kKc;
  const int c_begin = blockIdx.z * g.kchunks_per_split;
  const int c_end = min(nch, c_begin + g.kchunks_per_split);
  if (warp == 0) tc::tmem_alloc(tslot, kNT);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_bf16(128, kNT);
  const uint32_t sbo = (kKc / 8) * 128;
  bool ok = true;
  int phase = 0;
  for (int c = c_begin; c < c_end; ++c) {
    load_tile(Aim, g.A, g.lda, g.M, m0, 128, c * kKc, g.Kd, tid);
    load_tile(Bim, g.B, g.ldb, g.N, n0, kNT, c * kKc, g.Kd, tid);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int ks = 0; ks < kKc / 16; ++ks)
        tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(Aim) + ks * 256, 128, sbo),
                     tc::smem_desc(tc::smem_u32(Bim) + ks * 256, 128, sbo), idesc, c > c_begin || ks > 0);
      tc::mma_commit(mbar);
    }
    if (!tc::mbar_wait(mbar, phase, 1 << 22)) ok = false;
    phase ^= 1;
    __syncthreads();   // the images may be overwritten by the next chunk
  }
  tc::fence_after();
  ok = __syncthreads_and(ok) != 0;   // one verdict per block: the TMEM loads below are warp-wide
  if (ok && c_end > c_begin && !g.staged) {
    // Straight from registers, one row per lane: fewest instructions, for
    // grids of about one block per SM, where each warp's stores are issued
    // and left to the memory system while the block has little else to do.
    const int row = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < kNT; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + c0, v);
      if (row >= g.M) continue;
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int col = n0 + c0 + e;
        if (col >= g.N) continue;
        float x = v[e];
        switch (g.mode) {
          case kStore: g.C[(size_t)row * g.ldc + col] = x; break;
          case kAtomic: atomicAdd(&g.C[(size_t)row * g.ldc + col], x); break;
          case kBias: g.C[(size_t)row * g.ldc + col] = x + g.bias[col]; break;
          case kBiasGelu: {
            const float p = x + g.bias[col];
            if (g.C) g.C[(size_t)row * g.ldc + col] = p;
            const bf16 h = __float2bfloat16_rn(gelu(p));
            if (g.H) g.H[(size_t)row * g.ldh + col] = h;
            if (g.HT) g.HT[(size_t)col * g.ldt + row] = h;
          } break;
          case kDGelu: {
            const float d = x * gelu_prime(g.pre[(size_t)row * g.ldp + col]);
            g.C[(size_t)row * g.ldc + col] = d;
            const bf16 h = __float2bfloat16_rn(d);
            if (g.H) g.H[(size_t)row * g.ldh + col] = h;
            if (g.HT) g.HT[(size_t)col * g.ldt + row] = h;
          } break;
        }
      }
    }
  } else if (ok && c_end > c_begin) {
    // The accumulator leaves TMEM with one row per lane.  Each warp stages its
    // 32 x 32 blocks in shared memory (the operand images are free now; pitch 33
    // keeps both access directions free of bank conflicts), so that C and H are
    // written along rows and the transposed copy HT along columns: every
    // global access of a warp covers consecutive addresses.
    float *buf = reinterpret_cast<float *>(smem) + warp * 32 * 33;
    const int rbase = m0 + 32 * warp;
    for (int c0 = 0; c0 < kNT; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
      for (int e = 0; e < 32; ++e) buf[lane * 33 + e] = v[e];
      __syncwarp();
      const int col = n0 + c0 + lane;
      const bool cok = col < g.N;
      for (int r = 0; r < 32 && rbase + r < g.M; ++r) {
        const int row = rbase + r;
        float x = buf[r * 33 + lane];
        if (cok) {
          switch (g.mode) {
            case kStore: g.C[(size_t)row * g.ldc + col] = x; break;
            case kAtomic: atomicAdd(&g.C[(size_t)row * g.ldc + col], x); break;
            case kBias: g.C[(size_t)row * g.ldc + col] = x + g.bias[col]; break;
            case kBiasGelu: {
              const float p = x + g.bias[col];
              if (g.C) g.C[(size_t)row * g.ldc + col] = p;   // the pre-activation, kept for training
              x = gelu(p);
              if (g.H) g.H[(size_t)row * g.ldh + col] = __float2bfloat16_rn(x);
            } break;
            case kDGelu: {
              x *= gelu_prime(g.pre[(size_t)row * g.ldp + col]);
              g.C[(size_t)row * g.ldc + col] = x;
              if (g.H) g.H[(size_t)row * g.ldh + col] = __float2bfloat16_rn(x);
            } break;
          }
        }
        buf[r * 33 + lane] = x;   // the value HT receives (rounded to BF16 there)
      }
      __syncwarp();
      if (g.HT && (g.mode == kBiasGelu || g.mode == kDGelu) && rbase + lane < g.M) {
#pragma unroll 4
        for (int e = 0; e < 32; ++e) {
          const int ce = n0 + c0 + e;
          if (ce < g.N) g.HT[(size_t)ce * g.ldt + rbase + lane] = __float2bfloat16_rn(buf[lane * 33 + e]);
        }
      }
      __syncwarp();
    }
  } else if (!ok && tid == 0 && g.err) {
    atomicOr(g.err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, kNT);
}

cudaError_t gemm(const GemmArgs &a0, int split, cudaStream_t st) {
  GemmArgs a = a0;
  const int nch = (a.Kd + kKc - 1) / kKc;
  if (split < 1) split = 1;
  if (split > nch) split = nch;
  a.kchunks_per_split = (nch + split - 1) / split;
  split = (nch + a.kchunks_per_split - 1) / a.kchunks_per_split;
  const size_t smem = tc::smem_for_tmem((size_t)(128 + kNT) * kKc * 2 + 64, kNT);
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.M + 127) / 128, (a.N + kNT - 1) / kNT, split);
  // staged (coalesced) stores pay once the grid fills the SMs several times
  // over (inference chunks); training batches launch about a block per SM
  a.staged = (int64_t)grid.x * grid.y * grid.z >= 1024 ? 1 : 0;
  gemm_bf16_kernel<<<grid, kGemmThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace prop
}  // namespace sdl

namespace sdl {
namespace prop {
namespace {

using omp_detail::warp_sum;

// Y [B][m] FP32 -> X [B][mp] BF16 and X^T [mp][ldt] BF16 (zero padding).
__global__ void to_bf16_kernel(const float *__restrict__ Y, int64_t B, int m, int mp, bf16 *X, bf16 *XT, int ldt) {
  const int64_t total = B * mp;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / mp;
    const int r = (int)(q - b * mp);
    const bf16 v = __float2bfloat16_rn(r < m ? Y[(size_t)b * m + r] : 0.f);
    X[q] = v;
    if (XT) XT[(size_t)r * ldt + b] = v;
  }
}

// Binary cross-entropy on the logits against support labels; dZ = (sigmoid(z) - t) / B.
__global__ void bce_kernel(const float *__restrict__ Z, int64_t B, int K, const int32_t *__restrict__ idx, int s,
                           float *dZ, bf16 *dZb, bf16 *dZT, int ldt, float *loss) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  const float invB = 1.f / (float)B;
  float acc = 0.f;
  for (int j = lane; j < K; j += 32) {
    float t = 0.f;
    for (int k = 0; k < s; ++k)
      if (idx[(size_t)b * s + k] == j) t = 1.f;
    const float z = Z[(size_t)b * K + j];
    acc += fmaxf(z, 0.f) - z * t + log1pf(expf(-fabsf(z)));
    const float d = (1.f / (1.f + expf(-z)) - t) * invB;
    dZ[(size_t)b * K + j] = d;
    const bf16 db = __float2bfloat16_rn(d);
    dZb[(size_t)b * K + j] = db;
    dZT[(size_t)j * ldt + b] = db;
  }
  acc = warp_sum(acc);
  if (lane == 0) atomicAdd(loss, acc * invB);
}

// out[j] += sum over rows of X[b][j]: blocks of 32 columns x 8 row lanes.
__global__ void colsum_kernel(const float *__restrict__ X, int64_t B, int n, int ld, float *out) {
  __shared__ float red[8][33];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  float acc = 0.f;
  if (col < n)
    for (int64_t b = (int64_t)blockIdx.y * 8 + rl; b < B; b += (int64_t)gridDim.y * 8) acc += X[(size_t)b * ld + col];
  red[rl][threadIdx.x & 31] = acc;
  __syncthreads();
  if (rl == 0 && col < n) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += red[q][threadIdx.x & 31];
    atomicAdd(&out[col], s);
  }
}

__global__ void adam_kernel(float *p, const float *__restrict__ g, float *mo, float *ve, int64_t n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float m1 = b1 * mo[q] + (1.f - b1) * gq;
    const float v1 = b2 * ve[q] + (1.f - b2) * gq * gq;
    mo[q] = m1;
    ve[q] = v1;
    p[q] -= lr * (m1 / bc1) / (sqrtf(v1 / bc2) + eps);
  }
}

// BF16 copies of the weights: W [out][in] (padded in) and, where given, W^T [in][out].
__global__ void weights_kernel(const float *__restrict__ W, int out, int in, int inp, bf16 *Wb, bf16 *WT) {
  const int64_t total = (int64_t)out * inp;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(q / inp), i = (int)(q - (int64_t)o * inp);
    const bf16 v = __float2bfloat16_rn(i < in ? W[(size_t)o * in + i] : 0.f);
    Wb[q] = v;
    if (WT && i < in) WT[(size_t)i * out + o] = v;
  }
}

// Top-c atoms by score for every signal (warp per signal, lowest index on ties).
__global__ void topk_kernel(const float *__restrict__ Z, int64_t n, int K, int c, int32_t *cand) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n) return;
  float v[32];
  const int kpl = (K + 31) >> 5;
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = (q < kpl && lane + 32 * q < K) ? Z[(size_t)b * K + lane + 32 * q] : -INFINITY;
  for (int r = 0; r < c; ++r) {
    float bv = -INFINITY;
    int bj = -1;
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q < kpl && v[q] > bv) { bv = v[q]; bj = lane + 32 * q; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > bv || (ov == bv && oj >= 0 && (bj < 0 || oj < bj))) { bv = ov; bj = oj; }
    }
    if (lane == 0) cand[(size_t)b * c + r] = bj;
    if (bj >= 0 && (bj & 31) == lane) {
#pragma unroll
      for (int q = 0; q < 32; ++q)
        if (q == (bj >> 5)) v[q] = -INFINITY;
    }
  }
}

// Subset of row i under offsets [L+1]: the largest t with offsets[t] <= i (an
// empty subset never qualifies, since the next one starts at the same row).
__device__ __forceinline__ int subset_of_row(const int64_t *__restrict__ offsets, int L, int64_t i) {
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// OMP restricted to c candidate atoms (lane j < c holds candidate j), Batch-OMP
// with the FP32 Gram of D, exact refit and one correction step on the support;
// flags signals whose residual norm exceeds eps_fb for the full-OMP fallback.
// offsets (device [L+1], or null for one dictionary): signal i is coded
// against dictionary t(i) of D [L][K][m] with Gram G [L][K][K], and its
// candidates are atom indices of that dictionary.
__global__ void romp_kernel(const float *__restrict__ D, const float *__restrict__ G, int m, int K,
                            const float *__restrict__ Y, int64_t n, int s, int c, const int32_t *__restrict__ cand,
                            float eps_fb, int32_t *idx, float *val, int32_t *nnz, float *resid2, int32_t *flag,
                            const int64_t *__restrict__ offsets, int L) {
  extern __shared__ __align__(16) float Lshared[];
  using namespace omp_detail;
  constexpr int M32 = kMaxM / 32;
  const int warp_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp_g >= n) return;
  const int64_t b = warp_g;
  if (offsets) {
    const int t = subset_of_row(offsets, L, b);
    D += (size_t)t * K * m;
    G += (size_t)t * K * K;
  }
  const int lp = odd_pitch(s);
  float *Ls = Lshared + (size_t)(threadIdx.x >> 5) * s * lp;   // per-warp factor scratch
  const int mu = (m + 31) >> 5;
  const float *ysig = Y + (size_t)b * m;
  const int cj = lane < c ? cand[(size_t)b * c + lane] : -1;
  // correlations of the candidates (each lane its own dot product)
  float a0 = 0.f;
  if (cj >= 0)
    for (int r = 0; r < m; ++r) a0 = fmaf(D[(size_t)cj * m + r], ysig[r], a0);
  float yl[M32];
#pragma unroll
  for (int u = 0; u < M32; ++u) yl[u] = (u < mu && lane + 32 * u < m) ? ysig[lane + 32 * u] : 0.f;
  bool avail = cj >= 0;
  int k = 0, Sl = -1;
  float a0Sl = 0.f, xl = 0.f;
  while (k < s) {
    float av = a0;
    for (int p = 0; p < k; ++p) {
      const float xp = __shfl_sync(0xffffffffu, xl, p);
      const int Sp = __shfl_sync(0xffffffffu, Sl, p);
      if (cj >= 0) av = fmaf(-G[(size_t)cj * K + Sp], xp, av);
    }
    float bv = avail ? fabsf(av) : -1.f;
    int bj = avail ? cj : -1;   // candidate atom, ties to the lowest atom index
    int bl = avail ? lane : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ov > bv || (ov == bv && oj >= 0 && (bj < 0 || oj < bj))) { bv = ov; bj = oj; bl = ol; }
    }
    if (bj < 0 || !(bv > 0.f)) break;
    const int best = bj;
    const float a0b = __shfl_sync(0xffffffffu, a0, bl);
    const float gS = lane < k ? G[(size_t)best * K + Sl] : 0.f;
    const float w = lower_solve(Ls, lp, k, gS, lane);
    const float gbb = G[(size_t)best * K + best];
    const float piv2 = gbb - warp_sum(lane < k ? w * w : 0.f);
    if (!(piv2 > kOmpPivotRelF32 * gbb) || !(piv2 > 0.f)) break;
    if (lane < k) Ls[k * lp + lane] = w;
    if (lane == k) {
      Ls[k * lp + k] = 1.f / sqrtf(piv2);
      Sl = best;
      a0Sl = a0b;
    }
    if (lane == bl) avail = false;
    __syncwarp();
    ++k;
    xl = upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, a0Sl, lane), lane);
  }
  float res2 = warp_sum([&] { float a = 0.f; for (int u = 0; u < M32; ++u) a = fmaf(yl[u], yl[u], a); return a; }());
  if (k > 0) {
    // exact refit from D (the Gram entries are the FP32 Gram of D) and one correction step
    const float bl2 = support_dots(D, m, mu, k, Sl, yl, lane);
    xl = upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, bl2, lane), lane);
    float rloc[M32];
    support_residual(D, ysig, m, mu, k, Sl, xl, rloc, lane);
    const float cr = support_dots(D, m, mu, k, Sl, rloc, lane);
    xl += upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, cr, lane), lane);
    support_residual(D, ysig, m, mu, k, Sl, xl, rloc, lane);
    float racc = 0.f;
#pragma unroll
    for (int u = 0; u < M32; ++u) racc = fmaf(rloc[u], rloc[u], racc);
    res2 = warp_sum(racc);
  }
  if (lane < s) {
    idx[(size_t)b * s + lane] = lane < k ? Sl : -1;
    val[(size_t)b * s + lane] = lane < k ? xl : 0.f;
  }
  if (lane == 0) {
    nnz[b] = k;
    resid2[b] = res2;
    flag[b] = res2 > eps_fb * eps_fb ? 1 : 0;
  }
}

// Fallback bookkeeping.  Signals grouped by subset.  Pass 1 counts the flagged signals of
// each subset into cnt[t] and their total into cnt[L]; pass 2 places flagged
// signal i at list[foff[t] + k], k its arrival rank within subset t (the order
// inside a subset is free: every signal is coded on its own).  The lanes of a
// warp that flag signals of one subset share one atomic (rows of a warp are
// consecutive, so they are nearly always in one subset).
__global__ void count_flags_kernel(const int32_t *__restrict__ flag, const int64_t *__restrict__ offsets, int L,
                                   int64_t n, int32_t *cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_up = (n + 31) / 32 * 32;    // whole warps stay in the loop together
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_up; q += stride) {
    const bool f = q < n && flag[q] != 0;
    const unsigned act = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int t = subset_of_row(offsets, L, q);
      const unsigned grp = __match_any_sync(act, t);
      if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cnt[t], __popc(grp));
    }
    if ((threadIdx.x & 31) == 0 && act) atomicAdd(&cnt[L], __popc(act));
  }
}

__global__ void place_flags_kernel(const int32_t *__restrict__ flag, const int64_t *__restrict__ offsets, int L,
                                   int64_t n, const int64_t *__restrict__ foff, int32_t *pos, int32_t *list) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_up = (n + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_up; q += stride) {
    const bool f = q < n && flag[q] != 0;
    const unsigned act = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int t = subset_of_row(offsets, L, q);
      const unsigned grp = __match_any_sync(act, t);
      const int leader = __ffs(grp) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&pos[t], __popc(grp));
      base = __shfl_sync(grp, base, leader);
      const int rank = __popc(grp & ((1u << lane) - 1u));
      list[foff[t] + base + rank] = (int32_t)q;
    }
  }
}

__global__ void gather_rows_kernel(const float *__restrict__ Y, int m, const int32_t *__restrict__ list,
                                   const int32_t *__restrict__ count, float *Yf) {
  const int64_t total = (int64_t)(*count) * m;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / m;
    const int r = (int)(q - i * m);
    Yf[q] = Y[(size_t)list[i] * m + r];
  }
}

__global__ void scatter_codes_kernel(const int32_t *__restrict__ list, const int32_t *__restrict__ count, int s,
                                     const int32_t *__restrict__ fi, const float *__restrict__ fv,
                                     const int32_t *__restrict__ fn, const float *__restrict__ fr, int32_t *idx,
                                     float *val, int32_t *nnz, float *resid2) {
  const int64_t total = (int64_t)(*count) * s;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / s;
    const int k = (int)(q - i * s);
    const int64_t dst = list[i];
    idx[(size_t)dst * s + k] = fi[q];
    val[(size_t)dst * s + k] = fv[q];
    if (k == 0) {
      nnz[dst] = fn[i];
      if (resid2) resid2[dst] = fr[i];
    }
  }
}

inline unsigned nblocks(int64_t items, int per, unsigned cap = 8192) {
  int64_t b = (items + per - 1) / per;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

}  // namespace
}  // namespace prop
}  // namespace sdl

// ------------------------------------------------------------- host side ----
struct sdl_proposer {
  int device = 0;
  int m = 0, h1 = 0, h2 = 0, K = 0, mp = 0;
  int64_t nparams = 0;
  int64_t step = 0;
  float *params = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  sdl::prop::bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2T = nullptr, *W3T = nullptr;
  // batch buffers (capacity cap rows)
  int64_t cap = 0;
  sdl::prop::bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr;
  sdl::prop::bf16 *dZb = nullptr, *dZT = nullptr, *dA2b = nullptr, *dA2T = nullptr, *dA1T = nullptr;
  float *A1 = nullptr, *A2 = nullptr, *Z = nullptr, *dZ = nullptr, *dA2 = nullptr, *dA1 = nullptr;
  float *loss = nullptr;
  int32_t *err = nullptr;
};

namespace sdl {
namespace prop {
namespace {

void free_batch(sdl_proposer *p) {
  void *bufs[] = {p->X, p->XT, p->H1, p->H1T, p->H2, p->H2T, p->dZb, p->dZT, p->dA2b, p->dA2T, p->dA1T,
                  p->A1, p->A2, p->Z, p->dZ, p->dA2, p->dA1};
  for (void *b : bufs) if (b) cudaFree(b);
  p->X = p->XT = p->H1 = p->H1T = p->H2 = p->H2T = p->dZb = p->dZT = p->dA2b = p->dA2T = p->dA1T = nullptr;
  p->A1 = p->A2 = p->Z = p->dZ = p->dA2 = p->dA1 = nullptr;
  p->cap = 0;
}

// Grow the batch buffers to hold `rows` (rounded up to 64) rows; synchronises.
cudaError_t ensure_batch(sdl_proposer *p, int64_t rows, cudaStream_t st) {
  const int64_t want = (rows + 63) / 64 * 64;
  if (want <= p->cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  free_batch(p);
  const int64_t B = want;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
  };
  const size_t h = sizeof(bf16), f = sizeof(float);
  alloc((void **)&p->X, h * B * p->mp);   alloc((void **)&p->XT, h * B * p->mp);
  alloc((void **)&p->H1, h * B * p->h1);  alloc((void **)&p->H1T, h * B * p->h1);
  alloc((void **)&p->H2, h * B * p->h2);  alloc((void **)&p->H2T, h * B * p->h2);
  alloc((void **)&p->dZb, h * B * p->K);  alloc((void **)&p->dZT, h * B * p->K);
  alloc((void **)&p->dA2b, h * B * p->h2); alloc((void **)&p->dA2T, h * B * p->h2);
  alloc((void **)&p->dA1T, h * B * p->h1);
  alloc((void **)&p->A1, f * B * p->h1);  alloc((void **)&p->A2, f * B * p->h2);
  alloc((void **)&p->Z, f * B * p->K);    alloc((void **)&p->dZ, f * B * p->K);
  alloc((void **)&p->dA2, f * B * p->h2); alloc((void **)&p->dA1, f * B * p->h1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(p);
    return e;
  }
  p->cap = B;
  return cudaSuccess;
}

struct Offsets { int64_t W1, b1, W2, b2, W3, b3, total; };
Offsets offsets_of(const sdl_proposer *p) {
  Offsets o;
  o.W1 = 0; o.b1 = o.W1 + (int64_t)p->h1 * p->m; o.W2 = o.b1 + p->h1;
  o.b2 = o.W2 + (int64_t)p->h2 * p->h1; o.W3 = o.b2 + p->h2; o.b3 = o.W3 + (int64_t)p->K * p->h2;
  o.total = o.b3 + p->K;
  return o;
}

cudaError_t refresh_weights(sdl_proposer *p, cudaStream_t st) {
  const Offsets o = offsets_of(p);
  weights_kernel<<<nblocks((int64_t)p->h1 * p->mp, 256), 256, 0, st>>>(p->params + o.W1, p->h1, p->m, p->mp, p->W1b, nullptr);
  weights_kernel<<<nblocks((int64_t)p->h2 * p->h1, 256), 256, 0, st>>>(p->params + o.W2, p->h2, p->h1, p->h1, p->W2b, p->W2T);
  weights_kernel<<<nblocks((int64_t)p->K * p->h2, 256), 256, 0, st>>>(p->params + o.W3, p->K, p->h2, p->h2, p->W3b, p->W3T);
  return cudaGetLastError();
}

// Forward pass of B rows of Y (B <= cap): logits in p->Z.  training: also keep
// the transposed activations the weight gradients need.
cudaError_t forward(sdl_proposer *p, const float *Y, int64_t B, bool training, cudaStream_t st) {
  const Offsets o = offsets_of(p);
  const int ldt = (int)p->cap;
  to_bf16_kernel<<<nblocks(B * p->mp, 256), 256, 0, st>>>(Y, B, p->m, p->mp, p->X, training ? p->XT : nullptr, ldt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GemmArgs g{};
  g.err = p->err;
  g.A = p->X; g.lda = p->mp; g.B = p->W1b; g.ldb = p->mp; g.M = (int)B; g.N = p->h1; g.Kd = p->mp;
  g.mode = kBiasGelu; g.C = training ? p->A1 : nullptr; g.ldc = p->h1; g.bias = p->params + o.b1;
  g.H = p->H1; g.ldh = p->h1; g.HT = training ? p->H1T : nullptr; g.ldt = ldt;
  if ((e = gemm(g, 1, st)) != cudaSuccess) return e;
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->H1; g.lda = p->h1; g.B = p->W2b; g.ldb = p->h1; g.M = (int)B; g.N = p->h2; g.Kd = p->h1;
  g.mode = kBiasGelu; g.C = training ? p->A2 : nullptr; g.ldc = p->h2; g.bias = p->params + o.b2;
  g.H = p->H2; g.ldh = p->h2; g.HT = training ? p->H2T : nullptr; g.ldt = ldt;
  if ((e = gemm(g, 1, st)) != cudaSuccess) return e;
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->H2; g.lda = p->h2; g.B = p->W3b; g.ldb = p->h2; g.M = (int)B; g.N = p->K; g.Kd = p->h2;
  g.mode = kBias; g.C = p->Z; g.ldc = p->K; g.bias = p->params + o.b3;
  return gemm(g, 1, st);
}

int split_for(int M, int N, int num_sms) {
  const int tiles = ((M + 127) / 128) * ((N + kNT - 1) / kNT);
  int sp = (num_sms + tiles - 1) / tiles;
  return sp < 1 ? 1 : sp;
}

// Loss and gradient of the batch (forward must have run with training = true).
cudaError_t backward(sdl_proposer *p, const int32_t *idx, int s, int64_t B, int num_sms, cudaStream_t st) {
  const Offsets o = offsets_of(p);
  const int ldt = (int)p->cap;
  cudaError_t e = cudaMemsetAsync(p->grad, 0, sizeof(float) * p->nparams, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(p->loss, 0, sizeof(float), st)) != cudaSuccess) return e;
  bce_kernel<<<nblocks(B, 8, 1u << 30), 256, 0, st>>>(p->Z, B, p->K, idx, s, p->dZ, p->dZb, p->dZT, ldt, p->loss);
  const unsigned ry = nblocks(B, 8 * 64, 64);
  colsum_kernel<<<dim3((p->K + 31) / 32, ry), 256, 0, st>>>(p->dZ, B, p->K, p->K, p->grad + o.b3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  GemmArgs g{};
  g.err = p->err;
  // gW3 = dZ^T H2
  g.A = p->dZT; g.lda = ldt; g.B = p->H2T; g.ldb = ldt; g.M = p->K; g.N = p->h2; g.Kd = (int)B;
  g.mode = kAtomic; g.C = p->grad + o.W3; g.ldc = p->h2;
  if ((e = gemm(g, split_for(p->K, p->h2, num_sms), st)) != cudaSuccess) return e;
  // dA2 = (dZ W3) * gelu'(A2)
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->dZb; g.lda = p->K; g.B = p->W3T; g.ldb = p->K; g.M = (int)B; g.N = p->h2; g.Kd = p->K;
  g.mode = kDGelu; g.pre = p->A2; g.ldp = p->h2; g.C = p->dA2; g.ldc = p->h2;
  g.H = p->dA2b; g.ldh = p->h2; g.HT = p->dA2T; g.ldt = ldt;
  if ((e = gemm(g, 1, st)) != cudaSuccess) return e;
  colsum_kernel<<<dim3((p->h2 + 31) / 32, ry), 256, 0, st>>>(p->dA2, B, p->h2, p->h2, p->grad + o.b2);
  // gW2 = dA2^T H1
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->dA2T; g.lda = ldt; g.B = p->H1T; g.ldb = ldt; g.M = p->h2; g.N = p->h1; g.Kd = (int)B;
  g.mode = kAtomic; g.C = p->grad + o.W2; g.ldc = p->h1;
  if ((e = gemm(g, split_for(p->h2, p->h1, num_sms), st)) != cudaSuccess) return e;
  // dA1 = (dA2 W2) * gelu'(A1)
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->dA2b; g.lda = p->h2; g.B = p->W2T; g.ldb = p->h2; g.M = (int)B; g.N = p->h1; g.Kd = p->h2;
  g.mode = kDGelu; g.pre = p->A1; g.ldp = p->h1; g.C = p->dA1; g.ldc = p->h1;
  g.H = nullptr; g.HT = p->dA1T; g.ldt = ldt;
  if ((e = gemm(g, 1, st)) != cudaSuccess) return e;
  colsum_kernel<<<dim3((p->h1 + 31) / 32, ry), 256, 0, st>>>(p->dA1, B, p->h1, p->h1, p->grad + o.b1);
  // gW1 = dA1^T X
  g = GemmArgs{};
  g.err = p->err;
  g.A = p->dA1T; g.lda = ldt; g.B = p->XT; g.ldb = ldt; g.M = p->h1; g.N = p->m; g.Kd = (int)B;
  g.mode = kAtomic; g.C = p->grad + o.W1; g.ldc = p->m;
  return gemm(g, split_for(p->h1, p->m, num_sms), st);
}

}  // namespace
}  // namespace prop
}  // namespace sdl

using namespace sdl;
using namespace sdl::prop;

namespace {
sdl_status perr(sdl_ctx *ctx, sdl_status st, const char *msg) { return set_error(ctx, st, msg); }
sdl_status pcuda(sdl_ctx *ctx, cudaError_t e, const char *what) { return check_cuda(ctx, e, what); }
bool al16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }
}  // namespace

extern "C" {

sdl_status sdl_proposer_create(sdl_ctx *ctx, int m, int h1, int h2, int K, const float *params,
                               sdl_proposer **out) {
  if (!ctx || !out) return SDL_EINVAL;
  *out = nullptr;
  if (m < 1 || m > kMaxK || h1 < 8 || h2 < 8 || K < 1 || K > kMaxK || h1 % 8 || h2 % 8 || K % 8)
    return perr(ctx, SDL_EINVAL, "proposer sizes: 1 <= m <= 1024, h1, h2 multiples of 8, K <= 1024 multiple of 8");
  if (!al16(params)) return perr(ctx, SDL_EINVAL, "params must be a 16-byte aligned device pointer");
  sdl_proposer *p = new sdl_proposer();
  p->device = ctx->device;
  p->m = m; p->h1 = h1; p->h2 = h2; p->K = K; p->mp = (m + 7) / 8 * 8;
  const Offsets o = offsets_of(p);
  p->nparams = o.total;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
  };
  alloc((void **)&p->params, sizeof(float) * o.total);
  alloc((void **)&p->grad, sizeof(float) * o.total);
  alloc((void **)&p->am, sizeof(float) * o.total);
  alloc((void **)&p->av, sizeof(float) * o.total);
  alloc((void **)&p->W1b, sizeof(bf16) * (size_t)h1 * p->mp);
  alloc((void **)&p->W2b, sizeof(bf16) * (size_t)h2 * h1);
  alloc((void **)&p->W3b, sizeof(bf16) * (size_t)K * h2);
  alloc((void **)&p->W2T, sizeof(bf16) * (size_t)h1 * h2);
  alloc((void **)&p->W3T, sizeof(bf16) * (size_t)h2 * K);
  alloc((void **)&p->loss, sizeof(float) * 4);
  alloc((void **)&p->err, sizeof(int32_t) * 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->params, params, sizeof(float) * o.total, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = refresh_weights(p, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    sdl_proposer_destroy(p);
    return pcuda(ctx, e, "proposer create");
  }
  *out = p;
  return SDL_OK;
}

sdl_status sdl_proposer_destroy(sdl_proposer *p) {
  if (!p) return SDL_OK;
  free_batch(p);
  void *bufs[] = {p->params, p->grad, p->am, p->av, p->W1b, p->W2b, p->W3b, p->W2T, p->W3T, p->loss, p->err};
  for (void *b : bufs) if (b) cudaFree(b);
  delete p;
  return SDL_OK;
}

sdl_status sdl_proposer_get_params(sdl_ctx *ctx, const sdl_proposer *p, float *params) {
  if (!ctx || !p || !al16(params)) return SDL_EINVAL;
  return pcuda(ctx, cudaMemcpyAsync(params, p->params, sizeof(float) * p->nparams, cudaMemcpyDeviceToDevice,
                                    ctx->stream), "params copy");
}

sdl_status sdl_proposer_loss_grad(sdl_ctx *ctx, sdl_proposer *p, const float *Y, const int32_t *idx, int s,
                                  int64_t B, float *loss, float *grad) {
  if (!ctx || !p) return SDL_EINVAL;
  ctx->err.clear();
  if (B <= 0 || B % 8 || s < 1 || s > kMaxS || B >= ((int64_t)1 << 31))
    return perr(ctx, SDL_EINVAL, "batch must be a positive multiple of 8 and 1 <= s <= 32");
  if (!al16(Y) || !al16(idx) || (loss && !al16(loss)) || (grad && !al16(grad)))
    return perr(ctx, SDL_EINVAL, "device pointers must be 16-byte aligned");
  cudaStream_t st = ctx->stream;
  cudaError_t e = ensure_batch(p, B, st);
  if (e == cudaSuccess) e = forward(p, Y, B, true, st);
  if (e == cudaSuccess) e = backward(p, idx, s, B, ctx->num_sms, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, p->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, p->grad, sizeof(float) * p->nparams, cudaMemcpyDeviceToDevice, st);
  ctx->launches += 14;
  return pcuda(ctx, e, "proposer loss/grad");
}

sdl_status sdl_proposer_train_step(sdl_ctx *ctx, sdl_proposer *p, const float *Y, const int32_t *idx, int s,
                                   int64_t B, float lr, float *loss) {
  sdl_status stt = sdl_proposer_loss_grad(ctx, p, Y, idx, s, B, loss, nullptr);
  if (stt != SDL_OK) return stt;
  p->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)p->step), bc2 = 1.f - powf(b2, (float)p->step);
  adam_kernel<<<nblocks(p->nparams, 256, 4096), 256, 0, ctx->stream>>>(p->params, p->grad, p->am, p->av,
                                                                        p->nparams, lr, b1, b2, 1e-8f, bc1, bc2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = refresh_weights(p, ctx->stream);
  ctx->launches += 4;
  return pcuda(ctx, e, "proposer adam");
}

sdl_status sdl_proposer_scores(sdl_ctx *ctx, sdl_proposer *p, const float *Y, int64_t n, float *Z) {
  if (!ctx || !p) return SDL_EINVAL;
  ctx->err.clear();
  if (n < 0 || !al16(Y) || !al16(Z)) return perr(ctx, SDL_EINVAL, "bad arguments");
  const int64_t chunk = 65536;
  cudaStream_t st = ctx->stream;
  cudaError_t e = ensure_batch(p, n < chunk ? n : chunk, st);
  for (int64_t a = 0; a < n && e == cudaSuccess; a += chunk) {
    const int64_t b = n - a < chunk ? n - a : chunk;
    e = forward(p, Y + (size_t)a * p->m, b, false, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Z + (size_t)a * p->K, p->Z, sizeof(float) * b * p->K, cudaMemcpyDeviceToDevice, st);
    ctx->launches += 4;
  }
  return pcuda(ctx, e, "proposer scores");
}

}  // extern "C"

namespace sdl {

int proposer_m(const sdl_proposer *p) { return p->m; }
int proposer_K(const sdl_proposer *p) { return p->K; }

cudaError_t proposer_topk(sdl_proposer *p, const float *Y, int64_t n, int c, int32_t *cand, cudaStream_t st) {
  using namespace prop;
  const int64_t chunk = 65536;
  cudaError_t e = ensure_batch(p, n < chunk ? n : chunk, st);
  for (int64_t a = 0; a < n && e == cudaSuccess; a += chunk) {
    const int64_t b = n - a < chunk ? n - a : chunk;
    e = forward(p, Y + (size_t)a * p->m, b, false, st);
    if (e != cudaSuccess) break;
    topk_kernel<<<nblocks(b, 8, 1u << 30), 256, 0, st>>>(p->Z, b, p->K, c, cand + (size_t)a * c);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_romp(const float *D, const float *G, int m, int K, const float *Y, int64_t n, int s, int c,
                        const int32_t *cand, float eps_fb, int32_t *idx, float *val, int32_t *nnz, float *resid2,
                        int32_t *flag, const int64_t *offsets, int L, cudaStream_t st) {
  using namespace prop;
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * 8 * (size_t)s * omp_detail::odd_pitch(s);
  romp_kernel<<<nblocks(n, 8, 1u << 30), 256, smem, st>>>(D, G, m, K, Y, n, s, c, cand, eps_fb, idx, val, nnz,
                                                           resid2, flag, offsets, L);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const int32_t *flag, const int64_t *offsets, int L, int64_t n, int32_t *cnt,
                               cudaStream_t st) {
  using namespace prop;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (L + 1), st);
  if (e != cudaSuccess || n <= 0) return e;
  count_flags_kernel<<<nblocks(n, 256, 4096), 256, 0, st>>>(flag, offsets, L, n, cnt);
  return cudaGetLastError();
}

cudaError_t launch_place_flags(const int32_t *flag, const int64_t *offsets, int L, int64_t n, const int64_t *foff,
                               int32_t *pos, int32_t *list, cudaStream_t st) {
  using namespace prop;
  cudaError_t e = cudaMemsetAsync(pos, 0, sizeof(int32_t) * L, st);
  if (e != cudaSuccess || n <= 0) return e;
  place_flags_kernel<<<nblocks(n, 256, 4096), 256, 0, st>>>(flag, offsets, L, n, foff, pos, list);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float *Y, int m, const int32_t *list, const int32_t *count, int64_t nmax,
                               float *Yf, cudaStream_t st) {
  using namespace prop;
  gather_rows_kernel<<<nblocks(nmax * m, 256, 4096), 256, 0, st>>>(Y, m, list, count, Yf);
  return cudaGetLastError();
}

cudaError_t launch_scatter_codes(const int32_t *list, const int32_t *count, int64_t nmax, int s, const int32_t *fi,
                                 const float *fv, const int32_t *fn, const float *fr, int32_t *idx, float *val,
                                 int32_t *nnz, float *resid2, cudaStream_t st) {
  using namespace prop;
  scatter_codes_kernel<<<nblocks(nmax * s, 256, 4096), 256, 0, st>>>(list, count, s, fi, fv, fn, fr, idx, val, nnz,
                                                                     resid2);
  return cudaGetLastError();
}

}  // namespace sdl
