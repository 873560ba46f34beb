// OMP sparse coding on CUDA cores (Sec. 1; error-constrained stop of Sec. 3.2.2).
//
// Batch-OMP form: per signal the correlations alpha0 = D^T y are computed once
// (a small GEMM over a tile of signals, kept in shared memory), and after each
// selection the correlations are alpha = alpha0 - G[:, S] x_S, with G = D^T D
// and x_S from a progressively updated Cholesky factor of G_SS.  This reaches
// the same greedy choices as the residual form (d_j^T r = alpha_j exactly in
// real arithmetic) at K s instead of K m work per step.  After the loop the
// coefficients are recomputed on the support from y and D_S (exact Gram of the
// support, one step of iterative refinement) and ||y - D_S x||^2 is reported.
#include <float.h>
#include <math.h>

#include "omp_common.cuh"

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kJBlock = 256;   // atoms per GEMM pass (8 per lane: lane + 32 c)
constexpr int kKChunk = 16;    // signal entries per GEMM stage
constexpr int kDPitch = 20;    // staged atom row pitch (floats): 5 x 16 bytes, so the
                               // 16-byte loads of lanes 0..7 hit distinct bank groups

// ---------------------------------------------------------------- Gram ------
// G_t = D_t D_t^T for D_t stored [K][m]; one 64x64 tile of G per block.
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const T *__restrict__ D, int m, int K,
                                                   T *__restrict__ G) {
  const int t = blockIdx.z;
  const T *Dt = D + (size_t)t * K * m;
  T *Gt = G + (size_t)t * K * K;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  __shared__ T As[16][65];
  __shared__ T Bs[16][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
  for (int k0 = 0; k0 < m; k0 += 16) {
    for (int q = threadIdx.x; q < 64 * 16; q += 256) {
      const int row = q >> 4, kk = q & 15, gk = k0 + kk;
      const int gi = i0 + row, gj = j0 + row;
      As[kk][row] = (gi < K && gk < m) ? Dt[(size_t)gi * m + gk] : T(0);
      Bs[kk][row] = (gj < K && gk < m) ? Dt[(size_t)gj * m + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < K && gj < K) Gt[(size_t)gi * K + gj] = acc[r][c];
    }
}

// ------------------------------------------------------------------ OMP -----
// Shared-memory carve-up of one CUDA-core OMP block.
struct OmpLayout {
  int TS, K, m, s, lp;   // lp: odd row pitch of the per-warp Cholesky factor
  int yp;                // signal row pitch in shared memory (m rounded up to 16, zero padded)
  bool gcache;
  size_t a0, yt, uni, ls, total;
};

template <typename T>
__host__ __device__ inline OmpLayout omp_layout(int TS, int K, int m, int s, bool gcache) {
  OmpLayout L{};
  L.TS = TS; L.K = K; L.m = m; L.s = s; L.gcache = gcache;
  L.lp = odd_pitch(s);
  L.yp = (m + kKChunk - 1) / kKChunk * kKChunk;
  size_t off = 0;
  L.a0 = off;  off += align16(sizeof(T) * (size_t)TS * K);
  L.yt = off;  off += align16(sizeof(T) * (size_t)TS * L.yp);
  const size_t stage = sizeof(T) * (size_t)kJBlock * kDPitch;
  const size_t gcol = gcache ? sizeof(T) * (size_t)kWarps * s * K : 0;
  L.uni = off; off += align16(stage > gcol ? stage : gcol);
  L.ls = off;  off += align16(sizeof(T) * (size_t)kWarps * s * L.lp);
  L.total = off;
  return L;
}

// 16-byte shared/global vector of four T.
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };

// One block codes a tile of TS = 4 * 8 signals of one subset: the correlation
// tile alpha0 = Y_tile D^T is a register-tiled FFMA GEMM (4 signals x 8 atoms
// per thread) over D staged in chunks of 16 signal entries, read back as
// 4-entry vectors; then each warp runs the selection loop for its 4 signals.
template <typename T, int KPL, int MU>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (KPL <= 16 ? 3 : 2) : 1) omp_kernel(OmpArgs a, OmpLayout lay) {
  extern __shared__ __align__(16) unsigned char smem[];
  using V4 = typename Vec4<T>::type;
  constexpr int SPW = 4;
  const int TS = SPW * kWarps;
  const int K = a.K, m = a.m;
  const int yp = lay.yp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int64_t g = blockIdx.x;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)TS;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < TS ? (int)rows_left : TS;

  const T *__restrict__ Dt = static_cast<const T *>(a.D) + (size_t)t * K * m;
  const T *__restrict__ Gt = static_cast<const T *>(a.G) + (size_t)t * K * K;
  const T *__restrict__ Y = static_cast<const T *>(a.Y);

  T *a0 = reinterpret_cast<T *>(smem + lay.a0);     // [TS][K]
  T *yt = reinterpret_cast<T *>(smem + lay.yt);     // [TS][yp], zero beyond m
  T *uni = reinterpret_cast<T *>(smem + lay.uni);   // GEMM stage [256][kDPitch] / G columns [warps][s][K]

  for (int q = threadIdx.x; q < TS * yp; q += kThreads) {
    const int sig = q / yp, r = q - sig * yp;
    yt[q] = (sig < nsig && r < m) ? Y[(size_t)(row0 + sig) * m + r] : T(0);
  }
  // 16-byte global loads of D rows need m a multiple of 4 (D itself is
  // 16-byte aligned)
  const bool vec = (m & 3) == 0;

  // ---- alpha0[sig][j] = <y_sig, d_j>
  for (int jb = 0; jb < K; jb += kJBlock) {
    T acc[SPW][8];
#pragma unroll
    for (int r = 0; r < SPW; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = T(0);
    for (int k0 = 0; k0 < m; k0 += kKChunk) {
      __syncthreads();
      {   // thread jj stages entries k0 .. k0+15 of atom jb + jj (zero outside D)
        const int jj = threadIdx.x, gj = jb + jj;
        T *dst = uni + jj * kDPitch;
        const T *src = Dt + (size_t)gj * m + k0;
        if (vec) {
#pragma unroll
          for (int e = 0; e < kKChunk; e += 4) {
            V4 v;
            if (gj < K && k0 + e < m) v = *reinterpret_cast<const V4 *>(src + e);
            else v.x = v.y = v.z = v.w = T(0);
            *reinterpret_cast<V4 *>(dst + e) = v;
          }
        } else {
#pragma unroll
          for (int e = 0; e < kKChunk; ++e) dst[e] = (gj < K && k0 + e < m) ? src[e] : T(0);
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int kq = 0; kq < kKChunk; kq += 4) {
        V4 yv[SPW];
#pragma unroll
        for (int r = 0; r < SPW; ++r) yv[r] = *reinterpret_cast<const V4 *>(yt + (warp * SPW + r) * yp + k0 + kq);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const V4 dv = *reinterpret_cast<const V4 *>(uni + (lane + 32 * c) * kDPitch + kq);
#pragma unroll
          for (int r = 0; r < SPW; ++r) {
            acc[r][c] = fma(yv[r].x, dv.x, acc[r][c]);
            acc[r][c] = fma(yv[r].y, dv.y, acc[r][c]);
            acc[r][c] = fma(yv[r].z, dv.z, acc[r][c]);
            acc[r][c] = fma(yv[r].w, dv.w, acc[r][c]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < SPW; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = jb + lane + 32 * c;
        if (j < K) a0[(warp * SPW + r) * K + j] = acc[r][c];
      }
  }
  __syncthreads();   // staging is dead from here; the union holds G columns

  T *Ls = reinterpret_cast<T *>(smem + lay.ls) + (size_t)warp * a.s * lay.lp;
  code_warp_signals<T, KPL, MU, false>(a, a0, yt, yp, warp * SPW, SPW, nsig, row0, Dt, Gt, Ls,
                                       uni + (size_t)warp * a.s * K, lay.lp, lay.gcache ? a.s : 0);
}

}  // namespace

// ------------------------------------------------------------- launchers ----
template <typename T>
cudaError_t launch_gram(const T *D, int m, int K, int L, T *G, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    // 128 x 128 tiles when they give at least one block per SM of the GB300
    // (152: the batched local dictionaries), 64 x 64 tiles otherwise (a single
    // dictionary, where the smaller tiles spread over more SMs)
    constexpr int64_t kMinBigBlocks = 152;
    const int64_t big = (int64_t)L * ((K + 127) / 128) * ((K + 127) / 128);
    if (big >= kMinBigBlocks) return launch_gram_f32_tiles(reinterpret_cast<const float *>(D), m, K, L,
                                                 reinterpret_cast<float *>(G), st);
  }
  dim3 grid((K + 63) / 64, (K + 63) / 64, L);
  gram_kernel<T><<<grid, 256, 0, st>>>(D, m, K, G);
  return cudaGetLastError();
}

int omp_tile_signals() { return 32; }

template <typename T, int KPL, int MU>
static cudaError_t launch_omp_kpl(const OmpArgs &a, const OmpLayout &lay, cudaStream_t st) {
  auto kern = omp_kernel<T, KPL, MU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.total_tiles, kThreads, lay.total, st>>>(a, lay);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_omp(const OmpArgs &a, int num_sms, cudaStream_t st) {
  (void)num_sms;
  if (a.total_tiles <= 0) return cudaSuccess;
  // Tile: 32 signals (4 per warp).  The selected G columns are cached per warp
  // when they fit beside the correlation tile, else read from L2.
  const int TS = omp_tile_signals();
  const size_t limit = 227 * 1024;
  OmpLayout lay = omp_layout<T>(TS, a.K, a.m, a.s, true);
  if (lay.total > 112 * 1024) lay = omp_layout<T>(TS, a.K, a.m, a.s, false);
  if (lay.total > limit) return cudaErrorInvalidConfiguration;
  const int kpl = (a.K + 31) / 32;
  if (a.m <= 64) {
    if (kpl <= 4) return launch_omp_kpl<T, 4, 2>(a, lay, st);
    if (kpl <= 8) return launch_omp_kpl<T, 8, 2>(a, lay, st);
    if (kpl <= 16) return launch_omp_kpl<T, 16, 2>(a, lay, st);
    return launch_omp_kpl<T, 32, 2>(a, lay, st);
  }
  if (kpl <= 4) return launch_omp_kpl<T, 4, 8>(a, lay, st);
  if (kpl <= 8) return launch_omp_kpl<T, 8, 8>(a, lay, st);
  if (kpl <= 16) return launch_omp_kpl<T, 16, 8>(a, lay, st);
  return launch_omp_kpl<T, 32, 8>(a, lay, st);
}

template cudaError_t launch_gram<float>(const float *, int, int, int, float *, cudaStream_t);
template cudaError_t launch_gram<double>(const double *, int, int, int, double *, cudaStream_t);
template cudaError_t launch_omp<float>(const OmpArgs &, int, cudaStream_t);
template cudaError_t launch_omp<double>(const OmpArgs &, int, cudaStream_t);

}  // namespace sdl
