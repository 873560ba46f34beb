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

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kJBlock = 256;   // atoms per GEMM pass (8 per lane)
constexpr int kKChunk = 16;    // signal entries per GEMM stage

template <typename T> __device__ __forceinline__ T tsqrt(T v);
template <> __device__ __forceinline__ float tsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double tsqrt<double>(double v) { return sqrt(v); }

template <typename T> struct PivotRel;
template <> struct PivotRel<float> { static constexpr float v = kOmpPivotRelF32; };
template <> struct PivotRel<double> { static constexpr double v = kOmpPivotRelF64; };

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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
__device__ __forceinline__ int find_subset(const int32_t *__restrict__ tile_start, int L, int64_t g) {
  int lo = 0, hi = L;   // tile_start[lo] <= g < tile_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_start[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Shared-memory carve-up of one OMP block.
struct OmpLayout {
  int TS, K, m, s, lp;   // lp: odd row pitch of the per-warp Cholesky factor
  bool gcache;
  size_t a0, yt, uni, ls, total;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

constexpr int kStagePitch = kJBlock + 1;   // conflict-free transposed staging

template <typename T>
__host__ __device__ inline OmpLayout omp_layout(int TS, int K, int m, int s, bool gcache) {
  OmpLayout L{};
  L.TS = TS; L.K = K; L.m = m; L.s = s; L.gcache = gcache;
  L.lp = (s % 2 == 0) ? s + 1 : s + 2;
  size_t off = 0;
  L.a0 = off;  off += align16(sizeof(T) * (size_t)TS * K);
  L.yt = off;  off += align16(sizeof(T) * (size_t)TS * m);
  const size_t stage = sizeof(T) * (size_t)kKChunk * kStagePitch;
  const size_t gcol = gcache ? sizeof(T) * (size_t)kWarps * s * K : 0;
  L.uni = off; off += align16(stage > gcol ? stage : gcol);
  L.ls = off;  off += align16(sizeof(T) * (size_t)kWarps * s * L.lp);
  L.total = off;
  return L;
}

// Lane-distributed triangular solves with the per-warp factor L (row pitch lp):
// lane q holds entry q of the vector.  Column sweeps: one shuffle and one FMA
// per step, every lane busy.
template <typename T>
__device__ __forceinline__ T lower_solve(const T *L, int lp, int k, T b, int lane) {
  T z = T(0);
  for (int q = 0; q < k; ++q) {
    const T zq = __shfl_sync(0xffffffffu, b / L[q * lp + q], q);
    if (lane == q) z = zq;
    if (lane > q && lane < k) b = fma(-L[lane * lp + q], zq, b);
  }
  return z;
}

template <typename T>
__device__ __forceinline__ T upper_solve(const T *L, int lp, int k, T z, int lane) {
  T x = T(0);
  for (int q = k - 1; q >= 0; --q) {
    const T xq = __shfl_sync(0xffffffffu, z / L[q * lp + q], q);
    if (lane == q) x = xq;
    if (lane < q) z = fma(-L[q * lp + lane], xq, z);
  }
  return x;
}

// One block codes a tile of TS = 4 * 8 signals of one subset; each warp runs the
// selection loop for its 4 signals.  KPL = atoms per lane (K <= 32 KPL): the
// signal's alpha0 row lives in registers, atom j = lane + 32 c.  The support
// (atom, alpha0, coefficient, factor row) is spread one entry per lane.
template <typename T, int KPL>
__global__ void __launch_bounds__(kThreads) omp_kernel(OmpArgs a, OmpLayout lay) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int SPW = 4;
  const int TS = SPW * kWarps;
  const int K = a.K, m = a.m, s = a.s, lp = lay.lp;
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
  T *yt = reinterpret_cast<T *>(smem + lay.yt);     // [TS][m]
  T *uni = reinterpret_cast<T *>(smem + lay.uni);   // GEMM stage / G columns [warps][s][K]

  for (int q = threadIdx.x; q < TS * m; q += kThreads) {
    const int sig = q / m, r = q - sig * m;
    yt[q] = sig < nsig ? Y[(size_t)(row0 + sig) * m + r] : T(0);
  }

  // ---- alpha0[sig][j] = <y_sig, d_j>: register tile SPW signals x 8 atoms per thread
  for (int jb = 0; jb < K; jb += kJBlock) {
    T acc[SPW][8];
#pragma unroll
    for (int r = 0; r < SPW; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = T(0);
    for (int k0 = 0; k0 < m; k0 += kKChunk) {
      __syncthreads();
      for (int q = threadIdx.x; q < kKChunk * kJBlock; q += kThreads) {
        const int jj = q / kKChunk, kk = q - jj * kKChunk;
        const int gj = jb + jj, gk = k0 + kk;
        uni[kk * kStagePitch + jj] = (gj < K && gk < m) ? Dt[(size_t)gj * m + gk] : T(0);
      }
      __syncthreads();
      const int kmax = (m - k0) < kKChunk ? (m - k0) : kKChunk;
      for (int kk = 0; kk < kmax; ++kk) {
        T yv[SPW], dv[8];
#pragma unroll
        for (int r = 0; r < SPW; ++r) yv[r] = yt[(warp * SPW + r) * m + k0 + kk];
#pragma unroll
        for (int c = 0; c < 8; ++c) dv[c] = uni[kk * kStagePitch + lane + 32 * c];
#pragma unroll
        for (int r = 0; r < SPW; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = fma(yv[r], dv[c], acc[r][c]);
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

  T *Ls = reinterpret_cast<T *>(smem + lay.ls) + (size_t)warp * s * lp;
  T *gc = uni + (size_t)warp * s * K;
  const bool gcache = lay.gcache;
  const T eps = (T)a.eps;
  uint32_t valid = 0;   // bit c: atom lane + 32 c exists
#pragma unroll
  for (int c = 0; c < KPL; ++c)
    if (lane + 32 * c < K) valid |= 1u << c;

  for (int q = 0; q < SPW; ++q) {
    const int sig = warp * SPW + q;
    if (sig >= nsig) break;
    const int64_t gi = row0 + sig;
    const T *ysig = yt + sig * m;
    const T *arow = a0 + sig * K;
    T a0r[KPL];
#pragma unroll
    for (int c = 0; c < KPL; ++c) a0r[c] = (valid >> c) & 1u ? arow[lane + 32 * c] : T(0);

    T yn2 = T(0);
    for (int r = lane; r < m; r += 32) yn2 = fma(ysig[r], ysig[r], yn2);
    yn2 = warp_sum(yn2);

    uint32_t avail = valid;   // unselected existing atoms of this lane
    int k = 0;
    int Sl = -1;              // lane p: p-th selected atom
    T a0Sl = T(0), xl = T(0); // lane p: its alpha0 and coefficient
    T rn2 = yn2;
    while (k < s) {
      if (eps > T(0) && tsqrt(rn2) <= eps) break;
      // alpha = alpha0 - G[:, S] x_S, masked argmax |alpha| (lowest index on ties)
      T av[KPL];
#pragma unroll
      for (int c = 0; c < KPL; ++c) av[c] = a0r[c];
      for (int p = 0; p < k; ++p) {
        const T xp = __shfl_sync(0xffffffffu, xl, p);
        const T *gp = gcache ? gc + (size_t)p * K : Gt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * K;
#pragma unroll
        for (int c = 0; c < KPL; ++c)
          if ((valid >> c) & 1u) av[c] = fma(-gp[lane + 32 * c], xp, av[c]);
      }
      T bestv = T(-1);
      int best = -1;
#pragma unroll
      for (int c = 0; c < KPL; ++c) {
        const T v = fabs(av[c]);
        if (((avail >> c) & 1u) && v > bestv) { bestv = v; best = lane + 32 * c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bestv, o);
        const int oj = __shfl_xor_sync(0xffffffffu, best, o);
        if (ov > bestv || (ov == bestv && oj >= 0 && (best < 0 || oj < best))) {
          bestv = ov;
          best = oj;
        }
      }
      if (best < 0 || !(bestv > T(0))) break;
      T a0b = T(0);
#pragma unroll
      for (int c = 0; c < KPL; ++c)
        if (c == (best >> 5)) a0b = a0r[c];
      a0b = __shfl_sync(0xffffffffu, a0b, best & 31);
      // column `best` of G (= row, G symmetric)
      const T *gcol = Gt + (size_t)best * K;
      if (gcache) {
        T *dst = gc + (size_t)k * K;
        for (int j = lane; j < K; j += 32) dst[j] = gcol[j];
        __syncwarp();
        gcol = dst;
      }
      // progressive Cholesky: L w = G[S, best]; new row [w^T, sqrt(g_bb - w^T w)]
      const T gS = lane < k ? gcol[Sl] : T(0);
      const T w = lower_solve(Ls, lp, k, gS, lane);
      const T gbb = gcol[best];
      const T piv2 = gbb - warp_sum(lane < k ? w * w : T(0));
      if (!(piv2 > PivotRel<T>::v * gbb) || !(piv2 > T(0))) break;
      if (lane < k) Ls[k * lp + lane] = w;
      if (lane == k) {
        Ls[k * lp + k] = tsqrt(piv2);
        Sl = best;
        a0Sl = a0b;
      }
      if ((best & 31) == lane) avail &= ~(1u << (best >> 5));
      __syncwarp();
      ++k;
      xl = upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, a0Sl, lane), lane);
      if (eps > T(0) && k < s) {   // explicit residual for the error-constrained stop
        constexpr int M32 = kMaxM / 32;
        const int mu = (m + 31) >> 5;
        T rl[M32];
#pragma unroll
        for (int u = 0; u < M32; ++u) rl[u] = (u < mu && lane + 32 * u < m) ? ysig[lane + 32 * u] : T(0);
        for (int p = 0; p < k; ++p) {   // every lane runs the shuffles; rows are guarded inside
          const T *dp = Dt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * m;
          const T xp = __shfl_sync(0xffffffffu, xl, p);
#pragma unroll
          for (int u = 0; u < M32; ++u)
            if (u < mu && lane + 32 * u < m) rl[u] = fma(-dp[lane + 32 * u], xp, rl[u]);
        }
        T acc = T(0);
#pragma unroll
        for (int u = 0; u < M32; ++u) acc = fma(rl[u], rl[u], acc);
        rn2 = warp_sum(acc);
      }
    }

    // ---- one refinement step on the support: x += G_SS^{-1} D_S^T (y - D_S x)
    T res2 = yn2;
    if (k > 0) {
      constexpr int M32 = kMaxM / 32;
      const int mu = (m + 31) >> 5;
      for (int pass = 0; pass < 2; ++pass) {
        T rloc[M32];
#pragma unroll
        for (int u = 0; u < M32; ++u) rloc[u] = (u < mu && lane + 32 * u < m) ? ysig[lane + 32 * u] : T(0);
        for (int p = 0; p < k; ++p) {
          const T *dp = Dt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * m;
          const T xp = __shfl_sync(0xffffffffu, xl, p);
#pragma unroll
          for (int u = 0; u < M32; ++u)
            if (u < mu && lane + 32 * u < m) rloc[u] = fma(-dp[lane + 32 * u], xp, rloc[u]);
        }
        if (pass == 1) {
          T racc = T(0);
#pragma unroll
          for (int u = 0; u < M32; ++u) racc = fma(rloc[u], rloc[u], racc);
          res2 = warp_sum(racc);
          break;
        }
        T cl = T(0);   // lane p: d_{S_p}^T r
        for (int p = 0; p < k; ++p) {
          const T *dp = Dt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * m;
          T acc = T(0);
#pragma unroll
          for (int u = 0; u < M32; ++u)
            if (u < mu && lane + 32 * u < m) acc = fma(dp[lane + 32 * u], rloc[u], acc);
          acc = warp_sum(acc);
          if (lane == p) cl = acc;
        }
        xl += upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, cl, lane), lane);
      }
    }

    // ---- write the ELL row (lane p holds entry p)
    T *val = static_cast<T *>(a.val);
    if (lane < s) {
      a.idx[(size_t)gi * s + lane] = lane < k ? Sl : -1;
      val[(size_t)gi * s + lane] = lane < k ? xl : T(0);
    }
    if (lane == 0) {
      a.nnz[gi] = k;
      if (a.resid2) static_cast<T *>(a.resid2)[gi] = res2;
    }
    __syncwarp();
  }
}

}  // namespace

// ------------------------------------------------------------- launchers ----
template <typename T>
cudaError_t launch_gram(const T *D, int m, int K, int L, T *G, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  dim3 grid((K + 63) / 64, (K + 63) / 64, L);
  gram_kernel<T><<<grid, 256, 0, st>>>(D, m, K, G);
  return cudaGetLastError();
}

int omp_tile_signals() { return 32; }

template <typename T, int KPL>
static cudaError_t launch_omp_kpl(const OmpArgs &a, const OmpLayout &lay, cudaStream_t st) {
  auto kern = omp_kernel<T, KPL>;
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
  if (kpl <= 4) return launch_omp_kpl<T, 4>(a, lay, st);
  if (kpl <= 8) return launch_omp_kpl<T, 8>(a, lay, st);
  if (kpl <= 16) return launch_omp_kpl<T, 16>(a, lay, st);
  return launch_omp_kpl<T, 32>(a, lay, st);
}

template cudaError_t launch_gram<float>(const float *, int, int, int, float *, cudaStream_t);
template cudaError_t launch_gram<double>(const double *, int, int, int, double *, cudaStream_t);
template cudaError_t launch_omp<float>(const OmpArgs &, int, cudaStream_t);
template cudaError_t launch_omp<double>(const OmpArgs &, int, cudaStream_t);

}  // namespace sdl
