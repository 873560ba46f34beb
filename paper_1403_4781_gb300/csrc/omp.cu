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

// Shared-memory carve-up of one OMP block (sizes in elements of T unless noted).
struct OmpLayout {
  int TS, K, m, s;
  bool gcache;
  size_t a0, yt, uni, ls, xs, a0s, gss, bs, ss, cp, total;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline OmpLayout omp_layout(int TS, int K, int m, int s, bool gcache) {
  OmpLayout L{};
  L.TS = TS; L.K = K; L.m = m; L.s = s; L.gcache = gcache;
  size_t off = 0;
  L.a0 = off;  off += align16(sizeof(T) * (size_t)TS * K);
  L.yt = off;  off += align16(sizeof(T) * (size_t)TS * m);
  const size_t stage = sizeof(T) * (size_t)kKChunk * kJBlock;
  const size_t gcol = gcache ? sizeof(T) * (size_t)kWarps * s * K : 0;
  L.uni = off; off += align16(stage > gcol ? stage : gcol);
  L.ls = off;  off += align16(sizeof(T) * (size_t)kWarps * s * s);
  L.xs = off;  off += align16(sizeof(T) * (size_t)kWarps * s);
  L.a0s = off; off += align16(sizeof(T) * (size_t)kWarps * s);
  L.gss = off; off += align16(sizeof(T) * (size_t)kWarps * s * s);
  L.bs = off;  off += align16(sizeof(T) * (size_t)kWarps * s);
  L.ss = off;  off += align16(sizeof(int) * (size_t)kWarps * s);
  L.cp = off;  off += align16(sizeof(void *) * (size_t)kWarps * s);
  L.total = off;
  return L;
}

// Solve L L^T x = b for the p x p lower factor L (row stride ld); one thread.
template <typename T>
__device__ void chol_solve_serial(const T *L, int ld, int p, const T *b, T *x) {
  for (int q = 0; q < p; ++q) {
    T v = b[q];
    for (int r = 0; r < q; ++r) v -= L[q * ld + r] * x[r];
    x[q] = v / L[q * ld + q];
  }
  for (int q = p - 1; q >= 0; --q) {
    T v = x[q];
    for (int r = q + 1; r < p; ++r) v -= L[r * ld + q] * x[r];
    x[q] = v / L[q * ld + q];
  }
}

// One block codes a tile of TS signals of one subset.  SPW = signals per warp.
template <typename T, int SPW>
__global__ void __launch_bounds__(kThreads) omp_kernel(OmpArgs a, OmpLayout lay) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TS = SPW * kWarps;
  const int K = a.K, m = a.m, s = a.s;
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
  T *uni = reinterpret_cast<T *>(smem + lay.uni);   // GEMM stage [16][256] / G columns [warps][s][K]

  // ---- load the signal tile (zero rows past the subset end)
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
        uni[kk * kJBlock + jj] = (gj < K && gk < m) ? Dt[(size_t)gj * m + gk] : T(0);
      }
      __syncthreads();
      const int kmax = (m - k0) < kKChunk ? (m - k0) : kKChunk;
      for (int kk = 0; kk < kmax; ++kk) {
        T yv[SPW], dv[8];
#pragma unroll
        for (int r = 0; r < SPW; ++r) yv[r] = yt[(warp * SPW + r) * m + k0 + kk];
#pragma unroll
        for (int c = 0; c < 8; ++c) dv[c] = uni[kk * kJBlock + lane + 32 * c];
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
  __syncthreads();   // GEMM staging is dead from here; the union becomes G columns

  T *Ls = reinterpret_cast<T *>(smem + lay.ls) + (size_t)warp * s * s;
  T *xs = reinterpret_cast<T *>(smem + lay.xs) + (size_t)warp * s;
  T *a0S = reinterpret_cast<T *>(smem + lay.a0s) + (size_t)warp * s;
  T *Gss = reinterpret_cast<T *>(smem + lay.gss) + (size_t)warp * s * s;
  T *bs = reinterpret_cast<T *>(smem + lay.bs) + (size_t)warp * s;
  int *Ss = reinterpret_cast<int *>(smem + lay.ss) + (size_t)warp * s;
  const T **cp = reinterpret_cast<const T **>(smem + lay.cp) + (size_t)warp * s;
  T *gc = lay.gcache ? uni + (size_t)warp * s * K : nullptr;

  const int KPL = (K + 31) >> 5;   // atoms per lane (<= 32)
  const T eps = (T)a.eps;

  for (int q = 0; q < SPW; ++q) {
    const int sig = warp * SPW + q;
    if (sig >= nsig) break;
    const int64_t gi = row0 + sig;
    const T *ysig = yt + sig * m;
    const T *arow = a0 + sig * K;

    T yn2 = T(0);
    for (int r = lane; r < m; r += 32) yn2 = fma(ysig[r], ysig[r], yn2);
    yn2 = warp_sum(yn2);

    uint32_t selmask = 0;   // bit c: atom lane + 32 c selected
    int k = 0;
    T rn2 = yn2;
    while (k < s) {
      if (tsqrt(rn2) <= eps) break;   // rn2 is the explicit ||y - D_S x_S||^2
      // alpha_j = alpha0_j - sum_q G[j, S_q] x_q ; masked argmax |alpha_j|
      T bestv = T(-1);
      int best = -1;
      for (int c = 0; c < KPL; ++c) {
        const int j = lane + 32 * c;
        if (j >= K || ((selmask >> c) & 1u)) continue;
        T av = arow[j];
        for (int p = 0; p < k; ++p) av = fma(-cp[p][j], xs[p], av);
        const T v = fabs(av);
        if (v > bestv) { bestv = v; best = j; }
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
      // column `best` of G (row `best`, G symmetric)
      const T *gcol;
      if (gc) {
        T *dst = gc + (size_t)k * K;
        for (int j = lane; j < K; j += 32) dst[j] = Gt[(size_t)best * K + j];
        gcol = dst;
      } else {
        gcol = Gt + (size_t)best * K;
      }
      __syncwarp();
      // progressive Cholesky: new row [w^T, sqrt(g_bb - w^T w)], L w = G[S, best]
      int ok = 0;
      if (lane == 0) {
        T ww = T(0);
        for (int p = 0; p < k; ++p) {
          T v = gcol[Ss[p]];
          for (int r = 0; r < p; ++r) v -= Ls[p * s + r] * Ls[k * s + r];
          v /= Ls[p * s + p];
          Ls[k * s + p] = v;
          ww = fma(v, v, ww);
        }
        const T gbb = gcol[best];
        const T piv2 = gbb - ww;
        if (piv2 > PivotRel<T>::v * gbb && piv2 > T(0)) {
          ok = 1;
          Ls[k * s + k] = tsqrt(piv2);
          Ss[k] = best;
          cp[k] = gcol;
          a0S[k] = arow[best];
          chol_solve_serial(Ls, s, k + 1, a0S, xs);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) break;
      if ((best & 31) == lane) selmask |= 1u << (best >> 5);
      ++k;
      if (k < s) {   // explicit residual for the stop test of the next step
        T acc = T(0);
        for (int r = lane; r < m; r += 32) {
          T v = ysig[r];
          for (int p = 0; p < k; ++p) v = fma(-Dt[(size_t)Ss[p] * m + r], xs[p], v);
          acc = fma(v, v, acc);
        }
        rn2 = warp_sum(acc);
      }
    }

    // ---- refinement on the support: exact Gram of D_S, solve, one correction step
    T res2 = yn2;
    if (k > 0) {
      for (int p = 0; p < k; ++p) {
        const T *dp = Dt + (size_t)Ss[p] * m;
        for (int p2 = 0; p2 <= p; ++p2) {
          const T *dq = Dt + (size_t)Ss[p2] * m;
          T acc = T(0);
          for (int r = lane; r < m; r += 32) acc = fma(dp[r], dq[r], acc);
          acc = warp_sum(acc);
          if (lane == 0) Gss[p * s + p2] = acc;
        }
        T acc = T(0);
        for (int r = lane; r < m; r += 32) acc = fma(dp[r], ysig[r], acc);
        acc = warp_sum(acc);
        if (lane == 0) bs[p] = acc;
      }
      __syncwarp();
      int fact_ok = 1;
      if (lane == 0) {
        for (int p = 0; p < k && fact_ok; ++p) {
          T d = Gss[p * s + p];
          for (int r = 0; r < p; ++r) d -= Gss[p * s + r] * Gss[p * s + r];
          if (!(d > T(0))) { fact_ok = 0; break; }
          const T lpp = tsqrt(d);
          Gss[p * s + p] = lpp;
          for (int i = p + 1; i < k; ++i) {
            T v = Gss[i * s + p];
            for (int r = 0; r < p; ++r) v -= Gss[i * s + r] * Gss[p * s + r];
            Gss[i * s + p] = v / lpp;
          }
        }
        if (fact_ok) chol_solve_serial(Gss, s, k, bs, xs);
      }
      fact_ok = __shfl_sync(0xffffffffu, fact_ok, 0);
      __syncwarp();
      // (if the exact support Gram is not numerically positive, keep the Batch-OMP x)
      for (int pass = 0; pass < 2; ++pass) {
        // r = y - D_S x; pass 0: correction right-hand side; pass 1: final residual
        T racc = T(0);
        T rloc[kMaxM / 32];
#pragma unroll
        for (int u = 0; u < kMaxM / 32; ++u) {
          const int r = lane + 32 * u;
          T v = T(0);
          if (r < m) {
            v = ysig[r];
            for (int p = 0; p < k; ++p) v = fma(-Dt[(size_t)Ss[p] * m + r], xs[p], v);
          }
          rloc[u] = v;
          racc = fma(v, v, racc);
        }
        if (pass == 1 || !fact_ok) {
          res2 = warp_sum(racc);
          break;
        }
        for (int p = 0; p < k; ++p) {
          const T *dp = Dt + (size_t)Ss[p] * m;
          T acc = T(0);
#pragma unroll
          for (int u = 0; u < kMaxM / 32; ++u) {
            const int r = lane + 32 * u;
            if (r < m) acc = fma(dp[r], rloc[u], acc);
          }
          acc = warp_sum(acc);
          if (lane == 0) bs[p] = acc;
        }
        __syncwarp();
        if (lane == 0) {
          T dx[kMaxS];
          chol_solve_serial(Gss, s, k, bs, dx);
          for (int p = 0; p < k; ++p) xs[p] += dx[p];
        }
        __syncwarp();
      }
    }

    // ---- write the ELL row
    T *val = static_cast<T *>(a.val);
    for (int p = lane; p < s; p += 32) {
      a.idx[(size_t)gi * s + p] = p < k ? Ss[p] : -1;
      val[(size_t)gi * s + p] = p < k ? xs[p] : T(0);
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

template <typename T, int SPW>
static cudaError_t launch_omp_spw(const OmpArgs &a, const OmpLayout &lay, cudaStream_t st) {
  auto kern = omp_kernel<T, SPW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lay.total);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.total_tiles, kThreads, lay.total, st>>>(a, lay);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_omp(const OmpArgs &a, int num_sms, cudaStream_t st) {
  (void)num_sms;
  if (a.total_tiles <= 0) return cudaSuccess;
  // Tile size is fixed at 32 signals (4 per warp); the G-column cache is used
  // when it fits next to the correlation tile.
  const int TS = omp_tile_signals();
  const size_t limit = 227 * 1024;
  OmpLayout lay = omp_layout<T>(TS, a.K, a.m, a.s, true);
  if (lay.total > limit) lay = omp_layout<T>(TS, a.K, a.m, a.s, false);
  if (lay.total > limit) return cudaErrorInvalidConfiguration;
  return launch_omp_spw<T, 4>(a, lay, st);
}

template cudaError_t launch_gram<float>(const float *, int, int, int, float *, cudaStream_t);
template cudaError_t launch_gram<double>(const double *, int, int, int, double *, cudaStream_t);
template cudaError_t launch_omp<float>(const OmpArgs &, int, cudaStream_t);
template cudaError_t launch_omp<double>(const OmpArgs &, int, cudaStream_t);

}  // namespace sdl
