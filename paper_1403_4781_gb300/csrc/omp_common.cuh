// Device code shared by the OMP kernels (CUDA-core and tensor-core correlation
// front ends): tile-to-subset lookup, lane-distributed small triangular solves,
// and the per-warp Batch-OMP selection loop with its refinement on the support.
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "sdl_internal.cuh"

namespace sdl {
namespace omp_detail {

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

__device__ __forceinline__ int find_subset(const int32_t *__restrict__ tile_start, int L, int64_t g) {
  int lo = 0, hi = L;   // tile_start[lo] <= g < tile_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_start[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ inline int odd_pitch(int s) { return (s % 2 == 0) ? s + 1 : s + 2; }

// Lane-distributed triangular solves with a per-warp lower factor L (row pitch
// lp) whose diagonal slots hold the reciprocals 1 / L_qq: lane q holds entry q
// of the vector.  Column sweeps: one shuffle and one FMA per step, every lane
// busy.
template <typename T>
__device__ __forceinline__ T lower_solve(const T *L, int lp, int k, T b, int lane) {
  T z = T(0);
  for (int q = 0; q < k; ++q) {
    const T zq = __shfl_sync(0xffffffffu, b * L[q * lp + q], q);
    if (lane == q) z = zq;
    if (lane > q && lane < k) b = fma(-L[lane * lp + q], zq, b);
  }
  return z;
}

template <typename T>
__device__ __forceinline__ T upper_solve(const T *L, int lp, int k, T z, int lane) {
  T x = T(0);
  for (int q = k - 1; q >= 0; --q) {
    const T xq = __shfl_sync(0xffffffffu, z * L[q * lp + q], q);
    if (lane == q) x = xq;
    if (lane < q) z = fma(-L[q * lp + lane], xq, z);
  }
  return x;
}

// Warp argmax of per-lane candidates (bestv, best): the largest value, the
// lowest atom index among equal values; best < 0 marks a lane without one.
// FP32: non-negative floats order like their bit patterns read as unsigned
// integers, so two warp reductions do it; other types take shuffle rounds.
template <typename T>
__device__ __forceinline__ void warp_argmax(T &bestv, int &best) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, bestv, o);
    const int oj = __shfl_xor_sync(0xffffffffu, best, o);
    if (ov > bestv || (ov == bestv && oj >= 0 && (best < 0 || oj < best))) {
      bestv = ov;
      best = oj;
    }
  }
}
template <>
__device__ __forceinline__ void warp_argmax<float>(float &bestv, int &best) {
  const unsigned key = (best >= 0 && bestv > 0.f) ? __float_as_uint(bestv) : 0u;
  const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
  const unsigned cand = (key == kmax && best >= 0) ? (unsigned)best : 0xffffffffu;
  const unsigned bmin = __reduce_min_sync(0xffffffffu, cand);
  bestv = __uint_as_float(kmax);
  best = kmax == 0u ? -1 : (int)bmin;
}

// Lane-distributed dot products of the support atoms with a vector held as
// rloc[u] = v[lane + 32 u]: returns d_{S_p}^T v in lane p.
template <typename T, int M32>
__device__ __forceinline__ T support_dots(const T *Dt, int m, int mu, int k, int Sl, const T (&rloc)[M32], int lane) {
  T out = T(0);
  for (int p = 0; p < k; ++p) {
    const T *dp = Dt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * m;
    T acc = T(0);
#pragma unroll
    for (int u = 0; u < M32; ++u)
      if (u < mu && lane + 32 * u < m) acc = fma(dp[lane + 32 * u], rloc[u], acc);
    acc = warp_sum(acc);
    if (lane == p) out = acc;
  }
  return out;
}

// r = y - D_S x as rloc[u] = r[lane + 32 u].
template <typename T, int M32>
__device__ __forceinline__ void support_residual(const T *Dt, const T *ysig, int m, int mu, int k, int Sl, T xl,
                                                 T (&rloc)[M32], int lane) {
#pragma unroll
  for (int u = 0; u < M32; ++u) rloc[u] = (u < mu && lane + 32 * u < m) ? ysig[lane + 32 * u] : T(0);
  for (int p = 0; p < k; ++p) {
    const T *dp = Dt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * m;
    const T xp = __shfl_sync(0xffffffffu, xl, p);
#pragma unroll
    for (int u = 0; u < M32; ++u)
      if (u < mu && lane + 32 * u < m) rloc[u] = fma(-dp[lane + 32 * u], xp, rloc[u]);
  }
}

// Atom of entry c of a lane's KPL correlations: groups of four consecutive
// atoms, lane l holding atoms 4 l .. 4 l + 3 of every 128 (so a warp's 16-byte
// loads of one group cover 512 contiguous bytes).
__device__ __forceinline__ int lane_atom(int lane, int c) { return 128 * (c >> 2) + 4 * lane + (c & 3); }

// This lane's entries of a row (bit c of `valid`: entry c exists; missing
// entries read as zero); p points at the row's atom 4 lane.  vec: the rows are
// 16-byte aligned (K a multiple of 4), so each group loads as one vector.
template <int KPL>
__device__ __forceinline__ void span_load(const float *p, float (&v)[KPL], uint32_t valid, bool vec) {
#pragma unroll
  for (int c = 0; c < KPL; c += 4) {
    const float *q = p + 128 * (c >> 2);
    if (vec) {
      if ((valid >> c) & 1u) {
        const float4 t = *reinterpret_cast<const float4 *>(q);
        v[c] = t.x; v[c + 1] = t.y; v[c + 2] = t.z; v[c + 3] = t.w;
      } else {
        v[c] = v[c + 1] = v[c + 2] = v[c + 3] = 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c + e] = (valid >> (c + e)) & 1u ? q[e] : 0.f;
    }
  }
}
template <int KPL>
__device__ __forceinline__ void span_load(const double *p, double (&v)[KPL], uint32_t valid, bool vec) {
#pragma unroll
  for (int c = 0; c < KPL; c += 4) {
    const double *q = p + 128 * (c >> 2);
    if (vec) {
      if ((valid >> c) & 1u) {
        const double2 t0 = *reinterpret_cast<const double2 *>(q);
        const double2 t1 = *reinterpret_cast<const double2 *>(q + 2);
        v[c] = t0.x; v[c + 1] = t0.y; v[c + 2] = t1.x; v[c + 3] = t1.y;
      } else {
        v[c] = v[c + 1] = v[c + 2] = v[c + 3] = 0.0;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c + e] = (valid >> (c + e)) & 1u ? q[e] : 0.0;
    }
  }
}

// This lane's entries of a row whose every group exists and is 16-byte
// aligned: unconditional vector loads (no per-group tests).
template <int KPL>
__device__ __forceinline__ void span_load_full(const float *p, float (&v)[KPL]) {
#pragma unroll
  for (int c = 0; c < KPL; c += 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p + 128 * (c >> 2));
    v[c] = t.x; v[c + 1] = t.y; v[c + 2] = t.z; v[c + 3] = t.w;
  }
}

// This lane's entries of a half-precision row (four consecutive atoms per group
// load as one 8-byte vector when vec), widened to FP32.
template <int KPL>
__device__ __forceinline__ void span_load_h(const __half *p, float (&v)[KPL], uint32_t valid, bool vec) {
#pragma unroll
  for (int c = 0; c < KPL; c += 4) {
    const __half *q = p + 128 * (c >> 2);
    if (vec) {
      if ((valid >> c) & 1u) {
        const uint2 t = *reinterpret_cast<const uint2 *>(q);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[c] = a.x; v[c + 1] = a.y; v[c + 2] = b.x; v[c + 3] = b.y;
      } else {
        v[c] = v[c + 1] = v[c + 2] = v[c + 3] = 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c + e] = (valid >> (c + e)) & 1u ? __half2float(q[e]) : 0.f;
    }
  }
}

// The selection loop (Sec. 1 greedy choice, Batch-OMP form), refinement on the
// support and the ELL write-out for signals sig_begin .. sig_begin+sig_count-1
// of a tile, run by one warp.
//   a0     correlation tile alpha0 [tile signals][K] (shared or global memory)
//   ybase  signal 0 of the tile, row stride ypitch (shared or global memory)
//   MU     ceil(m / 32): signal entries per lane
//   Gt     the Gram matrix of D in T (FP32 or FP64 products)
//   Ls     per-warp [s][lp] factor scratch;  gc per-warp [gcn][K] cache of the
//          first gcn G columns of the support (the earliest picks are re-read by
//          the most later updates)
//   EXACT  alpha0 came from reduced-precision products: the refit takes D_S^T y
//          in T instead of alpha0 on the support
//   H16    (FP32 only) the running update alpha -= G[:, S] dx reads a
//          half-precision copy of G (G16t; the shared-memory cache gc holds
//          half columns too), the Cholesky entries still come from the FP32 Gt
// Lane l owns the atoms lane_atom(l, c), c < KPL: its correlations and the
// matching entries of each G column load as 16-byte vectors.
// Per step the correlations are kept as a running vector alpha = alpha0 -
// G[:, S] x_S in registers: after the support grows, alpha -= G[:, S] dx with dx
// the change of every coefficient.  The forward-solved vector z = L^{-1}
// alpha0_S grows by one entry per step, (alpha0_j - w^T z) / l for the new
// factor row [w^T, l], so only x = L^{-T} z is solved again.
template <typename T, int KPL, int MU, bool EXACT, bool H16 = false>
__device__ void code_warp_signals(const OmpArgs &a, const T *a0, const T *ybase, int ypitch, int sig_begin,
                                  int sig_count, int nsig, int64_t row0, const T *__restrict__ Dt,
                                  const T *__restrict__ Gt, T *Ls, void *gcv, int lp, int gcn,
                                  const __half *__restrict__ G16t = nullptr) {
  T *gc = static_cast<T *>(gcv);
  __half *gc16 = static_cast<__half *>(gcv);
  constexpr int M32 = MU;
  const int K = a.K, m = a.m, s = a.s;
  const int lane = threadIdx.x & 31;
  constexpr int mu = MU;
  const T eps = (T)a.eps;
  uint32_t valid = 0;   // bit c: atom lane_atom(lane, c) exists
#pragma unroll
  for (int c = 0; c < KPL; ++c)
    if (lane_atom(lane, c) < K) valid |= 1u << c;
  const bool vec = (K & 3) == 0;   // 16-byte aligned rows of alpha0 and G (warp-uniform)
  const int j0 = 4 * lane;         // this lane's first atom
  // every entry of this lane exists (K a multiple of 128 makes it every lane):
  // rows load without per-group tests
  const bool full = sizeof(T) == 4 && vec && valid == (KPL >= 32 ? 0xffffffffu : ((1u << KPL) - 1u));

  for (int q = 0; q < sig_count; ++q) {
    const int sig = sig_begin + q;
    if (sig >= nsig) break;
    const int64_t gi = row0 + sig;
    const T *ysig = ybase + (size_t)sig * ypitch;
    const T *arow = a0 + (size_t)sig * K;
    T av[KPL];   // running correlations of this lane's atoms
    if constexpr (sizeof(T) == 4) {
      if (full) span_load_full<KPL>(arow + j0, av);
      else span_load<KPL>(arow + j0, av, valid, vec);
    } else {
      span_load<KPL>(arow + j0, av, valid, vec);
    }

    T yn2 = T(0);
#pragma unroll
    for (int u = 0; u < M32; ++u)
      if (u < mu && lane + 32 * u < m) yn2 = fma(ysig[lane + 32 * u], ysig[lane + 32 * u], yn2);
    yn2 = warp_sum(yn2);

    uint32_t avail = valid;   // unselected existing atoms of this lane
    int k = 0;
    int Sl = -1;              // lane p: p-th selected atom
    T zl = T(0), xl = T(0);   // lane p: z_p and the coefficient x_p
    T rn2 = yn2;
    while (k < s) {
      if (eps > T(0) && tsqrt(rn2) <= eps) break;
      // masked argmax |alpha| (lowest index on ties)
      T bestv = T(-1);
      int best = -1;
#pragma unroll
      for (int c = 0; c < KPL; ++c) {
        const T v = fabs(av[c]);
        if (((avail >> c) & 1u) && v > bestv) { bestv = v; best = lane_atom(lane, c); }
      }
      warp_argmax<T>(bestv, best);
      if (best < 0 || !(bestv > T(0))) break;
      const T a0b = arow[best];
      // column `best` of G (= row, G symmetric); the cached copy serves the
      // updates of later steps only, so the last step reads it from L2
      const T *gcol = Gt + (size_t)best * K;
      if (k < gcn && k + 1 < s) {
        if constexpr (H16) {   // the update's half column; the FP32 entries below stay in L2
          const __half *src = G16t + (size_t)best * K;
          __half *dst = gc16 + (size_t)k * K;
          if (vec) {
            for (int j = 4 * lane; j < K; j += 128)
              *reinterpret_cast<uint2 *>(dst + j) = *reinterpret_cast<const uint2 *>(src + j);
          } else {
            for (int j = lane; j < K; j += 32) dst[j] = src[j];
          }
          __syncwarp();
        } else {
          T *dst = gc + (size_t)k * K;
          for (int j = lane; j < K; j += 32) dst[j] = gcol[j];
          __syncwarp();
          gcol = dst;
        }
      }
      // progressive Cholesky: L w = G[S, best]; new row [w^T, sqrt(g_bb - w^T w)]
      const T gS = lane < k ? gcol[Sl] : T(0);
      const T w = lower_solve(Ls, lp, k, gS, lane);
      const T gbb = gcol[best];
      const T piv2 = gbb - warp_sum(lane < k ? w * w : T(0));
      if (!(piv2 > PivotRel<T>::v * gbb) || !(piv2 > T(0))) break;
      const T wz = warp_sum(lane < k ? w * zl : T(0));
      const T rl = T(1) / tsqrt(piv2);
      if (lane < k) Ls[k * lp + lane] = w;
      if (lane == k) {
        Ls[k * lp + k] = rl;
        Sl = best;
        zl = (a0b - wz) * rl;
      }
      if (((best & 127) >> 2) == lane) avail &= ~(1u << (4 * (best >> 7) + (best & 3)));
      __syncwarp();
      ++k;
      const T xn = upper_solve(Ls, lp, k, zl, lane);
      if (k < s) {
        // alpha -= G[:, S] (x_new - x_old); the new atom's old coefficient is 0
        const T dl = xn - xl;
        for (int p = 0; p < k; ++p) {
          const T dp = __shfl_sync(0xffffffffu, dl, p);
          T g[KPL];
          if constexpr (H16) {
            const __half *gp = p < gcn ? gc16 + (size_t)p * K
                                       : G16t + (size_t)__shfl_sync(0xffffffffu, Sl, p) * K;
            span_load_h<KPL>(gp + j0, g, valid, vec);
          } else {
            const T *gp = p < gcn ? gc + (size_t)p * K : Gt + (size_t)__shfl_sync(0xffffffffu, Sl, p) * K;
            if constexpr (sizeof(T) == 4) {
              if (full) span_load_full<KPL>(gp + j0, g);
              else span_load<KPL>(gp + j0, g, valid, vec);
            } else {
              span_load<KPL>(gp + j0, g, valid, vec);
            }
          }
#pragma unroll
          for (int c = 0; c < KPL; ++c) av[c] = fma(-g[c], dp, av[c]);
        }
      }
      xl = xn;
      if (eps > T(0) && k < s) {   // explicit residual for the error-constrained stop
        T rl2[M32];
        support_residual(Dt, ysig, m, mu, k, Sl, xl, rl2, lane);
        T acc = T(0);
#pragma unroll
        for (int u = 0; u < M32; ++u) acc = fma(rl2[u], rl2[u], acc);
        rn2 = warp_sum(acc);
      }
    }

    // ---- refinement on the support
    T res2 = yn2;
    if (k > 0) {
      if (EXACT) {   // x = G_SS^{-1} D_S^T y with D_S^T y in T
        T yl[M32];
#pragma unroll
        for (int u = 0; u < M32; ++u) yl[u] = (u < mu && lane + 32 * u < m) ? ysig[lane + 32 * u] : T(0);
        const T bl = support_dots(Dt, m, mu, k, Sl, yl, lane);
        xl = upper_solve(Ls, lp, k, lower_solve(Ls, lp, k, bl, lane), lane);
      }
      // one correction step x += G_SS^{-1} c, c = D_S^T r, r = y - D_S x.  The
      // corrected residual's energy follows without another pass over D_S:
      // ||r - D_S G_SS^{-1} c||^2 = ||r||^2 - c^T G_SS^{-1} c = ||r||^2 - ||L^{-1} c||^2
      T rloc[M32];
      support_residual(Dt, ysig, m, mu, k, Sl, xl, rloc, lane);
      T racc = T(0);
#pragma unroll
      for (int u = 0; u < M32; ++u) racc = fma(rloc[u], rloc[u], racc);
      const T cl = support_dots(Dt, m, mu, k, Sl, rloc, lane);
      const T wl = lower_solve(Ls, lp, k, cl, lane);
      xl += upper_solve(Ls, lp, k, wl, lane);
      const T r2 = warp_sum(racc) - warp_sum(lane < k ? wl * wl : T(0));
      res2 = r2 > T(0) ? r2 : T(0);
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

}  // namespace omp_detail
}  // namespace sdl
