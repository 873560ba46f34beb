// MOD dictionary update (Sec. 1) with column renormalisation (Sec. 3.1), batched
// over subsets.  D_U = B_U A_UU^{-1}, A = X X^T, B = Y X^T, U = used atoms.
//
//  1. usage[t][j] = number of signals of subset t whose code uses atom j.
//  2. CSC transpose of the ELL codes (per subset, per atom: list of (signal, slot)).
//  3. One warp per (subset, atom j): B[:, j] = sum_i x_ij y_i and row j of A,
//     accumulated in FP64 from exact FP32 x FP32 products.  An unused atom gets
//     the identity row and B[:, j] = its previous value, which decouples it:
//     the solve then returns the previous atom unchanged.
//  4. FP64 blocked Cholesky of A (one block per subset, 32x32 tiles); a squared
//     pivot <= 1e-12 of its diagonal is a breakdown -> one retry with
//     A_UU + lambda I, lambda = 1e-10 tr(A_UU)/|U|.
//  5. FP64 blocked forward/back substitution, the m right-hand sides split over
//     blocks: B <- A^{-1} B (column j of B is atom j's m values).
//  6. Used atoms scaled to unit norm; zero or non-finite columns keep the old atom.
#include <cooperative_groups.h>
#include <math.h>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr int kModTile = 256;   // signals per block in the count / fill passes
constexpr int kNb = 32;         // Cholesky / solve tile

__device__ __forceinline__ int find_subset_tiles(const int32_t *__restrict__ tile_start, int L,
                                                 int64_t g) {
  int lo = 0, hi = L;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_start[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- 1 + 2: usage counts, scan, fill --------------------------------------
// Counts of one tile of signals are gathered in a shared-memory histogram first,
// so the global counters take one atomic per (tile, atom) instead of one per
// code entry (the merge's single subset would otherwise serialise many atomics
// on each of its K counters).
__global__ void mod_count_kernel(ModArgs a) {
  __shared__ int hist[1024];   // K <= 1024
  const int64_t g = blockIdx.x;
  const int t = find_subset_tiles(a.tile_start, a.L, g);
  const int K = a.K;
  for (int j = threadIdx.x; j < K; j += kModTile) hist[j] = 0;
  __syncthreads();
  const int64_t i = a.offsets[t] + (g - a.tile_start[t]) * kModTile + threadIdx.x;
  if (i < a.offsets[t + 1])
    for (int k = 0; k < a.s; ++k) {
      const int j = a.idx[(size_t)i * a.s + k];
      if (j >= 0 && j < K) atomicAdd_block(&hist[j], 1);
    }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += kModTile)
    if (hist[j] > 0) atomicAdd(&a.usage[(size_t)t * K + j], hist[j]);
}

// Exclusive scan of usage[t][0..K) -> ptr[t][0..K]; cursor = ptr.  K <= 1024.
__global__ void __launch_bounds__(1024) mod_scan_kernel(ModArgs a) {
  __shared__ int warp_tot[32];
  const int t = blockIdx.x;
  const int j = threadIdx.x;
  const int lane = j & 31, w = j >> 5;
  const int v = j < a.K ? a.usage[(size_t)t * a.K + j] : 0;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    warp_tot[lane] = x;   // inclusive over warps
  }
  __syncthreads();
  const int excl = incl - v + (w > 0 ? warp_tot[w - 1] : 0);
  if (j < a.K) {
    a.ptr[(size_t)t * (a.K + 1) + j] = excl;
    a.cursor[(size_t)t * a.K + j] = excl;
  }
  if (j == a.K - 1) a.ptr[(size_t)t * (a.K + 1) + a.K] = excl + v;
}

__global__ void mod_fill_kernel(ModArgs a) {
  const int64_t g = blockIdx.x;
  const int t = find_subset_tiles(a.tile_start, a.L, g);
  const int64_t i = a.offsets[t] + (g - a.tile_start[t]) * kModTile + threadIdx.x;
  if (i >= a.offsets[t + 1]) return;
  const int64_t base = a.offsets[t] * a.s;
  for (int k = 0; k < a.s; ++k) {
    const int j = a.idx[(size_t)i * a.s + k];
    if (j < 0 || j >= a.K) continue;
    const int pos = atomicAdd(&a.cursor[(size_t)t * a.K + j], 1);
    a.lsig[base + pos] = (int32_t)(i - a.offsets[t]);
    a.lslot[base + pos] = k;
    a.latom[base + pos] = j;
  }
}

// ---- 3: A and B accumulation, one warp per (subset, atom) --------------------
// The atom's list is walked in batches of 8 entries whose loads are all issued
// before any is consumed; M32 = ceil(m / 32) signal entries per lane.
template <typename T, int M32>
__global__ void __launch_bounds__(256) mod_accum_kernel(ModArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *arow_all = reinterpret_cast<double *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y;
  const int j = blockIdx.x * 8 + warp;
  if (j >= a.K) return;
  const int K = a.K, m = a.m, s = a.s;
  double *arow = arow_all + (size_t)warp * K;
  const T *__restrict__ Y = static_cast<const T *>(a.Y) + (size_t)a.offsets[t] * m;
  const T *__restrict__ val = static_cast<const T *>(a.val) + (size_t)a.offsets[t] * s;
  const int32_t *__restrict__ idx = a.idx + (size_t)a.offsets[t] * s;
  double *Arow_g = a.A + ((size_t)t * K + j) * K;
  double *Bcol = a.B + ((size_t)t * K + j) * m;
  const int c = a.usage[(size_t)t * K + j];
  if (c == 0) {
    const T *Dj = static_cast<const T *>(a.D) + ((size_t)t * K + j) * m;
    for (int q = lane; q < K; q += 32) Arow_g[q] = q == j ? 1.0 : 0.0;
    for (int r = lane; r < m; r += 32) Bcol[r] = (double)Dj[r];
    return;
  }
  for (int q = lane; q < K; q += 32) arow[q] = 0.0;
  __syncwarp();
  double b[M32];
#pragma unroll
  for (int u = 0; u < M32; ++u) b[u] = 0.0;
  const int64_t base = a.offsets[t] * s + a.ptr[(size_t)t * (K + 1) + j];
  constexpr int kB = 8;
  for (int e0 = 0; e0 < c; e0 += 32) {
    const int ne = (c - e0) < 32 ? (c - e0) : 32;
    int my_i = 0;
    double my_v = 0.0;
    if (lane < ne) {
      my_i = a.lsig[base + e0 + lane];
      my_v = (double)val[(size_t)my_i * s + a.lslot[base + e0 + lane]];
    }
    for (int eb = 0; eb < ne; eb += kB) {
      int ii[kB];
      double vv[kB];
      T yv[kB][M32];
      int j2[kB];
      double x2[kB];
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        ii[q] = __shfl_sync(0xffffffffu, my_i, (eb + q) & 31);
        vv[q] = __shfl_sync(0xffffffffu, my_v, (eb + q) & 31);
        if (eb + q >= ne) vv[q] = 0.0;
      }
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        const T *yi = Y + (size_t)ii[q] * m;
#pragma unroll
        for (int u = 0; u < M32; ++u) {
          const int r = lane + 32 * u;
          yv[q][u] = (r < m && eb + q < ne) ? yi[r] : T(0);
        }
        j2[q] = (lane < s && eb + q < ne) ? idx[(size_t)ii[q] * s + lane] : -1;
        x2[q] = (lane < s && eb + q < ne) ? (double)val[(size_t)ii[q] * s + lane] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kB; ++q)
#pragma unroll
        for (int u = 0; u < M32; ++u) b[u] = fma(vv[q], (double)yv[q][u], b[u]);
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        if (j2[q] >= 0 && j2[q] < K) arow[j2[q]] = fma(vv[q], x2[q], arow[j2[q]]);
        __syncwarp();
      }
    }
  }
  for (int q = lane; q < K; q += 32) Arow_g[q] = arow[q];
#pragma unroll
  for (int u = 0; u < M32; ++u) {
    const int r = lane + 32 * u;
    if (r < m) Bcol[r] = b[u];
  }
}

// ---- 3 (FP32 signals): A and B from the CSC entries, warps over entry ranges --
// Each warp takes 32 s consecutive CSC entries of a subset (atom-major, so a
// range spans few atoms).  B[:, j] = sum x_ij y_i is accumulated per run of
// equal atoms by compensated summation on the FP32 pipe -- each product x y of
// two floats is split exactly into p + e by an FMA, p is added with TwoSum and
// the errors are collected in a second float, so the run's sum is good to
// about 2^-48 of its terms' magnitudes -- and added to B in FP64 when the atom
// changes.  Every entry (i, j) adds x_ij x_ij2 (exact in FP64) to A[j][j2] for
// the atoms j2 <= j of its signal, so A's lower triangle is complete.  A and B
// start at zero; unused atoms get their identity row and previous value after.
struct DSum {
  float hi, lo;
};

// hi is the plain FP32 running sum; every rounding error it makes (TwoSum,
// exact) and every product's low part e go into lo, which stays about 2^-24 of
// the sum's magnitude per term, so its own rounding is negligible (compensated
// summation, no renormalisation per term).  Explicit _rn operations keep the
// compiler from contracting the sums with the product.
__device__ __forceinline__ void ds_add_product(DSum &a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = fmaf(x, y, -p);          // x y = p + e exactly
  const float s = __fadd_rn(a.hi, p);      // TwoSum(a.hi, p) = s + err exactly
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(e, err));
}

template <int MU>
__global__ void __launch_bounds__(256) mod_accum_ds_kernel(ModArgs a) {
  const int K = a.K, m = a.m, s = a.s;
  const int64_t g = blockIdx.x;
  const int t = find_subset_tiles(a.tile_start, a.L, g);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t E = a.ptr[(size_t)t * (K + 1) + K];
  const int64_t span = 32 * (int64_t)s;
  const int64_t e_lo = (g - a.tile_start[t]) * (int64_t)kModTile * s + warp * span;
  if (e_lo >= E) return;
  const int64_t e_hi = e_lo + span < E ? e_lo + span : E;
  const int64_t base = a.offsets[t] * s;
  const float *__restrict__ Yt = static_cast<const float *>(a.Y) + (size_t)a.offsets[t] * m;
  const float *__restrict__ vt = static_cast<const float *>(a.val) + (size_t)a.offsets[t] * s;
  const int32_t *__restrict__ it = a.idx + (size_t)a.offsets[t] * s;
  double *At = a.A + (size_t)t * K * K;
  double *Bt = a.B + (size_t)t * K * m;
  DSum acc[MU];
#pragma unroll
  for (int u = 0; u < MU; ++u) acc[u] = DSum{0.f, 0.f};
  int cur = -1;
  for (int64_t e0 = e_lo; e0 < e_hi; e0 += 32) {
    const int64_t e = e0 + lane;
    const bool ok = e < e_hi;
    const int i = ok ? a.lsig[base + e] : 0;
    const int j = ok ? a.latom[base + e] : -1;
    const int slot = ok ? a.lslot[base + e] : 0;
    const float x = ok ? vt[(size_t)i * s + slot] : 0.f;
    if (ok)
      for (int k = 0; k < s; ++k) {
        const int j2 = it[(size_t)i * s + k];
        if (j2 >= 0 && (j2 < j || (j2 == j && k != slot)))
          atomicAdd(&At[(size_t)j * K + j2], (double)x * (double)vt[(size_t)i * s + k]);
      }
    // the diagonal term x^2 of every entry, summed over the lanes of a run of
    // equal atoms (contiguous: the entries are atom-major) and added once, so
    // the diagonal counters do not serialise one atomic per entry
    {
      double d = (double)x * (double)x;
      const unsigned grp = __match_any_sync(0xffffffffu, j);
      const int lo = __ffs(grp) - 1, hi = 31 - __clz(grp);
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const double o = __shfl_down_sync(0xffffffffu, d, off);
        if (lane + off <= hi) d += o;
      }
      if (ok && lane == lo) atomicAdd(&At[(size_t)j * K + j], d);
    }
    // the entries' signal rows are loaded kB at a time (their loads in flight
    // together), then added in entry order
    constexpr int kB = MU <= 2 ? 8 : 1;   // wider rows: registers would cost occupancy
    const int nq = e_hi - e0 < 32 ? (int)(e_hi - e0) : 32;
    for (int q0 = 0; q0 < nq; q0 += kB) {
      float yb[kB][MU], xb[kB];
      int jb[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int q = q0 + b;   // < 32: kB divides 32
        const int jq = __shfl_sync(0xffffffffu, j, q);
        const int iq = __shfl_sync(0xffffffffu, i, q);
        xb[b] = __shfl_sync(0xffffffffu, x, q);
        jb[b] = q < nq ? jq : -2;   // -2: past the range
        const float *yr = Yt + (size_t)iq * m;
#pragma unroll
        for (int u = 0; u < MU; ++u) {
          const int r = lane + 32 * u;
          yb[b][u] = (q < nq && r < m) ? yr[r] : 0.f;
        }
      }
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        if (jb[b] == -2) break;   // warp-uniform
        if (jb[b] != cur) {       // warp-uniform
          if (cur >= 0)
#pragma unroll
            for (int u = 0; u < MU; ++u) {
              const int r = lane + 32 * u;
              if (r < m) atomicAdd(&Bt[(size_t)cur * m + r], (double)acc[u].hi + (double)acc[u].lo);
              acc[u] = DSum{0.f, 0.f};
            }
          cur = jb[b];
        }
#pragma unroll
        for (int u = 0; u < MU; ++u)
          if (lane + 32 * u < m) ds_add_product(acc[u], xb[b], yb[b][u]);
      }
    }
  }
  if (cur >= 0)
#pragma unroll
    for (int u = 0; u < MU; ++u) {
      const int r = lane + 32 * u;
      if (r < m) atomicAdd(&Bt[(size_t)cur * m + r], (double)acc[u].hi + (double)acc[u].lo);
    }
}

// Unused atoms: identity row of A (its off-diagonal entries stayed zero) and
// B = the previous atom, which decouples them in the solve.
template <typename T>
__global__ void mod_unused_kernel(ModArgs a) {
  const int t = blockIdx.y;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= a.K || a.usage[(size_t)t * a.K + j] != 0) return;
  if (lane == 0) a.A[((size_t)t * a.K + j) * a.K + j] = 1.0;
  const T *Dj = static_cast<const T *>(a.D) + ((size_t)t * a.K + j) * a.m;
  for (int r = lane; r < a.m; r += 32) a.B[((size_t)t * a.K + j) * a.m + r] = (double)Dj[r];
}

// ---- 4: FP64 blocked Cholesky, one block (256 threads) per subset -----------
// Lf receives the lower factor (upper part untouched).  status[t]: 0 ok,
// 1 ridge retry taken, 2 breakdown after the retry.
__global__ void __launch_bounds__(256) chol_kernel(const double *__restrict__ A, double *Lf,
                                                   const int32_t *__restrict__ usage, int K,
                                                   int32_t *status) {
  __shared__ double Dblk[kNb][kNb + 1];
  __shared__ double Pi[kNb][kNb + 1];
  __shared__ double Pj[kNb][kNb + 1];
  __shared__ double red[2][8];
  __shared__ int fail;
  const int t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double *At = A + (size_t)t * K * K;
  double *Lt = Lf + (size_t)t * K * K;
  const int32_t *ut = usage + (size_t)t * K;

  // ridge = 1e-10 tr(A_UU) / |U|
  double tr = 0.0, nu = 0.0;
  for (int j = tid; j < K; j += 256)
    if (ut[j] > 0) { tr += At[(size_t)j * K + j]; nu += 1.0; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    nu += __shfl_xor_sync(0xffffffffu, nu, o);
  }
  if (lane == 0) { red[0][warp] = tr; red[1][warp] = nu; }
  __syncthreads();
  double lambda = 0.0;
  {
    double T0 = 0.0, N0 = 0.0;
    for (int w = 0; w < 8; ++w) { T0 += red[0][w]; N0 += red[1][w]; }
    lambda = N0 > 0.0 ? kModRidge * T0 / N0 : 0.0;
  }

  int st = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double ridge = attempt == 0 ? 0.0 : lambda;
    // copy the lower triangle (with ridge on used diagonal entries)
    for (size_t q = tid; q < (size_t)K * K; q += 256) {
      const int i = (int)(q / K), j = (int)(q % K);
      if (j <= i) Lt[q] = At[q] + ((i == j && ut[i] > 0) ? ridge : 0.0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int kb = 0; kb < K; kb += kNb) {
      const int nb = (K - kb) < kNb ? (K - kb) : kNb;
      // (a) factor the diagonal block in shared memory (warp 0)
      for (int q = tid; q < kNb * kNb; q += 256) {
        const int r = q / kNb, c = q % kNb;
        Dblk[r][c] = (r < nb && c <= r) ? Lt[(size_t)(kb + r) * K + kb + c] : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        for (int c = 0; c < nb; ++c) {
          const double d = Dblk[c][c];
          const double diag0 = At[(size_t)(kb + c) * K + kb + c] + ((ut[kb + c] > 0) ? ridge : 0.0);
          const bool ok = (d > kModPivotRel * diag0) && (d > 0.0);
          if (!ok) { if (lane == 0) fail = 1; break; }
          const double lcc = sqrt(d);
          __syncwarp();
          if (lane == c) Dblk[c][c] = lcc;
          if (lane > c && lane < nb) Dblk[lane][c] /= lcc;
          __syncwarp();
          if (lane > c && lane < nb) {
            const double lr = Dblk[lane][c];
            for (int q = c + 1; q <= lane; ++q) Dblk[lane][q] -= lr * Dblk[q][c];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      if (fail) break;
      for (int q = tid; q < kNb * kNb; q += 256) {
        const int r = q / kNb, c = q % kNb;
        if (r < nb && c <= r) Lt[(size_t)(kb + r) * K + kb + c] = Dblk[r][c];
      }
      // (b) panel: rows below, X L_kk^T = P  (one thread per row, 32-wide row in registers)
      const int r0 = kb + nb;
      for (int i = r0 + tid; i < K; i += 256) {
        double x[kNb];
#pragma unroll
        for (int c = 0; c < kNb; ++c) x[c] = c < nb ? Lt[(size_t)i * K + kb + c] : 0.0;
#pragma unroll
        for (int c = 0; c < kNb; ++c) {
          if (c < nb) {
            double v = x[c];
#pragma unroll
            for (int q = 0; q < c; ++q) v = fma(-x[q], Dblk[c][q], v);
            x[c] = v / Dblk[c][c];
          }
        }
#pragma unroll
        for (int c = 0; c < kNb; ++c)
          if (c < nb) Lt[(size_t)i * K + kb + c] = x[c];
      }
      __syncthreads();
      // (c) trailing update of the lower triangle, 32x32 tiles (I >= J)
      const int ntile = (K - r0 + kNb - 1) / kNb;
      for (int ti = 0; ti < ntile; ++ti) {
        for (int tj = 0; tj <= ti; ++tj) {
          const int I0 = r0 + ti * kNb, J0 = r0 + tj * kNb;
          for (int q = tid; q < kNb * kNb; q += 256) {
            const int r = q / kNb, c = q % kNb;
            Pi[r][c] = (I0 + r < K && c < nb) ? Lt[(size_t)(I0 + r) * K + kb + c] : 0.0;
            Pj[r][c] = (J0 + r < K && c < nb) ? Lt[(size_t)(J0 + r) * K + kb + c] : 0.0;
          }
          __syncthreads();
          const int cx = tid & 31, ry = tid >> 5;   // 4 rows per thread: ry + 8 u
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
          for (int q = 0; q < kNb; ++q) {
            const double pj = Pj[cx][q];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(Pi[ry + 8 * u][q], pj, acc[u]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int gi = I0 + ry + 8 * u, gj = J0 + cx;
            if (gi < K && gj < K && gj <= gi) Lt[(size_t)gi * K + gj] -= acc[u];
          }
          __syncthreads();
        }
      }
    }
    __syncthreads();
    if (!fail) { st = attempt; break; }
    st = 2;
    __syncthreads();
  }
  if (tid == 0) status[t] = st;
}

// ---- 5: FP64 blocked solve A X = B for a chunk of RC right-hand-side rows ----
// B is [K][m] per subset (row j = atom j); the chunk holds entries r0..r0+RC-1
// of every row.  Z lives in shared memory: Z[j][c].
template <int RC>
__global__ void __launch_bounds__(256) solve_kernel(const double *__restrict__ Lf, double *B,
                                                    int K, int m, const int32_t *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *Z = reinterpret_cast<double *>(smem_raw);           // [K][RC]
  __shared__ double Lb[kNb][kNb + 1];
  const int t = blockIdx.x;
  if (status[t] == 2) return;
  const int rc0 = blockIdx.y * RC;
  const int tid = threadIdx.x;
  const double *Lt = Lf + (size_t)t * K * K;
  double *Bt = B + (size_t)t * K * m;
  for (int q = tid; q < K * RC; q += 256) {
    const int j = q / RC, c = q % RC;
    Z[q] = (rc0 + c < m) ? Bt[(size_t)j * m + rc0 + c] : 0.0;
  }
  __syncthreads();
  const int nblk = (K + kNb - 1) / kNb;
  // forward: L Z = B
  for (int b = 0; b < nblk; ++b) {
    const int j0 = b * kNb, nb = (K - j0) < kNb ? (K - j0) : kNb;
    // Z_b -= L[b, 0:j0] Z[0:j0]
    for (int o = tid; o < kNb * RC; o += 256) {
      const int r = o / RC, c = o % RC;
      if (r < nb && j0 > 0) {
        const double *lrow = Lt + (size_t)(j0 + r) * K;
        double acc0 = 0.0, acc1 = 0.0;
        int q = 0;
        for (; q + 1 < j0; q += 2) {
          acc0 = fma(lrow[q], Z[q * RC + c], acc0);
          acc1 = fma(lrow[q + 1], Z[(q + 1) * RC + c], acc1);
        }
        for (; q < j0; ++q) acc0 = fma(lrow[q], Z[q * RC + c], acc0);
        Z[(j0 + r) * RC + c] -= acc0 + acc1;
      }
    }
    for (int q = tid; q < kNb * kNb; q += 256) {
      const int r = q / kNb, c = q % kNb;
      Lb[r][c] = (r < nb && c <= r) ? Lt[(size_t)(j0 + r) * K + j0 + c] : 0.0;
    }
    __syncthreads();
    if (tid < RC) {
      for (int r = 0; r < nb; ++r) {
        double v = Z[(j0 + r) * RC + tid];
        for (int q = 0; q < r; ++q) v = fma(-Lb[r][q], Z[(j0 + q) * RC + tid], v);
        Z[(j0 + r) * RC + tid] = v / Lb[r][r];
      }
    }
    __syncthreads();
  }
  // backward: L^T X = Z
  for (int b = nblk - 1; b >= 0; --b) {
    const int j0 = b * kNb, nb = (K - j0) < kNb ? (K - j0) : kNb;
    const int j1 = j0 + nb;
    // Z_b -= L[j1:K, b]^T X[j1:K]
    for (int o = tid; o < kNb * RC; o += 256) {
      const int r = o / RC, c = o % RC;
      if (r < nb && j1 < K) {
        double acc0 = 0.0, acc1 = 0.0;
        int q = j1;
        for (; q + 1 < K; q += 2) {
          acc0 = fma(Lt[(size_t)q * K + j0 + r], Z[q * RC + c], acc0);
          acc1 = fma(Lt[(size_t)(q + 1) * K + j0 + r], Z[(q + 1) * RC + c], acc1);
        }
        for (; q < K; ++q) acc0 = fma(Lt[(size_t)q * K + j0 + r], Z[q * RC + c], acc0);
        Z[(j0 + r) * RC + c] -= acc0 + acc1;
      }
    }
    for (int q = tid; q < kNb * kNb; q += 256) {
      const int r = q / kNb, c = q % kNb;
      Lb[r][c] = (r < nb && c <= r) ? Lt[(size_t)(j0 + r) * K + j0 + c] : 0.0;
    }
    __syncthreads();
    if (tid < RC) {
      for (int r = nb - 1; r >= 0; --r) {
        double v = Z[(j0 + r) * RC + tid];
        for (int q = r + 1; q < nb; ++q) v = fma(-Lb[q][r], Z[(j0 + q) * RC + tid], v);
        Z[(j0 + r) * RC + tid] = v / Lb[r][r];
      }
    }
    __syncthreads();
  }
  for (int q = tid; q < K * RC; q += 256) {
    const int j = q / RC, c = q % RC;
    if (rc0 + c < m) Bt[(size_t)j * m + rc0 + c] = Z[q];
  }
}

// ---- 6: renormalise used atoms -----------------------------------------------
template <typename T>
__global__ void normalise_kernel(const double *__restrict__ B, const int32_t *__restrict__ usage,
                                 const int32_t *__restrict__ status, int K, int m, T *D) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y;
  const int j = blockIdx.x * 8 + warp;
  if (j >= K || status[t] == 2 || usage[(size_t)t * K + j] == 0) return;
  const double *b = B + ((size_t)t * K + j) * m;
  double acc = 0.0;
  for (int r = lane; r < m; r += 32) acc = fma(b[r], b[r], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const double nrm = sqrt(acc);
  if (!(nrm > 0.0) || !isfinite(nrm)) return;
  T *d = D + ((size_t)t * K + j) * m;
  for (int r = lane; r < m; r += 32) d[r] = (T)(b[r] / nrm);
}


// ---- 4-6 fused: FP64 Cholesky, solve and renormalisation by one thread-block
// cluster per subset.  A's lower triangle is cut into 16x16 tiles; tile (i, j)
// lives in the shared memory of cluster rank (i + j) mod C.  Each right-looking
// step k: the owner of (k, k) factors it; owners of the panel tiles (i, k)
// solve them against L_kk (read through distributed shared memory); every rank
// copies the finished panel column and updates the trailing tiles it owns.
// The right-hand sides (rows of B = atoms) are split by columns: rank c solves
// columns [c*mc, (c+1)*mc) of L L^T X = B alone, reading L tiles remotely.
// Atom norms are summed across ranks, then each rank writes its columns of the
// renormalised atoms.  A breakdown (squared pivot <= 1e-12 of its diagonal)
// restarts the factorisation once from A + lambda I (A is re-read from global
// memory, which the kernel never writes).
constexpr int kT = 16;            // tile edge
constexpr int kTP = kT + 1;       // padded row pitch (doubles)
constexpr int kTile = kT * kTP;   // doubles per stored tile

struct ClusterLayout {
  int R, C, mc, nown;
  size_t tiles, slot, own, panel, lkk, z, normp, dg, flag, total;
};

__host__ inline ClusterLayout cluster_layout(int K, int m, int C) {
  ClusterLayout L{};
  L.R = (K + kT - 1) / kT;
  L.C = C;
  L.mc = (m + C - 1) / C;
  int cnt[32] = {0};
  for (int i = 0; i < L.R; ++i)
    for (int j = 0; j <= i; ++j) cnt[(i + j) % C]++;
  L.nown = 0;
  for (int c = 0; c < C; ++c) L.nown = cnt[c] > L.nown ? cnt[c] : L.nown;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 15) & ~size_t(15); return o; };
  L.tiles = take(sizeof(double) * (size_t)L.nown * kTile);
  L.slot = take(sizeof(int) * (size_t)L.R * L.R);
  L.own = take(sizeof(int) * (size_t)L.nown);
  L.panel = take(sizeof(double) * (size_t)2 * L.R * kTile);   // two panel buffers (steps k even / odd)
  L.lkk = take(sizeof(double) * 2 * kTile);                    // two L_kk buffers
  L.z = take(sizeof(double) * (size_t)L.R * kT * L.mc);
  L.normp = take(sizeof(double) * (size_t)L.R * kT);
  L.dg = take(sizeof(double) * (size_t)L.R * kT);
  L.flag = take(sizeof(int) * 4);
  L.total = off;
  return L;
}

template <typename T, int C>
__global__ void __launch_bounds__(256) mod_solve_cluster_kernel(const double *__restrict__ A,
                                                                const double *__restrict__ B,
                                                                const int32_t *__restrict__ usage, int K,
                                                                int m, T *D, int32_t *status,
                                                                ClusterLayout lay) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = (int)cl.block_rank();
  const int t = blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = lay.R, mc = lay.mc;
  const int col0 = c * mc;
  const int ncol = m - col0 < mc ? (m - col0 > 0 ? m - col0 : 0) : mc;
  double *tiles = reinterpret_cast<double *>(smem_raw + lay.tiles);
  int *slot = reinterpret_cast<int *>(smem_raw + lay.slot);
  int *own = reinterpret_cast<int *>(smem_raw + lay.own);
  double *Pbuf = reinterpret_cast<double *>(smem_raw + lay.panel);   // [2][R][kTile]
  double *Lbuf = reinterpret_cast<double *>(smem_raw + lay.lkk);     // [2][kTile]
  double *Z = reinterpret_cast<double *>(smem_raw + lay.z);          // [R*kT][mc]
  double *normp = reinterpret_cast<double *>(smem_raw + lay.normp);
  double *dg = reinterpret_cast<double *>(smem_raw + lay.dg);        // original diagonal (+ ridge)
  int *flag = reinterpret_cast<int *>(smem_raw + lay.flag);
  const double *At = A + (size_t)t * K * K;
  const double *Bt = B + (size_t)t * K * m;
  const int32_t *ut = usage + (size_t)t * K;

  if (tid == 0) {
    int cnt[C];
    for (int q = 0; q < C; ++q) cnt[q] = 0;
    for (int i = 0; i < R; ++i)
      for (int j = 0; j <= i; ++j) {
        const int o = (i + j) % C;
        if (o == c) own[cnt[o]] = i * R + j;
        slot[i * R + j] = cnt[o]++;
      }
    flag[1] = cnt[c];
  }
  // ridge = 1e-10 tr(A_UU) / |U| (every rank computes the same value)
  __shared__ double red[2][8];
  double tr = 0.0, nu = 0.0;
  for (int j = tid; j < K; j += 256)
    if (ut[j] > 0) { tr += At[(size_t)j * K + j]; nu += 1.0; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    nu += __shfl_xor_sync(0xffffffffu, nu, o);
  }
  if (lane == 0) { red[0][warp] = tr; red[1][warp] = nu; }
  __syncthreads();
  double T0 = 0.0, N0 = 0.0;
  for (int w = 0; w < 8; ++w) { T0 += red[0][w]; N0 += red[1][w]; }
  const double lambda = N0 > 0.0 ? kModRidge * T0 / N0 : 0.0;
  const int nown = flag[1];
  auto owner = [&](int i, int j) { return (i + j) % C; };

  int st = 0;
  bool failed = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double ridge = attempt == 0 ? 0.0 : lambda;
    for (int g = tid; g < R * kT; g += 256)
      dg[g] = g < K ? At[(size_t)g * K + g] + (ut[g] > 0 ? ridge : 0.0) : 1.0;
    // load owned tiles (padding: identity on the diagonal) and own RHS columns
    for (int q = tid; q < nown * kT * kT; q += 256) {
      const int ot = q / (kT * kT), e = q % (kT * kT), r = e / kT, cc = e % kT;
      const int i = own[ot] / R, j = own[ot] % R;
      const int gi = i * kT + r, gj = j * kT + cc;
      double v;
      if (gi < K && gj < K) v = (gj <= gi) ? At[(size_t)gi * K + gj] + (gi == gj && ut[gi] > 0 ? ridge : 0.0) : 0.0;
      else v = (gi == gj) ? 1.0 : 0.0;
      tiles[(size_t)ot * kTile + r * kTP + cc] = v;
    }
    for (int q = tid; q < R * kT * mc; q += 256) {
      const int row = q / mc, cc = q % mc;
      Z[q] = (row < K && cc < ncol) ? Bt[(size_t)row * m + col0 + cc] : 0.0;
    }
    if (tid == 0) flag[0] = 0;
    cl.sync();
    failed = false;
    for (int k = 0; k < R; ++k) {
      const int okk = owner(k, k);
      double *Lkk = Lbuf + (size_t)(k & 1) * kTile;
      double *P = Pbuf + (size_t)(k & 1) * R * kTile;
      // (a) owner of (k, k): factor it (warp 0), then push L_kk into every rank
      if (c == okk) {
        double *Tk = tiles + (size_t)slot[k * R + k] * kTile;
        if (warp == 0) {
          for (int col = 0; col < kT; ++col) {
            const double d = Tk[col * kTP + col];
            if (!(d > kModPivotRel * dg[k * kT + col]) || !(d > 0.0)) {
              if (lane == 0) flag[0] = 1;
              break;
            }
            const double lcc = sqrt(d);
            __syncwarp();
            if (lane == col) Tk[col * kTP + col] = lcc;
            if (lane > col && lane < kT) Tk[lane * kTP + col] /= lcc;
            __syncwarp();
            if (lane > col && lane < kT) {
              const double lr = Tk[lane * kTP + col];
              for (int q = col + 1; q <= lane; ++q) Tk[lane * kTP + q] -= lr * Tk[q * kTP + col];
            }
            __syncwarp();
          }
        }
        __syncthreads();
        if (!flag[0]) {
          for (int q = tid; q < C * (kTile / 2); q += 256) {
            const int r2 = q / (kTile / 2), e = q % (kTile / 2);
            reinterpret_cast<double2 *>(cl.map_shared_rank(Lkk, r2))[e] = reinterpret_cast<const double2 *>(Tk)[e];
          }
        }
      }
      cl.sync();
      if (*cl.map_shared_rank(flag, okk)) failed = true;
      if (failed) break;   // uniform: every rank read the same flag after the sync
      // (b) panel tiles (i, k) owned here: X L_kk^T = T(i, k), one thread per tile row;
      //     each finished tile is pushed into slot i-k-1 of every rank's panel buffer
      for (int q = tid; q < (R - k - 1) * kT; q += 256) {
        const int i = k + 1 + q / kT, r = q % kT;
        if (owner(i, k) != c) continue;
        double *row = tiles + (size_t)slot[i * R + k] * kTile + r * kTP;
        double x[kT];
#pragma unroll
        for (int cc = 0; cc < kT; ++cc) x[cc] = row[cc];
#pragma unroll
        for (int cc = 0; cc < kT; ++cc) {
          double v = x[cc];
#pragma unroll
          for (int p = 0; p < cc; ++p) v = fma(-x[p], Lkk[cc * kTP + p], v);
          x[cc] = v / Lkk[cc * kTP + cc];
        }
#pragma unroll
        for (int cc = 0; cc < kT; ++cc) row[cc] = x[cc];
      }
      __syncthreads();
      for (int ot = 0; ot < nown; ++ot) {
        const int i = own[ot] / R, j = own[ot] % R;
        if (j != k || i <= k) continue;
        const double2 *src = reinterpret_cast<const double2 *>(tiles + (size_t)ot * kTile);
        for (int q = tid; q < C * (kTile / 2); q += 256) {
          const int r2 = q / (kTile / 2), e = q % (kTile / 2);
          reinterpret_cast<double2 *>(cl.map_shared_rank(P, r2) + (size_t)(i - k - 1) * kTile)[e] = src[e];
        }
      }
      cl.sync();
      // forward substitution on own columns, step k: Z_k <- L_kk^{-1} Z_k
      if (tid < ncol) {
        for (int r = 0; r < kT; ++r) {
          double v = Z[(k * kT + r) * mc + tid];
          for (int p = 0; p < r; ++p) v = fma(-Lkk[r * kTP + p], Z[(k * kT + p) * mc + tid], v);
          Z[(k * kT + r) * mc + tid] = v / Lkk[r * kTP + r];
        }
      }
      __syncthreads();
      // (d) Z_i -= L_ik Z_k for i > k (own columns)
      for (int q = tid; q < (R - k - 1) * kT * ncol; q += 256) {
        const int ii = q / (kT * ncol), e = q % (kT * ncol), r = e / ncol, cc = e % ncol;
        const double *Pi = P + (size_t)ii * kTile + r * kTP;
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p < kT; ++p) acc = fma(Pi[p], Z[(k * kT + p) * mc + cc], acc);
        Z[((k + 1 + ii) * kT + r) * mc + cc] -= acc;
      }
      // (e) trailing update of owned tiles (i, j), k < j <= i: T(i,j) -= P_i P_j^T
      for (int ot = 0; ot < nown; ++ot) {
        const int i = own[ot] / R, j = own[ot] % R;
        if (j <= k) continue;
        const int r = tid >> 4, cc = tid & 15;
        if (j == i && cc > r) continue;
        const double *Pi = P + (size_t)(i - k - 1) * kTile + r * kTP;
        const double *Pj = P + (size_t)(j - k - 1) * kTile + cc * kTP;
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
        for (int p = 0; p < kT; p += 2) {
          acc0 = fma(Pi[p], Pj[p], acc0);
          acc1 = fma(Pi[p + 1], Pj[p + 1], acc1);
        }
        tiles[(size_t)ot * kTile + r * kTP + cc] -= acc0 + acc1;
      }
      __syncthreads();
    }
    if (!failed) { st = attempt; break; }
    st = 2;
    cl.sync();   // nobody still reads the flag before it is reset
  }

  if (!failed) {
    // backward substitution on own columns: L^T X = Z (L tiles pulled, no cluster sync)
    double *P = Pbuf;
    for (int k = R - 1; k >= 0; --k) {
      {   // pull row k of L (tiles (k, 0..k)), four remote loads in flight per thread
        constexpr int h = kTile / 2;
        const int n2 = (k + 1) * h;
        double2 *dst = reinterpret_cast<double2 *>(P);
        for (int q0 = tid; q0 < n2; q0 += 4 * 256) {
          double2 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * 256;
            if (q < n2) {
              const int j = q / h, e = q - j * h;
              v[u] = reinterpret_cast<const double2 *>(cl.map_shared_rank(tiles, owner(k, j)) +
                                                       (size_t)slot[k * R + j] * kTile)[e];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u * 256 < n2) dst[q0 + u * 256] = v[u];
        }
      }
      __syncthreads();
      const double *Lk = P + (size_t)k * kTile;
      if (tid < ncol) {
        for (int r = kT - 1; r >= 0; --r) {
          double v = Z[(k * kT + r) * mc + tid];
          for (int p = r + 1; p < kT; ++p) v = fma(-Lk[p * kTP + r], Z[(k * kT + p) * mc + tid], v);
          Z[(k * kT + r) * mc + tid] = v / Lk[r * kTP + r];
        }
      }
      __syncthreads();
      for (int q = tid; q < k * kT * ncol; q += 256) {
        const int jj = q / (kT * ncol), e = q % (kT * ncol), r = e / ncol, cc = e % ncol;
        const double *Lkj = P + (size_t)jj * kTile;
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p < kT; ++p) acc = fma(Lkj[p * kTP + r], Z[(k * kT + p) * mc + cc], acc);
        Z[(jj * kT + r) * mc + cc] -= acc;
      }
      __syncthreads();
    }
    // partial squared norms of every atom over own columns
    for (int row = tid; row < R * kT; row += 256) {
      double acc = 0.0;
      for (int cc = 0; cc < ncol; ++cc) acc = fma(Z[row * mc + cc], Z[row * mc + cc], acc);
      normp[row] = acc;
    }
  }
  cl.sync();
  if (!failed) {
    for (int row = tid; row < K; row += 256) {
      double part[C];
#pragma unroll
      for (int r2 = 0; r2 < C; ++r2) part[r2] = cl.map_shared_rank(normp, r2)[row];
      double n2 = 0.0;
#pragma unroll
      for (int r2 = 0; r2 < C; ++r2) n2 += part[r2];
      dg[row] = sqrt(n2);
    }
    __syncthreads();
    for (int q = tid; q < K * ncol; q += 256) {
      const int row = q / ncol, cc = q % ncol;
      const double nrm = dg[row];
      if (ut[row] == 0 || !(nrm > 0.0) || !isfinite(nrm)) continue;   // keep the previous atom
      D[((size_t)t * K + row) * m + col0 + cc] = (T)(Z[row * mc + cc] / nrm);
    }
  }
  if (c == 0 && tid == 0) status[t] = st;
  cl.sync();   // keep this block's shared memory alive until every rank is done reading it
}
}  // namespace

int mod_tile_signals() { return kModTile; }

template <typename T>
cudaError_t launch_mod_accum(const ModArgs &a, cudaStream_t st) {
  cudaError_t e;
  if (a.L <= 0) return cudaSuccess;
  e = cudaMemsetAsync(a.usage, 0, sizeof(int32_t) * (size_t)a.L * a.K, st);
  if (e != cudaSuccess) return e;
  if (a.total_tiles > 0) {
    mod_count_kernel<<<(unsigned)a.total_tiles, kModTile, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  mod_scan_kernel<<<a.L, 1024, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.total_tiles > 0) {
    mod_fill_kernel<<<(unsigned)a.total_tiles, kModTile, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (sizeof(T) == 4) {
    // FP32 signals: zeroed A and B, entry-range warps, then the unused atoms
    e = cudaMemsetAsync(a.A, 0, sizeof(double) * (size_t)a.L * a.K * a.K, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.B, 0, sizeof(double) * (size_t)a.L * a.K * a.m, st);
    if (e != cudaSuccess) return e;
    if (a.total_tiles > 0) {
      auto kern = a.m <= 64 ? mod_accum_ds_kernel<2> : mod_accum_ds_kernel<8>;
      kern<<<(unsigned)a.total_tiles, kModTile, 0, st>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mod_unused_kernel<T><<<dim3((a.K + 7) / 8, a.L), 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(double) * 8 * (size_t)a.K;
  dim3 grid((a.K + 7) / 8, a.L);
  auto kern = a.m <= 32 ? mod_accum_kernel<T, 1>
            : a.m <= 64 ? mod_accum_kernel<T, 2>
            : a.m <= 128 ? mod_accum_kernel<T, 4> : mod_accum_kernel<T, 8>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mod_chol(const ModArgs &a, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  chol_kernel<<<a.L, 256, 0, st>>>(a.A, a.Lf, a.usage, a.K, a.status);
  return cudaGetLastError();
}

cudaError_t launch_mod_solve(const ModArgs &a, int num_sms, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  cudaError_t e;
  // right-hand-side chunk: enough blocks to cover the SMs twice
  int rc = 16;
  while (rc > 1 && (int64_t)a.L * ((a.m + rc - 1) / rc) < 2 * (int64_t)num_sms) rc >>= 1;
  const size_t sm = sizeof(double) * (size_t)a.K * rc;
  dim3 grid(a.L, (a.m + rc - 1) / rc);
  switch (rc) {
#define SDL_SOLVE_CASE(R)                                                                 \
  case R:                                                                                 \
    e = cudaFuncSetAttribute(solve_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)sm);                                                    \
    if (e != cudaSuccess) return e;                                                       \
    solve_kernel<R><<<grid, 256, sm, st>>>(a.Lf, a.B, a.K, a.m, a.status);                \
    break;
    SDL_SOLVE_CASE(16)
    SDL_SOLVE_CASE(8)
    SDL_SOLVE_CASE(4)
    SDL_SOLVE_CASE(2)
    SDL_SOLVE_CASE(1)
#undef SDL_SOLVE_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


template <typename T, int C>
static cudaError_t launch_cluster_c(const ModArgs &a, const ClusterLayout &lay, cudaStream_t st) {
  auto kern = mod_solve_cluster_kernel<T, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.L * C));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = lay.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  e = cudaLaunchKernelEx(&cfg, kern, (const double *)a.A, (const double *)a.B, (const int32_t *)a.usage,
                         a.K, a.m, static_cast<T *>(a.D), a.status, lay);
  return e;
}

template <typename T>
cudaError_t launch_mod_solve_cluster(const ModArgs &a, int cluster, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  if (a.K > 512) return cudaErrorNotSupported;
  const size_t limit = 227 * 1024;
  // requested size first, then the larger sizes (less shared memory per rank)
  const int order[3] = {cluster, 16, 8};
  for (int q = 0; q < 3; ++q) {
    const int C = order[q];
    if (C != 4 && C != 8 && C != 16) continue;
    ClusterLayout lay = cluster_layout(a.K, a.m, C);
    if (lay.total > limit) continue;
    cudaError_t e = C == 16 ? launch_cluster_c<T, 16>(a, lay, st)
                  : C == 8 ? launch_cluster_c<T, 8>(a, lay, st) : launch_cluster_c<T, 4>(a, lay, st);
    if (e != cudaErrorNotSupported) return e;
  }
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_mod_normalise(const ModArgs &a, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  dim3 grid((a.K + 7) / 8, a.L);
  normalise_kernel<T><<<grid, 256, 0, st>>>(a.B, a.usage, a.status, a.K, a.m, static_cast<T *>(a.D));
  return cudaGetLastError();
}

template cudaError_t launch_mod_accum<float>(const ModArgs &, cudaStream_t);
template cudaError_t launch_mod_accum<double>(const ModArgs &, cudaStream_t);
template cudaError_t launch_mod_normalise<float>(const ModArgs &, cudaStream_t);
template cudaError_t launch_mod_normalise<double>(const ModArgs &, cudaStream_t);
template cudaError_t launch_mod_solve_cluster<float>(const ModArgs &, int, cudaStream_t);
template cudaError_t launch_mod_solve_cluster<double>(const ModArgs &, int, cudaStream_t);

}  // namespace sdl
