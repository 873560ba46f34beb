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
__global__ void mod_count_kernel(ModArgs a) {
  const int64_t g = blockIdx.x;
  const int t = find_subset_tiles(a.tile_start, a.L, g);
  const int64_t i = a.offsets[t] + (g - a.tile_start[t]) * kModTile + threadIdx.x;
  if (i >= a.offsets[t + 1]) return;
  for (int k = 0; k < a.s; ++k) {
    const int j = a.idx[(size_t)i * a.s + k];
    if (j >= 0 && j < a.K) atomicAdd(&a.usage[(size_t)t * a.K + j], 1);
  }
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
  }
}

// ---- 3: A and B accumulation, one warp per (subset, atom) --------------------
template <typename T>
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
  double b[kMaxM / 32];
#pragma unroll
  for (int u = 0; u < kMaxM / 32; ++u) b[u] = 0.0;
  const int64_t base = a.offsets[t] * s + a.ptr[(size_t)t * (K + 1) + j];
  for (int e0 = 0; e0 < c; e0 += 32) {
    const int ne = (c - e0) < 32 ? (c - e0) : 32;
    int my_i = 0, my_k = 0;
    if (lane < ne) {
      my_i = a.lsig[base + e0 + lane];
      my_k = a.lslot[base + e0 + lane];
    }
    for (int e = 0; e < ne; ++e) {
      const int i = __shfl_sync(0xffffffffu, my_i, e);
      const int k = __shfl_sync(0xffffffffu, my_k, e);
      const double v = (double)val[(size_t)i * s + k];
      const T *yi = Y + (size_t)i * m;
#pragma unroll
      for (int u = 0; u < kMaxM / 32; ++u) {
        const int r = lane + 32 * u;
        if (r < m) b[u] = fma(v, (double)yi[r], b[u]);
      }
      if (lane < s) {
        const int j2 = idx[(size_t)i * s + lane];
        if (j2 >= 0 && j2 < K) arow[j2] = fma(v, (double)val[(size_t)i * s + lane], arow[j2]);
      }
      __syncwarp();
    }
  }
  for (int q = lane; q < K; q += 32) Arow_g[q] = arow[q];
#pragma unroll
  for (int u = 0; u < kMaxM / 32; ++u) {
    const int r = lane + 32 * u;
    if (r < m) Bcol[r] = b[u];
  }
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
  const size_t sm = sizeof(double) * 8 * (size_t)a.K;
  e = cudaFuncSetAttribute(mod_accum_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((a.K + 7) / 8, a.L);
  mod_accum_kernel<T><<<grid, 256, sm, st>>>(a);
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

}  // namespace sdl
