// OMP in two kernels for FP32 data (Sec. 1; error-constrained stop of Sec.
// 3.2.2), the default FP32 form: an FFMA correlation GEMM writes alpha0 = D^T y
// of 128-signal tiles to the same global scratch the BF16 path uses, then the
// shared selection kernel codes the signals from there.  The fused kernel
// (omp.cu) keeps a 32-signal correlation tile in shared memory, which leaves
// one to three blocks per SM for the latency-bound selection loop; here the
// selection runs with little shared memory at full occupancy and the GEMM runs
// with full-size register tiles, at the cost of writing and reading alpha0
// (4K bytes per signal each way).  The products are FP32 FMAs over the signal
// entries in order, like the fused kernel's, so the codes are the same and no
// refit is needed.
#include "omp_common.cuh"

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kGThreads = 256;
constexpr int kGM = 128;      // signals per block (the tile of the plan)
constexpr int kGN = 128;      // atoms per block
constexpr int kGK = 16;       // signal entries per stage
constexpr int kGPitch = 132;  // staged row pitch (floats): 16-byte aligned rows

// out[r][j0 + c] = <y_r, d_(j0 + c)> for the rows r < nsig of a 128-row tile
// (row r at Yt + r m) against atoms j0 .. j0 + 127 of Dt ([K][m]); row r of the
// output at out + r ldo.  Thread (ty, tx) of a 16 x 16 grid owns rows 4 ty +
// {0..3} and 64 + 4 ty + {0..3} and atoms 4 tx + {0..3} and 64 + 4 tx + {0..3}:
// an 8 x 8 register tile fed by four 16-byte shared-memory reads per entry.
// Stages of 16 entries are double-buffered, the next stage's global loads held
// in registers during the products.  Each product is an ordered chain of FP32
// FMAs over the entries, as in the fused OMP kernel.  kAbs: store |product|.
template <bool kAbs = false>
__device__ __forceinline__ void tile_products(const float *__restrict__ Yt, int nsig, const float *__restrict__ Dt,
                                              int K, int m, int j0, float *out, int64_t ldo) {
  __shared__ __align__(16) float Ys[2][kGK][kGPitch];
  __shared__ __align__(16) float Ds[2][kGK][kGPitch];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool vec = (m & 3) == 0;

  // loader: thread tid stages row (tid >> 1) of both operands, entries
  // 8 (tid & 1) .. 8 (tid & 1) + 7 of the stage
  const int lrow = tid >> 1, lk = (tid & 1) * 8;
  const bool yok = lrow < nsig, dok = j0 + lrow < K;
  const float *ysrc = Yt + (size_t)(yok ? lrow : 0) * m;
  const float *dsrc = Dt + (size_t)(dok ? j0 + lrow : 0) * m;
  float yr[8], dr[8];
  auto fetch = [&](int k0) {
    const int kb = k0 + lk;
    if (vec && kb + 8 <= m) {
      const float4 y0 = yok ? *reinterpret_cast<const float4 *>(ysrc + kb) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 y1 = yok ? *reinterpret_cast<const float4 *>(ysrc + kb + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 d0 = dok ? *reinterpret_cast<const float4 *>(dsrc + kb) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 d1 = dok ? *reinterpret_cast<const float4 *>(dsrc + kb + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      yr[0] = y0.x; yr[1] = y0.y; yr[2] = y0.z; yr[3] = y0.w;
      yr[4] = y1.x; yr[5] = y1.y; yr[6] = y1.z; yr[7] = y1.w;
      dr[0] = d0.x; dr[1] = d0.y; dr[2] = d0.z; dr[3] = d0.w;
      dr[4] = d1.x; dr[5] = d1.y; dr[6] = d1.z; dr[7] = d1.w;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        yr[e] = (yok && kb + e < m) ? ysrc[kb + e] : 0.f;
        dr[e] = (dok && kb + e < m) ? dsrc[kb + e] : 0.f;
      }
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      Ys[buf][lk + e][lrow] = yr[e];
      Ds[buf][lk + e][lrow] = dr[e];
    }
  };

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  const int nst = (m + kGK - 1) / kGK;
  fetch(0);
  stage(0);
  __syncthreads();
  for (int st = 0; st < nst; ++st) {
    const int buf = st & 1;
    if (st + 1 < nst) fetch((st + 1) * kGK);
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 ya = *reinterpret_cast<const float4 *>(&Ys[buf][kk][4 * ty]);
      const float4 yb = *reinterpret_cast<const float4 *>(&Ys[buf][kk][64 + 4 * ty]);
      const float4 da = *reinterpret_cast<const float4 *>(&Ds[buf][kk][4 * tx]);
      const float4 db = *reinterpret_cast<const float4 *>(&Ds[buf][kk][64 + 4 * tx]);
      const float yv[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
      const float dv[8] = {da.x, da.y, da.z, da.w, db.x, db.y, db.z, db.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(yv[r], dv[c], acc[r][c]);
    }
    if (st + 1 < nst) stage(buf ^ 1);
    __syncthreads();
  }

  if (kAbs) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fabsf(acc[r][c]);
  }
  const bool vstore = (K & 3) == 0 && (ldo & 3) == 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int row = (r < 4 ? 4 * ty : 64 + 4 * ty) + (r & 3);
    if (row >= nsig) continue;
    float *orow = out + (size_t)row * ldo;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + (h == 0 ? 4 * tx : 64 + 4 * tx);
      if (vstore && j + 4 <= K) {
        *reinterpret_cast<float4 *>(orow + j) =
            make_float4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (j + e < K) orow[j + e] = acc[r][4 * h + e];
      }
    }
  }
}

// alpha0 of one 128-signal tile of the plan against 128 atoms, into the
// scratch (signal r of the tile at a0c + ((g - tile0) 128 + r) K).  The atom
// blocks of a tile are consecutive blocks, so the tile's signals come from
// DRAM once and from L2 for the other atom blocks.
__global__ void __launch_bounds__(kGThreads) corr_f32_kernel(OmpArgs a, float *a0c, int64_t tile0, int nb) {
  const int K = a.K, m = a.m;
  const int64_t g = tile0 + blockIdx.x / nb;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)kGM;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < kGM ? (int)rows_left : kGM;
  const int j0 = (int)(blockIdx.x % nb) * kGN;
  tile_products(static_cast<const float *>(a.Y) + (size_t)row0 * m, nsig,
                static_cast<const float *>(a.D) + (size_t)t * K * m, K, m, j0,
                a0c + (size_t)(g - tile0) * kGM * K, K);
}

// Correlation features F[i][j] = |<d_(t(i), j), y_i>| of every signal against
// its own subset's dictionary (the input of a dictionary-conditioned support
// proposer): the same tile products, stored as absolute values straight into
// row i - row_base of F (pitch K), no scratch.
__global__ void __launch_bounds__(kGThreads) corr_abs_kernel(OmpArgs a, float *F, int64_t tile0, int64_t row_base,
                                                              int nb) {
  const int K = a.K, m = a.m;
  const int64_t g = tile0 + blockIdx.x / nb;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)kGM;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < kGM ? (int)rows_left : kGM;
  const int j0 = (int)(blockIdx.x % nb) * kGN;
  tile_products<true>(static_cast<const float *>(a.Y) + (size_t)row0 * m, nsig,
                      static_cast<const float *>(a.D) + (size_t)t * K * m, K, m, j0,
                      F + (size_t)(row0 - row_base) * K, K);
}

// The Gram matrices G_t = D_t D_t^T of L dictionaries [L][K][m] into [L][K][K]:
// the same tile products with the atoms of D_t as the rows.  Block b covers
// subset b / (nt nb), row tile (b / nb) mod nt and atom block b mod nb.
__global__ void __launch_bounds__(kGThreads) gram_f32_kernel(const float *__restrict__ D, int K, int m, int nt,
                                                             int nb, float *G) {
  const int64_t b = blockIdx.x;
  const int t = (int)(b / ((int64_t)nt * nb));
  const int rt = (int)((b / nb) % nt);
  const int j0 = (int)(b % nb) * kGN;
  const int r0 = rt * kGM;
  const int nrow = K - r0 < kGM ? K - r0 : kGM;
  const float *Dt = D + (size_t)t * K * m;
  tile_products(Dt + (size_t)r0 * m, nrow, Dt, K, m, j0, G + ((size_t)t * K + r0) * K, K);
}

}  // namespace

cudaError_t launch_gram_f32_tiles(const float *D, int m, int K, int L, float *G, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  const int nt = (K + kGM - 1) / kGM, nb = (K + kGN - 1) / kGN;
  gram_f32_kernel<<<(unsigned)((int64_t)L * nt * nb), kGThreads, 0, st>>>(D, K, m, nt, nb, G);
  return cudaGetLastError();
}

cudaError_t launch_corr_features(const OmpArgs &a, int64_t tile0, int64_t ntile, int64_t row_base, float *F,
                                 cudaStream_t st) {
  if (ntile <= 0) return cudaSuccess;
  const int nb = (a.K + kGN - 1) / kGN;
  corr_abs_kernel<<<(unsigned)(ntile * nb), kGThreads, 0, st>>>(a, F, tile0, row_base, nb);
  return cudaGetLastError();
}

cudaError_t launch_omp_split_f32(const OmpArgs &a, float *a0c, cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  const int64_t chunk = omp_tc_chunk_tiles(a.K, a.total_tiles, a.a0_cap);
  for (int64_t g0 = 0; g0 < a.total_tiles; g0 += chunk) {
    const int64_t nt = a.total_tiles - g0 < chunk ? a.total_tiles - g0 : chunk;
    const int nb = (a.K + kGN - 1) / kGN;
    corr_f32_kernel<<<(unsigned)(nt * nb), kGThreads, 0, st>>>(a, a0c, g0, nb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_omp_select(a, a0c, g0, nt, false, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sdl
