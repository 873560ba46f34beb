// BF16 tensor-core front end of OMP (Sec. 1) and of the Gram matrix.
//
// The correlations alpha0 = D^T y are the dense contraction of the coding pass
// (2 m K products per signal) and G = D^T D that of each dictionary, so the
// BF16 path runs both on the 5th-generation tensor cores: tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulation) with the accumulator tile in
// tensor memory, operands in shared memory in the canonical K-major layout.
// Dictionary tiles are streamed in by bulk TMA copies of a pre-laid-out BF16
// image of D; the signal tile is converted from FP32 in the kernel.  The
// correlation kernel writes alpha0 of 128-signal tiles to a global scratch (in
// chunks of at most 1 GiB); the selection kernel then runs the shared selection
// loop from there with little shared memory per block.  The Gram is formed
// from a two-term BF16 split of D (hi + lo, three products), accurate to about
// 2^-16 where one BF16 product would give 2^-8, so the selection's Cholesky
// factor of G_SS also serves the correction step of the coefficients on the
// support (residuals from D_S and y in FP32), which removes the BF16 rounding
// they inherit from alpha0: that rounding affects only which atoms are chosen.
#include "omp_common.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kWaitLimit = 1 << 22;   // polls of a bounded mbarrier wait

// D [L][K][m] FP32 -> BF16 images [L][Kp][mp] (zero padding rows / columns):
// hi = bf16(d) and, when lo is not null, lo = bf16(d - hi), the next eight
// significant bits, so that hi + lo carries d to about 2^-16.
__global__ void bf16_image_kernel(const float *__restrict__ D, int K, int m, int Kp, int mp, int L,
                                  unsigned char *__restrict__ img, unsigned char *__restrict__ lo_img) {
  const int kc8 = mp >> 3;
  const int64_t total = (int64_t)L * Kp * kc8;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / ((int64_t)Kp * kc8);
    const int rem = (int)(q - t * Kp * kc8);
    const int r = rem / kc8, kc = rem - r * kc8;
    const float *src = D + ((size_t)t * K + r) * m;
    uint32_t packed[4], packed_lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k0 = kc * 8 + 2 * e;
      const float x0 = (r < K && k0 < m) ? src[k0] : 0.f;
      const float x1 = (r < K && k0 + 1 < m) ? src[k0 + 1] : 0.f;
      const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
      packed[e] = *reinterpret_cast<const uint32_t *>(&h);
      packed_lo[e] = *reinterpret_cast<const uint32_t *>(&l);
    }
    const size_t off = (size_t)t * Kp * mp * 2 + tc::image_offset(r, kc * 8, mp);
    *reinterpret_cast<uint4 *>(img + off) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    if (lo_img)
      *reinterpret_cast<uint4 *>(lo_img + off) = make_uint4(packed_lo[0], packed_lo[1], packed_lo[2], packed_lo[3]);
  }
}

// Gram tile G[128 rows][128 cols] of subset blockIdx.z on the tensor cores from
// the split images: hi hi^T + hi lo^T + lo hi^T accumulated in one TMEM tile
// (the dropped terms are about 2^-18 of each product).  all4: the hi and lo
// row and column tiles are loaded in one round of bulk copies; otherwise three
// rounds through one pair of buffers, each round's products finished before the
// next round's loads overwrite the operands.
constexpr int kGramNG = 128;

__global__ void __launch_bounds__(128) gram_tc_kernel(const unsigned char *__restrict__ hi,
                                                      const unsigned char *__restrict__ lo, int K, int Kp, int mp,
                                                      bool all4, float *__restrict__ G, int32_t *err,
                                                      __half *__restrict__ G16) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = blockIdx.z, bx = blockIdx.x, by = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t tile = (size_t)128 * mp * 2;   // one 128-row operand tile (kGramNG == 128)
  unsigned char *Aim = smem;
  unsigned char *Bim = smem + tile;
  unsigned char *Alo = smem + 2 * tile;   // all4: the lo tiles too, one round of loads
  unsigned char *Blo = smem + 3 * tile;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (all4 ? 4 : 2) * tile);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
  if (warp == 0) tc::tmem_alloc(tslot, kGramNG);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const size_t sub = (size_t)t * Kp * mp * 2;
  const int rowsA = min(128, Kp - 128 * bx), rowsB = min(kGramNG, Kp - kGramNG * by);
  const uint32_t idesc = tc::idesc_bf16(128, kGramNG);
  const uint32_t sbo = (uint32_t)(mp >> 3) * 128;
  bool ok = true;
  auto mma_tiles = [&](const unsigned char *A, const unsigned char *B, bool acc) {
    for (int ks = 0; ks < (mp >> 4); ++ks)
      tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(A) + ks * 256, 128, sbo),
                   tc::smem_desc(tc::smem_u32(B) + ks * 256, 128, sbo), idesc, acc || ks > 0);
  };
  const size_t arow = (size_t)128 * bx * mp * 2, brow = (size_t)kGramNG * by * mp * 2;
  const uint32_t abytes = (uint32_t)rowsA * mp * 2, bbytes = (uint32_t)rowsB * mp * 2;
  // every decision below is made block-wide (barrier with a vote), so all
  // threads leave together
  if (all4) {   // the four tiles at once, then the three products
    if (tid == 0) {
      tc::mbar_expect_tx(&mbar[0], 2 * (abytes + bbytes));
      tc::bulk_g2s(Aim, hi + sub + arow, abytes, &mbar[0]);
      tc::bulk_g2s(Bim, hi + sub + brow, bbytes, &mbar[0]);
      tc::bulk_g2s(Alo, lo + sub + arow, abytes, &mbar[0]);
      tc::bulk_g2s(Blo, lo + sub + brow, bbytes, &mbar[0]);
    }
    if (__syncthreads_or(!tc::mbar_wait(&mbar[0], 0, kWaitLimit))) {
      if (tid == 0) tc::mbar_wait(&mbar[0], 0, kWaitLimit);   // drain copies in flight (bounded)
      ok = false;
    } else {
      if (tid == 0) {
        tc::fence_after();
        mma_tiles(Aim, Bim, false);
        mma_tiles(Aim, Blo, true);
        mma_tiles(Alo, Bim, true);
        tc::mma_commit(&mbar[1]);
      }
      ok = !__syncthreads_or(!tc::mbar_wait(&mbar[1], 0, kWaitLimit));
    }
  } else {   // three rounds through one pair of tile buffers
    for (int round = 0; round < 3; ++round) {
      const unsigned char *a = (round == 2 ? lo : hi) + sub;
      const unsigned char *b = (round == 1 ? lo : hi) + sub;
      const uint32_t par = (uint32_t)(round & 1);
      if (tid == 0) {
        tc::mbar_expect_tx(&mbar[0], abytes + bbytes);
        tc::bulk_g2s(Aim, a + arow, abytes, &mbar[0]);
        tc::bulk_g2s(Bim, b + brow, bbytes, &mbar[0]);
      }
      if (__syncthreads_or(!tc::mbar_wait(&mbar[0], par, kWaitLimit))) {
        if (tid == 0) tc::mbar_wait(&mbar[0], par, kWaitLimit);   // drain copies in flight (bounded)
        ok = false;
        break;
      }
      if (tid == 0) {
        tc::fence_after();
        mma_tiles(Aim, Bim, round > 0);
        tc::mma_commit(&mbar[1]);
      }
      // the products have read the operands: the next round may overwrite them
      if (__syncthreads_or(!tc::mbar_wait(&mbar[1], par, kWaitLimit))) {
        ok = false;
        break;
      }
    }
  }
  tc::fence_after();
  if (ok) {
    const int row = 128 * bx + 32 * warp + lane;
    for (int c0 = 0; c0 < kGramNG; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + c0, v);
      if (row < K) {
        float *grow = G + ((size_t)t * K + row) * K;
        __half *hrow = G16 ? G16 + ((size_t)t * K + row) * K : nullptr;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int col = kGramNG * by + c0 + e;
          if (col < K) {
            grow[col] = v[e];
            if (hrow) hrow[col] = __float2half_rn(v[e]);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, kGramNG);
}

// ---- correlations: alpha0 = Y D^T of 128-signal tiles into global memory ----
// One block per tile of 128 signals (the MMA's M), 8 warps.  The signal tile is
// converted to a BF16 K-major image once (16-byte loads, eight warps so many
// loads are in flight); dictionary tiles of 128 atoms stream in by bulk copies
// into two buffers, and their products go to two TMEM accumulators, so the MMA
// of tile nt+1 runs while tile nt is read out.  Warps w and w + 4 read the TMEM
// lanes of rows 32 (w mod 4) .. + 31, each half of the columns.  Row r of the
// tile's alpha0 block (atoms in order) is written to a0 + r * K.
constexpr int kCorrThreads = 256;
constexpr int kCorrNT = 128;

struct CorrLayout {
  size_t aim, bim, bar, total;
};

inline CorrLayout corr_layout(int mp) {
  CorrLayout L{};
  size_t off = 0;
  L.aim = off; off += (size_t)128 * mp * 2;
  L.bim = off; off += (size_t)2 * kCorrNT * mp * 2;
  L.bar = off; off += 64;
  L.total = off;
  return L;
}

__global__ void __launch_bounds__(kCorrThreads) corr_tc_kernel(OmpArgs a, CorrLayout lay, float *a0c, int64_t tile0) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, mp = a.mp, Kp = a.Kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t g = tile0 + blockIdx.x;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)128;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < 128 ? (int)rows_left : 128;
  const float *__restrict__ Y = static_cast<const float *>(a.Y);
  const unsigned char *sub = static_cast<const unsigned char *>(a.Dimg) + (size_t)t * Kp * mp * 2;
  unsigned char *Aim = smem + lay.aim;
  unsigned char *Bim = smem + lay.bim;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bar);   // [0,1] loads, [2,3] MMA commits
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 4);
  int *fail = reinterpret_cast<int *>(bar + 5);
  constexpr int NT = kCorrNT;
  const size_t btile = (size_t)NT * mp * 2;
  const int ntiles = (K + NT - 1) / NT;
  auto tile_bytes = [&](int nt) { return (uint32_t)min(NT, Kp - nt * NT) * (uint32_t)mp * 2u; };

  if (warp == 0) tc::tmem_alloc(tslot, 2 * NT);
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) tc::mbar_init(&bar[q], 1);
    tc::mbar_fence_init();
    *fail = 0;
    for (int nt = 0; nt < 2 && nt < ntiles; ++nt) {
      tc::mbar_expect_tx(&bar[nt], tile_bytes(nt));
      tc::bulk_g2s(Bim + nt * btile, sub + (size_t)nt * NT * mp * 2, tile_bytes(nt), &bar[nt]);
    }
  }
  // signal tile -> BF16 A image (rows beyond the tile are zero); item q is
  // entries 8 kc .. 8 kc + 7 of row r
  const int kc8 = mp >> 3;
  const bool vec = (m & 3) == 0;   // 16-byte aligned rows
  constexpr int kU = 4;            // items whose loads are in flight together
  for (int q0 = tid; q0 < 128 * kc8; q0 += kU * kCorrThreads) {
    float f[kU][8];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = q0 + u * kCorrThreads;
      const int r = q / kc8, k0 = (q - r * kc8) * 8;
      const float *yr = Y + (size_t)(row0 + r) * m + k0;
      if (q < 128 * kc8 && r < nsig && vec && k0 + 8 <= m) {
        const float4 u0 = *reinterpret_cast<const float4 *>(yr);
        const float4 u1 = *reinterpret_cast<const float4 *>(yr + 4);
        f[u][0] = u0.x; f[u][1] = u0.y; f[u][2] = u0.z; f[u][3] = u0.w;
        f[u][4] = u1.x; f[u][5] = u1.y; f[u][6] = u1.z; f[u][7] = u1.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) f[u][e] = (q < 128 * kc8 && r < nsig && k0 + e < m) ? yr[e] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = q0 + u * kCorrThreads;
      if (q >= 128 * kc8) break;
      const int r = q / kc8, kc = q - r * kc8;
      uint32_t packed[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(f[u][2 * e], f[u][2 * e + 1]);
        packed[e] = *reinterpret_cast<uint32_t *>(&b2);
      }
      *reinterpret_cast<uint4 *>(Aim + tc::image_offset(r, kc * 8, mp)) =
          make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_bf16(128, NT);
  const uint32_t sbo = (uint32_t)kc8 * 128;
  // tile nt's product into TMEM columns (nt & 1) * 128 (thread 0)
  auto issue = [&](int nt) {
    const int b = nt & 1;
    if (!tc::mbar_wait(&bar[b], (nt >> 1) & 1, kWaitLimit)) { *fail = 1; return; }
    tc::fence_after();
    const uint32_t bsm = tc::smem_u32(Bim + b * btile);
    for (int ks = 0; ks < (mp >> 4); ++ks)
      tc::mma_bf16(tbase + (uint32_t)(b * NT), tc::smem_desc(tc::smem_u32(Aim) + ks * 256, 128, sbo),
                   tc::smem_desc(bsm + ks * 256, 128, sbo), idesc, ks > 0);
    tc::mma_commit(&bar[2 + b]);
  };
  if (tid == 0) issue(0);
  const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32 quarter .. + 31
  const int row = 32 * quarter + lane;
  float *arow = a0c + ((size_t)(g - tile0) * 128 + row) * K;
  int nt = 0;
  for (; nt < ntiles; ++nt) {
    const int b = nt & 1;
    if (tid == 0 && nt + 1 < ntiles && !*fail) issue(nt + 1);
    if (!tc::mbar_wait(&bar[2 + b], (nt >> 1) & 1, kWaitLimit)) *fail = 1;
    __syncthreads();
    if (*fail) break;
    tc::fence_after();
    for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2); c0 += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * NT + c0), v);
      const int col0 = nt * NT + c0;
      if (row < nsig) {
        if (col0 + 32 <= K && (K & 3) == 0) {
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<float4 *>(arow + col0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (col0 + e < K) arow[col0 + e] = v[e];
        }
      }
    }
    tc::fence_before();
    __syncthreads();   // buffer b (TMEM columns and B image) is free again
    if (tid == 0 && nt + 2 < ntiles) {
      tc::mbar_expect_tx(&bar[b], tile_bytes(nt + 2));
      tc::bulk_g2s(Bim + b * btile, sub + (size_t)(nt + 2) * NT * mp * 2, tile_bytes(nt + 2), &bar[b]);
    }
  }
  if (*fail) {
    // wait (bounded) for the bulk copies still in flight before the shared
    // memory is given back: loads of tiles nt .. nt + 1 may be outstanding
    if (tid == 0) {
      for (int q = nt; q < nt + 2 && q < ntiles; ++q) tc::mbar_wait(&bar[q & 1], (q >> 1) & 1, kWaitLimit);
      if (a.err) atomicOr(a.err, 1);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 2 * NT);
}

// ---- selection: the Batch-OMP loop and exact refit from alpha0 in global memory
// A block covers a quarter (32 signals, 4 per warp) of a 128-signal tile; shared
// memory holds only the per-warp factors and, when it fits, the G-column cache,
// so many blocks share an SM to hide the loop's latency.
constexpr int kSelThreads = 256;

struct SelLayout {
  int lp;
  int gcn;   // G columns of the support cached per warp
  size_t ls, gc, total;
};

// Per-warp factor scratch, then as many of the support's G columns per warp as
// fit the shared memory one block gets at the occupancy its registers allow
// (the first picks' columns: column p is re-read by the s - 1 - p later
// updates, so caching the first few saves most of the L2 reads).
inline SelLayout sel_layout(int K, int s, int regs, bool h16) {
  const int rr = (regs + 7) & ~7;
  int blocks = 65536 / (kSelThreads * (rr > 0 ? rr : 8));
  blocks = blocks < 1 ? 1 : (blocks > 8 ? 8 : blocks);
  const size_t budget = (size_t)228 * 1024 / blocks - 1024;
  SelLayout L{};
  L.lp = odd_pitch(s);
  const size_t ls = align16(sizeof(float) * (size_t)8 * s * L.lp);
  const size_t col = (h16 ? 2 : sizeof(float)) * (size_t)8 * K;   // one column for every warp
  const int fit = budget > ls ? (int)((budget - ls) / col) : 0;
  L.gcn = fit < s - 1 ? fit : (s > 1 ? s - 1 : 0);
  size_t off = 0;
  L.ls = off; off += ls;
  L.gc = off; off += align16(col * L.gcn);
  L.total = off;
  return L;
}

template <int KPL, int MU, bool EXACT, bool H16>
__global__ void __launch_bounds__(kSelThreads, KPL <= 8 ? 4 : (KPL <= 16 ? 3 : 2)) omp_select_kernel(OmpArgs a, SelLayout lay, const float *a0c,
                                                                 int64_t tile0) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, s = a.s;
  const int warp = threadIdx.x >> 5;
  const int64_t g = tile0 + blockIdx.x / 4;
  const int quarter = blockIdx.x & 3;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)128 + quarter * 32;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  if (rows_left <= 0) return;   // whole block: nothing below is a block-wide barrier
  const int nsig = rows_left < 32 ? (int)rows_left : 32;
  const float *__restrict__ Dt = static_cast<const float *>(a.D) + (size_t)t * K * m;
  const float *__restrict__ Gt = static_cast<const float *>(a.G) + (size_t)t * K * K;
  const float *a0 = a0c + ((size_t)(g - tile0) * 128 + quarter * 32) * K;
  float *Ls = reinterpret_cast<float *>(smem + lay.ls) + (size_t)warp * s * lay.lp;
  void *gc = nullptr;
  if (lay.gcn > 0)
    gc = H16 ? static_cast<void *>(reinterpret_cast<__half *>(smem + lay.gc) + (size_t)warp * lay.gcn * K)
             : static_cast<void *>(reinterpret_cast<float *>(smem + lay.gc) + (size_t)warp * lay.gcn * K);
  const __half *G16t = H16 ? static_cast<const __half *>(a.G16) + (size_t)t * K * K : nullptr;
  code_warp_signals<float, KPL, MU, EXACT, H16>(a, a0, static_cast<const float *>(a.Y) + (size_t)row0 * m, m,
                                               warp * 4, 4, nsig, row0, Dt, Gt, Ls, gc, lay.lp, lay.gcn, G16t);
}

template <int KPL, int MU, bool EXACT, bool H16>
cudaError_t launch_select(const OmpArgs &a, const float *a0c, int64_t tile0, int64_t ntile, cudaStream_t st) {
  auto kern = omp_select_kernel<KPL, MU, EXACT, H16>;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const SelLayout lay = sel_layout(a.K, a.s, fa.numRegs, H16);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(ntile * 4), kSelThreads, lay.total, st>>>(a, lay, a0c, tile0);
  return cudaGetLastError();
}

template <bool EXACT, bool H16>
cudaError_t select_dispatch(const OmpArgs &a, const float *a0c, int64_t g0, int64_t nt, cudaStream_t st) {
  const int kpl = (a.K + 31) / 32;
  if (a.m <= 64) {
    return kpl <= 4 ? launch_select<4, 2, EXACT, H16>(a, a0c, g0, nt, st)
         : kpl <= 8 ? launch_select<8, 2, EXACT, H16>(a, a0c, g0, nt, st)
         : kpl <= 16 ? launch_select<16, 2, EXACT, H16>(a, a0c, g0, nt, st)
                     : launch_select<32, 2, EXACT, H16>(a, a0c, g0, nt, st);
  }
  return kpl <= 4 ? launch_select<4, 8, EXACT, H16>(a, a0c, g0, nt, st)
       : kpl <= 8 ? launch_select<8, 8, EXACT, H16>(a, a0c, g0, nt, st)
       : kpl <= 16 ? launch_select<16, 8, EXACT, H16>(a, a0c, g0, nt, st)
                   : launch_select<32, 8, EXACT, H16>(a, a0c, g0, nt, st);
}

}  // namespace

cudaError_t launch_bf16_image(const float *D, int K, int m, int L, void *img, void *lo_img, cudaStream_t st) {
  const int Kp = round16(K), mp = round16(m);
  const int64_t total = (int64_t)L * Kp * (mp >> 3);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  bf16_image_kernel<<<blocks, 256, 0, st>>>(D, K, m, Kp, mp, L, static_cast<unsigned char *>(img),
                                            static_cast<unsigned char *>(lo_img));
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(const void *hi, const void *lo, int K, int m, int L, float *G, int32_t *err,
                           cudaStream_t st, void *G16) {
  if (L <= 0) return cudaSuccess;
  const int Kp = round16(K), mp = round16(m);
  const size_t tile = (size_t)128 * mp * 2;
  const bool all4 = 4 * tile + 64 <= 200 * 1024;   // the four tiles fit: one round of loads
  const size_t smem = tc::smem_for_tmem((all4 ? 4 : 2) * tile + 64, kGramNG);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((Kp + 127) / 128, (Kp + kGramNG - 1) / kGramNG, L);
  gram_tc_kernel<<<grid, 128, smem, st>>>(static_cast<const unsigned char *>(hi),
                                          static_cast<const unsigned char *>(lo), K, Kp, mp, all4, G, err,
                                          static_cast<__half *>(G16));
  return cudaGetLastError();
}

cudaError_t launch_omp_select(const OmpArgs &a, const float *a0c, int64_t tile0, int64_t ntile, bool exact,
                              cudaStream_t st, bool h16) {
  if (exact) return select_dispatch<true, false>(a, a0c, tile0, ntile, st);
  return h16 && a.G16 ? select_dispatch<false, true>(a, a0c, tile0, ntile, st)
                      : select_dispatch<false, false>(a, a0c, tile0, ntile, st);
}

int omp_tc_tile_signals(int K, int m, int s) {
  (void)K;
  (void)m;
  (void)s;
  return 128;
}

// Tiles per chunk of the alpha0 scratch (at most cap bytes, 0: 1 GiB; at least
// one tile).
int64_t omp_tc_chunk_tiles(int K, int64_t total_tiles, int64_t cap) {
  const int64_t per = (int64_t)128 * K * (int64_t)sizeof(float);
  int64_t c = (cap > 0 ? cap : ((int64_t)1 << 30)) / per;
  if (c < 1) c = 1;
  return c < total_tiles ? c : (total_tiles > 0 ? total_tiles : 1);
}

cudaError_t launch_omp_tc(const OmpArgs &a, float *a0c, cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  const CorrLayout cl = corr_layout(a.mp);
  const size_t csm = tc::smem_for_tmem(cl.total, 2 * kCorrNT);
  if (csm > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(corr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
  if (e != cudaSuccess) return e;
  const int64_t chunk = omp_tc_chunk_tiles(a.K, a.total_tiles, a.a0_cap);
  for (int64_t g0 = 0; g0 < a.total_tiles; g0 += chunk) {
    const int64_t nt = a.total_tiles - g0 < chunk ? a.total_tiles - g0 : chunk;
    corr_tc_kernel<<<(unsigned)nt, kCorrThreads, csm, st>>>(a, cl, a0c, g0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the coefficients from alpha0 on the support carry its BF16 rounding; the
    // selection loop's FP32 correction step (residual from D_S and y in FP32,
    // solved with the factor of the FP32 Gram, within 2^-16 of the exact one)
    // removes it to about 2^-16 kappa(G_SS) of that rounding, so no separate
    // refit from D_S^T y is needed
    if ((e = launch_omp_select(a, a0c, g0, nt, false, st, a.G16 != nullptr)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sdl
