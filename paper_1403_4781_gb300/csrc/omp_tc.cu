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
// A persistent block per SM runs its tiles of 128 signals (the MMA's M) in
// turn, each as ceil(K / 256) work items: one pass of 256 atoms (the MMA's N
// and one 256-column TMEM accumulator) each.  The dictionary comes from its slab image
// ([L][mp/64][Kp][64] BF16, Kp = K rounded up to 256: the 256 atoms x 64
// entries of one pass and block are one contiguous 32 KB slab).  Four roles
// meet only at mbarriers:
//   warps 0-3  convert each tile's signal entries once, 64 at a time, from
//              FP32 into 16 KB BF16 block images (two sets of four, one set per
//              tile, alternating, so a tile's image serves all of its passes);
//              thread (w, lane) takes row lane & 7 of 8-row groups w, w + 4,
//              w + 8, w + 12 and entry groups lane >> 3 and + 4, so a
//              quarter-warp's 16-byte stores fill 128 contiguous bytes (no bank
//              conflict); the next block's loads fly while the thread waits for
//              a free set;
//   warp 8     streams each pass's slabs into two stages by bulk copies;
//   warp 9     issues per block four 128 x 256 x 16 MMAs into the item's
//              accumulator (two, alternating by item), freeing each stage by
//              tcgen05.commit and a tile's image set after its last pass;
//   warps 4-7  read a finished accumulator out while the next item's products
//              run into the other one: warp 4 + q owns TMEM lanes (tile rows)
//              32 q .. 32 q + 31, passes each 32-column slice through a padded
//              transpose buffer and stores it as four 128-byte row segments per
//              instruction.
// Every wait is bounded: a role that gives up sets the block's fail flag and
// the error word; the others leave at their next check or bounded wait, the
// loader waits for its copies in flight, the issuer for its products, and the
// tensor memory is freed.
constexpr int kC16Threads = 320;
constexpr int kC16NT = 256;                                 // atoms per item
constexpr int kC16KB = 64;                                  // signal entries per block
constexpr int kC16Stages = 2;                               // dictionary slab stages
constexpr int kC16ABlks = 4;                                // signal blocks per image set (m <= 256)
constexpr uint32_t kC16Slab = (uint32_t)kC16NT * kC16KB * 2;   // 32 KB
constexpr uint32_t kC16ABlk = 128u * kC16KB * 2;               // 16 KB
constexpr int kC16Pitch = 36;   // floats per row of a read-out transpose buffer (32 + 4: no bank conflict)

inline int round64c(int x) { return (x + 63) & ~63; }
inline int round256c(int x) { return (x + 255) & ~255; }

struct C16Job {
  OmpArgs a;                 // K, m, L, Y and the tile plan
  const unsigned char *img;  // slab image of D
  float *out;                // alpha0 scratch: row (g - tile0) * 128 + r of tile g
  int64_t tile0, ntile;
  int nblk, Kp, npass;       // 64-entry blocks, K rounded up to 256, items per tile
  int32_t *err;
  int wait_limit;            // polls of a bounded wait
  int leave;                 // 1: the loader leaves at once (a test of the bounded waits)
};

struct C16Tile {
  int t;              // dictionary
  const float *rows;  // row 0 of the tile (pitch m)
  int nrow;           // valid rows
  float *out;         // output row 0 (pitch K)
};

__device__ __forceinline__ C16Tile c16_tile(const C16Job &j, int64_t g) {
  C16Tile T;
  T.t = find_subset(j.a.tile_start, j.a.L, g);
  const int64_t row0 = j.a.offsets[T.t] + (g - j.a.tile_start[T.t]) * (int64_t)128;
  const int64_t left = j.a.offsets[T.t + 1] - row0;
  T.rows = static_cast<const float *>(j.a.Y) + (size_t)row0 * j.a.m;
  T.nrow = left < 128 ? (int)left : 128;
  T.out = j.out + (size_t)(g - j.tile0) * 128 * j.a.K;
  return T;
}

struct C16Bars {
  uint64_t full_b[kC16Stages], empty_b[kC16Stages];
  uint64_t full_a[2][kC16ABlks], empty_a[2];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t done;
  uint32_t tslot;
  int fail;
};

constexpr size_t kC16A = 0;                                             // two signal image sets
constexpr size_t kC16B = kC16A + 2 * kC16ABlks * (size_t)kC16ABlk;      // slab stages
constexpr size_t kC16T = kC16B + kC16Stages * (size_t)kC16Slab;         // read-out transpose buffers
constexpr size_t kC16Bar = kC16T + 4 * 32 * kC16Pitch * sizeof(float);
constexpr size_t kC16Smem = kC16Bar + sizeof(C16Bars);

__global__ void __launch_bounds__(kC16Threads, 1) corr16_kernel(C16Job j) {
  extern __shared__ __align__(1024) unsigned char smem[];
  C16Bars *bars = reinterpret_cast<C16Bars *>(smem + kC16Bar);
  volatile int *fail = &bars->fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = j.a.K, m = j.a.m, nblk = j.nblk;
  const int npass = j.npass;

  if (warp == 9) tc::tmem_alloc(&bars->tslot, 2 * kC16NT);
  if (tid == 0) {
    for (int q = 0; q < kC16Stages; ++q) {
      tc::mbar_init(&bars->full_b[q], 1);
      tc::mbar_init(&bars->empty_b[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      for (int b = 0; b < kC16ABlks; ++b) tc::mbar_init(&bars->full_a[q][b], 128);
      tc::mbar_init(&bars->empty_a[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bars->acc_full[q], 1);
      tc::mbar_init(&bars->acc_empty[q], 128);
    }
    tc::mbar_init(&bars->done, 1);
    bars->fail = 0;
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = bars->tslot;
  auto give_up = [&]() {
    *fail = 1;
    if (j.err) atomicOr(j.err, 1);
  };

  if (warp < 4) {
    // ---- converters
    const int rr = lane & 7, gq = lane >> 3;
    const bool vec = (m & 3) == 0 && (reinterpret_cast<uintptr_t>(j.a.Y) & 15) == 0;
    float4 v[4][2][2];   // [row group i][entry group gq + 4 h][half]
    auto load = [&](const C16Tile &T, int b) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 8 * (warp + 4 * i) + rr;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = b * kC16KB + 8 * (gq + 4 * h);
          const float *src = T.rows + (size_t)r * m + k;
          const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (r >= T.nrow || k >= m) {
            v[i][h][0] = z;
            v[i][h][1] = z;
          } else if (vec) {   // k + 4 <= m; entries k + 4 .. exist only if k + 8 <= m
            v[i][h][0] = __ldg(reinterpret_cast<const float4 *>(src));
            v[i][h][1] = k + 8 <= m ? __ldg(reinterpret_cast<const float4 *>(src + 4)) : z;
          } else {
            float e[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) e[q] = k + q < m ? src[q] : 0.f;
            v[i][h][0] = make_float4(e[0], e[1], e[2], e[3]);
            v[i][h][1] = make_float4(e[4], e[5], e[6], e[7]);
          }
        }
      }
    };
    bool stop = false;
    if ((int64_t)blockIdx.x < j.ntile) load(c16_tile(j, j.tile0 + blockIdx.x), 0);
    uint32_t tk = 0;   // tiles converted
    for (int64_t tt = blockIdx.x; tt < j.ntile && !stop; tt += gridDim.x, ++tk) {
      const C16Tile T = c16_tile(j, j.tile0 + tt);
      const int set = (int)(tk & 1);
      // the products of every pass of the tile two back read this set
      if (tk >= 2 && !tc::mbar_wait(&bars->empty_a[set], ((tk >> 1) - 1) & 1, j.wait_limit)) {
        give_up();
        break;
      }
      for (int b = 0; b < nblk; ++b) {
        if (*fail) {
          stop = true;
          break;
        }
        unsigned char *A = smem + kC16A + (size_t)(set * kC16ABlks + b) * kC16ABlk;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float4 x = v[i][h][0], y = v[i][h][1];
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(x.x, x.y), p1 = __floats2bfloat162_rn(x.z, x.w);
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(y.x, y.y), p3 = __floats2bfloat162_rn(y.z, y.w);
            const uint32_t off = (uint32_t)((warp + 4 * i) * 1024 + (gq + 4 * h) * 128 + rr * 16);
            *reinterpret_cast<uint4 *>(A + off) =
                make_uint4(*reinterpret_cast<const uint32_t *>(&p0), *reinterpret_cast<const uint32_t *>(&p1),
                           *reinterpret_cast<const uint32_t *>(&p2), *reinterpret_cast<const uint32_t *>(&p3));
          }
        }
        tc::fence_proxy_async();
        tc::mbar_arrive(&bars->full_a[set][b]);
        if (b + 1 < nblk)
          load(T, b + 1);
        else if (tt + gridDim.x < j.ntile)
          load(c16_tile(j, j.tile0 + tt + gridDim.x), 0);
      }
    }
  } else if (warp < 8) {
    // ---- read-out: warp 4 + q owns TMEM lanes (tile rows) 32 q .. 32 q + 31
    const int q = warp & 3;
    float *tb = reinterpret_cast<float *>(smem + kC16T) + (size_t)q * 32 * kC16Pitch;
    const bool vst = (K & 3) == 0;
    const int sub = lane >> 3, c4 = 4 * (lane & 7);   // write phase: row 4 jj + sub, columns c4 .. c4 + 3
    uint32_t cnt = 0;   // items read out
    const int64_t nit = ((j.ntile - blockIdx.x + gridDim.x - 1) / gridDim.x) * npass;   // this block's items
    for (int64_t k = 0; k < nit; ++k, ++cnt) {
      const int64_t tt = blockIdx.x + (k / npass) * (int64_t)gridDim.x;
      const int p = (int)(k % npass);
      const int acc = cnt & 1;
      const bool got = tc::mbar_wait(&bars->acc_full[acc], (cnt >> 1) & 1, j.wait_limit);
      if (!__all_sync(0xffffffffu, got)) {   // the TMEM loads below need the whole warp
        give_up();
        break;
      }
      if (__any_sync(0xffffffffu, *fail != 0)) break;
      tc::fence_after();
      const C16Tile T = c16_tile(j, j.tile0 + tt);
      const int c0 = p * kC16NT;
      const int ncol = K - c0 < kC16NT ? K - c0 : kC16NT;
      for (int c = 0; c < ncol; c += 32) {
        float x[32];
        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kC16NT + c), x);
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          *reinterpret_cast<float4 *>(tb + lane * kC16Pitch + e) = make_float4(x[e], x[e + 1], x[e + 2], x[e + 3]);
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int rl = 4 * jj + sub, row = 32 * q + rl, col = c + c4;
          const float4 y = *reinterpret_cast<const float4 *>(tb + rl * kC16Pitch + c4);
          if (row >= T.nrow) continue;
          float *o = T.out + (size_t)row * K + c0 + col;
          if (vst && col + 4 <= ncol) {
            *reinterpret_cast<float4 *>(o) = y;
          } else {
            if (col < ncol) o[0] = y.x;
            if (col + 1 < ncol) o[1] = y.y;
            if (col + 2 < ncol) o[2] = y.z;
            if (col + 3 < ncol) o[3] = y.w;
          }
        }
        __syncwarp();
      }
      tc::fence_before();
      tc::mbar_arrive(&bars->acc_empty[acc]);
    }
  } else if (warp == 8) {
    // ---- loader: the pass's slabs (32 KB each) into the stages
    if (lane == 0 && !j.leave) {
      uint32_t c = 0;   // slabs issued
      bool stop = false;
      const int64_t nit = ((j.ntile - blockIdx.x + gridDim.x - 1) / gridDim.x) * npass;
      for (int64_t k = 0; k < nit && !stop; ++k) {
        const int64_t g = j.tile0 + blockIdx.x + (k / npass) * (int64_t)gridDim.x;
        const int t = find_subset(j.a.tile_start, j.a.L, g);
        const int p = (int)(k % npass);
        for (int b = 0; b < nblk; ++b) {
          const int s = (int)(c % kC16Stages);
          const uint32_t u = c / kC16Stages;
          if (u >= 1 && !tc::mbar_wait(&bars->empty_b[s], (u - 1) & 1, j.wait_limit)) {
            give_up();
            stop = true;
            break;
          }
          if (*fail) {
            stop = true;
            break;
          }
          const size_t src = ((size_t)t * nblk + b) * (size_t)j.Kp * kC16KB * 2 + (size_t)p * kC16Slab;
          tc::mbar_expect_tx(&bars->full_b[s], kC16Slab);
          tc::bulk_g2s(smem + kC16B + (size_t)s * kC16Slab, j.img + src, kC16Slab, &bars->full_b[s]);
          ++c;
        }
      }
      // the shared memory outlives no copy: wait (bounded) for the last slab
      // issued into every stage
      for (int s = 0; s < kC16Stages; ++s)
        if (c > (uint32_t)s) tc::mbar_wait(&bars->full_b[s], ((c - 1 - s) / kC16Stages) & 1, j.wait_limit);
    }
  } else {
    // ---- issuer: four 128 x 256 x 16 products per block into the item's accumulator
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(128, kC16NT);
      const uint32_t abase = tc::smem_u32(smem + kC16A), bbase = tc::smem_u32(smem + kC16B);
      uint32_t c = 0, cnt = 0, tk = 0;   // slabs, items, tiles
      bool stop = false;
      for (int64_t tt = blockIdx.x; tt < j.ntile && !stop; tt += gridDim.x, ++tk) {
        const int set = (int)(tk & 1);
        const uint32_t par = (tk >> 1) & 1;
        for (int p = 0; p < npass && !stop; ++p, ++cnt) {
          const int acc = cnt & 1;
          if (cnt >= 2 && !tc::mbar_wait(&bars->acc_empty[acc], ((cnt >> 1) - 1) & 1, j.wait_limit)) {
            give_up();
            stop = true;
            break;
          }
          tc::fence_after();
          const uint32_t d = tbase + (uint32_t)(acc * kC16NT);
          for (int b = 0; b < nblk; ++b) {
            const int s = (int)(c % kC16Stages);
            if (*fail || !tc::mbar_wait(&bars->full_a[set][b], par, j.wait_limit) ||
                !tc::mbar_wait(&bars->full_b[s], (c / kC16Stages) & 1, j.wait_limit)) {
              if (!*fail) give_up();
              stop = true;
              break;
            }
            tc::fence_after();
            const uint32_t a_s = abase + (uint32_t)(set * kC16ABlks + b) * kC16ABlk, b_s = bbase + (uint32_t)s * kC16Slab;
#pragma unroll
            for (int ks = 0; ks < kC16KB / 16; ++ks) {
              const uint32_t o = (uint32_t)ks * 256;
              tc::mma_bf16(d, tc::smem_desc(a_s + o, 128, 1024), tc::smem_desc(b_s + o, 128, 1024), idesc,
                           b > 0 || ks > 0);
            }
            tc::mma_commit(&bars->empty_b[s]);
            ++c;
          }
          if (stop) break;
          tc::mma_commit(&bars->acc_full[acc]);
        }
        if (stop) break;
        // every pass of the tile has read its image set
        tc::mma_commit(&bars->empty_a[set]);
      }
      // every product issued has finished before the tensor memory is freed
      tc::mma_commit(&bars->done);
      if (!tc::mbar_wait(&bars->done, 0, j.wait_limit)) give_up();
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 9) tc::tmem_dealloc(tbase, 2 * kC16NT);
}

// ---- selection: the Batch-OMP loop and exact refit from alpha0 in global memory
// A block of 8 warps covers 8 spw signals of a 128-signal tile (spw signals per
// warp, 16 / spw blocks per tile); shared memory holds only the per-warp
// factors and, when it fits, the G-column cache, so many blocks share an SM to
// hide the loop's latency.
constexpr int kSelThreads = 256;

struct SelLayout {
  int lp;
  int gcn;   // G columns of the support cached per warp
  size_t ls, gc, total;
};

// Per-warp factor scratch, then as many of the support's G columns per warp as
// fit the shared memory one block gets at the occupancy its registers allow
// (the first picks' columns: column p is re-read by the s - 1 - p later
// updates, so caching the first few saves most of the L2 reads), at most cap
// columns when cap > 0 and none when cap < 0.
inline SelLayout sel_layout(int K, int s, int regs, bool h16, int cap) {
  const int rr = (regs + 7) & ~7;
  int blocks = 65536 / (kSelThreads * (rr > 0 ? rr : 8));
  blocks = blocks < 1 ? 1 : (blocks > 8 ? 8 : blocks);
  const size_t budget = (size_t)228 * 1024 / blocks - 1024;
  SelLayout L{};
  L.lp = odd_pitch(s);
  const size_t ls = align16(sizeof(float) * (size_t)8 * s * L.lp);
  const size_t col = (h16 ? 2 : sizeof(float)) * (size_t)8 * K;   // one column for every warp
  int fit = budget > ls ? (int)((budget - ls) / col) : 0;
  if (cap < 0) fit = 0;
  else if (cap > 0 && fit > cap) fit = cap;
  L.gcn = fit < s - 1 ? fit : (s > 1 ? s - 1 : 0);
  size_t off = 0;
  L.ls = off; off += ls;
  L.gc = off; off += align16(col * L.gcn);
  L.total = off;
  return L;
}

// Signals per warp of the selection kernel: 1, 2 or 4 (default 4).
inline int sel_spw(const OmpArgs &a) { return a.sel_spw == 1 || a.sel_spw == 2 ? a.sel_spw : 4; }

template <int KPL, int MU, bool EXACT, bool H16>
__global__ void __launch_bounds__(kSelThreads, KPL <= 8 ? 4 : (KPL <= 16 ? 3 : 2)) omp_select_kernel(OmpArgs a, SelLayout lay, const float *a0c,
                                                                 int64_t tile0, int spw) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, s = a.s;
  const int warp = threadIdx.x >> 5;
  const int bpt = 16 / spw, nb = 8 * spw;   // blocks per tile, signals per block
  const int64_t g = tile0 + blockIdx.x / bpt;
  const int part = blockIdx.x % bpt;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)128 + part * nb;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  if (rows_left <= 0) return;   // whole block: nothing below is a block-wide barrier
  const int nsig = rows_left < nb ? (int)rows_left : nb;
  const float *__restrict__ Dt = static_cast<const float *>(a.D) + (size_t)t * K * m;
  const float *__restrict__ Gt = static_cast<const float *>(a.G) + (size_t)t * K * K;
  const float *a0 = a0c + ((size_t)(g - tile0) * 128 + part * nb) * K;
  float *Ls = reinterpret_cast<float *>(smem + lay.ls) + (size_t)warp * s * lay.lp;
  void *gc = nullptr;
  if (lay.gcn > 0)
    gc = H16 ? static_cast<void *>(reinterpret_cast<__half *>(smem + lay.gc) + (size_t)warp * lay.gcn * K)
             : static_cast<void *>(reinterpret_cast<float *>(smem + lay.gc) + (size_t)warp * lay.gcn * K);
  const __half *G16t = H16 ? static_cast<const __half *>(a.G16) + (size_t)t * K * K : nullptr;
  code_warp_signals<float, KPL, MU, EXACT, H16>(a, a0, static_cast<const float *>(a.Y) + (size_t)row0 * m, m,
                                               warp * spw, spw, nsig, row0, Dt, Gt, Ls, gc, lay.lp, lay.gcn, G16t);
}

template <int KPL, int MU, bool EXACT, bool H16>
cudaError_t launch_select(const OmpArgs &a, const float *a0c, int64_t tile0, int64_t ntile, cudaStream_t st) {
  auto kern = omp_select_kernel<KPL, MU, EXACT, H16>;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const SelLayout lay = sel_layout(a.K, a.s, fa.numRegs, H16, a.sel_gcn);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  const int spw = sel_spw(a);
  kern<<<(unsigned)(ntile * (16 / spw)), kSelThreads, lay.total, st>>>(a, lay, a0c, tile0, spw);
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

cudaError_t launch_omp_tc(const OmpArgs &a, const void *img, float *a0c, int num_sms, const X3Wait &w,
                          cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  const size_t smem = tc::smem_for_tmem(kC16Smem, 2 * kC16NT);   // all 512 TMEM columns: one block per SM
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(corr16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  C16Job j{};
  j.a = a;
  j.img = static_cast<const unsigned char *>(img);
  j.out = a0c;
  j.nblk = round64c(a.m) / kC16KB;
  j.Kp = round256c(a.K);
  j.npass = (a.K + kC16NT - 1) / kC16NT;
  if (j.nblk > kC16ABlks) return cudaErrorInvalidValue;   // m <= 256: a tile's image fits one set
  j.err = a.err;
  j.wait_limit = w.limit > 0 ? w.limit : 1;
  j.leave = w.leave;
  const int64_t sms = num_sms > 0 ? num_sms : 1;
  const int64_t chunk = omp_tc_chunk_tiles(a.K, a.total_tiles, a.a0_cap);
  for (int64_t g0 = 0; g0 < a.total_tiles; g0 += chunk) {
    j.tile0 = g0;
    j.ntile = a.total_tiles - g0 < chunk ? a.total_tiles - g0 : chunk;
    corr16_kernel<<<(unsigned)(j.ntile < sms ? j.ntile : sms), kC16Threads, smem, st>>>(j);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the coefficients from alpha0 on the support carry its BF16 rounding; the
    // selection loop's FP32 correction step (residual from D_S and y in FP32,
    // solved with the factor of the FP32 Gram, within 2^-16 of the exact one)
    // removes it to about 2^-16 kappa(G_SS) of that rounding, so no separate
    // refit from D_S^T y is needed
    if ((e = launch_omp_select(a, a0c, g0, j.ntile, false, st, a.G16 != nullptr)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sdl
