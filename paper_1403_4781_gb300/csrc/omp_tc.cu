// BF16 tensor-core front end of OMP (Sec. 1) and of the Gram matrix.
//
// The correlations alpha0 = D^T y and the Gram G = D^T D are dense contractions,
// so the BF16 path runs them on the 5th-generation tensor cores: tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulation) with the accumulator tile in
// tensor memory, operands in shared memory in the canonical K-major layout.
// Dictionary tiles are streamed in by bulk TMA copies of a pre-laid-out BF16
// image of D; the signal tile is converted from FP32 in the kernel.  After the
// readout of alpha0 into shared memory each warp runs the shared selection loop
// and then refits the coefficients on the support exactly in FP32 from D (one
// refinement step), so the BF16 rounding affects only which atoms are chosen.
#include "omp_common.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kTcThreads = 256;
constexpr int kWaitLimit = 1 << 22;   // polls of a bounded mbarrier wait

// D [L][K][m] FP32 -> BF16 image [L][Kp][mp]; zero padding rows / columns.
__global__ void bf16_image_kernel(const float *__restrict__ D, int K, int m, int Kp, int mp, int L,
                                  unsigned char *__restrict__ img) {
  const int kc8 = mp >> 3;
  const int64_t total = (int64_t)L * Kp * kc8;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / ((int64_t)Kp * kc8);
    const int rem = (int)(q - t * Kp * kc8);
    const int r = rem / kc8, kc = rem - r * kc8;
    const float *src = D + ((size_t)t * K + r) * m;
    uint32_t packed[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k0 = kc * 8 + 2 * e;
      const float lo = (r < K && k0 < m) ? src[k0] : 0.f;
      const float hi = (r < K && k0 + 1 < m) ? src[k0 + 1] : 0.f;
      __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
      packed[e] = *reinterpret_cast<uint32_t *>(&b2);
    }
    *reinterpret_cast<uint4 *>(img + (size_t)t * Kp * mp * 2 + tc::image_offset(r, kc * 8, mp)) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// G tile [128 rows][NG cols] of subset blockIdx.z from the BF16 image.
__global__ void __launch_bounds__(128) gram_tc_kernel(const unsigned char *__restrict__ img, int K, int Kp, int mp,
                                                      int NG, float *__restrict__ G, int32_t *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = blockIdx.z, bx = blockIdx.x, by = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *Aim = smem;
  unsigned char *Bim = smem + (size_t)128 * mp * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (size_t)(128 + NG) * mp * 2);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
  const uint32_t ncols = NG <= 128 ? 128u : 256u;
  if (warp == 0) tc::tmem_alloc(tslot, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const unsigned char *sub = img + (size_t)t * Kp * mp * 2;
  const int rowsA = min(128, Kp - 128 * bx), rowsB = min(NG, Kp - NG * by);
  if (tid == 0) {
    tc::mbar_expect_tx(&mbar[0], (uint32_t)(rowsA + rowsB) * mp * 2);
    tc::bulk_g2s(Aim, sub + (size_t)128 * bx * mp * 2, (uint32_t)rowsA * mp * 2, &mbar[0]);
    tc::bulk_g2s(Bim, sub + (size_t)NG * by * mp * 2, (uint32_t)rowsB * mp * 2, &mbar[0]);
  }
  bool ok = tc::mbar_wait(&mbar[0], 0, kWaitLimit);
  if (ok && tid == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, NG);
    const uint32_t sbo = (uint32_t)(mp >> 3) * 128;
    for (int ks = 0; ks < (mp >> 4); ++ks)
      tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(Aim) + ks * 256, 128, sbo),
                   tc::smem_desc(tc::smem_u32(Bim) + ks * 256, 128, sbo), idesc, ks > 0);
    tc::mma_commit(&mbar[1]);
  }
  __syncthreads();
  if (ok) ok = tc::mbar_wait(&mbar[1], 0, kWaitLimit);
  tc::fence_after();
  if (ok) {
    const int row = 128 * bx + 32 * warp + lane;
    for (int c0 = 0; c0 < NG; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + c0, v);
      if (row < K) {
        float *grow = G + ((size_t)t * K + row) * K;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int col = NG * by + c0 + e;
          if (col < K) grow[col] = v[e];
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

struct TcLayout {
  int TS, NT, lp;
  bool gcache;
  size_t a0, uni, ls, gx, bar, total;
};

TcLayout tc_layout(int TS, int NT, int K, int mp, int s, bool gcache) {
  TcLayout L{};
  L.TS = TS; L.NT = NT; L.gcache = gcache;
  L.lp = odd_pitch(s);
  size_t off = 0;
  L.uni = off;   // first: 1024-aligned operand images / G-column cache
  const size_t imgs = (size_t)(128 + NT) * mp * 2;
  const size_t gcol = gcache ? sizeof(float) * (size_t)8 * s * K : 0;
  off += align16(imgs > gcol ? imgs : gcol);
  L.a0 = off;  off += align16(sizeof(float) * (size_t)TS * K);
  L.ls = off;  off += align16(sizeof(float) * (size_t)8 * s * L.lp);
  L.gx = off;  off += align16(sizeof(float) * (size_t)8 * s * L.lp);
  L.bar = off; off += 64;
  L.total = off;
  return L;
}

// Prefer layouts that let two blocks share an SM (the selection loop is latency
// bound and wants warps), then the largest signal tile.
bool pick_tc_layout(int K, int mp, int s, TcLayout *out) {
  const size_t limits[2] = {113 * 1024, 227 * 1024};
  const int tss[4] = {128, 64, 32, 16}, nts[3] = {256, 128, 64};
  for (int li = 0; li < 2; ++li)
    for (int ti = 0; ti < 4; ++ti)
      for (int ni = 0; ni < 3; ++ni)
        for (int gcv = 1; gcv >= 0; --gcv) {
          TcLayout L = tc_layout(tss[ti], nts[ni], K, mp, s, gcv == 1);
          if (L.total <= limits[li]) { *out = L; return true; }
        }
  return false;
}

// One block codes TS signals of one subset: alpha0 tile on the tensor cores
// (one M=128 MMA row block, N-tiles of NT atoms), then the selection loop.
template <int KPL, int MU>
__global__ void __launch_bounds__(kTcThreads) omp_tc_kernel(OmpArgs a, TcLayout lay) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, s = a.s, mp = a.mp, Kp = a.Kp, TS = lay.TS, NT = lay.NT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t g = blockIdx.x;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)TS;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < TS ? (int)rows_left : TS;
  const float *__restrict__ Dt = static_cast<const float *>(a.D) + (size_t)t * K * m;
  const float *__restrict__ Gt = static_cast<const float *>(a.G) + (size_t)t * K * K;
  const float *__restrict__ Y = static_cast<const float *>(a.Y);
  const unsigned char *sub = static_cast<const unsigned char *>(a.Dimg) + (size_t)t * Kp * mp * 2;
  float *a0 = reinterpret_cast<float *>(smem + lay.a0);
  unsigned char *Aim = smem + lay.uni;
  unsigned char *Bim = Aim + (size_t)128 * mp * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + lay.bar);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
  int *fail = reinterpret_cast<int *>(mbar + 3);
  const uint32_t ncols = (uint32_t)NT;

  if (warp == 0) tc::tmem_alloc(tslot, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
    *fail = 0;
  }
  // signal tile -> BF16 A image (rows beyond the tile are zero)
  const int kc8 = mp >> 3;
  for (int q = tid; q < 128 * kc8; q += kTcThreads) {
    const int r = q / kc8, kc = q - r * kc8;
    uint32_t packed[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k0 = kc * 8 + 2 * e;
      const float *yr = Y + (size_t)(row0 + r) * m;
      const float lo = (r < nsig && k0 < m) ? yr[k0] : 0.f;
      const float hi = (r < nsig && k0 + 1 < m) ? yr[k0 + 1] : 0.f;
      __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
      packed[e] = *reinterpret_cast<uint32_t *>(&b2);
    }
    *reinterpret_cast<uint4 *>(Aim + tc::image_offset(r, kc * 8, mp)) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_bf16(128, NT);
  const uint32_t sbo = (uint32_t)kc8 * 128;
  const int ntiles = (K + NT - 1) / NT;
  for (int nt = 0; nt < ntiles; ++nt) {
    const int rows = min(NT, Kp - nt * NT);
    if (tid == 0) {
      tc::mbar_expect_tx(&mbar[0], (uint32_t)rows * mp * 2);
      tc::bulk_g2s(Bim, sub + (size_t)nt * NT * mp * 2, (uint32_t)rows * mp * 2, &mbar[0]);
    }
    if (!tc::mbar_wait(&mbar[0], nt & 1, kWaitLimit)) *fail = 1;
    __syncthreads();
    if (*fail) break;
    if (tid == 0) {
      tc::fence_after();
      for (int ks = 0; ks < (mp >> 4); ++ks)
        tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(Aim) + ks * 256, 128, sbo),
                     tc::smem_desc(tc::smem_u32(Bim) + ks * 256, 128, sbo), idesc, ks > 0);
      tc::mma_commit(&mbar[1]);
    }
    if (!tc::mbar_wait(&mbar[1], nt & 1, kWaitLimit)) *fail = 1;
    __syncthreads();
    if (*fail) break;
    tc::fence_after();
    {   // warp w: TMEM lanes 32 (w % 4) .., columns of half w / 4
      const int rq = (warp & 3) * 32, cb = (warp >> 2) * (NT >> 1);
      const int row = rq + lane;
      for (int c0 = cb; c0 < cb + (NT >> 1); c0 += 32) {
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)rq << 16) + c0, v);
        if (row < TS) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int col = nt * NT + c0 + e;
            if (col < K) a0[(size_t)row * K + col] = v[e];
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();   // TMEM and the B image are free for the next tile
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
  if (*fail) {
    if (tid == 0 && a.err) atomicOr(a.err, 1);
    return;
  }
  float *Ls = reinterpret_cast<float *>(smem + lay.ls) + (size_t)warp * s * lay.lp;
  float *Gx = reinterpret_cast<float *>(smem + lay.gx) + (size_t)warp * s * lay.lp;
  float *gc = reinterpret_cast<float *>(smem + lay.uni) + (size_t)warp * s * K;
  const int spw = TS / 8;
  code_warp_signals<float, KPL, MU, true>(a, a0, Y + (size_t)row0 * m, m, warp * spw, spw, nsig, row0, Dt, Gt, Ls, Gx, gc,
                                      lay.lp, lay.gcache);
}

template <int KPL, int MU>
cudaError_t launch_omp_tc_kpl(const OmpArgs &a, const TcLayout &lay, cudaStream_t st) {
  auto kern = omp_tc_kernel<KPL, MU>;
  const size_t smem = tc::smem_for_tmem(lay.total, lay.NT);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.total_tiles, kTcThreads, smem, st>>>(a, lay);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bf16_image(const float *D, int K, int m, int L, void *img, cudaStream_t st) {
  const int Kp = round16(K), mp = round16(m);
  const int64_t total = (int64_t)L * Kp * (mp >> 3);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  bf16_image_kernel<<<blocks, 256, 0, st>>>(D, K, m, Kp, mp, L, static_cast<unsigned char *>(img));
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(const void *img, int K, int m, int L, float *G, int32_t *err, cudaStream_t st) {
  const int Kp = round16(K), mp = round16(m);
  const int NG = Kp > 128 ? 256 : 128;
  const size_t smem = tc::smem_for_tmem((size_t)(128 + NG) * mp * 2 + 64, NG <= 128 ? 128 : 256);
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((Kp + 127) / 128, (Kp + NG - 1) / NG, L);
  gram_tc_kernel<<<grid, 128, smem, st>>>(static_cast<const unsigned char *>(img), K, Kp, mp, NG, G, err);
  return cudaGetLastError();
}

int omp_tc_tile_signals(int K, int m, int s) {
  TcLayout lay;
  return pick_tc_layout(K, round16(m), s, &lay) ? lay.TS : 0;
}

cudaError_t launch_omp_tc(const OmpArgs &a, cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  TcLayout lay;
  if (!pick_tc_layout(a.K, a.mp, a.s, &lay)) return cudaErrorInvalidConfiguration;
  const int kpl = (a.K + 31) / 32;
  if (a.m <= 64) {
    if (kpl <= 4) return launch_omp_tc_kpl<4, 2>(a, lay, st);
    if (kpl <= 8) return launch_omp_tc_kpl<8, 2>(a, lay, st);
    if (kpl <= 16) return launch_omp_tc_kpl<16, 2>(a, lay, st);
    return launch_omp_tc_kpl<32, 2>(a, lay, st);
  }
  if (kpl <= 4) return launch_omp_tc_kpl<4, 8>(a, lay, st);
  if (kpl <= 8) return launch_omp_tc_kpl<8, 8>(a, lay, st);
  if (kpl <= 16) return launch_omp_tc_kpl<16, 8>(a, lay, st);
  return launch_omp_tc_kpl<32, 8>(a, lay, st);
}

}  // namespace sdl
