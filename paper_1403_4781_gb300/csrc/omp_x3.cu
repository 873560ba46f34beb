// FP32-accurate tensor-core correlations and Gram for OMP (SDL_PREC_F32X3),
// and the single-product TF32 correlations (SDL_PREC_TF32).
//
// OMP's first step ranks alpha0 = D^T y (Sec. 1) and the Batch-OMP update
// reads G = D^T D; the FP32 path forms both with FMA chains on the CUDA cores.
// Here they run on the tensor cores with kind::tf32 products, each operand
// split in two TF32 parts (hi = tf32(x), lo = tf32(x - hi): hi + lo carries x
// to about 2^-22) and x.z = x_hi z_hi + x_hi z_lo + x_lo z_hi accumulated in
// FP32 in tensor memory.  The dropped x_lo z_lo and the two splits leave under
// 3 2^-22 of each |x_i z_i|, below the FP32 sum's own rounding bound (m 2^-24
// at m >= 64), so the selection that follows (the FP32 selection kernel with
// its refit and refinement step on the support) meets the FP32 parity bar.
// The TF32 precision (SDL_PREC_TF32) takes the correlations from hi hi^T
// alone (one product; each operand rounded to 11 significant bits, so within
// 2 2^-11 of each |x_i z_i|) and keeps the three-product Gram, whose factor
// lets the selection's FP32 correction step on the support remove that
// rounding from the coefficients.
//
// Layout.  Operands are K-major canonical images of 32-bit elements without
// swizzle: core matrices of 8 rows x 16 bytes (four elements), 128 bytes apart
// along K, 8-row groups 1 KB apart, in blocks of 32 signal entries (four
// K-steps of eight).  The dictionary's hi and lo images are [L][mp/32][Kp][32]
// floats (Kp = K rounded up to 128, zero padding), so 128 atoms of one block
// are one contiguous 16 KB bulk copy.
//
// Kernel.  A work item is a tile of 128 rows (signals, or atoms for the Gram)
// against one pass of up to 256 atoms; a persistent block of 10 warps runs
// items in turn with four roles that meet only at mbarriers:
//   warps 0-3  convert the tile's rows, 32 entries at a time, into the hi and
//              lo A images (two buffers), the next block's loads in flight
//              while they wait for a free buffer;
//   warp 8     streams the dictionary's 128-atom chunks (hi + lo, 32 KB) into
//              four stages by bulk copies;
//   warp 9     issues per chunk four K-steps of three 128 x 128 x 8 MMAs into
//              the pass's TMEM accumulator (two of 256 columns, alternating by
//              item), freeing each stage and A buffer by tcgen05.commit;
//   warps 4-7  read a finished accumulator out (warp 4 + q owns TMEM lanes
//              32 q .. 32 q + 31) into the item's rows of the output while the
//              next item's products run into the other accumulator.
// Every wait is bounded: a role that gives up sets the block's fail flag and
// the error word; the others leave at their next check or bounded wait, the
// loader waits for its copies in flight, the issuer for its products, and the
// tensor memory is freed.
#include "omp_common.cuh"
#include "tc_ptx.cuh"

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kX3Threads = 320;
constexpr int kX3NT = 128;                     // atoms per chunk (the MMA's N)
constexpr int kX3KB = 32;                      // signal entries per block
constexpr int kX3Pass = 256;                   // atoms per item (one accumulator)
constexpr int kX3Stages = 4;                   // dictionary chunk stages
constexpr uint32_t kX3Slab = 128u * kX3KB * 4; // one 128-row block image (hi or lo): 16 KB

inline int round32(int x) { return (x + 31) & ~31; }
inline int round128(int x) { return (x + 127) & ~127; }

// TF32 value nearest to x (ties away from zero), as an FP32 bit pattern.
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (r, k), k < 32, in a block image of 32-bit elements.
__host__ __device__ inline uint32_t x3_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Instruction descriptor of kind::tf32: FP32 accumulate (bit 4), TF32 A and B
// (format 2 at bits 7 and 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc) : "memory");
}

// D [L][K][m] FP32 -> hi and lo images [L][mp/32][Kp][32] (zero padding).
// Thread item q: four consecutive entries of one row.
__global__ void x3_image_kernel(const float *__restrict__ D, int K, int m, int Kp, int mp, int L,
                                unsigned char *__restrict__ hi, unsigned char *__restrict__ lo) {
  const int ng = mp >> 2;
  const int64_t total = (int64_t)L * Kp * ng;
  const int nblk = mp / kX3KB;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / ((int64_t)Kp * ng);
    const int rem = (int)(q - t * Kp * ng);
    const int r = rem / ng, k0 = (rem - r * ng) * 4;
    const float *src = D + ((size_t)t * K + r) * m;
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = (r < K && k0 + e < m) ? src[k0 + e] : 0.f;
      h[e] = tf32_rn(x);
      l[e] = tf32_rn(x - h[e]);
    }
    const int b = k0 / kX3KB;
    const size_t off = ((size_t)t * nblk + b) * (size_t)Kp * kX3KB * 4 + x3_offset(r, k0 % kX3KB);
    *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// What the kernel reads and writes.  Tiles are the 128-signal tiles of the OMP
// plan (tile0 .. tile0 + ntile - 1, output rows in the alpha0 scratch) or, for
// the Gram, 128-atom tiles of every dictionary (output rows of G).
struct X3Job {
  OmpArgs a;                 // K, m, L; OMP: Y and the tile plan; Gram: D
  const unsigned char *hi;   // dictionary images [L][nblk][Kp][32]
  const unsigned char *lo;
  float *out;                // alpha0 scratch (rows of K) or G [L][K][K]
  int64_t tile0, ntile;
  int nblk, Kp, npass, tpd;  // blocks of 32 entries, padded K, items per tile, Gram tiles per dictionary
  int32_t *err;
  int wait_limit;            // polls of a bounded wait
  int leave;                 // 1: the loader leaves at once (a test of the bounded waits)
};

struct X3Tile {
  int t;              // dictionary
  const float *rows;  // row 0 of the tile (pitch m)
  int nrow;           // valid rows
  float *out;         // output row 0 (pitch K)
};

template <bool GRAM>
__device__ __forceinline__ X3Tile x3_tile(const X3Job &j, int64_t g) {
  X3Tile T;
  const int K = j.a.K, m = j.a.m;
  if (GRAM) {
    T.t = (int)(g / j.tpd);
    const int r0 = (int)(g - (int64_t)T.t * j.tpd) * 128;
    T.rows = static_cast<const float *>(j.a.D) + ((size_t)T.t * K + r0) * m;
    T.nrow = K - r0 < 128 ? K - r0 : 128;
    T.out = j.out + ((size_t)T.t * K + r0) * K;
  } else {
    T.t = find_subset(j.a.tile_start, j.a.L, g);
    const int64_t row0 = j.a.offsets[T.t] + (g - j.a.tile_start[T.t]) * (int64_t)128;
    const int64_t left = j.a.offsets[T.t + 1] - row0;
    T.rows = static_cast<const float *>(j.a.Y) + (size_t)row0 * m;
    T.nrow = left < 128 ? (int)left : 128;
    T.out = j.out + (size_t)(g - j.tile0) * 128 * K;
  }
  return T;
}

struct X3Bars {
  uint64_t full_b[kX3Stages], empty_b[kX3Stages];
  uint64_t full_a[2], empty_a[2];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t done;
  uint32_t tslot;
  int fail;
};

constexpr size_t kX3A = 0;                                  // 2 x (hi, lo) block images
constexpr size_t kX3B = 4 * (size_t)kX3Slab;                // 4 stages x (hi, lo) chunks
constexpr size_t kX3Bar = kX3B + 2 * kX3Stages * (size_t)kX3Slab;
constexpr size_t kX3Smem = kX3Bar + sizeof(X3Bars);


// NP = 3: the three products of the split; NP = 1: hi hi^T alone (one TF32
// product, SDL_PREC_TF32), the lo images neither formed nor loaded.
template <bool GRAM, int NP>
__global__ void __launch_bounds__(kX3Threads, 1) corr_x3_kernel(X3Job j) {
  extern __shared__ __align__(1024) unsigned char smem[];
  X3Bars *bars = reinterpret_cast<X3Bars *>(smem + kX3Bar);
  volatile int *fail = &bars->fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = j.a.K, m = j.a.m, nblk = j.nblk;
  const int64_t nitem = j.ntile * j.npass;

  if (warp == 9) tc::tmem_alloc(&bars->tslot, 2 * kX3Pass);
  if (tid == 0) {
    for (int q = 0; q < kX3Stages; ++q) {
      tc::mbar_init(&bars->full_b[q], 1);
      tc::mbar_init(&bars->empty_b[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bars->full_a[q], 128);
      tc::mbar_init(&bars->empty_a[q], 1);
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
  // 128-atom chunks of item pass p (the last pass may hold fewer than 256 atoms)
  auto chunks_of = [&](int p) { return K - p * kX3Pass > kX3NT ? 2 : 1; };

  if (warp < 4) {
    // ---- converters: item u of thread (warp, lane) is row 8 (warp + 4 (u / 2)) +
    // (lane & 7) and entries 4 ((lane >> 3) + 4 (u & 1)) .. + 3 of each block,
    // so the eight lanes of a quarter-warp store 128 contiguous bytes (rows 0-7
    // of one core matrix: no bank conflict)
    const int rr = lane & 7, gq = lane >> 3;
    auto row_of = [&](int u) { return 8 * (warp + 4 * (u >> 1)) + rr; };
    auto grp_of = [&](int u) { return gq + 4 * (u & 1); };
    const bool vec = (m & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(GRAM ? j.a.D : j.a.Y) & 15) == 0;   // 16-byte rows
    float4 v[8];
    auto load = [&](const X3Tile &T, int b) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = row_of(i), k = b * kX3KB + 4 * grp_of(i);
        const float *src = T.rows + (size_t)r * m + k;
        if (r >= T.nrow || k >= m) {
          v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (vec) {   // k + 4 <= m when m is a multiple of 4
          v[i] = __ldg(reinterpret_cast<const float4 *>(src));
        } else {
          v[i] = make_float4(src[0], k + 1 < m ? src[1] : 0.f, k + 2 < m ? src[2] : 0.f, k + 3 < m ? src[3] : 0.f);
        }
      }
    };
    uint32_t cnt = 0;   // blocks converted
    bool stop = false;
    if ((int64_t)blockIdx.x < nitem) load(x3_tile<GRAM>(j, j.tile0 + blockIdx.x / j.npass), 0);
    for (int64_t it = blockIdx.x; it < nitem && !stop; it += gridDim.x) {
      const X3Tile T = x3_tile<GRAM>(j, j.tile0 + it / j.npass);
      for (int b = 0; b < nblk; ++b) {
        const int ab = cnt & 1;
        if (cnt >= 2 && !tc::mbar_wait(&bars->empty_a[ab], ((cnt >> 1) - 1) & 1, j.wait_limit)) {
          give_up();
          stop = true;
          break;
        }
        if (*fail) {
          stop = true;
          break;
        }
        unsigned char *Ah = smem + kX3A + (size_t)ab * 2 * kX3Slab;
        unsigned char *Al = Ah + kX3Slab;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t off = x3_offset(row_of(i), 4 * grp_of(i));
          const float4 h = make_float4(tf32_rn(v[i].x), tf32_rn(v[i].y), tf32_rn(v[i].z), tf32_rn(v[i].w));
          *reinterpret_cast<float4 *>(Ah + off) = h;
          if (NP == 3) {
            const float4 l = make_float4(tf32_rn(v[i].x - h.x), tf32_rn(v[i].y - h.y), tf32_rn(v[i].z - h.z),
                                         tf32_rn(v[i].w - h.w));
            *reinterpret_cast<float4 *>(Al + off) = l;
          }
        }
        tc::fence_proxy_async();
        tc::mbar_arrive(&bars->full_a[ab]);
        ++cnt;
        // the next block's loads fly while this thread waits for a free buffer
        if (b + 1 < nblk)
          load(T, b + 1);
        else if (it + gridDim.x < nitem)
          load(x3_tile<GRAM>(j, j.tile0 + (it + gridDim.x) / j.npass), 0);
      }
    }
  } else if (warp < 8) {
    // ---- read-out: warp 4 + q owns TMEM lanes (tile rows) 32 q .. 32 q + 31
    const int q = warp & 3, row = 32 * q + lane;
    const bool vst = (K & 3) == 0;
    uint32_t cnt = 0;
    for (int64_t it = blockIdx.x; it < nitem; it += gridDim.x, ++cnt) {
      const int acc = cnt & 1;
      const bool got = tc::mbar_wait(&bars->acc_full[acc], (cnt >> 1) & 1, j.wait_limit);
      if (!__all_sync(0xffffffffu, got)) {   // the TMEM loads below need the whole warp
        give_up();
        break;
      }
      if (__any_sync(0xffffffffu, *fail != 0)) break;
      tc::fence_after();
      const X3Tile T = x3_tile<GRAM>(j, j.tile0 + it / j.npass);
      const int c0 = (int)(it % j.npass) * kX3Pass;
      const int ncol = K - c0 < kX3Pass ? K - c0 : kX3Pass;
      float *orow = T.out + (size_t)row * K + c0;
      const bool ok = row < T.nrow;
      for (int c = 0; c < ncol; c += 32) {
        float x[32];
        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kX3Pass + c), x);
        if (!ok) continue;
        if (vst && c + 32 <= ncol) {
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<float4 *>(orow + c + e) = make_float4(x[e], x[e + 1], x[e + 2], x[e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (c + e < ncol) orow[c + e] = x[e];
        }
      }
      tc::fence_before();
      tc::mbar_arrive(&bars->acc_empty[acc]);
    }
  } else if (warp == 8) {
    // ---- loader: the dictionary's chunks (hi and lo, 16 KB each) into the stages
    if (lane == 0 && !j.leave) {
      uint32_t c = 0;   // chunks issued
      bool stop = false;
      for (int64_t it = blockIdx.x; it < nitem && !stop; it += gridDim.x) {
        const int64_t g = j.tile0 + it / j.npass;
        const int t = GRAM ? (int)(g / j.tpd) : find_subset(j.a.tile_start, j.a.L, g);
        const int p = (int)(it % j.npass), nch = chunks_of(p);
        for (int b = 0; b < nblk && !stop; ++b) {
          const size_t slab = ((size_t)t * nblk + b) * (size_t)j.Kp * kX3KB * 4;
          for (int ch = 0; ch < nch; ++ch) {
            const int s = c % kX3Stages;
            const uint32_t u = c / kX3Stages;
            if (u >= 1 && !tc::mbar_wait(&bars->empty_b[s], (u - 1) & 1, j.wait_limit)) {
              give_up();
              stop = true;
              break;
            }
            if (*fail) {
              stop = true;
              break;
            }
            const size_t src = slab + (size_t)(p * kX3Pass + ch * kX3NT) * kX3KB * 4;
            unsigned char *dst = smem + kX3B + (size_t)s * 2 * kX3Slab;
            tc::mbar_expect_tx(&bars->full_b[s], (NP == 3 ? 2 : 1) * kX3Slab);
            tc::bulk_g2s(dst, j.hi + src, kX3Slab, &bars->full_b[s]);
            if (NP == 3) tc::bulk_g2s(dst + kX3Slab, j.lo + src, kX3Slab, &bars->full_b[s]);
            ++c;
          }
        }
      }
      // the shared memory outlives no copy: wait (bounded) for the last chunk
      // issued into every stage
      for (int s = 0; s < kX3Stages; ++s)
        if (c > (uint32_t)s) tc::mbar_wait(&bars->full_b[s], ((c - 1 - s) / kX3Stages) & 1, j.wait_limit);
    }
  } else {
    // ---- issuer: three kind::tf32 products per K-step into the item's accumulator
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, kX3NT);
      const uint32_t abase = tc::smem_u32(smem + kX3A), bbase = tc::smem_u32(smem + kX3B);
      uint32_t c = 0, nbk = 0, cnt = 0;
      bool stop = false;
      for (int64_t it = blockIdx.x; it < nitem && !stop; it += gridDim.x, ++cnt) {
        const int acc = cnt & 1, nch = chunks_of((int)(it % j.npass));
        if (cnt >= 2 && !tc::mbar_wait(&bars->acc_empty[acc], ((cnt >> 1) - 1) & 1, j.wait_limit)) {
          give_up();
          break;
        }
        tc::fence_after();
        for (int b = 0; b < nblk && !stop; ++b) {
          const int ab = nbk & 1;
          if (*fail || !tc::mbar_wait(&bars->full_a[ab], (nbk >> 1) & 1, j.wait_limit)) {
            if (!*fail) give_up();
            stop = true;
            break;
          }
          tc::fence_after();
          const uint32_t ahi = abase + (uint32_t)ab * 2 * kX3Slab, alo = ahi + kX3Slab;
          for (int ch = 0; ch < nch; ++ch) {
            const int s = c % kX3Stages;
            if (!tc::mbar_wait(&bars->full_b[s], (c / kX3Stages) & 1, j.wait_limit)) {
              give_up();
              stop = true;
              break;
            }
            tc::fence_after();
            const uint32_t bhi = bbase + (uint32_t)s * 2 * kX3Slab, blo = bhi + kX3Slab;
            const uint32_t d = tbase + (uint32_t)(acc * kX3Pass + ch * kX3NT);
#pragma unroll
            for (int ks = 0; ks < kX3KB / 8; ++ks) {
              const uint32_t o = (uint32_t)ks * 256;
              const uint64_t dah = tc::smem_desc(ahi + o, 128, 1024), dal = tc::smem_desc(alo + o, 128, 1024);
              const uint64_t dbh = tc::smem_desc(bhi + o, 128, 1024), dbl = tc::smem_desc(blo + o, 128, 1024);
              mma_tf32(d, dah, dbh, idesc, b > 0 || ks > 0);
              if (NP == 3) {
                mma_tf32(d, dah, dbl, idesc, true);
                mma_tf32(d, dal, dbh, idesc, true);
              }
            }
            tc::mma_commit(&bars->empty_b[s]);
            ++c;
          }
          if (stop) break;
          tc::mma_commit(&bars->empty_a[ab]);
          ++nbk;
        }
        if (stop) break;
        tc::mma_commit(&bars->acc_full[acc]);
      }
      // every product issued has finished before the tensor memory is freed
      tc::mma_commit(&bars->done);
      if (!tc::mbar_wait(&bars->done, 0, j.wait_limit)) give_up();
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 9) tc::tmem_dealloc(tbase, 2 * kX3Pass);
}

template <bool GRAM, int NP>
cudaError_t launch_x3(const X3Job &j, int num_sms, cudaStream_t st) {
  const int64_t nitem = j.ntile * j.npass;
  if (nitem <= 0) return cudaSuccess;
  auto kern = corr_x3_kernel<GRAM, NP>;
  // the block takes all 512 TMEM columns: one block per SM
  const size_t smem = tc::smem_for_tmem(kX3Smem, 2 * kX3Pass);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t sms = num_sms > 0 ? num_sms : 1;
  const unsigned grid = (unsigned)(nitem < sms ? nitem : sms);
  kern<<<grid, kX3Threads, smem, st>>>(j);
  return cudaGetLastError();
}

X3Job x3_job(const OmpArgs &a, const void *hi, const void *lo, float *out, int32_t *err, const X3Wait &w) {
  X3Job j{};
  j.a = a;
  j.hi = static_cast<const unsigned char *>(hi);
  j.lo = static_cast<const unsigned char *>(lo);
  j.out = out;
  j.nblk = round32(a.m) / kX3KB;
  j.Kp = round128(a.K);
  j.npass = (a.K + kX3Pass - 1) / kX3Pass;
  j.tpd = (a.K + 127) / 128;
  j.err = err;
  j.wait_limit = w.limit > 0 ? w.limit : 1;
  j.leave = w.leave;
  return j;
}

}  // namespace

size_t x3_image_bytes(int L, int K, int m) { return (size_t)L * round128(K) * round32(m) * 4; }

cudaError_t launch_x3_image(const float *D, int K, int m, int L, void *hi, void *lo, cudaStream_t st) {
  const int Kp = round128(K), mp = round32(m);
  const int64_t total = (int64_t)L * Kp * (mp >> 2);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  x3_image_kernel<<<blocks, 256, 0, st>>>(D, K, m, Kp, mp, L, static_cast<unsigned char *>(hi),
                                          static_cast<unsigned char *>(lo));
  return cudaGetLastError();
}

cudaError_t launch_gram_x3(const float *D, const void *hi, const void *lo, int K, int m, int L, float *G,
                           int32_t *err, int num_sms, const X3Wait &w, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  OmpArgs a{};
  a.D = D;
  a.K = K;
  a.m = m;
  a.L = L;
  X3Job j = x3_job(a, hi, lo, G, err, w);
  j.tile0 = 0;
  j.ntile = (int64_t)L * j.tpd;
  return launch_x3<true, 3>(j, num_sms, st);
}

cudaError_t launch_omp_x3(const OmpArgs &a, const void *hi, const void *lo, float *a0c, int num_sms,
                          const X3Wait &w, cudaStream_t st, bool single) {
  if (a.total_tiles <= 0) return cudaSuccess;
  X3Job j = x3_job(a, hi, lo, a0c, a.err, w);
  const int64_t chunk = omp_tc_chunk_tiles(a.K, a.total_tiles, a.a0_cap);
  for (int64_t g0 = 0; g0 < a.total_tiles; g0 += chunk) {
    j.tile0 = g0;
    j.ntile = a.total_tiles - g0 < chunk ? a.total_tiles - g0 : chunk;
    cudaError_t e = single ? launch_x3<false, 1>(j, num_sms, st) : launch_x3<false, 3>(j, num_sms, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_omp_select(a, a0c, g0, j.ntile, false, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sdl
