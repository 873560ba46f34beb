// Residual-form OMP on the tensor cores (BF16 path, s <= 16).
//
// OMP's greedy step (Sec. 1) ranks |d_j^T r| over the atoms.  The Batch-OMP
// form of the selection kernel gets these from alpha0 = D^T y and a running
// update through the Gram matrix, which costs every signal one K-float Gram
// column per support pair (s(s-1)/2 of them) and thousands of warp
// instructions of selection loop.  This kernel recomputes D^T r itself at every
// step: for a tile of 128 signals the residuals, rounded to BF16, form the A
// operand of tcgen05.mma (kind::f16, FP32 accumulation in tensor memory), and
// the dictionary streams through as the B operand in slabs of 256 atoms x 64
// signal entries (32 KB), so every product is a 128 x 256 x 16 MMA (the
// smallest N whose own work exceeds the tensor core's issue cost).  Four roles
// meet only at mbarriers:
//   warp 4      loads the slabs of every step in order into NS stages by bulk
//               copies (D does not change, so it runs ahead across steps);
//   warp 5      issues a chunk's products (its nblk slabs, four K-steps each)
//               into one of two 256-column TMEM accumulators, alternating by
//               chunk, once the step's A operand is written;
//   warps 0-3   consumer thread i owns signal i of the tile, which is TMEM lane
//               i: it reads its correlations straight from TMEM chunk by chunk
//               for the masked argmax, and keeps its support, the Cholesky
//               factor of G_SS (rows grown one per step, from the FP32 Gram)
//               and its coefficients.  The residual r = y - D_S x is formed in
//               FP32 from y and the FP32 atoms, warp-cooperatively for eight
//               signals at a time (lanes over the signal entries, so the atom
//               rows load coalesced), together with the right-hand side d_j^T y
//               of each new atom, so the coefficients are the FP32
//               least-squares fit on the support; after the last step one
//               correction step x += G_SS^{-1} D_S^T r refines them, as on the
//               Batch-OMP path.
// The last chunk's accumulator completes only when every product of the step
// has read the A operand, so the consumers write the next step's operand right
// after reading it.  Every wait is bounded; a role that gives up sets the
// block's fail flag and the error word, the others leave at their next check or
// bounded wait, the loader waits for its copies in flight and the issuer for
// its products before the tensor memory is freed.
//
// The correlations a step compares are those of the BF16-rounded residual, so
// their error is about 2^-8 of sum_i |d_ji r_i| at that step, where the
// Batch-OMP form carries the 2^-8 sum_i |d_ji y_i| of alpha0 into every step.
#include "omp_common.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace sdl {
namespace {

using namespace omp_detail;

constexpr int kRtcConsumers = 128;    // four warps: thread i owns signal i of the tile (TMEM lane i)
constexpr int kRtcThreads = 192;      // and the loader and issuer warps
constexpr int kRtcNT = 256;           // atoms per chunk (the MMA's N)
constexpr int kRtcKB = 64;            // signal entries per slab (four K-steps of 16)
constexpr uint32_t kRtcSlab = (uint32_t)kRtcNT * kRtcKB * 2;   // 32 KB
constexpr int kRtcWait = 1 << 26;     // polls of a bounded mbarrier wait (test_wait: tens of ns each)
constexpr int kMaxStages = 4;

inline int round64i(int x) { return (x + 63) & ~63; }
inline int round256i(int x) { return (x + 255) & ~255; }

// Byte offset of BF16 element (r, k), k < 64, in a 64-entry block: 8-row
// groups of 1 KB, core matrices of 8 rows x 16 bytes 128 bytes apart along K.
__host__ __device__ inline uint32_t blk_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct RtcLayout {
  int NS;                   // slab stages
  size_t aim, bim, lfac, bar, total;
};

// Barrier block: full/empty per stage, tfull/tempty per accumulator, aready
// (the step's A operand is written), done (the issuer's last products), then
// the TMEM address, the failure, go and stop flags.
struct RtcBars {
  uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2], aready, done;
  uint32_t tslot;
  int fail, go, stop;
};

// A operand (128 x mp BF16 in 64-entry blocks of 16 KB), NS slab stages, the
// packed lower Cholesky factors of the 128 signals ([entry][signal] floats;
// entry p (p + 1) / 2 + q holds L_pq, the diagonal slot 1 / L_pp), barriers.
inline RtcLayout rtc_layout(int mp, int smax, int NS) {
  RtcLayout L{};
  L.NS = NS;
  size_t off = 0;
  L.aim = off;  off += (size_t)128 * mp * 2;
  L.bim = off;  off += (size_t)NS * kRtcSlab;
  L.lfac = off; off += (size_t)smax * (smax + 1) / 2 * kRtcConsumers * sizeof(float);
  L.bar = off;  off += (sizeof(RtcBars) + 15) & ~size_t(15);
  L.total = off;
  return L;
}

__device__ __forceinline__ int tri(int p, int q) { return p * (p + 1) / 2 + q; }

// Entries 8 gg .. 8 gg + 7 of a length-m row (zero beyond m); vec: 16-byte
// aligned rows (m a multiple of 4).
__device__ __forceinline__ void load8(const float *row, int gg, int m, bool vec, float (&v)[8]) {
  const int k0 = 8 * gg;
  if (vec && k0 + 8 <= m) {
    const float4 a = *reinterpret_cast<const float4 *>(row + k0);
    const float4 b = *reinterpret_cast<const float4 *>(row + k0 + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = k0 + e < m ? row[k0 + e] : 0.f;
  }
}

// Sum over the four lanes that share a signal (lanes l, l^8, l^16, l^24).
__device__ __forceinline__ float sum4(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// Eight BF16 entries of an A-operand row into the blocked image.
__device__ __forceinline__ void store8(unsigned char *Aim, int row, int gg, const float (&v)[8]) {
  uint32_t packed[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    packed[e] = *reinterpret_cast<uint32_t *>(&b2);
  }
  const int k = 8 * gg;
  *reinterpret_cast<uint4 *>(Aim + (size_t)(k >> 6) * (128 * kRtcKB * 2) + blk_offset(row, k & 63)) =
      make_uint4(packed[0], packed[1], packed[2], packed[3]);
}

// Signal status: active (awaiting a pick), picked this step (coefficients and
// residual pending), stopping this step without a pick, done (code written).
enum : int { kActive = 0, kPicked = 1, kStopping = 3, kDone = 2 };

template <int SMAX>
__device__ __forceinline__ int reg_at(const int (&v)[SMAX], int i) {
  int out = -1;
#pragma unroll
  for (int p = 0; p < SMAX; ++p)
    if (p == i) out = v[p];
  return out;
}

// D [L][K][m] FP32 -> BF16 image [L][mp/64][Kp][64] (Kp = K rounded up to 256,
// zero padding): 256 atoms of one 64-entry block are one contiguous slab.
__global__ void rtc_image_kernel(const float *__restrict__ D, int K, int m, int Kp, int mp, int L,
                                 unsigned char *__restrict__ img) {
  const int kg = mp >> 3;
  const int nblk = mp / kRtcKB;
  const int64_t total = (int64_t)L * Kp * kg;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / ((int64_t)Kp * kg);
    const int rem = (int)(q - t * Kp * kg);
    const int r = rem / kg, gg = rem - r * kg;
    const float *src = D + ((size_t)t * K + r) * m;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (r < K && 8 * gg + e < m) ? src[8 * gg + e] : 0.f;
    uint32_t packed[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      packed[e] = *reinterpret_cast<uint32_t *>(&b2);
    }
    const int k = 8 * gg;
    const size_t off = ((size_t)t * nblk + (k >> 6)) * (size_t)Kp * kRtcKB * 2 + blk_offset(r, k & 63);
    *reinterpret_cast<uint4 *>(img + off) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// One block per 128-signal tile: consumer warps 0..3 (thread i owns signal i),
// loader warp 4, issuer warp 5.  SMAX: the largest sparsity the registers hold
// (s <= SMAX); UMAX: 8-entry groups of the signal per lane in the
// warp-cooperative residual passes (mp / 32).
template <int SMAX, int UMAX>
__global__ void __launch_bounds__(kRtcThreads, 1) omp_rtc_kernel(OmpArgs a, RtcLayout lay,
                                                                 const unsigned char *__restrict__ img) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, s = a.s, NS = lay.NS;
  const int mp = (m + 63) & ~63, Kp = (K + 255) & ~255;
  const int nblk = mp / kRtcKB, nch = Kp / kRtcNT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t g = blockIdx.x;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)128;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < 128 ? (int)rows_left : 128;
  const float *__restrict__ Y = static_cast<const float *>(a.Y);
  const float *__restrict__ Dt = static_cast<const float *>(a.D) + (size_t)t * K * m;
  const float *__restrict__ Gt = static_cast<const float *>(a.G) + (size_t)t * K * K;
  const unsigned char *sub = img + (size_t)t * nblk * Kp * kRtcKB * 2;
  float *val_out = static_cast<float *>(a.val);
  float *r2_out = static_cast<float *>(a.resid2);
  unsigned char *Aim = smem + lay.aim;
  unsigned char *Bim = smem + lay.bim;
  float *Lf = reinterpret_cast<float *>(smem + lay.lfac);
  RtcBars *B = reinterpret_cast<RtcBars *>(smem + lay.bar);
  volatile int *fail = &B->fail;
  volatile int *go = &B->go;
  volatile int *stop = &B->stop;
  const bool vec = (m & 3) == 0;
  const float eps = (float)a.eps;
  const int kg = mp >> 3;                        // 8-entry groups of a padded signal
  const int64_t total_slabs = (int64_t)s * nch * nblk;

  if (warp == 5) tc::tmem_alloc(&B->tslot, 2 * kRtcNT);
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      tc::mbar_init(&B->full[q], 1);
      tc::mbar_init(&B->empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&B->tfull[q], 1);
      tc::mbar_init(&B->tempty[q], kRtcConsumers);
    }
    tc::mbar_init(&B->aready, kRtcConsumers);
    tc::mbar_init(&B->done, 1);
    tc::mbar_fence_init();
    B->fail = 0;
    B->go = 0;
    B->stop = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = B->tslot;

  if (warp == 4) {
    // ---- loader: every step's slabs in order, NS stages ahead of the products
    if (lane == 0) {
      int64_t lq = 0;
      bool ok = true;
      for (; lq < total_slabs; ++lq) {
        const int st = (int)(lq % NS);
        if (lq >= NS) {   // the stage's previous slab must have been multiplied, unless the steps ended
          const uint32_t par = (uint32_t)(((lq / NS) - 1) & 1);
          bool got = false;
          for (int it = 0; it < kRtcWait && !got; ++it) {
            got = tc::mbar_poll(&B->empty[st], par, 1);
            if (!got && (*stop || *fail)) break;
          }
          if (!got) {
            if (!*stop) ok = false;
            break;
          }
        }
        const int sl = (int)(lq % ((int64_t)nch * nblk));
        const int c = sl / nblk, b = sl - c * nblk;
        tc::mbar_expect_tx(&B->full[st], kRtcSlab);
        tc::bulk_g2s(Bim + (size_t)st * kRtcSlab, sub + ((size_t)b * Kp + (size_t)c * kRtcNT) * kRtcKB * 2, kRtcSlab,
                     &B->full[st]);
      }
      if (!ok) {
        *fail = 1;
        if (a.err) atomicOr(a.err, 1);
      }
      // the shared memory outlives no copy: the last slab issued into every stage
      for (int st = 0; st < NS; ++st)
        if (lq > st) {
          const int64_t last = st + (int64_t)NS * ((lq - 1 - st) / NS);
          tc::mbar_poll(&B->full[st], (uint32_t)((last / NS) & 1), kRtcWait);
        }
    }
  } else if (warp == 5) {
    // ---- issuer: per step, once the A operand is written, every chunk's
    // products into the accumulator the chunk's parity picks
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(128, kRtcNT);
      int64_t q = 0, cq = 0;
      bool ok = true;
      for (int step = 0; step < s && ok; ++step) {
        if (!tc::mbar_poll(&B->aready, (uint32_t)(step & 1), kRtcWait)) {
          ok = false;
          break;
        }
        if (!*go || *fail) break;
        tc::fence_after();
        for (int c = 0; c < nch && ok; ++c) {
          const int acc = (int)(cq & 1);
          if (cq >= 2 && !tc::mbar_poll(&B->tempty[acc], (uint32_t)(((cq >> 1) - 1) & 1), kRtcWait)) {
            ok = false;
            break;
          }
          tc::fence_after();
          for (int b = 0; b < nblk; ++b) {
            const int st = (int)(q % NS);
            if (!tc::mbar_poll(&B->full[st], (uint32_t)((q / NS) & 1), kRtcWait)) {
              ok = false;
              break;
            }
            tc::fence_after();
            const uint32_t asb = tc::smem_u32(Aim) + (uint32_t)b * (128 * kRtcKB * 2);
            const uint32_t bsb = tc::smem_u32(Bim) + (uint32_t)st * kRtcSlab;
#pragma unroll
            for (int ks = 0; ks < kRtcKB / 16; ++ks)
              tc::mma_bf16(tbase + (uint32_t)(acc * kRtcNT), tc::smem_desc(asb + ks * 256, 128, 1024),
                           tc::smem_desc(bsb + ks * 256, 128, 1024), idesc, b > 0 || ks > 0);
            tc::mma_commit(&B->empty[st]);
            ++q;
          }
          if (!ok) break;
          tc::mma_commit(&B->tfull[acc]);
          ++cq;
        }
      }
      if (!ok) {
        *fail = 1;
        if (a.err) atomicOr(a.err, 1);
      }
      *stop = 1;   // no more products: a loader waiting on a stage may leave
      // every product issued has finished before the tensor memory is freed
      tc::mma_commit(&B->done);
      tc::mbar_poll(&B->done, 0, kRtcWait);
    }
  } else {
    // ---- consumers: thread tid owns signal row tid of the tile
    int S[SMAX];
    float x[SMAX], z[SMAX];
#pragma unroll
    for (int p = 0; p < SMAX; ++p) {
      S[p] = -1;
      x[p] = 0.f;
      z[p] = 0.f;
    }
    int status = tid < nsig ? kActive : kDone;
    float wz = 0.f, rl = 0.f;   // the step's new factor row: w^T z and 1 / l

    // step 0's operand: bf16(y) of every signal, and ||y||^2 to its owner.
    // Lanes l, l^8, l^16, l^24 share signal 8 grp + (l & 7) of the warp, each
    // holding its 8-entry groups gsub + 4u (gsub = l >> 3).
    const int gsub = lane >> 3;
    float yn2 = 0.f;
    for (int grp = 0; grp < 4; ++grp) {
      const int ow = grp * 8 + (lane & 7);
      const int row = warp * 32 + ow;
      const float *yrow = Y + (size_t)(row0 + (row < nsig ? row : 0)) * m;
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        const int gg = gsub + 4 * u;
        if (gg >= kg) continue;
        float v[8];
        if (row < nsig) {
          load8(yrow, gg, m, vec, v);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.f;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) acc = fmaf(v[e], v[e], acc);
        store8(Aim, row, gg, v);
      }
      acc = sum4(acc);
      if (gsub == grp) yn2 = acc;   // this lane owns the signal
    }
    // error-constrained stop before the first pick: ||y|| <= eps codes nothing
    if (status == kActive && eps > 0.f && sqrtf(yn2) <= eps) status = kStopping;

    int64_t cq = 0;   // chunks read (the accumulators alternate by it)
    for (int step = 0; step < s; ++step) {
      // the A operand (bf16 residuals) is complete: hand it to the issuer
      tc::fence_proxy_async();
      const bool act = tc::named_any(1, kRtcConsumers, status == kActive) && !*fail;
      if (tid == 0) *go = act ? 1 : 0;
      tc::mbar_arrive(&B->aready);
      float best = 0.f;   // a pick needs |d_j^T r| > 0
      int bj = -1;
      if (act) {
        // D^T r chunk by chunk from the accumulators: masked argmax, lowest
        // index on ties (columns are visited in increasing atom order)
        for (int c = 0; c < nch; ++c, ++cq) {
          const int acc = (int)(cq & 1);
          bool ok = !*fail && tc::mbar_poll(&B->tfull[acc], (uint32_t)((cq >> 1) & 1), kRtcWait);
          ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
          if (!ok) *fail = 1;
          tc::fence_after();
          if (ok) {
            for (int cc = 0; cc < kRtcNT; cc += 32) {
              if (c * kRtcNT + cc >= K) break;   // warp-uniform
              float v[32];
              tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * kRtcNT + cc), v);
              if (status == kActive) {
                const int j0 = c * kRtcNT + cc;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  const float av = fabsf(v[e]);
                  const int j = j0 + e;
                  if (av > best && j < K) {
                    bool in = false;
#pragma unroll
                    for (int p = 0; p < SMAX; ++p) in |= (p < step && S[p] == j);
                    if (!in) {
                      best = av;
                      bj = j;
                    }
                  }
                }
              }
            }
          }
          tc::fence_before();
          tc::mbar_arrive(&B->tempty[acc]);   // this accumulator may be overwritten
        }
        if (*fail) bj = -1;
      }

      // ---- the pick's Cholesky row (thread per signal): L w = G[S, j],
      // l = sqrt(g_jj - w^T w); the pivot test of the Batch-OMP loop
      if (status == kActive) {
        if (bj < 0) {
          status = kStopping;
        } else {
          const float *grow = Gt + (size_t)bj * K;
          float w[SMAX];
          float wtw = 0.f, wzz = 0.f;
#pragma unroll
          for (int p = 0; p < SMAX; ++p) {
            w[p] = 0.f;
            if (p < step) {
              float acc = grow[S[p]];
#pragma unroll
              for (int q = 0; q < p; ++q) acc = fmaf(-Lf[tri(p, q) * kRtcConsumers + tid], w[q], acc);
              w[p] = acc * Lf[tri(p, p) * kRtcConsumers + tid];
              wtw = fmaf(w[p], w[p], wtw);
              wzz = fmaf(w[p], z[p], wzz);
            }
          }
          const float gbb = grow[bj];
          const float piv2 = gbb - wtw;
          if (!(piv2 > kOmpPivotRelF32 * gbb) || !(piv2 > 0.f)) {
            status = kStopping;
          } else {
#pragma unroll
            for (int p = 0; p < SMAX; ++p)
              if (p < step) Lf[tri(step, p) * kRtcConsumers + tid] = w[p];
            rl = 1.f / sqrtf(piv2);
            Lf[tri(step, step) * kRtcConsumers + tid] = rl;
            wz = wzz;
#pragma unroll
            for (int p = 0; p < SMAX; ++p)
              if (p == step) S[p] = bj;
            status = kPicked;
          }
        }
      }

      // ---- coefficients and residuals, eight signals per warp at a time (every
      // lane runs every pass; the shuffles below are warp-wide).  The step's
      // products are done (the last chunk was read), so the operand rows may
      // be overwritten for the next step.
      for (int grp = 0; grp < 4; ++grp) {
        const int ow = grp * 8 + (lane & 7);   // lane that owns this lane's signal
        const int row = warp * 32 + ow;
        const bool mine = gsub == grp;
        const int st = __shfl_sync(0xffffffffu, status, ow);
        const bool work = st == kPicked || st == kStopping;
        const int natoms = st == kPicked ? step + 1 : step;
        const float *yrow = Y + (size_t)(row0 + (work ? row : 0)) * m;
        float r[UMAX][8];
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
          const int gg = gsub + 4 * u;
          if (work && gg < kg) {
            load8(yrow, gg, m, vec, r[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) r[u][e] = 0.f;
          }
        }
        // right-hand side of the new atom, d_j^T y in FP32
        const int jn = __shfl_sync(0xffffffffu, reg_at<SMAX>(S, step), ow);
        float bp = 0.f;
        if (st == kPicked) {
          const float *dj = Dt + (size_t)jn * m;
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            const int gg = gsub + 4 * u;
            if (gg >= kg) continue;
            float d[8];
            load8(dj, gg, m, vec, d);
#pragma unroll
            for (int e = 0; e < 8; ++e) bp = fmaf(d[e], r[u][e], bp);
          }
        }
        const float bsum = sum4(bp);
        if (mine && status == kPicked) {
          // z grows by one entry; x = L^{-T} z on the support
#pragma unroll
          for (int p = 0; p < SMAX; ++p)
            if (p == step) z[p] = (bsum - wz) * rl;
#pragma unroll
          for (int p = SMAX - 1; p >= 0; --p) {
            if (p <= step) {
              float acc = z[p];
#pragma unroll
              for (int q = p + 1; q < SMAX; ++q)
                if (q <= step) acc = fmaf(-Lf[tri(q, p) * kRtcConsumers + tid], x[q], acc);
              x[p] = acc * Lf[tri(p, p) * kRtcConsumers + tid];
            }
          }
        }
        // r = y - D_S x in FP32
#pragma unroll
        for (int p = 0; p < SMAX; ++p) {
          const float xp = __shfl_sync(0xffffffffu, x[p], ow);
          const int sp = __shfl_sync(0xffffffffu, S[p], ow);
          if (work && p < natoms) {
            const float *dp = Dt + (size_t)sp * m;
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
              const int gg = gsub + 4 * u;
              if (gg >= kg) continue;
              float d[8];
              load8(dp, gg, m, vec, d);
#pragma unroll
              for (int e = 0; e < 8; ++e) r[u][e] = fmaf(-d[e], xp, r[u][e]);
            }
          }
        }
        float rp = 0.f;
#pragma unroll
        for (int u = 0; u < UMAX; ++u)
#pragma unroll
          for (int e = 0; e < 8; ++e) rp = fmaf(r[u][e], r[u][e], rp);
        const float rsum = sum4(rp);   // the same value in the signal's four lanes
        const bool fin = st == kStopping ||
                         (st == kPicked && (step + 1 == s || (eps > 0.f && sqrtf(rsum) <= eps)));
        if (st == kPicked && !fin) {   // the next step's operand row
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            const int gg = gsub + 4 * u;
            if (gg < kg) store8(Aim, row, gg, r[u]);
          }
        } else if (work) {             // a finished signal's row stays zero from now on
          const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int u = 0; u < UMAX; ++u) {
            const int gg = gsub + 4 * u;
            if (gg < kg) store8(Aim, row, gg, zero);
          }
        }
        // finished signals: one correction step x += G_SS^{-1} D_S^T r, whose
        // residual energy is ||r||^2 - ||L^{-1} D_S^T r||^2, then the ELL row
        float cvec[SMAX];
#pragma unroll
        for (int p = 0; p < SMAX; ++p) {
          const int sp = __shfl_sync(0xffffffffu, S[p], ow);
          float part = 0.f;
          if (fin && p < natoms) {
            const float *dp = Dt + (size_t)sp * m;
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
              const int gg = gsub + 4 * u;
              if (gg >= kg) continue;
              float d[8];
              load8(dp, gg, m, vec, d);
#pragma unroll
              for (int e = 0; e < 8; ++e) part = fmaf(d[e], r[u][e], part);
            }
          }
          cvec[p] = sum4(part);
        }
        if (mine && fin) {
          float wq[SMAX], dx[SMAX];
          float wn2 = 0.f;
#pragma unroll
          for (int p = 0; p < SMAX; ++p) {
            wq[p] = 0.f;
            if (p < natoms) {
              float acc = cvec[p];
#pragma unroll
              for (int q = 0; q < p; ++q) acc = fmaf(-Lf[tri(p, q) * kRtcConsumers + tid], wq[q], acc);
              wq[p] = acc * Lf[tri(p, p) * kRtcConsumers + tid];
              wn2 = fmaf(wq[p], wq[p], wn2);
            }
          }
#pragma unroll
          for (int p = SMAX - 1; p >= 0; --p) {
            dx[p] = 0.f;
            if (p < natoms) {
              float acc = wq[p];
#pragma unroll
              for (int q = p + 1; q < SMAX; ++q)
                if (q < natoms) acc = fmaf(-Lf[tri(q, p) * kRtcConsumers + tid], dx[q], acc);
              dx[p] = acc * Lf[tri(p, p) * kRtcConsumers + tid];
            }
          }
          const int64_t gi = row0 + row;
#pragma unroll
          for (int p = 0; p < SMAX; ++p) {
            if (p < s) {
              a.idx[(size_t)gi * s + p] = p < natoms ? S[p] : -1;
              val_out[(size_t)gi * s + p] = p < natoms ? x[p] + dx[p] : 0.f;
            }
          }
          a.nnz[gi] = natoms;
          const float res2 = rsum - wn2;
          if (r2_out) r2_out[gi] = res2 > 0.f ? res2 : 0.f;
          status = kDone;
        } else if (mine && st == kPicked) {
          status = kActive;
        }
      }
      if (!act) break;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 5) tc::tmem_dealloc(tbase, 2 * kRtcNT);
}

template <int SMAX, int UMAX>
cudaError_t launch_rtc(const OmpArgs &a, const void *img, cudaStream_t st) {
  auto kern = omp_rtc_kernel<SMAX, UMAX>;
  const int mp = round64i(a.m);
  // the most slab stages (2 .. 4) that fit one block's shared memory
  RtcLayout lay{};
  bool found = false;
  for (int ns = kMaxStages; ns >= 2 && !found; --ns)
    if (rtc_layout(mp, SMAX, ns).total <= 227 * 1024) {
      lay = rtc_layout(mp, SMAX, ns);
      found = true;
    }
  if (!found) return cudaErrorInvalidConfiguration;
  // the block takes all 512 TMEM columns: one block per SM
  const size_t smem = tc::smem_for_tmem(lay.total, 2 * kRtcNT);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.total_tiles, kRtcThreads, smem, st>>>(a, lay, static_cast<const unsigned char *>(img));
  return cudaGetLastError();
}

template <int SMAX>
cudaError_t rtc_dispatch_m(const OmpArgs &a, const void *img, cudaStream_t st) {
  const int mp = round64i(a.m);
  if (mp <= 64) return launch_rtc<SMAX, 2>(a, img, st);
  if (mp <= 128) return launch_rtc<SMAX, 4>(a, img, st);
  return launch_rtc<SMAX, 8>(a, img, st);
}

}  // namespace

bool omp_rtc_supported(int K, int m, int s) { return s >= 1 && s <= 16 && m >= 1 && m <= 256 && K >= 1 && K <= 4096; }

size_t rtc_image_bytes(int L, int K, int m) { return (size_t)L * round256i(K) * round64i(m) * 2; }

cudaError_t launch_rtc_image(const float *D, int K, int m, int L, void *img, cudaStream_t st) {
  const int Kp = round256i(K), mp = round64i(m);
  const int64_t total = (int64_t)L * Kp * (mp >> 3);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  rtc_image_kernel<<<blocks, 256, 0, st>>>(D, K, m, Kp, mp, L, static_cast<unsigned char *>(img));
  return cudaGetLastError();
}

cudaError_t launch_omp_rtc(const OmpArgs &a, const void *img, cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  if (!omp_rtc_supported(a.K, a.m, a.s)) return cudaErrorInvalidValue;
  if (a.s <= 4) return rtc_dispatch_m<4>(a, img, st);
  if (a.s <= 8) return rtc_dispatch_m<8>(a, img, st);
  return rtc_dispatch_m<16>(a, img, st);
}

}  // namespace sdl
