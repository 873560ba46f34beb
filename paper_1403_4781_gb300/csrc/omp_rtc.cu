// Residual-form OMP on the tensor cores (BF16 path, s <= 16).
//
// OMP's greedy step (Sec. 1) ranks |d_j^T r| over the atoms.  The Batch-OMP
// form of the selection kernel gets these from alpha0 = D^T y and a running
// update through the Gram matrix, which costs every signal one K-float Gram
// column per support pair (s(s+1)/2 of them) and several thousand warp
// instructions of selection loop.  This kernel recomputes D^T r itself at every
// step: for a tile of 128 signals the residuals, rounded to BF16, form the A
// operand of tcgen05.mma (kind::f16, FP32 accumulation in tensor memory) and
// the dictionary streams through as the B operand in chunks of NT atoms.  A
// producer warp keeps NS chunks in flight (bulk copies from the dictionary's
// BF16 image into a ring of shared-memory stages, running ahead across step
// boundaries, since D does not change) and issues each chunk's products into
// one of two TMEM accumulators; full/empty mbarriers gate every hand-over, so
// no block-wide barrier sits in the chunk loop.  Consumer thread i owns signal i of the tile,
// which is TMEM lane i: it reads its correlations straight from TMEM for the
// masked argmax, and keeps its support, the Cholesky factor of G_SS (rows
// grown one per step, from the FP32 Gram) and its coefficients.  The residual
// r = y - D_S x is formed in FP32 from y and the FP32 atoms, warp-cooperatively
// for eight signals at a time (lanes over the signal entries, so the atom rows
// load coalesced and the BF16 rows store into the canonical operand layout
// without bank conflicts); the right-hand side d_j^T y of each new atom is
// formed there too, in FP32, so the coefficients are the FP32 least-squares
// fit on the support.  After the last step one correction step x += G_SS^{-1}
// D_S^T r refines them, as on the Batch-OMP path.
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
constexpr int kRtcThreads = 160;      // and one producer warp
constexpr int kRtcWait = 1 << 26;     // polls of a bounded mbarrier wait (test_wait: tens of ns each)

constexpr int kMaxStages = 8;

struct RtcLayout {
  int NT;                   // atoms per dictionary chunk (the MMA's N)
  int NS;                   // chunk stages in flight
  size_t aim, bim, lfac, bar, total;
};

// Barrier block: full[kMaxStages] (chunk landed), empty[kMaxStages] (its
// products are done), tfull[2] (accumulator ready), tempty[2] (accumulator
// read by every consumer), aready (the step's A operand is written), then the
// TMEM address, the failure flag and the step's go flag.
struct RtcBars {
  uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2], aready;
  uint32_t tslot;
  int fail, go;
};

// A operand (128 x mp BF16), NS dictionary chunks (NT x mp BF16 each), the
// packed lower Cholesky factors of the 128 signals ([entry][signal] floats;
// entry p (p + 1) / 2 + q holds L_pq, the diagonal slot 1 / L_pp), barriers.
inline RtcLayout rtc_layout(int mp, int smax, int NT, int NS) {
  RtcLayout L{};
  L.NT = NT;
  L.NS = NS;
  size_t off = 0;
  L.aim = off;  off += (size_t)128 * mp * 2;
  L.bim = off;  off += (size_t)NS * NT * mp * 2;
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

// One block per 128-signal tile: consumer warps 0..3 (thread i owns signal i)
// and producer warp 4.  SMAX: the largest sparsity the registers hold
// (s <= SMAX); UMAX: 8-entry groups of the signal per lane in the
// warp-cooperative residual passes (ceil(mp / 32)).
template <int SMAX, int UMAX>
__global__ void __launch_bounds__(kRtcThreads) omp_rtc_kernel(OmpArgs a, RtcLayout lay) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, m = a.m, mp = a.mp, Kp = a.Kp, s = a.s, NT = lay.NT, NS = lay.NS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t g = blockIdx.x;
  const int t = find_subset(a.tile_start, a.L, g);
  const int64_t row0 = a.offsets[t] + (g - a.tile_start[t]) * (int64_t)128;
  const int64_t rows_left = a.offsets[t + 1] - row0;
  const int nsig = rows_left < 128 ? (int)rows_left : 128;
  const float *__restrict__ Y = static_cast<const float *>(a.Y);
  const float *__restrict__ Dt = static_cast<const float *>(a.D) + (size_t)t * K * m;
  const float *__restrict__ Gt = static_cast<const float *>(a.G) + (size_t)t * K * K;
  const unsigned char *sub = static_cast<const unsigned char *>(a.Dimg) + (size_t)t * Kp * mp * 2;
  float *val_out = static_cast<float *>(a.val);
  float *r2_out = static_cast<float *>(a.resid2);
  unsigned char *Aim = smem + lay.aim;
  unsigned char *Bim = smem + lay.bim;
  float *Lf = reinterpret_cast<float *>(smem + lay.lfac);
  RtcBars *B = reinterpret_cast<RtcBars *>(smem + lay.bar);
  volatile int *fail = &B->fail;
  volatile int *go = &B->go;
  const size_t btile = (size_t)NT * mp * 2;
  const int nchunks = (K + NT - 1) / NT;
  const int64_t qtotal = (int64_t)s * nchunks;   // chunk loads of a run through all s steps
  const bool vec = (m & 3) == 0;
  const float eps = (float)a.eps;
  const int kg = mp >> 3;                        // 8-entry groups of a padded signal
  const uint32_t idesc = tc::idesc_bf16(128, NT);
  const uint32_t sbo = (uint32_t)kg * 128;
  const uint32_t ncols = 2 * NT < 32 ? 32u : (uint32_t)(2 * NT);

  if (warp == 0) tc::tmem_alloc(&B->tslot, ncols);
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
    tc::mbar_fence_init();
    B->fail = 0;
    B->go = 0;
  }
  // every chunk stage starts zero: a last chunk shorter than NT leaves rows of
  // its stage unwritten, whose products land in columns past K (never read)
  for (int i = tid; i < (int)((size_t)NS * btile / 16); i += kRtcThreads)
    reinterpret_cast<uint4 *>(Bim)[i] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = B->tslot;

  if (warp == 4) {
    // ---- producer: chunk loads NS - 1 ahead, products into alternating
    // accumulators; the step's products wait for its A operand (aready)
    if (lane == 0) {
      int64_t lq = 0, q = 0;   // chunk loads issued; chunks multiplied
      bool ok = true;
      auto load = [&](int64_t r) {
        const int st = (int)(r % NS), c = (int)(r % nchunks);
        const uint32_t bytes = (uint32_t)min(NT, Kp - c * NT) * (uint32_t)mp * 2u;
        tc::mbar_expect_tx(&B->full[st], bytes);
        tc::bulk_g2s(Bim + st * btile, sub + (size_t)c * NT * mp * 2, bytes, &B->full[st]);
      };
      for (; lq < NS - 1 && lq < qtotal; ++lq) load(lq);
      for (int step = 0; step < s && ok; ++step) {
        if (!tc::mbar_poll(&B->aready, (uint32_t)(step & 1), kRtcWait)) {
          ok = false;
          break;
        }
        if (!*go) break;
        for (int c = 0; c < nchunks && ok; ++c) {
          const int st = (int)(q % NS), acc = (int)(q & 1);
          if (!tc::mbar_poll(&B->full[st], (uint32_t)((q / NS) & 1), kRtcWait) ||
              (q >= 2 && !tc::mbar_poll(&B->tempty[acc], (uint32_t)(((q >> 1) - 1) & 1), kRtcWait))) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t bsm = tc::smem_u32(Bim + st * btile);
          for (int ks = 0; ks < (mp >> 4); ++ks)
            tc::mma_bf16(tbase + (uint32_t)(acc * NT), tc::smem_desc(tc::smem_u32(Aim) + ks * 256, 128, sbo),
                         tc::smem_desc(bsm + ks * 256, 128, sbo), idesc, ks > 0);
          tc::mma_commit(&B->empty[st]);
          tc::mma_commit(&B->tfull[acc]);
          ++q;
          // refill: chunk lq takes the stage of chunk lq - NS, whose products
          // are done or queued right behind the ones just issued
          while (ok && lq < qtotal && lq < q + NS - 1) {
            if (lq >= NS && !tc::mbar_poll(&B->empty[lq % NS], (uint32_t)(((lq / NS) - 1) & 1), kRtcWait)) {
              ok = false;
              break;
            }
            load(lq++);
          }
        }
      }
      if (!ok) *fail = 1;
      // wind down (bounded waits): loads that no product consumed, then the
      // last products
      for (int64_t r = q; r < lq; ++r) tc::mbar_poll(&B->full[r % NS], (uint32_t)((r / NS) & 1), kRtcWait);
      if (q > 0) tc::mbar_poll(&B->empty[(q - 1) % NS], (uint32_t)(((q - 1) / NS) & 1), kRtcWait);
      if (*fail && a.err) atomicOr(a.err, 1);
    }
    __syncwarp();   // lanes 1..31 wait for lane 0 here, then meet the block at the end
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
        uint32_t packed[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc = fmaf(v[2 * e], v[2 * e], acc);
          acc = fmaf(v[2 * e + 1], v[2 * e + 1], acc);
          __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          packed[e] = *reinterpret_cast<uint32_t *>(&b2);
        }
        *reinterpret_cast<uint4 *>(Aim + tc::image_offset(row, 8 * gg, mp)) =
            make_uint4(packed[0], packed[1], packed[2], packed[3]);
      }
      acc = sum4(acc);
      if (gsub == grp) yn2 = acc;   // this lane owns the signal
    }
    // error-constrained stop before the first pick: ||y|| <= eps codes nothing
    if (status == kActive && eps > 0.f && sqrtf(yn2) <= eps) status = kStopping;

    for (int step = 0; step < s; ++step) {
      // the A operand (bf16 residuals) is complete: hand it to the producer
      tc::fence_proxy_async();
      const bool act = tc::named_any(1, kRtcConsumers, status == kActive) && !*fail;
      if (tid == 0) *go = act ? 1 : 0;
      tc::mbar_arrive(&B->aready);
      float best = 0.f;   // a pick needs |d_j^T r| > 0
      int bj = -1;
      if (act) {
        // D^T r chunk by chunk from the accumulators: masked argmax, lowest
        // index on ties (columns are visited in increasing atom order)
        for (int c = 0; c < nchunks; ++c) {
          const int64_t q = (int64_t)step * nchunks + c;
          const int acc = (int)(q & 1);
          bool ok = !*fail && tc::mbar_poll(&B->tfull[acc], (uint32_t)((q >> 1) & 1), kRtcWait);
          ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
          if (!ok) *fail = 1;
          tc::fence_after();
          if (ok) {
            for (int cc = 0; cc < NT; cc += 16) {
              float v[16];
              tc::tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * NT + cc), v);
              if (status == kActive) {
                const int j0 = c * NT + cc;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
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
      // lane runs every pass; the shuffles below are warp-wide)
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
            if (gg >= kg) continue;
            uint32_t packed[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              __nv_bfloat162 b2 = __floats2bfloat162_rn(r[u][2 * e], r[u][2 * e + 1]);
              packed[e] = *reinterpret_cast<uint32_t *>(&b2);
            }
            *reinterpret_cast<uint4 *>(Aim + tc::image_offset(row, 8 * gg, mp)) =
                make_uint4(packed[0], packed[1], packed[2], packed[3]);
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
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

template <int SMAX, int UMAX>
cudaError_t launch_rtc(const OmpArgs &a, cudaStream_t st) {
  auto kern = omp_rtc_kernel<SMAX, UMAX>;
  // (atoms per chunk, stages): the first that lets two blocks share an SM (one
  // block's residual passes then overlap the other's products), else the
  // first that fits one block
  static const int two[][2] = {{32, 4}, {16, 6}, {32, 3}, {16, 4}, {16, 3}};
  static const int one[][2] = {{64, 4}, {32, 6}, {32, 4}, {16, 6}, {16, 4}, {16, 3}, {16, 2}};
  const size_t sm_total = 228 * 1024, sm_block = 227 * 1024;
  RtcLayout lay{};
  bool found = false;
  for (const auto &c : two)
    if (!found && 2 * (rtc_layout(a.mp, SMAX, c[0], c[1]).total + 1024) <= sm_total) {
      lay = rtc_layout(a.mp, SMAX, c[0], c[1]);
      found = true;
    }
  for (const auto &c : one)
    if (!found && rtc_layout(a.mp, SMAX, c[0], c[1]).total <= sm_block) {
      lay = rtc_layout(a.mp, SMAX, c[0], c[1]);
      found = true;
    }
  if (!found) return cudaErrorInvalidConfiguration;
  const size_t smem = tc::smem_for_tmem(lay.total, 2 * lay.NT < 32 ? 32 : 2 * lay.NT);
  if (smem > sm_block) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.total_tiles, kRtcThreads, smem, st>>>(a, lay);
  return cudaGetLastError();
}

template <int SMAX>
cudaError_t rtc_dispatch_m(const OmpArgs &a, cudaStream_t st) {
  if (a.mp <= 64) return launch_rtc<SMAX, 2>(a, st);
  if (a.mp <= 128) return launch_rtc<SMAX, 4>(a, st);
  return launch_rtc<SMAX, 8>(a, st);
}

}  // namespace

bool omp_rtc_supported(int K, int m, int s) { return s >= 1 && s <= 16 && m >= 1 && m <= 256 && K >= 1 && K <= 4096; }

cudaError_t launch_omp_rtc(const OmpArgs &a, cudaStream_t st) {
  if (a.total_tiles <= 0) return cudaSuccess;
  if (!omp_rtc_supported(a.K, a.m, a.s)) return cudaErrorInvalidValue;
  if (a.s <= 4) return rtc_dispatch_m<4>(a, st);
  if (a.s <= 8) return rtc_dispatch_m<8>(a, st);
  return rtc_dispatch_m<16>(a, st);
}

}  // namespace sdl
