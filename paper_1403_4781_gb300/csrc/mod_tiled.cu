// MOD solve (Sec. 1): D_U^T = (X X^T)_UU^{-1} (Y X^T)_U^T in FP64, with the
// renormalisation of Sec. 3.1, for a batch of independent subsets.
//
// One thread-block cluster of C blocks per subset; the subset's matrices live in
// an L2-resident scratch M of (K + m) rows x K columns:
//   rows 0..K-1   the lower triangle of A = X X^T (overwritten by its factor L),
//   rows K..K+m-1 the right-hand sides B^T (row r holds coordinate r of every
//                 atom's B column), which the right-looking factorisation carries
//                 along as extra rows: they end up as W = B^T L^{-T}.
// The matrix is cut into TS x TS tiles.  Step k of the factorisation: every
// tile below the diagonal tile (k, k) is multiplied by the inverse of its
// factor (the panel); every trailing tile (i, j), j > k, subtracts
// panel_i panel_j^T.  The block that updates tile (k+1, k+1) does so first,
// factors and inverts it at once in its shared memory and pushes the inverse
// (and the breakdown verdict) into every block of the cluster through
// distributed shared memory, while the other blocks go on with their trailing
// tiles; so the latency-bound diagonal factorisation runs once per step and
// off the critical path of the other blocks.  The backward sweep then forms
// X^T = W L^{-1} tile column by tile column from the kept inverses.  Each
// step's tile tasks are dealt round-robin to the cluster's blocks, which load
// the next task's tiles while multiplying the current one, and meet at a
// cluster barrier between dependent steps.  Several clusters share each SM, so
// one subset's barrier waits overlap another subset's tile products on the
// FP64 pipe.
//
// Breakdown (a squared pivot <= 1e-12 of its original diagonal, or not
// positive) restarts the factorisation once from A + lambda I on the used
// atoms, lambda = 1e-10 tr(A_UU) / |U|.  Unused atoms carry the identity row in
// A and their previous value in B, so they come back unchanged and are not
// renormalised.
#include <cooperative_groups.h>
#include <math.h>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr int kTThreads = 256;

// The FP32 pass's 64 x 64 tiles (R = float, TS = 64) multiply 4 x 4 register
// micro-tiles from transposed operands (A^T and B^T rows in shared memory, two
// 16-byte loads per 16 FMAs), where the other tiles' products read 1.25
// shared-memory words per FMA; their rows are padded to 68 floats so that the
// 16-byte loads stay aligned.
template <typename R, int TS>
constexpr bool kMicro = sizeof(R) == 4 && TS == 64;
template <typename R, int TS>
constexpr int kPitch = kMicro<R, TS> ? TS + 4 : TS + 1;

// R: the arithmetic type of the factorisation (double; float for the FP32
// pass of the checked mixed-precision solve below).  The micro-tiled products
// hold a and b transposed, and v as the transposes of the inverses.
template <typename R, int TS>
struct TiledSmem {
  static constexpr int P = kPitch<R, TS>;
  R a[TS][P];                // A operand; the diagonal factor during factor_diag
  R b[TS][P];                // B operand; the inverse during factor_diag
  R v[2][TS][P];             // inverses of diagonal factors k (v[k & 1]), pushed by their owner
  R invd[TS];
  R dg[TS];
  R col[TS];                 // factor_diag: the scaled column of the current step
  int fail;
  int verdict[2];            // breakdown verdict of diagonal tile k (verdict[k & 1]), pushed by its owner
};

struct TGeom {
  int K, m, R, RT, TS;
  __device__ int64_t row(int i, int r) const {
    return i < R ? (int64_t)i * TS + r : (int64_t)K + (int64_t)(i - R) * TS + r;
  }
  __device__ int rows_in(int i) const {
    const int v = i < R ? K - i * TS : m - (i - R) * TS;
    return v < TS ? v : TS;
  }
  __device__ int cols_in(int j) const {
    const int v = K - j * TS;
    return v < TS ? v : TS;
  }
};

// A TS x TS operand in global memory: p[r * ld + c] for r < nr, c < nc, zero
// elsewhere.
template <typename R>
struct Opnd {
  const R *p;
  int ld, nr, nc;
};

template <typename R, int TS>
__device__ __forceinline__ Opnd<R> tile_of(const R *Mt, const TGeom &g, int i, int j) {
  return Opnd<R>{Mt + g.row(i, 0) * g.K + (int64_t)j * TS, g.K, g.rows_in(i), g.cols_in(j)};
}

// One tile task: out (=|-=) A B^T with B staged as given (bt: from the
// transpose of its source; bsm: B is the inverse held in shared memory).
template <typename R>
struct TileTask {
  Opnd<R> a, b, o;
  bool bt, bsm, sub, lower;
};

// Thread-to-element map shared by the loads, the products and the stores:
// element u of this thread is (tid / TS + (256 / TS) u, tid mod TS).
template <typename R, int TS>
__device__ __forceinline__ void fetch(const Opnd<R> &o, R (&r)[TS * TS / kTThreads]) {
  constexpr int U = TS * TS / kTThreads, RS = kTThreads / TS;
  const int cc = threadIdx.x % TS, r0 = threadIdx.x / TS;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int rr = r0 + RS * u;
    r[u] = (rr < o.nr && cc < o.nc) ? __ldcg(o.p + (int64_t)rr * o.ld + cc) : R(0);
  }
}
template <typename R, int TS>
__device__ __forceinline__ void commit(R (*S)[kPitch<R, TS>], const R (&r)[TS * TS / kTThreads], bool t) {
  constexpr int U = TS * TS / kTThreads, RS = kTThreads / TS;
  const int cc = threadIdx.x % TS, r0 = threadIdx.x / TS;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (t) S[cc][r0 + RS * u] = r[u];
    else S[r0 + RS * u][cc] = r[u];
  }
}

// For this thread's outputs (r_u, c): acc[u] = sum_q As[r_u][q] Bs[c][q], or,
// with sub, acc[u] = old[u] - sum_q As[r_u][q] Bs[c][q] (the subtraction folded
// into the fused multiply-adds).
template <typename R, int TS>
__device__ __forceinline__ void tile_product(const R (*As)[kPitch<R, TS>], const R (*Bs)[kPitch<R, TS>], bool sub,
                                             const R (&old)[TS * TS / kTThreads], R (&acc)[TS * TS / kTThreads]) {
  constexpr int U = TS * TS / kTThreads, RS = kTThreads / TS;
  const int c = threadIdx.x % TS, r0 = threadIdx.x / TS;
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = sub ? old[u] : R(0);
  if (sub) {
#pragma unroll 8
    for (int q = 0; q < TS; ++q) {
      const R bv = Bs[c][q];
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = fma(-As[r0 + RS * u][q], bv, acc[u]);
    }
  } else {
#pragma unroll 8
    for (int q = 0; q < TS; ++q) {
      const R bv = Bs[c][q];
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = fma(As[r0 + RS * u][q], bv, acc[u]);
    }
  }
}

// The micro-tiled map (R = float, TS = 64): thread (warp w, lane l) owns
// output rows 4 ri .. 4 ri + 3 and columns 4 ci .. 4 ci + 3, ri = 4 (w / 2) +
// l / 8, ci = 8 (w mod 2) + l mod 8, element (a, b) in slot 4 a + b; a warp's
// 16-byte operand loads then touch 4 (A) and 8 (B) distinct chunks of one
// shared-memory row.
__device__ __forceinline__ int micro_ri() { return ((threadIdx.x >> 6) << 2) + ((threadIdx.x & 31) >> 3); }
__device__ __forceinline__ int micro_ci() { return (((threadIdx.x >> 5) & 1) << 3) + (threadIdx.x & 7); }

// Output tile elements in the micro map (zero outside the tile).
__device__ __forceinline__ void fetch_micro(const Opnd<float> &o, float (&r)[16]) {
  const int r0 = 4 * micro_ri(), c0 = 4 * micro_ci();
  const bool vec = (o.ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(o.p) & 15) == 0) && c0 + 4 <= o.nc;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int rr = r0 + a;
    if (rr < o.nr && vec) {
      const float4 v = __ldcg(reinterpret_cast<const float4 *>(o.p + (int64_t)rr * o.ld + c0));
      r[4 * a] = v.x; r[4 * a + 1] = v.y; r[4 * a + 2] = v.z; r[4 * a + 3] = v.w;
    } else {
#pragma unroll
      for (int b = 0; b < 4; ++b)
        r[4 * a + b] = (rr < o.nr && c0 + b < o.nc) ? __ldcg(o.p + (int64_t)rr * o.ld + c0 + b) : 0.f;
    }
  }
}

// acc = (old -) A B^T over the tile's 64 products, As[q][r] = A(r, q) and
// Bs[q][c] = B(c, q).  The products are summed from zero and old is added
// last, so that its loads (issued just before) complete under the products.
__device__ __forceinline__ void tile_product_micro(const float (*As)[68], const float (*Bs)[68], bool sub,
                                                   const float (&old)[16], float (&acc)[16]) {
  const int r0 = 4 * micro_ri(), c0 = 4 * micro_ci();
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = 0.f;
  // two copies of the loop, so that the sign is the FMA's own operand modifier
  if (sub) {
#pragma unroll 1
    for (int q = 0; q < 64; ++q) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[q][r0]);
      const float4 bv = *reinterpret_cast<const float4 *>(&Bs[q][c0]);
      const float a[4] = {av.x, av.y, av.z, av.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[4 * i + k] = fmaf(-a[i], b[k], acc[4 * i + k]);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = old[u] + acc[u];
  } else {
#pragma unroll 1
    for (int q = 0; q < 64; ++q) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[q][r0]);
      const float4 bv = *reinterpret_cast<const float4 *>(&Bs[q][c0]);
      const float a[4] = {av.x, av.y, av.z, av.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[4 * i + k] = fmaf(a[i], b[k], acc[4 * i + k]);
    }
  }
}

__device__ __forceinline__ void put_micro(const TileTask<float> &t, const float (&acc)[16]) {
  const int r0 = 4 * micro_ri(), c0 = 4 * micro_ci();
  float *base = const_cast<float *>(t.o.p);
  const bool vec = (t.o.ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(base) & 15) == 0) && c0 + 4 <= t.o.nc &&
                   !(t.lower && c0 + 3 > r0);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int rr = r0 + a;
    if (rr >= t.o.nr) continue;
    if (vec && (!t.lower || c0 + 3 <= rr)) {
      *reinterpret_cast<float4 *>(base + (int64_t)rr * t.o.ld + c0) =
          make_float4(acc[4 * a], acc[4 * a + 1], acc[4 * a + 2], acc[4 * a + 3]);
    } else {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + b;
        if (c < t.o.nc && (!t.lower || c <= rr)) base[(int64_t)rr * t.o.ld + c] = acc[4 * a + b];
      }
    }
  }
}

template <typename R, int TS>
__device__ __forceinline__ void put(const TileTask<R> &t, const R (&acc)[TS * TS / kTThreads]) {
  constexpr int U = TS * TS / kTThreads, RS = kTThreads / TS;
  const int c = threadIdx.x % TS, r0 = threadIdx.x / TS;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int r = r0 + RS * u;
    if (r < t.o.nr && c < t.o.nc && (!t.lower || c <= r))
      const_cast<R *>(t.o.p)[(int64_t)r * t.o.ld + c] = acc[u];
  }
}

// Run tasks first, first + C, ... < n of one step; the operands (and the old
// output) of the next task are loaded into registers while the current one is
// multiplied.  Tasks of one step never read a tile another task of the step
// writes.  vs: the inverse used by tasks whose B operand is in shared memory.
template <typename R, int TS, class Desc>
__device__ __forceinline__ void run_step(TiledSmem<R, TS> &sm, const R (*vs)[kPitch<R, TS>], int n, int first, int C,
                                         Desc desc) {
  constexpr int U = TS * TS / kTThreads;
  constexpr bool MI = kMicro<R, TS>;
  if (first >= n) return;
  // the output tile's old values in the product's map
  auto fetch_o = [&](const Opnd<R> &o, R (&r)[U]) {
    if constexpr (MI) fetch_micro(o, r);
    else fetch<R, TS>(o, r);
  };
  TileTask<R> cur = desc(first);
  R ra[U], rb[U], ro[U];
  fetch<R, TS>(cur.a, ra);
  if (!cur.bsm) fetch<R, TS>(cur.b, rb);
  if (!MI && cur.sub) fetch_o(cur.o, ro);
  for (int q = first; q < n; q += C) {
    __syncthreads();
    // the micro-tiled product reads A^T and B^T (B^T is the staged source
    // itself when B comes from the transpose of its source)
    commit<R, TS>(sm.a, ra, MI);
    if (!cur.bsm) commit<R, TS>(sm.b, rb, MI ? !cur.bt : cur.bt);
    __syncthreads();
    const bool more = q + C < n;
    TileTask<R> nxt = cur;
    R rn[U];
    if (more) {
      nxt = desc(q + C);
      fetch<R, TS>(nxt.a, ra);
      if (!nxt.bsm) fetch<R, TS>(nxt.b, rb);
      if (!MI && nxt.sub) fetch_o(nxt.o, rn);
    }
    // the micro-tiled tasks load their old outputs here (registers)
    if (MI && cur.sub) fetch_o(cur.o, ro);
    R acc[U];
    if constexpr (MI) {
      tile_product_micro(sm.a, cur.bsm ? vs : sm.b, cur.sub, ro, acc);
      put_micro(cur, acc);
    } else {
      tile_product<R, TS>(sm.a, cur.bsm ? vs : sm.b, cur.sub, ro, acc);
      put<R, TS>(cur, acc);
    }
    if (more) {
      cur = nxt;
      if (!MI)
#pragma unroll
        for (int u = 0; u < U; ++u) ro[u] = rn[u];
    }
  }
}

// Breakdown rule of the factorisation in FP32: a squared pivot at most this
// fraction of its diagonal leaves fewer than ~10 significant bits after
// K-term FP32 updates, so such a subset goes to the FP64 solve instead.
constexpr float kModPivotRel32 = 1e-3f;

template <typename R>
__device__ __forceinline__ R pivot_rel() { return sizeof(R) == 8 ? (R)kModPivotRel : (R)kModPivotRel32; }

template <typename R, int TS>
__device__ __forceinline__ void pivot(TiledSmem<R, TS> &sm, int c, R d) {
  if (!(d > pivot_rel<R>() * sm.dg[c]) || !(d > R(0))) {
    sm.fail = 1;
    return;
  }
  const R inv = rsqrt(d);
  sm.a[c][c] = d * inv;
  sm.invd[c] = inv;
}

// Factor the diagonal tile (k, k) into sm.a and invert the factor into sm.b
// (zero above the diagonal, identity on padding).  Returns false on breakdown.
template <typename R, int TS>
__device__ bool factor_diag(TiledSmem<R, TS> &sm, const R *Mt, const TGeom &g, int k, const double *At,
                            const int32_t *ut, double ridge) {
  const int tid = threadIdx.x;
  const int nb = g.cols_in(k);
  const int64_t base = (int64_t)k * TS;
  __syncthreads();
  for (int e = tid; e < TS * TS; e += kTThreads) {
    const int r = e / TS, c = e % TS;
    R v;
    if (r < nb && c < nb) v = c <= r ? __ldcg(Mt + (base + r) * g.K + base + c) : R(0);
    else v = r == c ? R(1) : R(0);
    sm.a[r][c] = v;
    sm.b[r][c] = r == c ? R(1) : R(0);
  }
  if (tid < TS)
    sm.dg[tid] = tid < nb ? (R)(At[(base + tid) * g.K + base + tid] + (ut[base + tid] > 0 ? ridge : 0.0)) : R(1);
  if (tid == 0) sm.fail = 0;
  __syncthreads();
  if (tid == 0) pivot(sm, 0, sm.a[0][0]);
  __syncthreads();
  // One sweep over the columns factors the tile and inverts the factor: once
  // column c of L is final, row c of V = L^{-1} is (the unit row minus the
  // earlier rows' contributions) / L_cc, and its contributions to the rows
  // below are subtracted in the same phase as the trailing update.
  for (int c = 0; c < TS; ++c) {
    if (sm.fail) break;   // uniform: read after a barrier
    if (tid > c && tid < TS) {
      const R l = sm.a[tid][c] * sm.invd[c];
      sm.a[tid][c] = l;
      sm.col[tid] = l;   // read below from consecutive words
    }
    if (tid >= TS && tid - TS <= c) sm.b[c][tid - TS] *= sm.invd[c];
    __syncthreads();
    // rank-1 update of the trailing triangle (the thread that updates the next
    // diagonal entry takes its pivot) and elimination of V's column block
    for (int e = tid; e < TS * TS; e += kTThreads) {
      const int r = e / TS, q = e % TS;
      if (q > c && q <= r) {
        const R v = fma(-sm.col[r], sm.col[q], sm.a[r][q]);
        if (r == c + 1 && q == c + 1) pivot(sm, c + 1, v);
        else sm.a[r][q] = v;
      }
      if (r > c && q <= c) sm.b[r][q] = fma(-sm.col[r], sm.b[c][q], sm.b[r][q]);
    }
    __syncthreads();
  }
  if (sm.fail) return false;
  return true;
}

// Status of a subset whose FP32 pass (factorisation below, or the check of
// its solution) left it to the FP64 solve.
constexpr int kModDeferred = 4;

// R = double: the FP64 solve with the ridge retry and the renormalisation; with
// only_deferred set it solves only the subsets the FP32 pass left to it.
// R = float: the FP32 pass of the checked mixed-precision solve: one attempt,
// the unnormalised solution left in the scratch for the check, breakdown
// recorded as kModDeferred (no ridge: the FP64 solve takes that subset).
template <typename T, int TS, typename R>
__global__ void __launch_bounds__(kTThreads, kMicro<R, TS> ? 2 : 3) mod_tiled_kernel(const double *__restrict__ A,
                                                                 const double *__restrict__ B,
                                                                 const int32_t *__restrict__ usage, int K, int m,
                                                                 int C, int light, int only_deferred, R *M, R *V,
                                                                 T *D, int32_t *status, int32_t *status_max) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  constexpr bool kF32 = sizeof(R) == 4;
  constexpr int P = kPitch<R, TS>;
  extern __shared__ __align__(16) unsigned char tiled_dyn[];
  TiledSmem<R, TS> &sm = *reinterpret_cast<TiledSmem<R, TS> *>(tiled_dyn);
  __shared__ double red[2][kTThreads / 32];
  const int rank = (int)cl.block_rank();
  const int t = blockIdx.x / C;
  // every block of the cluster reads the same word: all leave or none
  if (only_deferred && status[t] != kModDeferred) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TGeom g;
  g.K = K; g.m = m; g.TS = TS;
  g.R = (K + TS - 1) / TS;
  g.RT = g.R + (m + TS - 1) / TS;
  const int R_ = g.R, RT = g.RT, Rm = RT - R_;
  const double *At = A + (size_t)t * K * K;
  const double *Bt = B + (size_t)t * K * m;
  const int32_t *ut = usage + (size_t)t * K;
  R *Mt = M + (size_t)t * (K + m) * K;
  R *Vt = V + (size_t)t * R_ * TS * TS;

  double tr = 0.0, nu = 0.0;
  for (int j = tid; j < K; j += kTThreads)
    if (ut[j] > 0) { tr += At[(size_t)j * K + j]; nu += 1.0; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    nu += __shfl_xor_sync(0xffffffffu, nu, o);
  }
  if (lane == 0) { red[0][warp] = tr; red[1][warp] = nu; }
  __syncthreads();
  double T0 = 0.0, N0 = 0.0;
  for (int w = 0; w < kTThreads / 32; ++w) { T0 += red[0][w]; N0 += red[1][w]; }
  const double lambda = N0 > 0.0 ? kModRidge * T0 / N0 : 0.0;

  // Factor diagonal tile kk, keep its inverse for the backward sweep and push
  // inverse and verdict into every block of the cluster.
  double ridge = 0.0;
  auto own_diag = [&](int kk) {
    const bool ok = factor_diag<R, TS>(sm, Mt, g, kk, At, ut, ridge);
    const int par = kk & 1;
    for (int r2 = 0; r2 < C; ++r2) {
      R *dst = &cl.map_shared_rank(&sm.v[0][0][0], r2)[(size_t)par * TS * P];
      for (int e = tid; e < TS * TS; e += kTThreads) {
        const int r = e / TS, c = e % TS;
        if (kMicro<R, TS>) dst[c * P + r] = sm.b[r][c];   // the micro-tiled product reads V^T
        else dst[r * P + c] = sm.b[r][c];
      }
      if (tid == 0) cl.map_shared_rank(&sm.verdict[0], r2)[par] = ok ? 0 : 1;
    }
    for (int e = tid; e < TS * TS; e += kTThreads) Vt[(size_t)kk * TS * TS + e] = sm.b[e / TS][e % TS];
  };

  int st = 2;
  bool failed = true;
  // the FP32 pass makes one attempt: a breakdown goes to the FP64 solve
  for (int attempt = 0; attempt < (kF32 ? 1 : 2) && failed; ++attempt) {
    ridge = attempt == 0 ? 0.0 : lambda;
    // M <- [lower(A) + ridge on used diagonal entries; B^T]
    const int64_t total = (int64_t)(K + m) * K;
    for (int64_t q = (int64_t)rank * kTThreads + tid; q < total; q += (int64_t)C * kTThreads) {
      const int r = (int)(q / K), c = (int)(q % K);
      if (r < K) {
        if (c <= r) Mt[q] = (R)(At[(size_t)r * K + c] + ((r == c && ut[r] > 0) ? ridge : 0.0));
      } else {
        Mt[q] = (R)Bt[(size_t)c * m + (r - K)];
      }
    }
    cl.sync();
    // diagonal tile 0: factored by block 0, its inverse and verdict pushed to every block
    if (rank == 0) own_diag(0);
    cl.sync();
    failed = false;
    for (int k = 0; k < R_; ++k) {
      if (sm.verdict[k & 1]) { failed = true; break; }   // uniform: every block holds the pushed verdict
      const R (*vk)[P] = sm.v[k & 1];
      // panel: tile (i, k) <- tile (i, k) V_k^T for every tile row below k
      run_step<R, TS>(sm, vk, RT - k - 1, rank, C, [&](int q) {
        const Opnd<R> p = tile_of<R, TS>(Mt, g, k + 1 + q, k);
        return TileTask<R>{p, p, p, false, true, false, false};
      });
      cl.sync();
      // trailing: tile (i, j) -= panel_i panel_j^T, k < j <= i, j a column of A.
      // Task q enumerates (i, j) row by row (row i holds min(i, R - 1) - k
      // tasks), so task 0 is the next diagonal tile; its owner takes it first,
      // factors it at once and pushes the inverse while the other blocks go on
      // with their trailing tiles.
      const int ntr = (R_ - k - 1) * (R_ - k) / 2 + Rm * (R_ - k - 1);
      auto trail = [&](int q) {
        int i = k + 1, w = 1;
        while (q >= w) {
          q -= w;
          ++i;
          w = (i < R_ ? i : R_ - 1) - k;
        }
        const int j = k + 1 + q;
        return TileTask<R>{tile_of<R, TS>(Mt, g, i, k), tile_of<R, TS>(Mt, g, j, k), tile_of<R, TS>(Mt, g, i, j),
                           false, false, true, i == j};
      };
      if (ntr > 0) {
        const int owner = (k + 1) % C;
        if (light && C > 1) {
          // every block has an SM to itself: the owner's latency-bound diagonal
          // factorisation would lengthen the step, so it takes no other tile
          if (rank == owner) {
            run_step<R, TS>(sm, vk, 1, 0, C, trail);
            __syncthreads();   // the updated diagonal tile is in global memory
            own_diag(k + 1);
          } else {
            run_step<R, TS>(sm, vk, ntr, 1 + (rank - owner - 1 + C) % C, C - 1, trail);
          }
        } else if (rank == owner) {
          run_step<R, TS>(sm, vk, 1, 0, C, trail);
          __syncthreads();   // the updated diagonal tile is in global memory
          own_diag(k + 1);
          run_step<R, TS>(sm, vk, ntr, C, C, trail);
        } else {
          run_step<R, TS>(sm, vk, ntr, (rank - owner + C) % C, C, trail);
        }
      }
      cl.sync();
    }
    if (!failed) st = attempt;
    cl.sync();
  }

  if (!failed) {
    // backward sweep on the right-hand-side rows: X^T = W L^{-1}
    for (int k = R_ - 1; k >= 0; --k) {
      run_step<R, TS>(sm, sm.v[0], Rm, rank, C, [&](int q) {
        const Opnd<R> w = tile_of<R, TS>(Mt, g, R_ + q, k);
        return TileTask<R>{w, Opnd<R>{Vt + (size_t)k * TS * TS, TS, TS, TS}, w, true, false, false, false};
      });
      cl.sync();
      if (k > 0)
        run_step<R, TS>(sm, sm.v[0], Rm * k, rank, C, [&](int q) {
          const int rb = q / k, i = q % k;
          return TileTask<R>{tile_of<R, TS>(Mt, g, R_ + rb, k), tile_of<R, TS>(Mt, g, k, i),
                             tile_of<R, TS>(Mt, g, R_ + rb, i), true, false, true, false};
        });
      cl.sync();
    }
    // renormalise the used atoms (atom j = column j of the right-hand-side
    // rows); the FP32 pass leaves that to the check
    for (int j = rank * kTThreads + tid; j < K && !kF32; j += C * kTThreads) {
      if (ut[j] == 0) continue;   // unused: keeps the previous atom
      const R *xj = Mt + (size_t)K * K + j;
      double n2 = 0.0;
      for (int r = 0; r < m; ++r) {
        const double v = __ldcg(xj + (size_t)r * K);
        n2 = fma(v, v, n2);
      }
      const double nrm = sqrt(n2);
      if (!(nrm > 0.0) || !isfinite(nrm)) continue;
      const double inv = 1.0 / nrm;
      T *dj = D + ((size_t)t * K + j) * m;
      for (int r = 0; r < m; ++r) dj[r] = (T)(__ldcg(xj + (size_t)r * K) * inv);
    }
  }
  if (rank == 0 && tid == 0) {
    if (kF32) {
      status[t] = failed ? kModDeferred : 0;   // folded by the check or the FP64 solve
    } else {
      status[t] = st;
      if (status_max) atomicMax(status_max, st);
    }
  }
}

// ---- the wide form: one subset's tile tasks spread over G blocks anywhere on
// the GPU (a cooperative launch keeps them all resident), for few subsets, where
// a cluster of at most 16 SMs leaves the rest of the GPU idle while the
// single system's FP64 work runs on its 2 DFMA per clock per SM.  The steps and
// their tile tasks are the cluster form's; the blocks of a subset meet at a
// barrier in global memory instead of the cluster barrier, and the inverse of
// each diagonal factor and its breakdown verdict travel through global memory
// (every block loads the inverse into its shared memory after the barrier).

// Barrier words of one subset's group of blocks (zeroed before the launch).
struct WideSync {
  unsigned int count, gen;
  int verdict[2];
  int fail;
  int pad[3];
};

__device__ __forceinline__ unsigned int vload(const unsigned int *p) {
  return *reinterpret_cast<const volatile unsigned int *>(p);
}
__device__ __forceinline__ int vload(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Barrier of the nb blocks of a group: the arrivals count up, the last one
// resets the count and moves the generation on, the others wait (bounded) for
// the generation to change.  Global writes before it are visible to every
// block of the group after it.  False when some block of the group gave up.
__device__ bool wide_sync(WideSync *w, int nb, long long spin) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = vload(&w->gen);
    __threadfence();
    if (atomicAdd(&w->count, 1u) == (unsigned int)nb - 1) {
      atomicExch(&w->count, 0u);
      __threadfence();
      atomicAdd(&w->gen, 1u);
    } else {
      long long it = 0;
      while (vload(&w->gen) == g) {
        if (++it > spin || vload(&w->fail)) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (!ok) atomicExch(&w->fail, 1);
    ok_s = ok && !vload(&w->fail);
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T, int TS>
__global__ void __launch_bounds__(kTThreads, 2) mod_wide_kernel(const double *__restrict__ A,
                                                                const double *__restrict__ B,
                                                                const int32_t *__restrict__ usage, int K, int m,
                                                                int G, double *M, double *V, WideSync *sync, T *D,
                                                                int32_t *status, int32_t *status_max,
                                                                long long spin, int absent) {
  __shared__ TiledSmem<double, TS> sm;
  __shared__ double red[2][kTThreads / 32];
  const int rank = blockIdx.x % G;
  const int t = blockIdx.x / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TGeom g;
  g.K = K; g.m = m; g.TS = TS;
  g.R = (K + TS - 1) / TS;
  g.RT = g.R + (m + TS - 1) / TS;
  const int R = g.R, RT = g.RT, Rm = RT - R;
  const double *At = A + (size_t)t * K * K;
  const double *Bt = B + (size_t)t * K * m;
  const int32_t *ut = usage + (size_t)t * K;
  double *Mt = M + (size_t)t * (K + m) * K;
  double *Vt = V + (size_t)t * R * TS * TS;
  WideSync *ws = sync + t;
  // test of the bounded waits: the block of rank `absent` leaves at once, so
  // the others' first barrier wait runs out (status 3, SDL_ETIMEOUT)
  if (rank == absent) return;

  double tr = 0.0, nu = 0.0;
  for (int j = tid; j < K; j += kTThreads)
    if (ut[j] > 0) { tr += At[(size_t)j * K + j]; nu += 1.0; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    nu += __shfl_xor_sync(0xffffffffu, nu, o);
  }
  if (lane == 0) { red[0][warp] = tr; red[1][warp] = nu; }
  __syncthreads();
  double T0 = 0.0, N0 = 0.0;
  for (int w = 0; w < kTThreads / 32; ++w) { T0 += red[0][w]; N0 += red[1][w]; }
  const double lambda = N0 > 0.0 ? kModRidge * T0 / N0 : 0.0;

  // factor diagonal tile kk; its inverse and verdict go to global memory
  double ridge = 0.0;
  auto own_diag = [&](int kk) {
    const bool okd = factor_diag<double, TS>(sm, Mt, g, kk, At, ut, ridge);
    for (int e = tid; e < TS * TS; e += kTThreads) Vt[(size_t)kk * TS * TS + e] = sm.b[e / TS][e % TS];
    if (tid == 0) ws->verdict[kk & 1] = okd ? 0 : 1;
  };
  // every block's shared copy of the inverse of diagonal factor k
  auto load_inv = [&](int k) {
    for (int e = tid; e < TS * TS; e += kTThreads) sm.v[0][e / TS][e % TS] = __ldcg(Vt + (size_t)k * TS * TS + e);
    __syncthreads();
  };

  bool alive = true;   // false once a barrier gave up: every block then leaves
  int st = 2;
  bool failed = true;
  for (int attempt = 0; attempt < 2 && failed && alive; ++attempt) {
    ridge = attempt == 0 ? 0.0 : lambda;
    const int64_t total = (int64_t)(K + m) * K;
    for (int64_t q = (int64_t)rank * kTThreads + tid; q < total; q += (int64_t)G * kTThreads) {
      const int r = (int)(q / K), c = (int)(q % K);
      if (r < K) {
        if (c <= r) Mt[q] = At[(size_t)r * K + c] + ((r == c && ut[r] > 0) ? ridge : 0.0);
      } else {
        Mt[q] = Bt[(size_t)c * m + (r - K)];
      }
    }
    if (!(alive = wide_sync(ws, G, spin))) break;
    if (rank == 0) own_diag(0);
    if (!(alive = wide_sync(ws, G, spin))) break;
    failed = false;
    for (int k = 0; k < R; ++k) {
      if (vload(&ws->verdict[k & 1])) { failed = true; break; }   // the same value in every block
      load_inv(k);
      const double (*vk)[TS + 1] = sm.v[0];
      run_step<double, TS>(sm, vk, RT - k - 1, rank, G, [&](int q) {
        const Opnd<double> p = tile_of<double, TS>(Mt, g, k + 1 + q, k);
        return TileTask<double>{p, p, p, false, true, false, false};
      });
      if (!(alive = wide_sync(ws, G, spin))) break;
      const int ntr = (R - k - 1) * (R - k) / 2 + Rm * (R - k - 1);
      auto trail = [&](int q) {
        int i = k + 1, w = 1;
        while (q >= w) {
          q -= w;
          ++i;
          w = (i < R ? i : R - 1) - k;
        }
        const int j = k + 1 + q;
        return TileTask<double>{tile_of<double, TS>(Mt, g, i, k), tile_of<double, TS>(Mt, g, j, k), tile_of<double, TS>(Mt, g, i, j), false, false,
                        true, i == j};
      };
      if (ntr > 0) {
        // the owner of the next diagonal tile updates and factors it and, with
        // other blocks in the group, takes no other tile; they share the rest
        const int owner = (k + 1) % G;
        if (rank == owner) {
          run_step<double, TS>(sm, vk, 1, 0, G, trail);
          __syncthreads();   // the updated diagonal tile is in global memory
          own_diag(k + 1);
          if (G == 1) run_step<double, TS>(sm, vk, ntr, 1, 1, trail);
        } else {
          run_step<double, TS>(sm, vk, ntr, 1 + (rank - owner - 1 + G) % G, G - 1, trail);
        }
      }
      if (!(alive = wide_sync(ws, G, spin))) break;
    }
    if (!failed && alive) st = attempt;
    if (alive && !(alive = wide_sync(ws, G, spin))) break;
  }

  if (!failed && alive) {
    // backward sweep on the right-hand-side rows: X^T = W L^{-1}
    for (int k = R - 1; k >= 0 && alive; --k) {
      run_step<double, TS>(sm, sm.v[0], Rm, rank, G, [&](int q) {
        const Opnd<double> w = tile_of<double, TS>(Mt, g, R + q, k);
        return TileTask<double>{w, Opnd<double>{Vt + (size_t)k * TS * TS, TS, TS, TS}, w, true, false, false, false};
      });
      if (!(alive = wide_sync(ws, G, spin))) break;
      if (k > 0)
        run_step<double, TS>(sm, sm.v[0], Rm * k, rank, G, [&](int q) {
          const int rb = q / k, i = q % k;
          return TileTask<double>{tile_of<double, TS>(Mt, g, R + rb, k), tile_of<double, TS>(Mt, g, k, i), tile_of<double, TS>(Mt, g, R + rb, i),
                          true, false, true, false};
        });
      if (!(alive = wide_sync(ws, G, spin))) break;
    }
    if (alive) {
      for (int j = rank * kTThreads + tid; j < K; j += G * kTThreads) {
        if (ut[j] == 0) continue;   // unused: keeps the previous atom
        const double *xj = Mt + (size_t)K * K + j;
        double n2 = 0.0;
        for (int r = 0; r < m; ++r) {
          const double v = __ldcg(xj + (size_t)r * K);
          n2 = fma(v, v, n2);
        }
        const double nrm = sqrt(n2);
        if (!(nrm > 0.0) || !isfinite(nrm)) continue;
        const double inv = 1.0 / nrm;
        T *dj = D + ((size_t)t * K + j) * m;
        for (int r = 0; r < m; ++r) dj[r] = (T)(__ldcg(xj + (size_t)r * K) * inv);
      }
    }
  }
  if (rank == 0 && tid == 0) {
    // a barrier that gave up: status 3 (the atoms may be partly updated)
    const int code = alive ? st : 3;
    status[t] = code;
    if (status_max) atomicMax(status_max, code);
  }
}

}  // namespace

// Scratch per subset: M ((K + m) x K), room for the inverses of every tile
// edge, and the wide form's barrier words (4 doubles).
static size_t tiled_sub_doubles(int K, int m) {
  const int R = (K + 15) / 16;   // the smaller tile needs the most inverse blocks
  return (size_t)(K + m) * K + (size_t)R * 16 * 16 + (size_t)((K + 31) / 32) * 32 * 32 +
         (size_t)((K + 63) / 64) * 64 * 64 / 2;   // the FP32 pass's 64 x 64 inverses (floats)
}
size_t mod_tiled_scratch_doubles(int L, int K, int m) { return (size_t)L * (tiled_sub_doubles(K, m) + 4); }

// Dynamic shared memory of the tiled kernel: its tile buffers, grown where a
// cap of at most `cap` blocks per SM is asked for (0: no cap) to more than
// 1/(cap + 1) of the SM's 228 KB with the static part included.
template <typename R, int TS>
static size_t cap_smem(int cap) {
  const size_t need = sizeof(TiledSmem<R, TS>);
  if (cap <= 0) return need;
  const size_t stat = 2 * sizeof(double) * (kTThreads / 32) + 64;
  const size_t want = (size_t)228 * 1024 / (size_t)(cap + 1) + 1024;
  return want > stat + need ? want - stat : need;
}

template <typename T, int TS, typename R>
static cudaError_t launch_tiled_ts(const ModArgs &a, int C, int cap, int num_sms, int only_deferred,
                                   cudaStream_t st) {
  auto kern = mod_tiled_kernel<T, TS, R>;
  cudaError_t e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  const size_t dyn = cap_smem<R, TS>(cap);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((int64_t)a.L * C));
  cfg.blockDim = dim3(kTThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the FP32 pass lays its scratch out in floats over the same bytes
  R *M = reinterpret_cast<R *>(a.Lf);
  R *V = M + (size_t)a.L * (a.K + a.m) * a.K;
  const int light = (int64_t)a.L * C <= num_sms ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, (const double *)a.A, (const double *)a.B, (const int32_t *)a.usage, a.K,
                            a.m, C, light, only_deferred, M, V, static_cast<T *>(a.D), a.status, a.status_max);
}

template <typename T, typename R, int TS>
static int max_clusters_ts(int C, int cap) {
  auto kern = mod_tiled_kernel<T, TS, R>;
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t dyn = cap_smem<R, TS>(cap);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kTThreads);
  cfg.dynamicSmemBytes = dyn;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
int mod_tiled_max_clusters(int ts, int C, int cap, bool f32) {
  if (f32)
    return ts == 16 ? max_clusters_ts<T, float, 16>(C, cap)
         : ts == 32 ? max_clusters_ts<T, float, 32>(C, cap)
         : ts == 64 ? max_clusters_ts<T, float, 64>(C, cap) : 0;
  return ts == 16 ? max_clusters_ts<T, double, 16>(C, cap)
       : ts == 32 ? max_clusters_ts<T, double, 32>(C, cap) : 0;
}

template <typename T>
cudaError_t launch_mod_tiled(const ModArgs &a, int ts, int C, int cap, int num_sms, cudaStream_t st,
                             bool only_deferred) {
  if (a.L <= 0) return cudaSuccess;
  if (C < 1 || C > 16 || (ts != 16 && ts != 32) || cap < 0 || cap > 3) return cudaErrorInvalidValue;
  const int od = only_deferred ? 1 : 0;
  return ts == 16 ? launch_tiled_ts<T, 16, double>(a, C, cap, num_sms, od, st)
                  : launch_tiled_ts<T, 32, double>(a, C, cap, num_sms, od, st);
}

template <typename T>
cudaError_t launch_mod_tiled32(const ModArgs &a, int ts, int C, int cap, int num_sms, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  if (C < 1 || C > 16 || (ts != 16 && ts != 32 && ts != 64) || cap < 0 || cap > 3) return cudaErrorInvalidValue;
  return ts == 16 ? launch_tiled_ts<T, 16, float>(a, C, cap, num_sms, 0, st)
       : ts == 32 ? launch_tiled_ts<T, 32, float>(a, C, cap, num_sms, 0, st)
                  : launch_tiled_ts<T, 64, float>(a, C, cap, num_sms, 0, st);
}

template <typename T, int TS>
static cudaError_t launch_wide_ts(const ModArgs &a, int G, long long spin, int absent, cudaStream_t st) {
  auto kern = mod_wide_kernel<T, TS>;
  double *M = a.Lf;
  double *V = a.Lf + (size_t)a.L * (a.K + a.m) * a.K;
  WideSync *sync = reinterpret_cast<WideSync *>(a.Lf + (size_t)a.L * tiled_sub_doubles(a.K, a.m));
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(WideSync) * (size_t)a.L, st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((int64_t)a.L * G));
  cfg.blockDim = dim3(kTThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every block resident: the barriers need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, (const double *)a.A, (const double *)a.B, (const int32_t *)a.usage, a.K,
                            a.m, G, M, V, sync, static_cast<T *>(a.D), a.status, a.status_max, spin, absent);
}

template <typename T>
int mod_wide_max_blocks(int ts, int num_sms) {
  int per = 0;
  const cudaError_t e = ts == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mod_wide_kernel<T, 16>, kTThreads, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mod_wide_kernel<T, 32>, kTThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * num_sms;
}

template <typename T>
cudaError_t launch_mod_wide(const ModArgs &a, int ts, int G, long long spin, int absent, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  if (G < 1 || (ts != 16 && ts != 32) || spin < 1) return cudaErrorInvalidValue;
  return ts == 16 ? launch_wide_ts<T, 16>(a, G, spin, absent, st) : launch_wide_ts<T, 32>(a, G, spin, absent, st);
}

template cudaError_t launch_mod_wide<float>(const ModArgs &, int, int, long long, int, cudaStream_t);
template cudaError_t launch_mod_wide<double>(const ModArgs &, int, int, long long, int, cudaStream_t);
template int mod_wide_max_blocks<float>(int, int);
template int mod_wide_max_blocks<double>(int, int);
template cudaError_t launch_mod_tiled<float>(const ModArgs &, int, int, int, int, cudaStream_t, bool);
template cudaError_t launch_mod_tiled<double>(const ModArgs &, int, int, int, int, cudaStream_t, bool);
template cudaError_t launch_mod_tiled32<float>(const ModArgs &, int, int, int, int, cudaStream_t);
template int mod_tiled_max_clusters<float>(int, int, int, bool);
template int mod_tiled_max_clusters<double>(int, int, int, bool);

}  // namespace sdl
