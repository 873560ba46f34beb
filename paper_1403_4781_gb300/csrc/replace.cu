// Atom replacement, an alternative dictionary-update policy (the paper's MOD
// keeps unused atoms): after the MOD update, atom j of subset t with
// usage[t][j] < min_use, in increasing j, becomes y_i / ||y_i|| for the signal
// i of the subset with the largest squared residual of the coding pass that is
// not yet taken (lower i on ties; only resid2 > 0 qualifies, and such a signal
// is nonzero).  When no signal qualifies any more the remaining atoms keep
// their value.
//
// One block per subset.  The atoms to replace are listed in increasing order by
// a block scan; then one block-wide argmax over the subset's residuals per
// listed atom.  The signals taken so far are exactly those that rank at or
// before the previous pick in the order (resid2 descending, index ascending),
// so each argmax only admits signals ranking strictly after it: no mark array.
// The residuals of a subset stay in L2 across the rounds.  Usually no atom is
// listed and the block returns after the scan.
#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr int kRepThreads = 256;
constexpr int kRepWarps = kRepThreads / 32;

template <typename T>
__device__ __forceinline__ T rsqrt_exact(T v);
template <> __device__ __forceinline__ float rsqrt_exact<float>(float v) { return 1.0f / sqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_exact<double>(double v) { return 1.0 / sqrt(v); }

// (v, i) ranks before (bv, bi): larger residual, then lower index.
template <typename T>
__device__ __forceinline__ bool ranks_before(T v, int64_t i, T bv, int64_t bi) {
  return bi < 0 || v > bv || (v == bv && i < bi);
}

template <typename T>
__global__ void __launch_bounds__(kRepThreads) replace_atoms_kernel(const T *__restrict__ Y, int m,
                                                                    const int64_t *__restrict__ offsets,
                                                                    const int32_t *__restrict__ usage,
                                                                    const T *__restrict__ resid2, int min_use,
                                                                    T *__restrict__ D, int K, int32_t *rep) {
  __shared__ int16_t list[1024];   // K <= 1024
  __shared__ int wcount[kRepWarps];
  __shared__ T wv[kRepWarps];
  __shared__ long long wi[kRepWarps];
  __shared__ T pick_v;
  __shared__ long long pick_i;
  __shared__ T wsum[kRepWarps];
  const int t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t *ut = usage + (size_t)t * K;
  T *Dt = D + (size_t)t * K * m;
  if (rep)
    for (int j = tid; j < K; j += kRepThreads) rep[(size_t)t * K + j] = -1;

  // ---- atoms to replace, in increasing index: a contiguous chunk per thread
  const int per = (K + kRepThreads - 1) / kRepThreads;
  const int j0 = tid * per, j1 = min(j0 + per, K);
  int c = 0;
  for (int j = j0; j < j1; ++j) c += ut[j] < min_use;
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wcount[warp] = incl;
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kRepWarps; ++w) {
    base += w < warp ? wcount[w] : 0;
    total += wcount[w];
  }
  int pos = base + incl - c;
  for (int j = j0; j < j1; ++j)
    if (ut[j] < min_use) list[pos++] = (int16_t)j;
  __syncthreads();
  if (total == 0) return;   // block-uniform

  const int64_t a = offsets[t], b = offsets[t + 1];
  T pv = T(0);
  int64_t pi = -1;   // previous pick (none yet)
  for (int q = 0; q < total; ++q) {
    // ---- argmax of resid2 over the signals ranking after the previous pick
    T bv = T(0);
    int64_t bi = -1;
    for (int64_t i = a + tid; i < b; i += kRepThreads) {
      const T v = resid2[i];
      if (!(v > T(0))) continue;
      if (pi >= 0 && !(v < pv || (v == pv && i > pi))) continue;
      if (ranks_before(v, i, bv, bi)) { bv = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
      if (oi >= 0 && ranks_before(ov, (int64_t)oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      T v = T(0);
      int64_t i = -1;
      for (int w = 0; w < kRepWarps; ++w)
        if (wi[w] >= 0 && ranks_before(wv[w], (int64_t)wi[w], v, i)) { v = wv[w]; i = wi[w]; }
      pick_v = v;
      pick_i = i;
    }
    __syncthreads();
    pv = pick_v;
    pi = pick_i;
    if (pi < 0) break;   // block-uniform: no signal left
    // ---- atom list[q] = y_pi / ||y_pi||
    const T *y = Y + (size_t)pi * m;
    T acc = T(0);
    for (int r = tid; r < m; r += kRepThreads) acc = fma(y[r], y[r], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    T nrm2 = T(0);
#pragma unroll
    for (int w = 0; w < kRepWarps; ++w) nrm2 += wsum[w];
    const T inv = rsqrt_exact<T>(nrm2);
    const int j = list[q];
    for (int r = tid; r < m; r += kRepThreads) Dt[(size_t)j * m + r] = y[r] * inv;
    if (tid == 0 && rep) rep[(size_t)t * K + j] = (int32_t)pi;
    __syncthreads();   // wv / wi / wsum / pick are rewritten by the next round
  }
}

}  // namespace

template <typename T>
cudaError_t launch_replace_atoms(const T *Y, int m, const int64_t *offsets, int L, const int32_t *usage,
                                 const T *resid2, int min_use, T *D, int K, int32_t *rep, cudaStream_t st) {
  if (L <= 0 || min_use <= 0) return cudaSuccess;
  if (K > 1024) return cudaErrorInvalidValue;
  replace_atoms_kernel<T><<<L, kRepThreads, 0, st>>>(Y, m, offsets, usage, resid2, min_use, D, K, rep);
  return cudaGetLastError();
}

template cudaError_t launch_replace_atoms<float>(const float *, int, const int64_t *, int, const int32_t *,
                                                 const float *, int, float *, int, int32_t *, cudaStream_t);
template cudaError_t launch_replace_atoms<double>(const double *, int, const int64_t *, int, const int32_t *,
                                                  const double *, int, double *, int, int32_t *, cudaStream_t);

}  // namespace sdl
