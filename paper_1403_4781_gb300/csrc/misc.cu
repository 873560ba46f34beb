// Algorithm 1 plumbing (split gather, scaled stack, initial atoms) and the
// metrics of Sec. 3.1 / Table 1 (residual energy, atom recovery).
#include <math.h>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Algorithm 1 step 1: Yp[i] = Y[perm[i]], one warp per signal.
template <typename T>
__global__ void split_kernel(const T *__restrict__ Y, int m, int64_t N, const int64_t *__restrict__ perm,
                             T *__restrict__ Yp) {
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const int64_t src = perm[i];
  if (src < 0 || src >= N) return;   // rejected on the host; never reached for a permutation
  for (int r = lane; r < m; r += 32) Yp[(size_t)i * m + r] = Y[(size_t)src * m + r];
}

// Unit-normalised copy of a signal (or of a fill column where pick < 0).
template <typename T>
__global__ void init_dict_kernel(const T *__restrict__ Y, int m, const int64_t *__restrict__ pick,
                                 const T *__restrict__ fill, int64_t count, T *__restrict__ D) {
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= count) return;
  const int64_t p = pick[c];
  const T *src = p >= 0 ? Y + (size_t)p * m : fill + (size_t)c * m;
  double acc = 0.0;
  for (int r = lane; r < m; r += 32) acc = fma((double)src[r], (double)src[r], acc);
  acc = warp_sum(acc);
  const double nrm = sqrt(acc);
  for (int r = lane; r < m; r += 32)
    D[(size_t)c * m + r] = nrm > 0.0 ? (T)((double)src[r] / nrm) : T(0);
}

// Algorithm 1 step 3: Ytilde[t*K1 + j] = xfro[t] * D^(t)[j].
template <typename T>
__global__ void stack_kernel(const T *__restrict__ Dloc, const double *__restrict__ xfro, int m, int K1,
                             int L, T *__restrict__ Yt) {
  const int64_t total = (int64_t)L * K1 * m;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / ((int64_t)K1 * m);
    Yt[q] = (T)((double)Dloc[q] * xfro[t]);
  }
}

// Merge initial atoms: unit-normalised stacked columns Ytilde[pick[j]].
template <typename T>
__global__ void pick_init_kernel(const T *__restrict__ Yt, int m, const int32_t *__restrict__ pick, int K,
                                 T *__restrict__ D) {
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= K) return;
  const T *src = Yt + (size_t)pick[j] * m;
  double acc = 0.0;
  for (int r = lane; r < m; r += 32) acc = fma((double)src[r], (double)src[r], acc);
  acc = warp_sum(acc);
  const double nrm = sqrt(acc);
  for (int r = lane; r < m; r += 32)
    D[(size_t)j * m + r] = nrm > 0.0 ? (T)((double)src[r] / nrm) : T(0);
}

// Compensated FP32 sum (a hi + lo pair): each term, or each exact product
// x y = p + e (one FMA gives e), is added with TwoSum and the rounding error
// carried in lo, so about 48 significant bits survive.  Accumulating FP32
// values this way runs on the FP32 pipe; FP64 additions of every term would
// load one SM's narrow FP64 pipe when a single subset has many codes.
struct CSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float p, float e) {
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    const float l = lo + (e + err);
    hi = s + l;
    lo = l - (hi - s);
  }
  __device__ __forceinline__ void add(float x) { add(x, 0.f); }
  __device__ __forceinline__ void add_sq(float x) {
    const float p = x * x;
    add(p, fmaf(x, x, -p));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Per-subset sums: rmse[t] = sqrt(sum resid2 / (m n_t)), xfro[t] = ||val||_F.
// One block per subset.  FP32 codes: per-thread compensated FP32 sums, added
// in FP64 across threads; FP64 codes: FP64 sums.
template <typename T>
__global__ void __launch_bounds__(1024) subset_stats_kernel(const T *__restrict__ resid2,
                                                           const T *__restrict__ val,
                                                           const int64_t *__restrict__ offsets, int m,
                                                           int s, double *rmse_out, int64_t rmse_stride,
                                                           double *xfro_out) {
  __shared__ double red[2][32];
  const int t = blockIdx.x;
  const int64_t a = offsets[t], b = offsets[t + 1];
  double r2 = 0.0, v2 = 0.0;
  if constexpr (sizeof(T) == 4) {
    CSum cr, cv;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) cr.add((float)resid2[i]);
    if (xfro_out)
      for (int64_t e = a * s + threadIdx.x; e < b * s; e += blockDim.x) cv.add_sq((float)val[e]);
    r2 = cr.value();
    v2 = cv.value();
  } else {
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) r2 += (double)resid2[i];
    if (xfro_out)
      for (int64_t e = a * s + threadIdx.x; e < b * s; e += blockDim.x) {
        const double v = (double)val[e];
        v2 = fma(v, v, v2);
      }
  }
  r2 = warp_sum(r2);
  v2 = warp_sum(v2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = r2; red[1][w] = v2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R = 0.0, V = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { R += red[0][q]; V += red[1][q]; }
    const double n = (double)(b - a);
    if (rmse_out) rmse_out[(size_t)t * rmse_stride] = n > 0 ? sqrt(R / ((double)m * n)) : 0.0;
    if (xfro_out) xfro_out[t] = sqrt(V);
  }
}

// ||Y - D X||_F^2 and ||Y||_F^2: one warp per signal, block partials, FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const T *__restrict__ Y, int m, int64_t n,
                                                       const T *__restrict__ D,
                                                       const int32_t *__restrict__ idx,
                                                       const T *__restrict__ val, int s, double *out2) {
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double r2 = 0.0, y2 = 0.0;
  if constexpr (sizeof(T) == 4) {
    // FP32 data: the residual entry y - sum_k d x_k and the two energies in
    // compensated FP32 (each product split exactly by an FMA), about 48
    // significant bits, on the FP32 pipe rather than the narrow FP64 one
    // The signal's code sits in the lanes (lane k: entry k, s <= 32) and
    // reaches the warp by shuffles; lane l holds entries l + 32 u (m <= 256) of
    // the residual, so every atom's column loads once, coalesced.
    CSum cr, cy;
    constexpr int MU = 8;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
      int jl = -1;
      float xl = 0.f;
      if (lane < s) {
        jl = idx[(size_t)i * s + lane];
        xl = (float)val[(size_t)i * s + lane];
      }
      CSum v[MU];
      float yv[MU];
#pragma unroll
      for (int u = 0; u < MU; ++u) {
        const int r = lane + 32 * u;
        yv[u] = r < m ? (float)Y[(size_t)i * m + r] : 0.f;
        v[u].hi = yv[u];
      }
      for (int k = 0; k < s; ++k) {
        const int j = __shfl_sync(0xffffffffu, jl, k);
        const float x = __shfl_sync(0xffffffffu, xl, k);
        if (j < 0) continue;   // warp-uniform
        const T *dj = D + (size_t)j * m;
#pragma unroll
        for (int u = 0; u < MU; ++u) {
          const int r = lane + 32 * u;
          if (r < m) {
            const float d = (float)dj[r];
            const float p = d * x;
            v[u].add(-p, -fmaf(d, x, -p));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < MU; ++u) {
        if (lane + 32 * u >= m) continue;
        const float h = v[u].hi, l = v[u].lo, p2 = h * h;
        cr.add(p2, fmaf(h, h, -p2) + 2.f * h * l);
        cy.add_sq(yv[u]);
      }
    }
    r2 = cr.value();
    y2 = cy.value();
  } else {
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
      for (int r = lane; r < m; r += 32) {
        const double y = (double)Y[(size_t)i * m + r];
        double v = y;
        for (int k = 0; k < s; ++k) {
          const int j = idx[(size_t)i * s + k];
          if (j >= 0) v = fma(-(double)D[(size_t)j * m + r], (double)val[(size_t)i * s + k], v);
        }
        r2 = fma(v, v, r2);
        y2 = fma(y, y, y2);
      }
    }
  }
  r2 = warp_sum(r2);
  y2 = warp_sum(y2);
  if (lane == 0) { red[0][w] = r2; red[1][w] = y2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R = 0.0, Q = 0.0;
    for (int q = 0; q < 8; ++q) { R += red[0][q]; Q += red[1][q]; }
    atomicAdd(out2, R);
    atomicAdd(out2 + 1, Q);
  }
}

// Sec. 3.1 recovery: warp per atom of D0, max_j |<d0_i, d_j>| >= thresh.
template <typename T>
__global__ void recovery_kernel(const T *__restrict__ D0, int K0, const T *__restrict__ D, int K, int m,
                                double thresh, int32_t *count) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= K0) return;
  double best = 0.0;
  for (int j = 0; j < K; ++j) {
    double acc = 0.0;
    for (int r = lane; r < m; r += 32) acc = fma((double)D0[(size_t)i * m + r], (double)D[(size_t)j * m + r], acc);
    acc = warp_sum(acc);
    best = fmax(best, fabs(acc));
  }
  if (lane == 0 && best >= thresh) atomicAdd(count, 1);
}

__global__ void status_max_kernel(const int32_t *__restrict__ status, int L, int32_t *out) {
  int v = 0;
  for (int t = threadIdx.x; t < L; t += blockDim.x) v = max(v, status[t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = max(r, red[q]);
    *out = r;
  }
}

unsigned blocks_for(int64_t items, int per_block) {
  const int64_t b = (items + per_block - 1) / per_block;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t launch_split(const T *Y, int m, int64_t N, const int64_t *perm, T *Yp, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  split_kernel<T><<<blocks_for(N, 8), 256, 0, st>>>(Y, m, N, perm, Yp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_dict(const T *Y, int m, const int64_t *pick, const T *fill, int64_t count, T *D,
                             cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  init_dict_kernel<T><<<blocks_for(count, 8), 256, 0, st>>>(Y, m, pick, fill, count, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stack(const T *Dloc, const double *xfro, int m, int K1, int L, T *Yt, cudaStream_t st) {
  const int64_t total = (int64_t)L * K1 * m;
  unsigned blocks = blocks_for(total, 256);
  if (blocks > 4096) blocks = 4096;
  stack_kernel<T><<<blocks, 256, 0, st>>>(Dloc, xfro, m, K1, L, Yt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pick_init(const T *Yt, int m, const int32_t *pick, int K, T *D, cudaStream_t st) {
  pick_init_kernel<T><<<blocks_for(K, 8), 256, 0, st>>>(Yt, m, pick, K, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_subset_stats(const T *resid2, const T *val, const int64_t *offsets, int L, int m, int s,
                                double *rmse_out, int64_t rmse_stride, double *xfro_out, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  // one block per subset: wide blocks where few subsets (the merge's one) must
  // each sum many codes, narrow ones where many subsets fill the GPU
  const int threads = L < 16 ? 1024 : 256;
  subset_stats_kernel<T><<<L, threads, 0, st>>>(resid2, val, offsets, m, s, rmse_out, rmse_stride, xfro_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const T *Y, int m, int64_t n, const T *D, const int32_t *idx, const T *val,
                            int s, double *out2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess || n <= 0) return e;
  unsigned blocks = blocks_for(n, 8);
  if (blocks > 1216) blocks = 1216;
  residual_kernel<T><<<blocks, 256, 0, st>>>(Y, m, n, D, idx, val, s, out2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recovery(const T *D0, int K0, const T *D, int K, int m, double thresh, int32_t *count,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  recovery_kernel<T><<<blocks_for(K0, 8), 256, 0, st>>>(D0, K0, D, K, m, thresh, count);
  return cudaGetLastError();
}

cudaError_t launch_status_max(const int32_t *status, int L, int32_t *out, cudaStream_t st) {
  status_max_kernel<<<1, 256, 0, st>>>(status, L, out);
  return cudaGetLastError();
}

#define SDL_INST(T)                                                                                     \
  template cudaError_t launch_split<T>(const T *, int, int64_t, const int64_t *, T *, cudaStream_t);      \
  template cudaError_t launch_init_dict<T>(const T *, int, const int64_t *, const T *, int64_t, T *,     \
                                           cudaStream_t);                                                \
  template cudaError_t launch_stack<T>(const T *, const double *, int, int, int, T *, cudaStream_t);      \
  template cudaError_t launch_pick_init<T>(const T *, int, const int32_t *, int, T *, cudaStream_t);      \
  template cudaError_t launch_subset_stats<T>(const T *, const T *, const int64_t *, int, int, int,      \
                                              double *, int64_t, double *, cudaStream_t);                \
  template cudaError_t launch_residual<T>(const T *, int, int64_t, const T *, const int32_t *, const T *, \
                                          int, double *, cudaStream_t);                                  \
  template cudaError_t launch_recovery<T>(const T *, int, const T *, int, int, double, int32_t *,        \
                                          cudaStream_t);
SDL_INST(float)
SDL_INST(double)
#undef SDL_INST

}  // namespace sdl
