// Image denoising with a learned dictionary (Sec. 3.2.2): every overlapping
// p x p patch of the noisy image is coded by the error-constrained OMP (the
// OMP kernels), its estimate is D x, and the denoised image holds at every pixel
// the mean of the estimates of the patches covering it.  These kernels cut the
// patches out of the image and put the estimates back together.
#include "sdl_internal.cuh"

namespace sdl {
namespace {

// out[i][u p + v] = img[(r + u) W + c + v] for patch i = r (W - p + 1) + c: one
// thread per output entry, so consecutive threads write consecutive entries.
template <typename T>
__global__ void __launch_bounds__(256) extract_patches_kernel(const T *__restrict__ img, int W, int p, int nc,
                                                              int64_t total, T *__restrict__ out) {
  const int m = p * p;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / m;
    const int e = (int)(q - i * m);
    const int r = (int)(i / nc), c = (int)(i - (int64_t)r * nc);
    const int u = e / p, v = e - u * p;
    out[q] = img[(size_t)(r + u) * W + (c + v)];
  }
}

// One thread per pixel (y, x): the mean over the covering patches (r, c),
// r in [max(0, y-p+1), min(y, H-p)], of sum_k val[i][k] D[idx[i][k]][(y-r) p + (x-c)].
// Codes end at the first -1 (ELL padding).
template <typename T>
__global__ void __launch_bounds__(256) patch_average_kernel(const T *__restrict__ D, int K,
                                                            const int32_t *__restrict__ idx,
                                                            const T *__restrict__ val, int s, int H, int W, int p,
                                                            T *__restrict__ out) {
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (int64_t)H * W) return;
  const int y = (int)(pix / W), x = (int)(pix - (int64_t)y * W);
  const int nr = H - p + 1, nc = W - p + 1, m = p * p;
  const int r0 = y - p + 1 > 0 ? y - p + 1 : 0, r1 = y < nr - 1 ? y : nr - 1;
  const int c0 = x - p + 1 > 0 ? x - p + 1 : 0, c1 = x < nc - 1 ? x : nc - 1;
  T acc = T(0);
  for (int r = r0; r <= r1; ++r)
    for (int c = c0; c <= c1; ++c) {
      const size_t i = (size_t)r * nc + c;
      const int e = (y - r) * p + (x - c);
      for (int k = 0; k < s; ++k) {
        const int j = idx[i * s + k];
        if (j < 0 || j >= K) break;
        acc = fma(val[i * s + k], D[(size_t)j * m + e], acc);
      }
    }
  out[pix] = acc / (T)((r1 - r0 + 1) * (c1 - c0 + 1));
}

// out2[0] += sum (a - b)^2, out2[1] += sum b^2: block partials, FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(256) sq_error_kernel(const T *__restrict__ a, const T *__restrict__ b, int64_t n,
                                                       double *out2) {
  __shared__ double red[2][8];
  double d2 = 0.0, b2 = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)a[q] - (double)b[q];
    d2 = fma(d, d, d2);
    b2 = fma((double)b[q], (double)b[q], b2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = d2; red[1][w] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double D2 = 0.0, B2 = 0.0;
    for (int q = 0; q < 8; ++q) { D2 += red[0][q]; B2 += red[1][q]; }
    atomicAdd(&out2[0], D2);
    atomicAdd(&out2[1], B2);
  }
}

unsigned grid_for(int64_t items) {
  int64_t b = (items + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

template <typename T>
cudaError_t launch_extract_patches(const T *img, int H, int W, int p, T *out, cudaStream_t st) {
  const int nc = W - p + 1;
  const int64_t total = (int64_t)(H - p + 1) * nc * p * p;
  if (total <= 0) return cudaSuccess;
  extract_patches_kernel<T><<<grid_for(total), 256, 0, st>>>(img, W, p, nc, total, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_patch_average(const T *D, int K, const int32_t *idx, const T *val, int s, int H, int W, int p,
                                 T *out, cudaStream_t st) {
  const int64_t n = (int64_t)H * W;
  if (n <= 0) return cudaSuccess;
  patch_average_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D, K, idx, val, s, H, W, p, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sq_error(const T *a, const T *b, int64_t n, double *out2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess || n <= 0) return e;
  sq_error_kernel<T><<<grid_for(n), 256, 0, st>>>(a, b, n, out2);
  return cudaGetLastError();
}

#define SDL_DENOISE_INST(T)                                                                                   \
  template cudaError_t launch_extract_patches<T>(const T *, int, int, int, T *, cudaStream_t);                 \
  template cudaError_t launch_patch_average<T>(const T *, int, const int32_t *, const T *, int, int, int, int, \
                                               T *, cudaStream_t);                                            \
  template cudaError_t launch_sq_error<T>(const T *, const T *, int64_t, double *, cudaStream_t);
SDL_DENOISE_INST(float)
SDL_DENOISE_INST(double)
#undef SDL_DENOISE_INST

}  // namespace sdl
