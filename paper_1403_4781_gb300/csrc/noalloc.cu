// Allocation-free variant of the FP32 OMP entry point.
//
// Some callers cannot call cudaMalloc at the point where they need a sparse
// code: processes whose device memory is entirely owned by another allocator
// (a framework's caching pool sized to the whole GPU), or latency-critical loops
// that must not take cudaMalloc's implicit device synchronisation.  For them,
// sdl_omp_noalloc runs the same Gram and Batch-OMP kernels as sdl_omp, but its
// scratch (the K x K Gram matrix and the one-subset tile plan) lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.  Nothing is allocated by the call: no cudaMalloc, no
// cudaFree, no context workspace.
#include <mutex>

#include "sdl_internal.cuh"

namespace sdl {
constexpr int kNoAllocMaxK = 512;                 // Gram of at most 512 x 512 floats
constexpr size_t kPlanBytes = 256;                // offsets[2] (int64) + tile_start[2] (int32)
constexpr size_t kGramBytes = sizeof(float) * kNoAllocMaxK * kNoAllocMaxK;
constexpr size_t kScratchBytes = kPlanBytes + kGramBytes;   // 1 MiB + 256 B
}  // namespace sdl

// The shared scratch of every sdl_omp_noalloc call on a device.  In host code
// this name is only a stand-in: device code may name it directly, host code
// must use the address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sdl::kScratchBytes];

namespace sdl {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (the current device),
// looked up once per device.
cudaError_t scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

// Writes the one-subset tile plan into the scratch header.
__global__ void noalloc_plan_kernel(unsigned char *scratch, int64_t n, int32_t tiles) {
  int64_t *offsets = reinterpret_cast<int64_t *>(scratch);
  int32_t *tile_start = reinterpret_cast<int32_t *>(scratch + 2 * sizeof(int64_t));
  offsets[0] = 0;
  offsets[1] = n;
  tile_start[0] = 0;
  tile_start[1] = tiles;
}

bool aligned16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace sdl

extern "C" sdl_status sdl_omp_noalloc(void *stream, const float *D, int m, int K, const float *Y,
                                      int64_t n, int s, double eps, int32_t *idx, float *val,
                                      int32_t *nnz, float *resid2) {
  using namespace sdl;
  if (K > kNoAllocMaxK || m > kMaxM) return SDL_ERANGE;
  if (m < 1 || K < 1 || n < 0 || s < 1 || s > kMaxS || s > m || s > K || !(eps >= 0.0) || eps > 1e300)
    return SDL_EINVAL;
  if (n == 0) return SDL_OK;
  const int tile = omp_tile_signals();
  const int64_t tiles = (n + tile - 1) / tile;
  if (tiles >= ((int64_t)1 << 31)) return SDL_ERANGE;
  if (!aligned16(D) || !aligned16(Y) || !aligned16(idx) || !aligned16(val) || !aligned16(nnz) ||
      (resid2 && !aligned16(resid2)))
    return SDL_EINVAL;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return SDL_ECUDA;
  }
  void *base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return SDL_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *scratch = static_cast<unsigned char *>(base);
  noalloc_plan_kernel<<<1, 1, 0, st>>>(scratch, n, (int32_t)tiles);
  float *G = reinterpret_cast<float *>(scratch + kPlanBytes);
  if (cudaGetLastError() != cudaSuccess || launch_gram<float>(D, m, K, 1, G, st) != cudaSuccess)
    return SDL_ECUDA;
  OmpArgs a{};
  a.D = D; a.G = G; a.Y = Y;
  a.offsets = reinterpret_cast<const int64_t *>(scratch);
  a.tile_start = reinterpret_cast<const int32_t *>(scratch + 2 * sizeof(int64_t));
  a.total_tiles = tiles;
  a.L = 1; a.m = m; a.K = K; a.s = s; a.eps = eps;
  a.idx = idx; a.val = val; a.nnz = nnz; a.resid2 = resid2;
  // Every shape within the limits fits the fused kernel's shared memory: at
  // K = 512, m = 256, s = 32 its tile needs about 138 KB of the 227 KB a block
  // may use.  So any launch error here is a CUDA failure, not a size limit.
  const cudaError_t e = launch_omp<float>(a, 0, st);
  return e == cudaSuccess ? SDL_OK : SDL_ECUDA;
}
