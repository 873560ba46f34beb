// Check of the FP32 pass of the MOD solve (Sec. 1: D = Y X^T (X X^T)^-1) for
// FP32 data, and the renormalisation of Sec. 3.1 of the subsets it accepts.
//
// The FP32 pass (mod_tiled_kernel with R = float) factors A = X X^T and
// solves D A = B in FP32.  Its error E = D_32 - D is not known, but E A =
// D_32 A - B is: for a probe u (m entries of +-1), u^T E = (u^T D_32 A - u^T B)
// A^-1, whose FP64 residual costs two K x K and two m x K matrix-vector
// products against the FP64 A and B, and whose A^-1 comes from the FP32
// factor.  Entry j of u^T E is u . e_j, e_j the
// error of atom j, and E[(u . e_j)^2] = |e_j|^2 over random signs (the
// Hutchinson identity), so P = 8 probes give every atom's squared error up
// to a chi-square factor with 8 degrees of freedom (about 2 % of atoms whose
// error is twice the tolerance pass, 1.5e-4 at four times).  A subset is
// accepted when every used atom's estimated error is at most tau of its norm
// (default 2e-5, the FP32 atom tolerance: an atom's largest entry error is at
// most its error norm, and the FP32 solve spreads its error over the m
// entries, so the entries stay well inside the tolerance); then its used atoms
// are renormalised and written.  Otherwise (and where the factorisation broke
// down, or an atom's norm is zero or not finite) the subset is marked for the
// FP64 solve, which then decides exactly as it would have alone.  The residual
// is formed in FP64; the two triangular solves that map it through the factor
// run in FP32 (an estimate is all that is needed).
//
// One block per subset, 256 threads; thread j mod 256 owns atoms j.
#include <math.h>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr int kCThreads = 256;
constexpr int kProbes = 8;
constexpr int kCJMax = 4;            // atoms per thread at most (K <= 1024)
constexpr int kModDeferredC = 4;     // the status the FP32 pass and this check leave for the FP64 solve

// +-1 of probe p at signal entry r of subset t: a 32-bit integer mix of the
// three counters (xorshift-multiply rounds), its lowest bit as the sign.
__device__ __forceinline__ float probe_sign(int t, int p, int r) {
  uint32_t x = (uint32_t)r * 0x9E3779B1u ^ (uint32_t)(p + 1) * 0x85EBCA77u ^ (uint32_t)(t + 1) * 0xC2B2AE3Du;
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return (x & 1u) ? -1.f : 1.f;
}

// Double-float arithmetic on the FP32 pipes (this part's FP64 pipe, conversions
// included, runs at 1/64 of its FP32 rate): a value is a compensated sum s + c,
// each addition an error-free TwoSum (Knuth) whose rounding error goes into c,
// each product of two hi + lo pairs exact in its hi * hi part (the FMA
// residual, Dekker/Kahan) with the cross terms added to c.  Explicit _rn
// operations keep the compiler from contracting the sums into FMAs.
struct DF {
  float s, c;
};
__device__ __forceinline__ void df_add(DF &a, float t) {
  const float s = __fadd_rn(a.s, t);
  const float bb = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(t, bb));
  a.s = s;
  a.c = __fadd_rn(a.c, err);
}
__device__ __forceinline__ void df_add_prod(DF &a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  df_add(a, p);
  a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ DF df_merge(DF a, DF b) {
  df_add(a, b.s);
  a.c = __fadd_rn(a.c, b.c);
  return a;
}
// A double as hi + lo floats by integer operations on its bits: hi its sign,
// exponent and top 23 fraction bits, lo the other 29 fraction bits (rounded to
// 24).  Values outside the float range count as zero (|a| < 2^-126; the
// normal equations' entries are far above it).
__device__ __forceinline__ void split_d(double a, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;
  if (fe <= 0 || fe >= 255) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
  const int le = e - 1075 + 127;   // 2^(e - 1075), the weight of the lowest fraction bit
  const float l = le > 0 ? __fmul_rn(__uint2float_rn((unsigned)(b & 0x1FFFFFFFull)), __uint_as_float((unsigned)le << 23))
                         : 0.f;
  lo = sign ? -l : l;
}

// CJ: atoms per thread (K <= 256 CJ).
template <typename T, int CJ>
__global__ void __launch_bounds__(kCThreads) mod_check_kernel(const double *__restrict__ A,
                                                              const double *__restrict__ B,
                                                              const int32_t *__restrict__ usage, int K, int m, int TS,
                                                              const float *__restrict__ M, const float *__restrict__ V,
                                                              T *D, int32_t *status, float tau) {
  extern __shared__ double sh[];
  __shared__ float Us[kProbes][256];
  __shared__ float Ys[kProbes][64];
  const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (status[t] == kModDeferredC) return;   // the FP32 factorisation broke down
  const int R = (K + TS - 1) / TS;
  const double *At = A + (size_t)t * K * K;
  const double *Bt = B + (size_t)t * K * m;
  const int32_t *ut = usage + (size_t)t * K;
  const float *Lt = M + (size_t)t * (K + m) * K;   // lower triangle: the FP32 factor
  const float *X = Lt + (size_t)K * K;              // row r: coordinate r of every atom
  const float *Vt = V + (size_t)t * R * TS * TS;    // inverses of the diagonal factor tiles
  float *Gh = reinterpret_cast<float *>(sh);   // [P][K]: u_p^T D_32 as hi + lo
  float *Gl = Gh + kProbes * K;
  float *Hs = Gl + kProbes * K;                // [P][K]: the row part of G A, compensated sum
  float *Hc = Hs + kProbes * K;
  float *Zs = Hc + kProbes * K;                // [P][K]: the residual, then A^-1 applied to it

  for (int e = tid; e < kProbes * m; e += kCThreads) Us[e / m][e % m] = probe_sign(t, e / m, e % m);
  __syncthreads();

  // G = U^T D_32 (hi + lo pairs) and the atoms' squared norms
  float n2[CJ];
#pragma unroll
  for (int q = 0; q < CJ; ++q) {
    const int j = tid + kCThreads * q;
    n2[q] = 0.f;
    if (j >= K) continue;
    DF g[kProbes];
#pragma unroll
    for (int p = 0; p < kProbes; ++p) g[p] = DF{0.f, 0.f};
    for (int r = 0; r < m; ++r) {
      const float x = X[(size_t)r * K + j];
      n2[q] = fmaf(x, x, n2[q]);
#pragma unroll
      for (int p = 0; p < kProbes; ++p) df_add(g[p], Us[p][r] < 0.f ? -x : x);
    }
#pragma unroll
    for (int p = 0; p < kProbes; ++p) {
      const float hi = __fadd_rn(g[p].s, g[p].c);
      Gh[p * K + j] = hi;
      Gl[p * K + j] = __fsub_rn(g[p].c, __fsub_rn(hi, g[p].s));
    }
  }
  __syncthreads();

  // H = G A from the lower triangle of A: the part below the diagonal of
  // column j by columns (row i's entries left of the diagonal, coalesced), the
  // part on and right of it by rows (warp-per-row sums into Hs, Hc)
  DF h[CJ][kProbes];
#pragma unroll
  for (int q = 0; q < CJ; ++q)
#pragma unroll
    for (int p = 0; p < kProbes; ++p) h[q][p] = DF{0.f, 0.f};
  for (int i0 = 1; i0 < K; i0 += 8) {
    double a[8][CJ];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int q = 0; q < CJ; ++q) {
        const int i = i0 + u, j = tid + kCThreads * q;
        a[u][q] = (i < K && j < i) ? __ldg(At + (size_t)i * K + j) : 0.0;
      }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u < K ? i0 + u : K - 1;
#pragma unroll
      for (int q = 0; q < CJ; ++q) {
        float ah, al;
        split_d(a[u][q], ah, al);
#pragma unroll
        for (int p = 0; p < kProbes; ++p) df_add_prod(h[q][p], ah, al, Gh[p * K + i], Gl[p * K + i]);
      }
    }
  }
  for (int i = warp; i < K; i += kCThreads / 32) {
    const double *ai = At + (size_t)i * K;
    DF d[kProbes];
#pragma unroll
    for (int p = 0; p < kProbes; ++p) d[p] = DF{0.f, 0.f};
    for (int c = lane; c <= i; c += 32) {
      float ah, al;
      split_d(__ldg(ai + c), ah, al);
#pragma unroll
      for (int p = 0; p < kProbes; ++p) df_add_prod(d[p], ah, al, Gh[p * K + c], Gl[p * K + c]);
    }
#pragma unroll
    for (int p = 0; p < kProbes; ++p)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const DF other{__shfl_xor_sync(0xffffffffu, d[p].s, o), __shfl_xor_sync(0xffffffffu, d[p].c, o)};
        d[p] = df_merge(d[p], other);
      }
    if (lane == 0)
#pragma unroll
      for (int p = 0; p < kProbes; ++p) {
        Hs[p * K + i] = d[p].s;
        Hc[p * K + i] = d[p].c;
      }
  }
  __syncthreads();
  // residual r_p = u_p^T D_32 A - u_p^T B (B is [K][m]: row j = atom j's
  // column); the large parts cancel exactly in the float differences of the
  // compensated sums, their corrections carry the rest
#pragma unroll
  for (int q = 0; q < CJ; ++q) {
    const int j = tid + kCThreads * q;
    if (j >= K) continue;
    DF bv[kProbes];
#pragma unroll
    for (int p = 0; p < kProbes; ++p) bv[p] = DF{0.f, 0.f};
    const double *bj = Bt + (size_t)j * m;
    for (int r = 0; r < m; ++r) {
      float bh, bl;
      split_d(__ldg(bj + r), bh, bl);
#pragma unroll
      for (int p = 0; p < kProbes; ++p) {
        const bool neg = Us[p][r] < 0.f;
        df_add(bv[p], neg ? -bh : bh);
        bv[p].c = __fadd_rn(bv[p].c, neg ? -bl : bl);
      }
    }
#pragma unroll
    for (int p = 0; p < kProbes; ++p) {
      const DF hp = df_merge(h[q][p], DF{Hs[p * K + j], Hc[p * K + j]});
      Zs[p * K + j] = __fadd_rn(__fsub_rn(hp.s, bv[p].s), __fsub_rn(hp.c, bv[p].c));
    }
  }
  __syncthreads();

  // z_p = r_p A^-1 = (L L^T)^-1 r_p in FP32 (an estimate is all that is
  // needed): forward L y = r, then backward L^T z = y, tile by tile with the
  // inverses of the diagonal factor tiles
  for (int k = 0; k < R; ++k) {
    const int k0 = k * TS, nb = K - k0 < TS ? K - k0 : TS;
    for (int e = tid; e < kProbes * TS; e += kCThreads) {
      const int p = e / TS, a = e % TS;
      float y = 0.f;
      if (a < nb)
        for (int c = 0; c <= a; ++c) y = fmaf(Vt[(size_t)k * TS * TS + a * TS + c], Zs[p * K + k0 + c], y);
      Ys[p][a] = y;
    }
    __syncthreads();
    for (int e = tid; e < kProbes * TS; e += kCThreads) {
      const int p = e / TS, a = e % TS;
      if (a < nb) Zs[p * K + k0 + a] = Ys[p][a];
    }
    for (int i = k0 + nb + tid; i < K; i += kCThreads) {
      const float *li = Lt + (size_t)i * K + k0;
      float acc[kProbes] = {};
      for (int c = 0; c < nb; ++c) {
        const float l = li[c];
#pragma unroll
        for (int p = 0; p < kProbes; ++p) acc[p] = fmaf(l, Ys[p][c], acc[p]);
      }
#pragma unroll
      for (int p = 0; p < kProbes; ++p) Zs[p * K + i] -= acc[p];
    }
    __syncthreads();
  }
  for (int k = R - 1; k >= 0; --k) {
    const int k0 = k * TS, nb = K - k0 < TS ? K - k0 : TS;
    for (int e = tid; e < kProbes * TS; e += kCThreads) {
      const int p = e / TS, a = e % TS;
      float z = 0.f;
      if (a < nb)
        for (int c = a; c < nb; ++c) z = fmaf(Vt[(size_t)k * TS * TS + c * TS + a], Zs[p * K + k0 + c], z);
      Ys[p][a] = z;
    }
    __syncthreads();
    for (int e = tid; e < kProbes * TS; e += kCThreads) {
      const int p = e / TS, a = e % TS;
      if (a < nb) Zs[p * K + k0 + a] = Ys[p][a];
    }
    for (int j = tid; j < k0; j += kCThreads) {
      float acc[kProbes] = {};
      for (int c = 0; c < nb; ++c) {
        const float l = Lt[(size_t)(k0 + c) * K + j];
#pragma unroll
        for (int p = 0; p < kProbes; ++p) acc[p] = fmaf(l, Ys[p][c], acc[p]);
      }
#pragma unroll
      for (int p = 0; p < kProbes; ++p) Zs[p * K + j] -= acc[p];
    }
    __syncthreads();
  }

  // every used atom's estimated error against tau of its norm
  bool ok = true;
#pragma unroll
  for (int q = 0; q < CJ; ++q) {
    const int j = tid + kCThreads * q;
    if (j >= K || ut[j] == 0) continue;
    double e2 = 0.0;
#pragma unroll
    for (int p = 0; p < kProbes; ++p) e2 = fma((double)Zs[p * K + j], (double)Zs[p * K + j], e2);
    e2 /= kProbes;
    const double lim = (double)tau * (double)tau * (double)n2[q];
    if (!(n2[q] > 0.f) || !isfinite(n2[q]) || !(e2 <= lim)) ok = false;
  }
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) status[t] = kModDeferredC;
    return;
  }
#pragma unroll
  for (int q = 0; q < CJ; ++q) {
    const int j = tid + kCThreads * q;
    if (j >= K || ut[j] == 0) continue;   // unused: keeps the previous atom
    // the norm again in FP64 for the scale (one pass over the atom)
    double s2 = 0.0;
    for (int r = 0; r < m; ++r) {
      const double x = X[(size_t)r * K + j];
      s2 = fma(x, x, s2);
    }
    const double inv = 1.0 / sqrt(s2);
    T *dj = D + ((size_t)t * K + j) * m;
    for (int r = 0; r < m; ++r) dj[r] = (T)((double)X[(size_t)r * K + j] * inv);
  }
  if (tid == 0) status[t] = 0;
}

}  // namespace

size_t mod_check_smem(int K) { return 5 * sizeof(float) * kProbes * (size_t)K; }

template <typename T>
cudaError_t launch_mod_check(const ModArgs &a, int ts, float tau, cudaStream_t st) {
  if (a.L <= 0) return cudaSuccess;
  if (a.K > kCThreads * kCJMax || a.m > 256 || (ts != 16 && ts != 32 && ts != 64)) return cudaErrorInvalidValue;
  const size_t smem = mod_check_smem(a.K);
  auto kern = a.K <= 2 * kCThreads ? mod_check_kernel<T, 2> : mod_check_kernel<T, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const float *M = reinterpret_cast<const float *>(a.Lf);
  const float *V = M + (size_t)a.L * (a.K + a.m) * a.K;
  kern<<<(unsigned)a.L, kCThreads, smem, st>>>(static_cast<const double *>(a.A), static_cast<const double *>(a.B),
                                               a.usage, a.K, a.m, ts, M, V, static_cast<T *>(a.D), a.status, tau);
  return cudaGetLastError();
}

template cudaError_t launch_mod_check<float>(const ModArgs &, int, float, cudaStream_t);

}  // namespace sdl
