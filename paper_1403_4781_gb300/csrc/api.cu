// C ABI entry points: argument checks, workspace, and the host-side order of
// kernels for OMP (Sec. 1), MOD (Sec. 1), and Algorithm 1 (split, local
// training, scaled-stack merge).  Every kernel runs on the context's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "sdl_internal.cuh"

namespace sdl {

sdl_status set_error(sdl_ctx *ctx, sdl_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return st;
}

sdl_status check_cuda(sdl_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SDL_OK;
  return set_error(ctx, SDL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void ws_reset(sdl_ctx *ctx) { ctx->ws.used = 0; }

static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Make sure the workspace holds `bytes`; regrowth synchronises the stream.
// Captured training loops refer to workspace addresses: drop them all.
static void clear_graphs(sdl_ctx *ctx) {
  for (auto &kv : ctx->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  ctx->graphs.clear();
  ctx->graph_seen.clear();
}

static sdl_status ws_reserve(sdl_ctx *ctx, size_t bytes) {
  ws_reset(ctx);
  if (bytes <= ctx->ws.cap) return SDL_OK;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return check_cuda(ctx, e, "workspace sync");
  clear_graphs(ctx);
  if (ctx->ws.base) cudaFree(ctx->ws.base);
  ctx->ws.base = nullptr;
  ctx->ws.cap = 0;
  size_t want = bytes + bytes / 8;
  e = cudaMalloc(&ctx->ws.base, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws.base = nullptr;
    return set_error(ctx, SDL_ENOMEM, "cannot allocate " + std::to_string(want) + " bytes of workspace");
  }
  ctx->ws.cap = want;
  return SDL_OK;
}

void *ws_alloc(sdl_ctx *ctx, size_t bytes) {
  const size_t b = round256(bytes ? bytes : 1);
  if (ctx->ws.used + b > ctx->ws.cap) return nullptr;
  void *p = ctx->ws.base + ctx->ws.used;
  ctx->ws.used += b;
  return p;
}

TilePlan make_tiles(const int64_t *offsets, int L, int tile) {
  TilePlan p;
  p.tile_start.resize((size_t)L + 1);
  int64_t acc = 0;
  for (int t = 0; t < L; ++t) {
    p.tile_start[t] = (int32_t)acc;
    acc += (offsets[t + 1] - offsets[t] + tile - 1) / tile;
  }
  p.tile_start[L] = (int32_t)acc;
  p.total_tiles = acc;
  return p;
}

namespace {

// Run one launcher; count its kernels and, when profiling is on, bracket it
// with a pair of events on the context stream.
template <class F>
cudaError_t timed(sdl_ctx *ctx, const char *name, int nkernels, F &&launch) {
  ctx->launches += nkernels;
  if (!ctx->prof.on) return launch();
  Prof &P = ctx->prof;
  int entry = -1;
  for (size_t q = 0; q < P.entries.size(); ++q)
    if (P.entries[q].name == name) { entry = (int)q; break; }
  if (entry < 0) {
    P.entries.push_back(ProfEntry{name, 0, 0, 0.0});
    entry = (int)P.entries.size() - 1;
  }
  cudaEvent_t ev[2];
  for (int q = 0; q < 2; ++q) {
    if (!P.pool.empty()) { ev[q] = P.pool.back(); P.pool.pop_back(); }
    else if (cudaEventCreate(&ev[q]) != cudaSuccess) return cudaGetLastError();
  }
  cudaEventRecord(ev[0], ctx->stream);
  cudaError_t e = launch();
  cudaEventRecord(ev[1], ctx->stream);
  P.entries[entry].launches += nkernels;
  P.entries[entry].calls += 1;
  P.pending.push_back(ProfPending{entry, ev[0], ev[1]});
  return e;
}

// Resolve pending event pairs into per-kernel totals (synchronises on them).
void prof_resolve(sdl_ctx *ctx) {
  Prof &P = ctx->prof;
  for (auto &q : P.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.e1) == cudaSuccess && cudaEventElapsedTime(&ms, q.e0, q.e1) == cudaSuccess)
      P.entries[q.entry].ms += ms;
    P.pool.push_back(q.e0);
    P.pool.push_back(q.e1);
  }
  P.pending.clear();
  cudaGetLastError();
}

// Cached number of clusters of the tiled solve (f32: its FP32 pass) that fit
// on the device at once.
template <typename T>
int tiled_occupancy(sdl_ctx *ctx, int ts, int C, int cap, bool f32 = false) {
  const int64_t key = ((int64_t)f32 << 40) | ((int64_t)(sizeof(T)) << 32) | ((int64_t)cap << 16) |
                      ((int64_t)ts << 8) | C;
  auto it = ctx->occ.find(key);
  if (it != ctx->occ.end()) return it->second;
  const int n = mod_tiled_max_clusters<T>(ts, C, cap, f32);
  ctx->occ[key] = n;
  return n;
}

// Tile edge and cluster size of the tiled FP64 solve from the shape alone.
// Few subsets: the factorisation's dependency chain dominates, so small tiles
// spread each subset over the largest cluster.  Many subsets: the largest
// cluster for which every subset's cluster is resident at once.
template <typename T>
void pick_tiled(sdl_ctx *ctx, int L, int *ts, int *C, bool f32 = false) {
  int t = ctx->opt_tile;
  int c = ctx->opt_cluster;
  if (t == 0) t = (int64_t)L * 8 <= ctx->num_sms ? 16 : 32;
  if (t == 64 && !f32) t = 32;   // 64 x 64 tiles: the FP32 pass only
  if (c == 0) {
    c = 1;
    const int cand[6] = {16, 8, 6, 4, 2, 1};
    for (int q = 0; q < 6; ++q) {
      const int n = tiled_occupancy<T>(ctx, t, cand[q], 0, f32);
      if (n >= L) { c = cand[q]; break; }
    }
  }
  *ts = t;
  *C = c;
}

// The checked mixed-precision solve of FP32 data: the FP32 pass (tile ts,
// clusters of C), the check that renormalises the subsets it accepts, then the
// FP64 solve of the subsets left to it (its shape from the shape rule; every
// other subset's blocks leave at once).
template <typename T>
cudaError_t run_mixed(sdl_ctx *ctx, const ModArgs &ma, int ts, int C, bool timed_parts) {
  if constexpr (sizeof(T) != 4) {   // FP32 data only
    return cudaErrorNotSupported;
  } else {
  cudaStream_t sm = ctx->stream;
  int ts64 = 32, C64 = 1;
  pick_tiled<T>(ctx, ma.L, &ts64, &C64);
  const bool single = ma.L == 1;
  auto r32 = [&] { return launch_mod_tiled32<T>(ma, ts, C, 0, ctx->num_sms, sm); };
  const float tau = (float)(ctx->opt_mod_check_ppb * 1e-9);
  auto chk = [&] { return launch_mod_check<T>(ma, ts, tau, sm); };
  auto r64 = [&] { return launch_mod_tiled<T>(ma, ts64, C64, 0, ctx->num_sms, sm, true); };
  cudaError_t e;
  if (!timed_parts) {
    if ((e = r32()) != cudaSuccess) return e;
    if ((e = chk()) != cudaSuccess) return e;
    return r64();
  }
  if ((e = timed(ctx, single ? "mod_solve_fp32_single" : "mod_solve_fp32", 1, r32)) != cudaSuccess) return e;
  if ((e = timed(ctx, "mod_check", 1, chk)) != cudaSuccess) return e;
  return timed(ctx, single ? "mod_solve_fp64_single" : "mod_solve_fp64", 1, r64);
  }
}

// Whether the checked FP32 pass applies to this call.
template <typename T>
bool mixed_allowed(const sdl_ctx *ctx, const ModArgs &ma) {
  return sizeof(T) == 4 && ctx->opt_mod_mixed && ma.K <= 1024 && ma.m <= 256;
}

// Autotuner of the tiled solve: on the first call for a shape (element type,
// subsets, K, m) that leaves the tile and cluster size automatic, every
// candidate tile edge and cluster size is run on the caller's own inputs (the
// solve reads A, B and the usage counts and rewrites only scratch, D and the
// status, so repeated runs give the same result) and timed with CUDA events;
// the fastest is cached in the context and run last.  For FP32 data the
// candidates include the checked FP32 pass with each tile and cluster size
// (timed with its check and the FP64 solve of what it leaves).  (Capping the
// blocks per SM to balance clusters over the SMs was measured slower at every
// shape tried: the FP64 pipe wants the warps more than the balance, so it is
// not a candidate.)  Skipped while the stream is being captured (the shape
// rule above is used then, with the checked FP32 pass where it applies) or
// when the option turns it off.
template <typename T>
cudaError_t run_tiled_tuned(sdl_ctx *ctx, const ModArgs &ma) {
  cudaStream_t sm = ctx->stream;
  int ts = 32, C = 1, cap = 0;
  const bool manual = ctx->opt_tile != 0 || ctx->opt_cluster != 0;
  const bool mix_ok = mixed_allowed<T>(ctx, ma);
  const std::string key = std::to_string(sizeof(T)) + ":" + std::to_string(ma.L) + ":" + std::to_string(ma.K) +
                          ":" + std::to_string(ma.m) + ":" + std::to_string((int)mix_ok);
  auto it = ctx->tuned.find(key);
  cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(sm, &capst) != cudaSuccess) {
    cudaGetLastError();
    capst = cudaStreamCaptureStatusActive;
  }
  int wide = 0, mixed = 0;
  if (!manual && it != ctx->tuned.end()) {
    ts = it->second.ts;
    C = it->second.C;
    cap = it->second.cap;
    wide = it->second.wide;
    mixed = it->second.mixed;
  } else if (manual || !ctx->opt_autotune || capst != cudaStreamCaptureStatusNone) {
    mixed = mix_ok ? 1 : 0;
    pick_tiled<T>(ctx, ma.L, &ts, &C, mixed != 0);
    if (manual) cap = ctx->opt_sm_blocks;
  } else {
    int best_ts = 0, best_c = 0, best_cap = 0, best_wide = 0, best_mixed = 0;
    float best = 3.4e38f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // best of two timed runs of one candidate
    auto time_it = [&](auto &&run) -> float {
      float ms_best = 3.4e38f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, sm);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, sm);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < ms_best) ms_best = ms;
      }
      return ms_best;
    };
    const int tiles[3] = {16, 32, 64};   // 64: the FP32 pass only
    const int cls[7] = {1, 2, 3, 4, 6, 8, 16};
    // the FP32 pass's tile and cluster size by the FP32 pass alone; then the
    // whole checked solve with that shape (its check and the FP64 solve of what
    // the check leaves do not depend on the shape) against the FP64 candidates
    int ts32 = 0, c32 = 0;
    float best32 = 3.4e38f;
    for (int pass = mix_ok ? 0 : 1; pass < 2 && e == cudaSuccess; ++pass) {
      const bool f32 = pass == 0;
      for (int a = 0; a < (f32 ? 3 : 2) && e == cudaSuccess; ++a)
        for (int b = 0; b < 7 && e == cudaSuccess; ++b) {
          const int t = tiles[a], c = cls[b], cp = 0;
          // a subset's cluster must fit on the device; small clusters for few
          // subsets leave most SMs idle and are not worth timing
          if (tiled_occupancy<T>(ctx, t, c, cp, f32) < 1) continue;
          if ((int64_t)ma.L * c * 4 < ctx->num_sms && c < 16) continue;
          const float ms = time_it([&] {
            ctx->launches += 1;
            return f32 ? launch_mod_tiled32<T>(ma, t, c, cp, ctx->num_sms, sm)
                       : launch_mod_tiled<T>(ma, t, c, cp, ctx->num_sms, sm);
          });
          if (e != cudaSuccess) break;
          if (f32 && ms < best32) { best32 = ms; ts32 = t; c32 = c; }
          if (!f32 && ms < best) { best = ms; best_ts = t; best_c = c; best_cap = cp; best_wide = 0; best_mixed = 0; }
        }
      if (f32 && ts32 > 0 && e == cudaSuccess) {   // the whole checked solve with the best FP32 shape
        const float msm = time_it([&] {
          ctx->launches += 3;
          return run_mixed<T>(ctx, ma, ts32, c32, false);
        });
        if (e == cudaSuccess && msm < best) {
          best = msm; best_ts = ts32; best_c = c32; best_cap = 0; best_wide = 0; best_mixed = 1;
        }
      }
    }
    // few subsets: the wide form, each subset's tile tasks over G blocks
    // anywhere on the GPU (its largest cluster holds at most 16 SMs)
    if ((int64_t)ma.L * 16 < ctx->num_sms)
      for (int a = 0; a < 2 && e == cudaSuccess; ++a)
        for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
          const int t = tiles[a];
          const int G = (int)((int64_t)ctx->num_sms * (f == 0 ? 1 : (f == 1 ? 2 : 4)) / (2 * ma.L));
          if (G <= 16 || (int64_t)ma.L * G > mod_wide_max_blocks<T>(t, ctx->num_sms)) continue;
          const float ms = time_it([&] {
            ctx->launches += 1;
            return launch_mod_wide<T>(ma, t, G, ctx->opt_wait_limit, -1, sm);
          });
          if (e == cudaSuccess && ms < best) {
            best = ms; best_ts = t; best_c = G; best_cap = 0; best_wide = 1; best_mixed = 0;
          }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    if (best_ts == 0) {
      mixed = mix_ok ? 1 : 0;
      pick_tiled<T>(ctx, ma.L, &ts, &C, mixed != 0);
    } else {
      ts = best_ts;
      C = best_c;
      cap = best_cap;
      wide = best_wide;
      mixed = best_mixed;
    }
    ctx->tuned[key] = sdl_ctx::TunedSolve{ts, C, cap, wide, mixed};
  }
  if (mixed) return run_mixed<T>(ctx, ma, ts, C, true);
  // the batched solve and the single-system (merge) solve are reported apart
  return timed(ctx, ma.L > 1 ? "mod_solve_fp64" : "mod_solve_fp64_single", 1, [&] {
    return wide ? launch_mod_wide<T>(ma, ts, C, ctx->opt_wait_limit, ctx->opt_wait_test ? 1 : -1, sm)
                : launch_mod_tiled<T>(ma, ts, C, cap, ctx->num_sms, sm);
  });
}

// FP64 Cholesky + solve + renormalisation: the tiled cluster kernel unless an
// option selects one of the other implementations.
template <typename T>
cudaError_t run_mod_solve(sdl_ctx *ctx, const ModArgs &ma) {
  cudaStream_t sm = ctx->stream;
  cudaError_t e = cudaErrorNotSupported;
  if (ctx->opt_mod_solve == 0 || ctx->opt_mod_solve == 3) return run_tiled_tuned<T>(ctx, ma);
  if (ctx->opt_mod_solve == 4)   // the wide form, tile edge and blocks per subset from the options
    return timed(ctx, ma.L > 1 ? "mod_solve_fp64" : "mod_solve_fp64_single", 1, [&] {
      const int G = ctx->opt_cluster > 0 ? ctx->opt_cluster : (ctx->num_sms + ma.L - 1) / ma.L;
      return launch_mod_wide<T>(ma, ctx->opt_tile ? ctx->opt_tile : 16, G, ctx->opt_wait_limit,
                                ctx->opt_wait_test ? 1 : -1, sm);
    });
  if (ma.K <= 512 && ctx->opt_mod_solve == 1)
    e = timed(ctx, "mod_solve_fp64", 1, [&] {
      return launch_mod_solve_cluster<T>(ma, ctx->opt_cluster ? ctx->opt_cluster : 16, sm);
    });
  if (e != cudaErrorNotSupported) return e;
  cudaGetLastError();
  e = timed(ctx, "chol_fp64", 1, [&] { return launch_mod_chol(ma, sm); });
  if (e != cudaSuccess) return e;
  e = timed(ctx, "solve_fp64", 1, [&] { return launch_mod_solve(ma, ctx->num_sms, sm); });
  if (e != cudaSuccess) return e;
  return timed(ctx, "normalise", 1, [&] { return launch_mod_normalise<T>(ma, sm); });
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool aligned16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

#define SDL_REQUIRE(cond, msg) \
  do {                         \
    if (!(cond)) return set_error(ctx, SDL_EINVAL, msg); \
  } while (0)

#define SDL_CUDA(expr, what)                                    \
  do {                                                          \
    cudaError_t e_ = (expr);                                    \
    if (e_ != cudaSuccess) return check_cuda(ctx, e_, what);    \
  } while (0)

sdl_status check_prec(sdl_ctx *ctx, sdl_precision prec) {
  if (prec == SDL_PREC_F64 || prec == SDL_PREC_F32 || prec == SDL_PREC_BF16 || prec == SDL_PREC_F32X3 ||
      prec == SDL_PREC_TF32)
    return SDL_OK;
  return set_error(ctx, SDL_EINVAL, "unknown precision");
}

// FP32 OMP form: the fused kernel (correlation tile in shared memory) or the
// correlation GEMM + selection kernel pair.  Automatic: the pair, which was
// the faster of the two at every shape measured (m 64..256, K 256..1024,
// s 2..16), by 1.2x at m = 64, K = 256, s = 2 and 2.2x at m = 256, K = 512.
bool omp_split_f32(const sdl_ctx *ctx, int K, int m, int s) {
  (void)K;
  (void)m;
  (void)s;
  return ctx->opt_omp_form != 1;
}

// Workspace of a tensor-core coding pass over n signals in L subsets: the two
// images of D (hi, then lo; BF16 or the larger TF32 layout), error word, and
// the correlation scratch (one chunk of 128-signal tiles).  The FP32 Gram
// lives in the caller's G.
size_t tc_image_bytes(int L, int K, int m) {
  const size_t bf16 = (size_t)L * round16(K) * round16(m) * 2, x3 = x3_image_bytes(L, K, m);
  const size_t rtc = rtc_image_bytes(L, K, m);
  const size_t mx = bf16 > x3 ? bf16 : x3;
  return mx > rtc ? mx : rtc;
}
size_t tc_a0_bytes(int L, int K, int64_t n) {
  const int64_t tiles = (n + 127) / 128 + L;
  return sizeof(float) * (size_t)omp_tc_chunk_tiles(K, tiles) * 128 * K;
}
// Half-precision copy of the Gram for the BF16 pass's running update.
size_t tc_g16_bytes(int L, int K) { return (size_t)L * K * K * 2; }
size_t tc_ws_bytes(int L, int K, int m, int64_t n) {
  return round256(3 * tc_image_bytes(L, K, m)) + round256(sizeof(int32_t) * 4) + round256(tc_a0_bytes(L, K, n)) +
         round256(tc_g16_bytes(L, K));
}

// Kernels of one two-kernel coding pass: a correlation and a selection launch
// per chunk of the scratch.
int split_kernels(const OmpArgs &oa) {
  const int64_t chunk = omp_tc_chunk_tiles(oa.K, oa.total_tiles, oa.a0_cap);
  return oa.total_tiles > 0 ? 2 * (int)((oa.total_tiles + chunk - 1) / chunk) : 0;
}

// Autotuner of the selection launch of the two-kernel coding passes: on the
// first call of a shape (tag, subsets, K, m, s, whether eps stops early, tiles
// rounded down to a power of two) with at least two 128-signal tiles per SM,
// the whole pass (correlations and selection, run()) is run once per selection
// shape (4, 2 or 1 signals per warp; the G-column cache as large as fits, or
// none) and timed with CUDA events, the pass of under 20 ms twice (best of
// two); the fastest shape is cached in the context.  Every shape computes the
// same codes (each signal's arithmetic and its order do not depend on it), so
// the timing runs cost only time.  Options set by hand, a stream being
// captured, or SDL_OPT_AUTOTUNE = 0: the cached shape, else 4 signals per warp
// and the cache as large as fits.
template <class Run>
cudaError_t tune_select(sdl_ctx *ctx, OmpArgs &oa, const char *tag, Run &&run) {
  const int gc_of[3] = {0, 0, -1};
  oa.sel_spw = ctx->opt_sel_spw != 0 ? ctx->opt_sel_spw : 4;
  oa.sel_gcn = gc_of[ctx->opt_sel_gcache];
  if (ctx->opt_sel_spw != 0 || ctx->opt_sel_gcache != 0) return cudaSuccess;
  int lg = 0;
  while (lg < 62 && ((int64_t)2 << lg) <= oa.total_tiles) ++lg;
  const std::string key = std::string(tag) + ":" + std::to_string(oa.L) + ":" + std::to_string(oa.K) + ":" +
                          std::to_string(oa.m) + ":" + std::to_string(oa.s) + ":" +
                          std::to_string(oa.eps > 0 ? 1 : 0) + ":" + std::to_string(lg);
  auto it = ctx->tuned_sel.find(key);
  if (it != ctx->tuned_sel.end()) {
    oa.sel_spw = it->second.spw;
    oa.sel_gcn = it->second.gcn;
    return cudaSuccess;
  }
  cudaStream_t sm = ctx->stream;
  cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(sm, &capst) != cudaSuccess) {
    cudaGetLastError();
    capst = cudaStreamCaptureStatusActive;
  }
  if (!ctx->opt_autotune || capst != cudaStreamCaptureStatusNone || oa.total_tiles < 2 * (int64_t)ctx->num_sms)
    return cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int spws[3] = {4, 2, 1}, gcns[2] = {0, -1};
  int best_spw = 4, best_gcn = 0;
  float best = 3.4e38f;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a)
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      oa.sel_spw = spws[a];
      oa.sel_gcn = gcns[b];
      float ms_best = 3.4e38f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, sm);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, sm);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < ms_best) ms_best = ms;
        if (ms_best >= 20.f) break;
      }
      if (e == cudaSuccess && ms_best < best) {
        best = ms_best;
        best_spw = spws[a];
        best_gcn = gcns[b];
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  oa.sel_spw = best_spw;
  oa.sel_gcn = best_gcn;
  if (e == cudaSuccess) ctx->tuned_sel[key] = sdl_ctx::TunedSelect{best_spw, best_gcn};
  return e;
}

// Bounds of the tensor-core kernels' mbarrier waits: SDL_OPT_WAIT_LIMIT
// polls, capped at 2^22 (each poll may suspend the thread for a while);
// SDL_OPT_WAIT_TEST makes their loader leave at once.
X3Wait x3_wait(const sdl_ctx *ctx) {
  const long long lim = ctx->opt_wait_limit < (1LL << 22) ? ctx->opt_wait_limit : (1LL << 22);
  return X3Wait{(int)(lim > 0 ? lim : 1), ctx->opt_wait_test ? 1 : 0};
}

// One BF16 coding pass: BF16 images of D (img holds hi, lo and the slab
// image), Gram and correlations on the tensor cores, selection loop with its
// FP32 correction step on the support.
cudaError_t run_omp_bf16(sdl_ctx *ctx, OmpArgs &oa, void *img, float *G, int32_t *err, float *a0c, void *G16) {
  // only form 3 reads the half-precision Gram copy in the running update
  if (ctx->opt_bf16_form != 3) G16 = nullptr;
  oa.G16 = G16;
  cudaStream_t sm = ctx->stream;
  // slots: the hi and lo images of the split Gram, then the slab image that
  // the correlation kernel and the residual form read
  void *lo = static_cast<unsigned char *>(img) + tc_image_bytes(oa.L, oa.K, oa.m);
  void *simg = static_cast<unsigned char *>(img) + 2 * tc_image_bytes(oa.L, oa.K, oa.m);
  oa.err = err;
  oa.G = G;
  cudaError_t e = timed(ctx, "bf16_image", 2, [&] {
    cudaError_t r = launch_bf16_image(static_cast<const float *>(oa.D), oa.K, oa.m, oa.L, img, lo, sm);
    return r != cudaSuccess ? r : launch_rtc_image(static_cast<const float *>(oa.D), oa.K, oa.m, oa.L, simg, sm);
  });
  if (e != cudaSuccess) return e;
  e = timed(ctx, "gram_tc", 1, [&] { return launch_gram_tc(img, lo, oa.K, oa.m, oa.L, G, err, sm, G16); });
  if (e != cudaSuccess) return e;
  if (ctx->opt_bf16_form == 2 && omp_rtc_supported(oa.K, oa.m, oa.s))
    return timed(ctx, "omp_rtc", 1, [&] { return launch_omp_rtc(oa, simg, sm); });
  auto pass = [&] { return launch_omp_tc(oa, simg, a0c, ctx->num_sms, x3_wait(ctx), sm); };
  e = tune_select(ctx, oa, G16 ? "bf16h" : "bf16", [&] {
    ctx->launches += split_kernels(oa);
    return pass();
  });
  if (e != cudaSuccess) return e;
  return timed(ctx, "omp_tc", split_kernels(oa), pass);
}

// One FP32-accurate tensor-core coding pass: TF32 hi and lo images of D (img
// holds hi, then lo), Gram and correlations as three TF32 products on the
// tensor cores, then the FP32 selection loop.  single: the correlations from
// one TF32 product (SDL_PREC_TF32), the Gram still from three.
cudaError_t run_omp_x3(sdl_ctx *ctx, OmpArgs &oa, void *img, float *G, int32_t *err, float *a0c,
                       bool single) {
  cudaStream_t sm = ctx->stream;
  void *lo = static_cast<unsigned char *>(img) + tc_image_bytes(oa.L, oa.K, oa.m);
  oa.err = err;
  oa.G = G;
  cudaError_t e = timed(ctx, "x3_image", 1, [&] {
    return launch_x3_image(static_cast<const float *>(oa.D), oa.K, oa.m, oa.L, img, lo, sm);
  });
  if (e != cudaSuccess) return e;
  e = timed(ctx, "gram_x3", 1, [&] {
    return launch_gram_x3(static_cast<const float *>(oa.D), img, lo, oa.K, oa.m, oa.L, G, err, ctx->num_sms,
                          x3_wait(ctx), sm);
  });
  if (e != cudaSuccess) return e;
  auto pass = [&] { return launch_omp_x3(oa, img, lo, a0c, ctx->num_sms, x3_wait(ctx), sm, single); };
  e = tune_select(ctx, oa, single ? "tf32" : "x3", [&] {
    ctx->launches += split_kernels(oa);
    return pass();
  });
  if (e != cudaSuccess) return e;
  return timed(ctx, single ? "omp_tf32" : "omp_x3", split_kernels(oa), pass);
}

// The FP32 two-kernel coding pass (correlation GEMM, then the selection
// kernel) with the tuned selection launch; the Gram is the caller's.
cudaError_t run_omp_split(sdl_ctx *ctx, OmpArgs &oa, float *a0c) {
  cudaStream_t sm = ctx->stream;
  auto pass = [&] { return launch_omp_split_f32(oa, a0c, sm); };
  cudaError_t e = tune_select(ctx, oa, "f32", [&] {
    ctx->launches += split_kernels(oa);
    return pass();
  });
  if (e != cudaSuccess) return e;
  return timed(ctx, "omp_split", split_kernels(oa), pass);
}

// Read back the error word of the tensor-core kernels (synchronises).
sdl_status tc_status(sdl_ctx *ctx, const int32_t *err) {
  SDL_CUDA(cudaMemcpyAsync(ctx->h_status, err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "err read");
  SDL_CUDA(cudaStreamSynchronize(ctx->stream), "err sync");
  if (*ctx->h_status != 0) return set_error(ctx, SDL_ETIMEOUT, "a bounded wait of a tensor-core kernel gave up");
  return SDL_OK;
}

sdl_status check_offsets(sdl_ctx *ctx, const int64_t *offsets, int L, bool nonempty) {
  SDL_REQUIRE(offsets != nullptr, "offsets is NULL");
  SDL_REQUIRE(L >= 1, "L must be >= 1");
  SDL_REQUIRE(offsets[0] == 0, "offsets[0] must be 0");
  for (int t = 0; t < L; ++t) {
    SDL_REQUIRE(offsets[t + 1] >= offsets[t], "offsets must be non-decreasing");
    if (nonempty) SDL_REQUIRE(offsets[t + 1] > offsets[t], "every subset must be non-empty");
  }
  SDL_REQUIRE(offsets[L] < ((int64_t)1 << 31), "at most 2^31-1 signals per call");
  return SDL_OK;
}

// Device copy of offsets and of a tile plan (pageable host -> device).
sdl_status upload_plan(sdl_ctx *ctx, const int64_t *offsets, int L, int tile, int64_t **d_off,
                       int32_t **d_tiles, int64_t *total_tiles) {
  TilePlan p = make_tiles(offsets, L, tile);
  if (p.total_tiles >= ((int64_t)1 << 31)) return set_error(ctx, SDL_EINVAL, "too many tiles");
  if (d_off) {
    *d_off = static_cast<int64_t *>(ws_alloc(ctx, sizeof(int64_t) * (L + 1)));
    SDL_CUDA(cudaMemcpyAsync(*d_off, offsets, sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice,
                             ctx->stream), "upload offsets");
  }
  *d_tiles = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (L + 1)));
  SDL_CUDA(cudaMemcpyAsync(*d_tiles, p.tile_start.data(), sizeof(int32_t) * (L + 1),
                           cudaMemcpyHostToDevice, ctx->stream), "upload tiles");
  *total_tiles = p.total_tiles;
  // the pageable source vector dies here: make the copy complete first
  SDL_CUDA(cudaStreamSynchronize(ctx->stream), "upload sync");
  return SDL_OK;
}

size_t elem_size(sdl_precision prec) { return prec == SDL_PREC_F64 ? 8 : 4; }

// Workspace bytes of one OMP pass over L dictionaries.
size_t omp_ws_bytes(sdl_precision prec, int L, int K) {
  return round256(elem_size(prec) * (size_t)L * K * K) + 2 * round256(sizeof(int64_t) * (L + 1));
}

size_t mod_ws_bytes(int L, int K, int m, int64_t n, int s) {
  size_t b = 0;
  b += round256(sizeof(int64_t) * (L + 1)) + round256(sizeof(int32_t) * (L + 1));
  b += round256(sizeof(int32_t) * (size_t)L * K);          // cursor
  b += round256(sizeof(int32_t) * (size_t)L * (K + 1));    // ptr
  b += 3 * round256(sizeof(int32_t) * (size_t)(n * s + 1));  // lsig, lslot, latom
  b += round256(sizeof(double) * (size_t)L * K * K);       // A
  b += round256(sizeof(double) * mod_tiled_scratch_doubles(L, K, m));   // factor scratch
  b += round256(sizeof(double) * (size_t)L * K * m);       // B
  b += round256(sizeof(int32_t) * (size_t)L);              // status
  b += round256(sizeof(int32_t) * (size_t)L * K);          // usage scratch
  b += round256(sizeof(int32_t) * 4);                      // status max
  return b;
}

// Carve the MOD scratch (after ws_reserve); offsets/tiles are uploaded here.
sdl_status mod_prepare(sdl_ctx *ctx, ModArgs &a, const int64_t *offsets_h, int L, int K, int m,
                       int s, int32_t *usage, int32_t **status_max) {
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  sdl_status st = upload_plan(ctx, offsets_h, L, mod_tile_signals(), &d_off, &d_tiles, &tiles);
  if (st != SDL_OK) return st;
  const int64_t n = offsets_h[L];
  a.offsets = d_off;
  a.tile_start = d_tiles;
  a.total_tiles = tiles;
  a.n = n;
  a.L = L; a.m = m; a.K = K; a.s = s;
  a.cursor = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)L * K));
  a.ptr = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)L * (K + 1)));
  a.lsig = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)(n * s + 1)));
  a.lslot = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)(n * s + 1)));
  a.latom = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)(n * s + 1)));
  a.A = static_cast<double *>(ws_alloc(ctx, sizeof(double) * (size_t)L * K * K));
  a.Lf = static_cast<double *>(ws_alloc(ctx, sizeof(double) * mod_tiled_scratch_doubles(L, K, m)));
  a.B = static_cast<double *>(ws_alloc(ctx, sizeof(double) * (size_t)L * K * m));
  a.status = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)L));
  int32_t *us = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)L * K));
  a.usage = usage ? usage : us;
  *status_max = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * 4));
  if (!a.cursor || !a.ptr || !a.lsig || !a.lslot || !a.latom || !a.A || !a.Lf || !a.B || !a.status || !us ||
      !*status_max)
    return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  return SDL_OK;
}

// Kernels one MOD accumulation launches: usage count, scan, CSC fill, the
// accumulation and, on the FP32 path, the unused-atom pass.  Without signals
// only the scan and the pass that sets the unused atoms run.
int mod_accum_kernels(bool f32, int64_t tiles) { return tiles > 0 ? (f32 ? 5 : 4) : 2; }

// Read back the worst MOD status of the last launch (synchronises).
sdl_status mod_status(sdl_ctx *ctx, const int32_t *status, int L, int32_t *d_max) {
  SDL_CUDA(timed(ctx, "status", 1, [&] { return launch_status_max(status, L, d_max, ctx->stream); }),
           "status reduce");
  SDL_CUDA(cudaMemcpyAsync(ctx->h_status, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
           "status read");
  SDL_CUDA(cudaStreamSynchronize(ctx->stream), "status sync");
  if (*ctx->h_status >= 3) return set_error(ctx, SDL_ETIMEOUT, "a bounded barrier wait of the FP64 solve gave up");
  if (*ctx->h_status >= 2)
    return set_error(ctx, SDL_ENOTPD,
                     "MOD normal equations not positive definite after the ridge retry");
  return SDL_OK;
}

sdl_status check_omp_shape(sdl_ctx *ctx, int m, int K, int s, double eps) {
  SDL_REQUIRE(m >= 1 && m <= kMaxM, "m must be in [1, 256]");
  SDL_REQUIRE(K >= 1 && K <= kMaxK, "K must be in [1, 1024]");
  SDL_REQUIRE(s >= 1 && s <= kMaxS && s <= m && s <= K, "s must be in [1, min(m, K, 32)]");
  SDL_REQUIRE(eps >= 0.0 && isfinite(eps), "eps must be finite and >= 0");
  return SDL_OK;
}

// Workspace of one training loop (Sec. 1, standard approach) over L subsets.
template <typename T>
size_t train_ws_bytes(int L, int K, int m, int64_t n, int s, int iters) {
  return omp_ws_bytes(sizeof(T) == 8 ? SDL_PREC_F64 : SDL_PREC_F32, L, K) + mod_ws_bytes(L, K, m, n, s) +
         tc_ws_bytes(L, K, m, n) +
         round256(sizeof(int32_t) * (size_t)n * s) + round256(sizeof(T) * (size_t)n * s) +
         round256(sizeof(int32_t) * (size_t)n) + round256(sizeof(T) * (size_t)n) +
         round256(sizeof(int32_t) * (size_t)(iters + 1)) + 4096;
}

// One training loop over L independent subsets; the workspace must already hold
// train_ws_bytes().  Per round: Gram, OMP, per-subset RMSE (and ||X||_F on the
// last round), MOD.  Synchronises once at the end to report a breakdown.
template <typename T>
sdl_status train_run(sdl_ctx *ctx, const T *Y, int m, const int64_t *offsets, int L, int K, int s,
                     double eps, int iters, T *D, double *xfro, double *rmse, sdl_precision tcp = SDL_PREC_F64) {
  // tcp: SDL_PREC_BF16, SDL_PREC_F32X3 or SDL_PREC_TF32 run the coding passes on the tensor cores
  const bool bf16 = sizeof(T) == 4 && tcp == SDL_PREC_BF16;
  const bool tf32 = sizeof(T) == 4 && tcp == SDL_PREC_TF32;
  const bool x3 = sizeof(T) == 4 && (tcp == SDL_PREC_F32X3 || tf32);
  const bool tc = bf16 || x3;
  const int64_t n = offsets[L];
  sdl_status st;
  OmpArgs oa{};
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  const bool split = !tc && sizeof(T) == 4 && omp_split_f32(ctx, K, m, s);
  const int tile = tc || split ? omp_tc_tile_signals(K, m, s) : omp_tile_signals();
  if (tile <= 0) return set_error(ctx, SDL_EINVAL, "shape too large for the tensor-core OMP kernel");
  if ((st = upload_plan(ctx, offsets, L, tile, &d_off, &d_tiles, &tiles)) != SDL_OK)
    return st;
  void *img = tc ? ws_alloc(ctx, 3 * tc_image_bytes(L, K, m)) : nullptr;
  int32_t *tc_err = tc ? static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * 4)) : nullptr;
  float *a0c = tc || split ? static_cast<float *>(ws_alloc(ctx, tc_a0_bytes(L, K, n))) : nullptr;
  void *g16 = bf16 && ctx->opt_bf16_form == 3 ? ws_alloc(ctx, tc_g16_bytes(L, K)) : nullptr;
  if ((split && !a0c) || (tc && (!img || !tc_err || !a0c)) || (bf16 && ctx->opt_bf16_form == 3 && !g16))
    return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  if (tc) SDL_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int32_t), ctx->stream), "err clear");
  T *G = static_cast<T *>(ws_alloc(ctx, sizeof(T) * (size_t)L * K * K));
  int32_t *idx = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n * s));
  T *val = static_cast<T *>(ws_alloc(ctx, sizeof(T) * (size_t)n * s));
  int32_t *nnz = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n));
  T *res2 = static_cast<T *>(ws_alloc(ctx, sizeof(T) * (size_t)n));
  int32_t *worst = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)(iters + 1)));
  if (!G || !idx || !val || !nnz || !res2 || !worst)
    return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  oa.D = D; oa.G = G; oa.Y = Y; oa.offsets = d_off; oa.tile_start = d_tiles; oa.total_tiles = tiles;
  oa.a0_cap = (int64_t)ctx->opt_a0_chunk_mb << 20;
  oa.L = L; oa.m = m; oa.K = K; oa.s = s; oa.eps = eps;
  oa.idx = idx; oa.val = val; oa.nnz = nnz; oa.resid2 = res2;
  ModArgs ma{};
  int32_t *d_max = nullptr;
  if ((st = mod_prepare(ctx, ma, offsets, L, K, m, s, nullptr, &d_max)) != SDL_OK) return st;
  ma.Y = Y; ma.idx = idx; ma.val = val; ma.D = D;
  // the tiled solve folds every iteration's worst status into worst[0]
  const bool tiled_folds_status = ctx->opt_mod_solve == 0 || ctx->opt_mod_solve == 3;
  ma.status_max = tiled_folds_status ? worst : nullptr;
  SDL_CUDA(cudaMemsetAsync(ma.status, 0, sizeof(int32_t) * L, ctx->stream), "status clear");
  SDL_CUDA(cudaMemsetAsync(worst, 0, sizeof(int32_t) * (iters + 1), ctx->stream), "status clear");
  if (xfro) SDL_CUDA(cudaMemsetAsync(xfro, 0, sizeof(double) * L, ctx->stream), "xfro clear");
  cudaStream_t sm = ctx->stream;
  auto run_loop = [&]() -> sdl_status {
    for (int it = 0; it < iters; ++it) {
      cudaError_t e;
      if (bf16) {
        e = run_omp_bf16(ctx, oa, img, reinterpret_cast<float *>(G), tc_err, a0c, g16);
      } else if (x3) {
        e = run_omp_x3(ctx, oa, img, reinterpret_cast<float *>(G), tc_err, a0c, tf32);
      } else if (split) {
        SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<T>(D, m, K, L, G, sm); }), "gram");
        e = run_omp_split(ctx, oa, a0c);
      } else {
        SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<T>(D, m, K, L, G, sm); }), "gram");
        e = timed(ctx, "omp", 1, [&] { return launch_omp<T>(oa, ctx->num_sms, sm); });
      }
      if (e == cudaErrorInvalidConfiguration)
        return set_error(ctx, SDL_EINVAL, "shape too large for the OMP kernel's shared memory");
      SDL_CUDA(e, "omp");
      SDL_CUDA(timed(ctx, "subset_stats", 1, [&] {
                 return launch_subset_stats<T>(res2, val, d_off, L, m, s, rmse ? rmse + it : nullptr, iters,
                                               it == iters - 1 ? xfro : nullptr, sm);
               }), "subset stats");
      SDL_CUDA(timed(ctx, "mod_accum", mod_accum_kernels(sizeof(T) == 4, ma.total_tiles),
                     [&] { return launch_mod_accum<T>(ma, sm); }), "mod accumulate");
      SDL_CUDA(run_mod_solve<T>(ctx, ma), "mod solve");
      if (ctx->opt_replace > 0)
        SDL_CUDA(timed(ctx, "replace", 1, [&] {
                   return launch_replace_atoms<T>(Y, m, ma.offsets, L, ma.usage, res2, ctx->opt_replace, D, K,
                                                  nullptr, sm);
                 }), "atom replacement");
      if (!tiled_folds_status)   // the other solve implementations only write status[]
        SDL_CUDA(timed(ctx, "status", 1, [&] { return launch_status_max(ma.status, L, worst + it, sm); }),
                 "status");
    }
    return SDL_OK;
  };
  // Graph replay: the loop's launches depend only on the pointers and sizes in
  // the key (the per-call plans are re-uploaded into the same workspace
  // addresses before it), so a key seen once eagerly is captured on its second
  // call and replayed from then on.
  const bool use_graph = ctx->opt_graph && !ctx->prof.on && iters > 0;
  if (!use_graph) {
    if ((st = run_loop()) != SDL_OK) return st;
  } else {
    char kb[512];
    snprintf(kb, sizeof(kb), "%zu:%d:%p:%p:%p:%p:%p:%p:%d:%d:%d:%d:%lld:%lld:%lld:%a:%d:%d:%d:%d:%d:%d:%d:%d:%lld:%d:%d:%d",
             sizeof(T), (int)bf16 + 2 * (int)x3 + 4 * (int)tf32, (const void *)Y, (void *)D, (void *)xfro, (void *)rmse, (void *)ctx->ws.base,
             (void *)d_off, m, K, s, L, (long long)n, (long long)tiles, (long long)ma.total_tiles, eps, iters,
             ctx->opt_mod_solve * 2 + ctx->opt_mod_mixed, ctx->opt_tile, ctx->opt_cluster * 4 + ctx->opt_sm_blocks,
             ctx->opt_autotune,
             (int)ctx->tuned.size(), (ctx->opt_replace * 4 + ctx->opt_omp_form) * 4 + ctx->opt_bf16_form,
             ctx->opt_wait_test, ctx->opt_wait_limit, ctx->opt_mod_check_ppb * 2048 + ctx->opt_a0_chunk_mb,
             ctx->opt_sel_spw * 4 + ctx->opt_sel_gcache, (int)ctx->tuned_sel.size());
    const std::string key(kb);
    auto hit = ctx->graphs.find(key);
    if (hit != ctx->graphs.end()) {
      SDL_CUDA(cudaGraphLaunch(hit->second.exec, sm), "graph launch");
      ctx->launches += hit->second.kernels;
    } else if (!ctx->graph_seen.count(key)) {
      if (ctx->graph_seen.size() >= 256) ctx->graph_seen.clear();
      ctx->graph_seen[key] = 1;
      if ((st = run_loop()) != SDL_OK) return st;
    } else {
      if (ctx->graphs.size() >= 16) clear_graphs(ctx);
      if (!ctx->capture_stream)
        SDL_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "capture stream");
      const int64_t before = ctx->launches;
      const cudaStream_t user = ctx->stream;
      SDL_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed), "graph capture");
      ctx->stream = sm = ctx->capture_stream;   // every launcher of the loop records into the capture
      st = run_loop();
      ctx->stream = sm = user;
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
      if (st != SDL_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st;
      }
      SDL_CUDA(ce, "graph capture end");
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      SDL_CUDA(ie, "graph instantiate");
      sdl_ctx::GraphEntry ent;
      ent.exec = exec;
      ent.kernels = ctx->launches - before;
      ctx->graphs[key] = ent;
      ctx->graph_seen[key] = 1;
      SDL_CUDA(cudaGraphLaunch(exec, sm), "graph launch");
    }
  }
  if (iters > 0) {
    if ((st = mod_status(ctx, worst, iters, d_max)) != SDL_OK) return st;
    if (tc) return tc_status(ctx, tc_err);
  }
  return SDL_OK;
}

}  // namespace
}  // namespace sdl

using namespace sdl;

extern "C" {

sdl_status sdl_create(sdl_ctx **out, int device, void *stream) {
  if (!out) return SDL_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SDL_EINVAL;
  }
  sdl_ctx *ctx = new sdl_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  DeviceGuard g(device);
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SDL_ECUDA;
  }
  *out = ctx;
  return SDL_OK;
}

sdl_status sdl_destroy(sdl_ctx *ctx) {
  if (!ctx) return SDL_OK;
  {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    prof_resolve(ctx);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    clear_graphs(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
  }
  delete ctx;
  return SDL_OK;
}

sdl_status sdl_set_stream(sdl_ctx *ctx, void *stream) {
  if (!ctx) return SDL_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return SDL_OK;
}

const char *sdl_last_error(const sdl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t sdl_workspace_bytes(const sdl_ctx *ctx) { return ctx ? ctx->ws.cap : 0; }

sdl_status sdl_omp_batched(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K, const void *Y,
                           const int64_t *offsets, int L, int s, double eps, int32_t *idx, void *val,
                           int32_t *nnz, void *resid2) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  if ((st = check_omp_shape(ctx, m, K, s, eps)) != SDL_OK) return st;
  if ((st = check_offsets(ctx, offsets, L, false)) != SDL_OK) return st;
  const int64_t n = offsets[L];
  if (n == 0) return SDL_OK;
  SDL_REQUIRE(aligned16(D) && aligned16(Y) && aligned16(idx) && aligned16(val) && aligned16(nnz) &&
                  (resid2 == nullptr || aligned16(resid2)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if ((st = ws_reserve(ctx, omp_ws_bytes(prec, L, K) + tc_ws_bytes(L, K, m, n) + 1024)) != SDL_OK) return st;
  OmpArgs a{};
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  const bool bf16 = prec == SDL_PREC_BF16, x3 = prec == SDL_PREC_F32X3 || prec == SDL_PREC_TF32;
  const bool split = prec == SDL_PREC_F32 && omp_split_f32(ctx, K, m, s);
  const int tile = bf16 || x3 || split ? omp_tc_tile_signals(K, m, s) : omp_tile_signals();
  if (tile <= 0) return set_error(ctx, SDL_EINVAL, "shape too large for the tensor-core OMP kernel");
  if ((st = upload_plan(ctx, offsets, L, tile, &d_off, &d_tiles, &tiles)) != SDL_OK)
    return st;
  void *G = ws_alloc(ctx, elem_size(prec) * (size_t)L * K * K);
  if (!G) return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  a.D = D; a.G = G; a.Y = Y; a.offsets = d_off; a.tile_start = d_tiles; a.total_tiles = tiles;
  a.a0_cap = (int64_t)ctx->opt_a0_chunk_mb << 20;
  a.L = L; a.m = m; a.K = K; a.s = s; a.eps = eps;
  a.idx = idx; a.val = val; a.nnz = nnz; a.resid2 = resid2;
  if (bf16 || x3) {
    void *img = ws_alloc(ctx, 3 * tc_image_bytes(L, K, m));
    int32_t *err = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * 4));
    float *a0c = static_cast<float *>(ws_alloc(ctx, tc_a0_bytes(L, K, n)));
    void *g16 = bf16 && ctx->opt_bf16_form == 3 ? ws_alloc(ctx, tc_g16_bytes(L, K)) : nullptr;
    if (!img || !err || !a0c || (bf16 && ctx->opt_bf16_form == 3 && !g16))
      return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
    SDL_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), ctx->stream), "err clear");
    cudaError_t e = bf16 ? run_omp_bf16(ctx, a, img, static_cast<float *>(G), err, a0c, g16)
                         : run_omp_x3(ctx, a, img, static_cast<float *>(G), err, a0c, prec == SDL_PREC_TF32);
    if (e == cudaErrorInvalidConfiguration)
      return set_error(ctx, SDL_EINVAL, "shape too large for the tensor-core OMP kernel");
    SDL_CUDA(e, bf16 ? "omp bf16" : (prec == SDL_PREC_TF32 ? "omp tf32" : "omp f32x3"));
    return tc_status(ctx, err);
  }
  if (prec == SDL_PREC_F64) {
    SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<double>(static_cast<const double *>(D), m, K, L, static_cast<double *>(G),
                                 ctx->stream); }), "gram");
    cudaError_t e = timed(ctx, "omp", 1, [&] { return launch_omp<double>(a, ctx->num_sms, ctx->stream); });
    if (e == cudaErrorInvalidConfiguration)
      return set_error(ctx, SDL_EINVAL, "shape too large for the FP64 OMP kernel's shared memory");
    SDL_CUDA(e, "omp");
  } else if (split) {
    float *a0c = static_cast<float *>(ws_alloc(ctx, tc_a0_bytes(L, K, n)));
    if (!a0c) return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
    SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<float>(static_cast<const float *>(D), m, K, L, static_cast<float *>(G),
                                ctx->stream); }), "gram");
    SDL_CUDA(run_omp_split(ctx, a, a0c), "omp");
  } else {
    SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<float>(static_cast<const float *>(D), m, K, L, static_cast<float *>(G),
                                ctx->stream); }), "gram");
    cudaError_t e = timed(ctx, "omp", 1, [&] { return launch_omp<float>(a, ctx->num_sms, ctx->stream); });
    if (e == cudaErrorInvalidConfiguration)
      return set_error(ctx, SDL_EINVAL, "shape too large for the OMP kernel's shared memory");
    SDL_CUDA(e, "omp");
  }
  return SDL_OK;
}

sdl_status sdl_omp(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K, const void *Y, int64_t n,
                   int s, double eps, int32_t *idx, void *val, int32_t *nnz, void *resid2) {
  if (!ctx) return SDL_EINVAL;
  if (n < 0) return set_error(ctx, SDL_EINVAL, "n must be >= 0");
  const int64_t offsets[2] = {0, n};
  return sdl_omp_batched(ctx, prec, D, m, K, Y, offsets, 1, s, eps, idx, val, nnz, resid2);
}

sdl_status sdl_mod_update_batched(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m,
                                  const int64_t *offsets, int L, const int32_t *idx, const void *val,
                                  int s, void *D, int K, int32_t *usage) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(m >= 1 && m <= kMaxM, "m must be in [1, 256]");
  SDL_REQUIRE(K >= 1 && K <= kMaxK, "K must be in [1, 1024]");
  SDL_REQUIRE(s >= 1 && s <= kMaxS, "s must be in [1, 32]");
  if ((st = check_offsets(ctx, offsets, L, false)) != SDL_OK) return st;
  const int64_t n = offsets[L];
  SDL_REQUIRE(aligned16(D) && (n == 0 || (aligned16(Y) && aligned16(idx) && aligned16(val))) &&
                  (usage == nullptr || aligned16(usage)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if ((st = ws_reserve(ctx, mod_ws_bytes(L, K, m, n, s) + 1024)) != SDL_OK) return st;
  ModArgs a{};
  int32_t *d_max = nullptr;
  if ((st = mod_prepare(ctx, a, offsets, L, K, m, s, usage, &d_max)) != SDL_OK) return st;
  a.Y = Y; a.idx = idx; a.val = val; a.D = D;
  SDL_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int32_t) * L, ctx->stream), "status clear");
  cudaStream_t sm = ctx->stream;
  const int nacc = mod_accum_kernels(prec != SDL_PREC_F64, a.total_tiles);
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "mod_accum", nacc, [&] { return launch_mod_accum<double>(a, sm); }), "mod accumulate");
  else
    SDL_CUDA(timed(ctx, "mod_accum", nacc, [&] { return launch_mod_accum<float>(a, sm); }), "mod accumulate");
  if (prec == SDL_PREC_F64) SDL_CUDA(run_mod_solve<double>(ctx, a), "mod solve");
  else SDL_CUDA(run_mod_solve<float>(ctx, a), "mod solve");
  return mod_status(ctx, a.status, L, d_max);
}

sdl_status sdl_replace_atoms(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, const int64_t *offsets,
                             int L, const int32_t *usage, const void *resid2, int min_use, void *D, int K,
                             int32_t *rep) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(prec != SDL_PREC_BF16, "atom replacement takes F32 or F64 data");
  SDL_REQUIRE(m >= 1 && m <= kMaxM, "m must be in [1, 256]");
  SDL_REQUIRE(K >= 1 && K <= kMaxK, "K must be in [1, 1024]");
  SDL_REQUIRE(min_use >= 0, "min_use must be >= 0");
  if ((st = check_offsets(ctx, offsets, L, false)) != SDL_OK) return st;
  const int64_t n = offsets[L];
  SDL_REQUIRE(n < ((int64_t)1 << 31), "more than 2^31 - 1 signals");
  SDL_REQUIRE(aligned16(D) && aligned16(usage) && (n == 0 || (aligned16(Y) && aligned16(resid2))) &&
                  (rep == nullptr || aligned16(rep)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if ((st = ws_reserve(ctx, 2 * round256(sizeof(int64_t) * (L + 1)) + 1024)) != SDL_OK) return st;
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  if ((st = upload_plan(ctx, offsets, L, 128, &d_off, &d_tiles, &tiles)) != SDL_OK) return st;
  cudaStream_t sm = ctx->stream;
  if (rep && min_use == 0)
    SDL_CUDA(cudaMemsetAsync(rep, 0xff, sizeof(int32_t) * (size_t)L * K, sm), "rep clear");
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "replace", min_use > 0 ? 1 : 0, [&] {
               return launch_replace_atoms<double>(static_cast<const double *>(Y), m, d_off, L, usage,
                                                   static_cast<const double *>(resid2), min_use,
                                                   static_cast<double *>(D), K, rep, sm);
             }), "atom replacement");
  else
    SDL_CUDA(timed(ctx, "replace", min_use > 0 ? 1 : 0, [&] {
               return launch_replace_atoms<float>(static_cast<const float *>(Y), m, d_off, L, usage,
                                                  static_cast<const float *>(resid2), min_use,
                                                  static_cast<float *>(D), K, rep, sm);
             }), "atom replacement");
  return SDL_OK;
}

sdl_status sdl_mod_update(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t n,
                          const int32_t *idx, const void *val, int s, void *D, int K, int32_t *usage) {
  if (!ctx) return SDL_EINVAL;
  if (n < 0) return set_error(ctx, SDL_EINVAL, "n must be >= 0");
  const int64_t offsets[2] = {0, n};
  return sdl_mod_update_batched(ctx, prec, Y, m, offsets, 1, idx, val, s, D, K, usage);
}

sdl_status sdl_split(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t N, const int64_t *perm,
                     void *Yp) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(m >= 1 && N >= 0, "m must be >= 1 and N >= 0");
  if (N == 0) return SDL_OK;
  SDL_REQUIRE(aligned16(Y) && aligned16(perm) && aligned16(Yp) && Y != Yp,
              "device pointers must be non-NULL, 16-byte aligned, and Yp must not alias Y");
  DeviceGuard g(ctx->device);
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "split", 1, [&] { return launch_split<double>(static_cast<const double *>(Y), m, N, perm, static_cast<double *>(Yp),
                                  ctx->stream); }), "split");
  else
    SDL_CUDA(timed(ctx, "split", 1, [&] { return launch_split<float>(static_cast<const float *>(Y), m, N, perm, static_cast<float *>(Yp),
                                 ctx->stream); }), "split");
  return SDL_OK;
}

sdl_status sdl_init_dict(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t nY,
                         const int64_t *pick, const void *fill, int64_t count, void *D) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(m >= 1 && count >= 0 && nY >= 0, "bad sizes");
  if (count == 0) return SDL_OK;
  SDL_REQUIRE(aligned16(pick) && aligned16(D) && (nY == 0 || aligned16(Y)) &&
                  (fill == nullptr || aligned16(fill)),
              "device pointers must be non-NULL and 16-byte aligned");
  (void)nY;
  DeviceGuard g(ctx->device);
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "init_dict", 1, [&] { return launch_init_dict<double>(static_cast<const double *>(Y), m, pick,
                                      static_cast<const double *>(fill), count, static_cast<double *>(D),
                                      ctx->stream); }), "init");
  else
    SDL_CUDA(timed(ctx, "init_dict", 1, [&] { return launch_init_dict<float>(static_cast<const float *>(Y), m, pick, static_cast<const float *>(fill),
                                     count, static_cast<float *>(D), ctx->stream); }), "init");
  return SDL_OK;
}

sdl_status sdl_local_train(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, const int64_t *offsets,
                           int L, int K1, int s1, double eps, int iters, void *D_local, double *xfro,
                           double *rmse) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  if ((st = check_omp_shape(ctx, m, K1, s1, eps)) != SDL_OK) return st;
  if ((st = check_offsets(ctx, offsets, L, true)) != SDL_OK) return st;
  SDL_REQUIRE(iters >= 0, "iters must be >= 0");
  SDL_REQUIRE(aligned16(Y) && aligned16(D_local) && aligned16(xfro) && (rmse == nullptr || aligned16(rmse)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  const int64_t n = offsets[L];
  if (prec == SDL_PREC_F64) {
    if ((st = ws_reserve(ctx, train_ws_bytes<double>(L, K1, m, n, s1, iters))) != SDL_OK) return st;
    return train_run<double>(ctx, static_cast<const double *>(Y), m, offsets, L, K1, s1, eps, iters,
                             static_cast<double *>(D_local), xfro, rmse);
  }
  if ((st = ws_reserve(ctx, train_ws_bytes<float>(L, K1, m, n, s1, iters))) != SDL_OK) return st;
  return train_run<float>(ctx, static_cast<const float *>(Y), m, offsets, L, K1, s1, eps, iters,
                          static_cast<float *>(D_local), xfro, rmse, prec);
}

sdl_status sdl_merge(sdl_ctx *ctx, sdl_precision prec, const void *D_local, const double *xfro, int m,
                     int K1, int L, const int32_t *pick, int K, int s2, double eps, int iters, void *D,
                     double *rmse) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  if ((st = check_omp_shape(ctx, m, K, s2, eps)) != SDL_OK) return st;
  SDL_REQUIRE(K1 >= 1 && L >= 1 && (int64_t)K1 * L < ((int64_t)1 << 31), "bad K1 or L");
  SDL_REQUIRE(iters >= 0, "iters must be >= 0");
  SDL_REQUIRE(aligned16(D_local) && aligned16(xfro) && (pick == nullptr || aligned16(pick)) && aligned16(D) &&
                  (rmse == nullptr || aligned16(rmse)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  const int64_t nt = (int64_t)K1 * L;
  const int64_t offsets[2] = {0, nt};
  const size_t es = elem_size(prec);
  const size_t train_b = prec == SDL_PREC_F64 ? train_ws_bytes<double>(1, K, m, nt, s2, iters)
                                              : train_ws_bytes<float>(1, K, m, nt, s2, iters);
  if ((st = ws_reserve(ctx, round256(es * (size_t)nt * m) + round256(sizeof(double)) + train_b)) != SDL_OK)
    return st;
  void *Yt = ws_alloc(ctx, es * (size_t)nt * m);       // Ytilde, carved before the training scratch
  double *xf_unused = static_cast<double *>(ws_alloc(ctx, sizeof(double)));
  if (!Yt || !xf_unused) return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  if (prec == SDL_PREC_F64) {
    SDL_CUDA(timed(ctx, "stack", 1, [&] { return launch_stack<double>(static_cast<const double *>(D_local), xfro, m, K1, L,
                                  static_cast<double *>(Yt), ctx->stream); }), "stack");
    if (pick)
      SDL_CUDA(timed(ctx, "pick_init", 1, [&] { return launch_pick_init<double>(static_cast<const double *>(Yt), m, pick, K, static_cast<double *>(D),
                                        ctx->stream); }), "merge init");
    return train_run<double>(ctx, static_cast<const double *>(Yt), m, offsets, 1, K, s2, eps, iters,
                             static_cast<double *>(D), xf_unused, rmse);
  }
  SDL_CUDA(timed(ctx, "stack", 1, [&] { return launch_stack<float>(static_cast<const float *>(D_local), xfro, m, K1, L, static_cast<float *>(Yt),
                               ctx->stream); }), "stack");
  if (pick)
    SDL_CUDA(timed(ctx, "pick_init", 1, [&] { return launch_pick_init<float>(static_cast<const float *>(Yt), m, pick, K, static_cast<float *>(D),
                                     ctx->stream); }), "merge init");
  return train_run<float>(ctx, static_cast<const float *>(Yt), m, offsets, 1, K, s2, eps, iters,
                          static_cast<float *>(D), xf_unused, rmse, prec);
}

sdl_status sdl_residual(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t n, const void *D,
                        int K, const int32_t *idx, const void *val, int s, double *out2) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(m >= 1 && m <= kMaxM && n >= 0 && K >= 1 && s >= 1 && s <= kMaxS,
              "bad sizes (m in [1, 256], s in [1, 32])");
  SDL_REQUIRE(aligned16(out2) && aligned16(D) && (n == 0 || (aligned16(Y) && aligned16(idx) && aligned16(val))),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "residual", 1, [&] { return launch_residual<double>(static_cast<const double *>(Y), m, n, static_cast<const double *>(D), idx,
                                     static_cast<const double *>(val), s, out2, ctx->stream); }), "residual");
  else
    SDL_CUDA(timed(ctx, "residual", 1, [&] { return launch_residual<float>(static_cast<const float *>(Y), m, n, static_cast<const float *>(D), idx,
                                    static_cast<const float *>(val), s, out2, ctx->stream); }), "residual");
  return SDL_OK;
}

sdl_status sdl_gram(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K, int L, void *G) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(m >= 1 && m <= kMaxM, "m must be in [1, 256]");
  SDL_REQUIRE(K >= 1 && K <= kMaxK, "K must be in [1, 1024]");
  SDL_REQUIRE(L >= 1, "L must be >= 1");
  SDL_REQUIRE(aligned16(D) && aligned16(G), "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  cudaStream_t sm = ctx->stream;
  if (prec == SDL_PREC_F64) {
    SDL_CUDA(timed(ctx, "gram", 1, [&] {
               return launch_gram<double>(static_cast<const double *>(D), m, K, L, static_cast<double *>(G), sm);
             }), "gram");
    return SDL_OK;
  }
  if (prec == SDL_PREC_F32) {
    SDL_CUDA(timed(ctx, "gram", 1, [&] {
               return launch_gram<float>(static_cast<const float *>(D), m, K, L, static_cast<float *>(G), sm);
             }), "gram");
    return SDL_OK;
  }
  if ((st = ws_reserve(ctx, round256(2 * tc_image_bytes(L, K, m)) + round256(sizeof(int32_t) * 4) + 1024)) !=
      SDL_OK)
    return st;
  void *img = ws_alloc(ctx, 2 * tc_image_bytes(L, K, m));
  int32_t *err = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * 4));
  if (!img || !err) return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  void *lo = static_cast<unsigned char *>(img) + tc_image_bytes(L, K, m);
  SDL_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), sm), "err clear");
  if (prec == SDL_PREC_F32X3 || prec == SDL_PREC_TF32) {   // TF32: the same FP32-accurate split Gram
    SDL_CUDA(timed(ctx, "x3_image", 1, [&] {
               return launch_x3_image(static_cast<const float *>(D), K, m, L, img, lo, sm);
             }), "tf32 image");
    SDL_CUDA(timed(ctx, "gram_x3", 1, [&] {
               return launch_gram_x3(static_cast<const float *>(D), img, lo, K, m, L, static_cast<float *>(G), err,
                                     ctx->num_sms, x3_wait(ctx), sm);
             }), "gram x3");
    return tc_status(ctx, err);
  }
  SDL_CUDA(timed(ctx, "bf16_image", 1, [&] {
             return launch_bf16_image(static_cast<const float *>(D), K, m, L, img, lo, sm);
           }), "bf16 image");
  cudaError_t e = timed(ctx, "gram_tc", 1, [&] {
    return launch_gram_tc(img, lo, K, m, L, static_cast<float *>(G), err, sm);
  });
  if (e == cudaErrorInvalidConfiguration) return set_error(ctx, SDL_EINVAL, "shape too large for the tensor-core Gram");
  SDL_CUDA(e, "gram tc");
  return tc_status(ctx, err);
}

sdl_status sdl_recovery(sdl_ctx *ctx, sdl_precision prec, const void *D0, int K0, const void *D, int K, int m,
                        double thresh, int32_t *count) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(K0 >= 1 && K >= 1 && m >= 1, "bad sizes");
  SDL_REQUIRE(aligned16(D0) && aligned16(D) && aligned16(count),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "recovery", 1, [&] { return launch_recovery<double>(static_cast<const double *>(D0), K0, static_cast<const double *>(D), K, m,
                                     thresh, count, ctx->stream); }), "recovery");
  else
    SDL_CUDA(timed(ctx, "recovery", 1, [&] { return launch_recovery<float>(static_cast<const float *>(D0), K0, static_cast<const float *>(D), K, m,
                                    thresh, count, ctx->stream); }), "recovery");
  return SDL_OK;
}

sdl_status sdl_extract_patches(sdl_ctx *ctx, sdl_precision prec, const void *img, int H, int W, int p,
                               void *patches) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(p >= 1 && p <= 16 && H >= p && W >= p, "need 1 <= p <= 16, p <= H, p <= W");
  SDL_REQUIRE(aligned16(img) && aligned16(patches), "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "extract_patches", 1, [&] {
               return launch_extract_patches<double>(static_cast<const double *>(img), H, W, p,
                                                     static_cast<double *>(patches), ctx->stream);
             }), "extract patches");
  else
    SDL_CUDA(timed(ctx, "extract_patches", 1, [&] {
               return launch_extract_patches<float>(static_cast<const float *>(img), H, W, p,
                                                    static_cast<float *>(patches), ctx->stream);
             }), "extract patches");
  return SDL_OK;
}

sdl_status sdl_patch_average(sdl_ctx *ctx, sdl_precision prec, const void *D, int K, const int32_t *idx,
                             const void *val, int s, int H, int W, int p, void *out) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(p >= 1 && p <= 16 && H >= p && W >= p && K >= 1 && s >= 1, "bad sizes");
  SDL_REQUIRE(aligned16(D) && aligned16(idx) && aligned16(val) && aligned16(out),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "patch_average", 1, [&] {
               return launch_patch_average<double>(static_cast<const double *>(D), K, idx,
                                                   static_cast<const double *>(val), s, H, W, p,
                                                   static_cast<double *>(out), ctx->stream);
             }), "patch average");
  else
    SDL_CUDA(timed(ctx, "patch_average", 1, [&] {
               return launch_patch_average<float>(static_cast<const float *>(D), K, idx,
                                                  static_cast<const float *>(val), s, H, W, p,
                                                  static_cast<float *>(out), ctx->stream);
             }), "patch average");
  return SDL_OK;
}

sdl_status sdl_sq_error(sdl_ctx *ctx, sdl_precision prec, const void *a, const void *b, int64_t n, double *out2) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  if ((st = check_prec(ctx, prec)) != SDL_OK) return st;
  SDL_REQUIRE(n >= 0, "bad size");
  SDL_REQUIRE(aligned16(out2) && (n == 0 || (aligned16(a) && aligned16(b))),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if (prec == SDL_PREC_F64)
    SDL_CUDA(timed(ctx, "sq_error", 1, [&] {
               return launch_sq_error<double>(static_cast<const double *>(a), static_cast<const double *>(b), n, out2,
                                              ctx->stream);
             }), "squared error");
  else
    SDL_CUDA(timed(ctx, "sq_error", 1, [&] {
               return launch_sq_error<float>(static_cast<const float *>(a), static_cast<const float *>(b), n, out2,
                                             ctx->stream);
             }), "squared error");
  return SDL_OK;
}

// One dictionary: the batched path with L = 1 and the proposer reading y.
sdl_status sdl_omp_proposed(sdl_ctx *ctx, sdl_proposer *p, const float *D, int m, int K, const float *Y, int64_t n,
                            int s, int ncand, double eps_fb, int32_t *idx, float *val, int32_t *nnz, float *resid2,
                            int64_t *n_fallback) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  if (n < 0) return set_error(ctx, SDL_EINVAL, "n must be >= 0");
  const int64_t offsets[2] = {0, n};
  return sdl_omp_proposed_batched(ctx, p, SDL_FEATURES_SIGNAL, D, m, K, Y, offsets, 1, s, ncand, eps_fb, idx, val,
                                  nnz, resid2, n_fallback);
}

sdl_status sdl_corr_features(sdl_ctx *ctx, const float *D, int m, int K, const float *Y, const int64_t *offsets,
                             int L, float *F) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  SDL_REQUIRE(m >= 1 && m <= kMaxM, "m must be in [1, 256]");
  SDL_REQUIRE(K >= 1 && K <= kMaxK, "K must be in [1, 1024]");
  if ((st = check_offsets(ctx, offsets, L, false)) != SDL_OK) return st;
  const int64_t n = offsets[L];
  if (n == 0) return SDL_OK;
  SDL_REQUIRE(aligned16(D) && aligned16(Y) && aligned16(F), "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  if ((st = ws_reserve(ctx, 2 * round256(sizeof(int64_t) * (L + 1)) + 1024)) != SDL_OK) return st;
  OmpArgs a{};
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  if ((st = upload_plan(ctx, offsets, L, 128, &d_off, &d_tiles, &tiles)) != SDL_OK) return st;
  a.D = D; a.Y = Y; a.offsets = d_off; a.tile_start = d_tiles; a.total_tiles = tiles;
  a.a0_cap = (int64_t)ctx->opt_a0_chunk_mb << 20;
  a.L = L; a.m = m; a.K = K;
  SDL_CUDA(timed(ctx, "corr_features", 1, [&] { return launch_corr_features(a, 0, tiles, 0, F, ctx->stream); }),
           "correlation features");
  return SDL_OK;
}

sdl_status sdl_omp_proposed_batched(sdl_ctx *ctx, sdl_proposer *p, int features, const float *D, int m, int K,
                                    const float *Y, const int64_t *offsets, int L, int s, int ncand, double eps_fb,
                                    int32_t *idx, float *val, int32_t *nnz, float *resid2, int64_t *n_fallback) {
  if (!ctx) return SDL_EINVAL;
  ctx->err.clear();
  sdl_status st;
  SDL_REQUIRE(p != nullptr && n_fallback != nullptr, "proposer and n_fallback must be given");
  SDL_REQUIRE(features == SDL_FEATURES_SIGNAL || features == SDL_FEATURES_CORR,
              "features must be SDL_FEATURES_SIGNAL or SDL_FEATURES_CORR");
  if ((st = check_omp_shape(ctx, m, K, s, 0.0)) != SDL_OK) return st;
  const bool corr = features == SDL_FEATURES_CORR;
  SDL_REQUIRE(proposer_m(p) == (corr ? K : m) && proposer_K(p) == K,
              "the proposer's sizes do not match: K outputs and m (signal) or K (correlation) inputs");
  SDL_REQUIRE(ncand >= s && ncand <= 32 && ncand <= K, "ncand must be in [s, min(32, K)]");
  SDL_REQUIRE(eps_fb >= 0.0 && isfinite(eps_fb), "eps_fb must be finite and >= 0");
  if ((st = check_offsets(ctx, offsets, L, false)) != SDL_OK) return st;
  *n_fallback = 0;
  const int64_t n = offsets[L];
  if (n == 0) return SDL_OK;
  SDL_REQUIRE(aligned16(D) && aligned16(Y) && aligned16(idx) && aligned16(val) && aligned16(nnz) &&
                  (resid2 == nullptr || aligned16(resid2)),
              "device pointers must be non-NULL and 16-byte aligned");
  DeviceGuard g(ctx->device);
  SDL_REQUIRE(g.ok, "cannot select the context device");
  const bool split = omp_split_f32(ctx, K, m, s);
  const int ftile = split ? omp_tc_tile_signals(K, m, s) : omp_tile_signals();
  // correlation features are formed per chunk of 512 tiles of 128 signals
  const int64_t kChunkTiles = 512;
  const int64_t frows = corr ? (n < kChunkTiles * 128 ? n : kChunkTiles * 128) : 0;
  const size_t plan_b = round256(sizeof(int64_t) * (L + 1)) + round256(sizeof(int32_t) * (L + 1));
  const size_t need = round256(sizeof(float) * (size_t)L * K * K) + round256(sizeof(int32_t) * (size_t)n * ncand) +
                      4 * round256(sizeof(int32_t) * (size_t)n) + round256(sizeof(int32_t) * (size_t)(2 * L + 1)) +
                      round256(sizeof(float) * (size_t)n * m) + 2 * round256(sizeof(int32_t) * (size_t)n * s) +
                      round256(sizeof(float) * (size_t)frows * K) + (split ? round256(tc_a0_bytes(L, K, n)) : 0) +
                      2 * plan_b + 4096;
  if ((st = ws_reserve(ctx, need)) != SDL_OK) return st;
  int64_t *d_off = nullptr;
  int32_t *d_tiles = nullptr;
  int64_t tiles = 0;
  if ((st = upload_plan(ctx, offsets, L, 128, &d_off, &d_tiles, &tiles)) != SDL_OK) return st;
  float *G = static_cast<float *>(ws_alloc(ctx, sizeof(float) * (size_t)L * K * K));
  int32_t *cand = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n * ncand));
  int32_t *flag = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n));
  int32_t *list = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n));
  int32_t *fn = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n));
  float *fr = static_cast<float *>(ws_alloc(ctx, sizeof(float) * (size_t)n));
  int32_t *cnt = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)(2 * L + 1)));
  float *Yf = static_cast<float *>(ws_alloc(ctx, sizeof(float) * (size_t)n * m));
  int32_t *fi = static_cast<int32_t *>(ws_alloc(ctx, sizeof(int32_t) * (size_t)n * s));
  float *fv = static_cast<float *>(ws_alloc(ctx, sizeof(float) * (size_t)n * s));
  float *F = corr ? static_cast<float *>(ws_alloc(ctx, sizeof(float) * (size_t)frows * K)) : nullptr;
  float *a0c = split ? static_cast<float *>(ws_alloc(ctx, tc_a0_bytes(L, K, n))) : nullptr;
  if (!G || !cand || !flag || !list || !fn || !fr || !cnt || !Yf || !fi || !fv || (corr && !F) || (split && !a0c))
    return set_error(ctx, SDL_ENOMEM, "workspace carve-up failed");
  int32_t *pos = cnt + L + 1;
  float *r2 = resid2 ? resid2 : fr;
  cudaStream_t sm = ctx->stream;
  if (!corr) {
    SDL_CUDA(timed(ctx, "proposer_topk", 5 * (int)((n + 65535) / 65536),
                   [&] { return proposer_topk(p, Y, n, ncand, cand, sm); }), "proposer scores");
  } else {
    // the rows of consecutive tiles are consecutive rows of Y
    const TilePlan plan = make_tiles(offsets, L, 128);
    auto subset_of_tile = [&](int64_t gt) {
      int lo = 0, hi = L - 1;   // largest t with tile_start[t] <= gt
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (plan.tile_start[mid] <= gt) lo = mid; else hi = mid - 1;
      }
      return lo;
    };
    OmpArgs fa{};
    fa.D = D; fa.Y = Y; fa.offsets = d_off; fa.tile_start = d_tiles; fa.total_tiles = tiles;
    fa.a0_cap = (int64_t)ctx->opt_a0_chunk_mb << 20;
    fa.L = L; fa.m = m; fa.K = K;
    for (int64_t g0 = 0; g0 < tiles; g0 += kChunkTiles) {
      const int64_t g1 = tiles - g0 < kChunkTiles ? tiles : g0 + kChunkTiles;
      const int t0 = subset_of_tile(g0), t1 = subset_of_tile(g1 - 1);
      const int64_t r0 = offsets[t0] + (g0 - plan.tile_start[t0]) * 128;
      const int64_t e1 = offsets[t1] + (g1 - plan.tile_start[t1]) * 128;
      const int64_t r1 = e1 < offsets[t1 + 1] ? e1 : offsets[t1 + 1];
      SDL_CUDA(timed(ctx, "corr_features", 1, [&] { return launch_corr_features(fa, g0, g1 - g0, r0, F, sm); }),
               "correlation features");
      SDL_CUDA(timed(ctx, "proposer_topk", 5, [&] { return proposer_topk(p, F, r1 - r0, ncand, cand + r0 * ncand, sm); }),
               "proposer scores");
    }
  }
  SDL_CUDA(timed(ctx, "gram", 1, [&] { return launch_gram<float>(D, m, K, L, G, sm); }), "gram");
  SDL_CUDA(timed(ctx, "omp_restricted", 1, [&] {
             return launch_romp(D, G, m, K, Y, n, s, ncand, cand, (float)eps_fb, idx, val, nnz, r2, flag, d_off, L,
                                sm);
           }), "restricted omp");
  SDL_CUDA(timed(ctx, "fallback_compact", 1, [&] { return launch_count_flags(flag, d_off, L, n, cnt, sm); }),
           "fallback count");
  std::vector<int32_t> hc((size_t)L + 1);
  SDL_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * (L + 1), cudaMemcpyDeviceToHost, sm), "count read");
  SDL_CUDA(cudaStreamSynchronize(sm), "count sync");
  const int64_t nf = hc[L];
  *n_fallback = nf;
  if (nf == 0) return SDL_OK;
  // full OMP on the flagged signals of each subset against its own dictionary
  std::vector<int64_t> fo((size_t)L + 1, 0);
  for (int t = 0; t < L; ++t) fo[t + 1] = fo[t] + hc[t];
  if (fo[L] != nf) return set_error(ctx, SDL_EINVAL, "fallback counts are inconsistent");
  int64_t *d_foff = nullptr;
  int32_t *d_ftiles = nullptr;
  int64_t ftiles = 0;
  if ((st = upload_plan(ctx, fo.data(), L, ftile, &d_foff, &d_ftiles, &ftiles)) != SDL_OK) return st;
  SDL_CUDA(timed(ctx, "fallback_compact", 1,
                 [&] { return launch_place_flags(flag, d_off, L, n, d_foff, pos, list, sm); }), "fallback place");
  SDL_CUDA(timed(ctx, "fallback_gather", 1, [&] { return launch_gather_rows(Y, m, list, cnt + L, nf, Yf, sm); }),
           "gather");
  OmpArgs a{};
  a.D = D; a.G = G; a.Y = Yf; a.offsets = d_foff; a.tile_start = d_ftiles; a.total_tiles = ftiles;
  a.L = L; a.m = m; a.K = K; a.s = s; a.eps = 0.0;
  a.idx = fi; a.val = fv; a.nnz = fn; a.resid2 = fr;
  if (split) {
    SDL_CUDA(timed(ctx, "omp_split", split_kernels(a), [&] { return launch_omp_split_f32(a, a0c, sm); }),
             "fallback omp");
  } else {
    SDL_CUDA(timed(ctx, "omp", 1, [&] { return launch_omp<float>(a, ctx->num_sms, sm); }), "fallback omp");
  }
  SDL_CUDA(timed(ctx, "fallback_scatter", 1, [&] {
             return launch_scatter_codes(list, cnt + L, nf, s, fi, fv, fn, fr, idx, val, nnz, resid2, sm);
           }), "scatter");
  return SDL_OK;
}

sdl_status sdl_profile_enable(sdl_ctx *ctx, int on) {
  if (!ctx) return SDL_EINVAL;
  ctx->prof.on = on != 0;
  return SDL_OK;
}

sdl_status sdl_profile_reset(sdl_ctx *ctx) {
  if (!ctx) return SDL_EINVAL;
  DeviceGuard g(ctx->device);
  prof_resolve(ctx);
  ctx->prof.entries.clear();
  return SDL_OK;
}

int sdl_profile_count(sdl_ctx *ctx) {
  if (!ctx) return -1;
  DeviceGuard g(ctx->device);
  prof_resolve(ctx);
  return (int)ctx->prof.entries.size();
}

sdl_status sdl_profile_entry(sdl_ctx *ctx, int i, const char **name, int64_t *launches, int64_t *calls,
                             double *total_ms) {
  if (!ctx || i < 0 || !name || !launches || !calls || !total_ms) return SDL_EINVAL;
  DeviceGuard g(ctx->device);
  prof_resolve(ctx);
  if (i >= (int)ctx->prof.entries.size()) return SDL_EINVAL;
  const ProfEntry &e = ctx->prof.entries[i];
  *name = e.name.c_str();
  *launches = e.launches;
  *calls = e.calls;
  *total_ms = e.ms;
  return SDL_OK;
}

int64_t sdl_launch_count(const sdl_ctx *ctx) { return ctx ? ctx->launches : -1; }

sdl_status sdl_set_option(sdl_ctx *ctx, int option, int64_t value) {
  if (!ctx) return SDL_EINVAL;
  switch (option) {
    case SDL_OPT_MOD_SOLVE:
      if (value < 0 || value > 4) return set_error(ctx, SDL_EINVAL, "SDL_OPT_MOD_SOLVE takes 0 to 4");
      ctx->opt_mod_solve = (int)value;
      return SDL_OK;
    case SDL_OPT_CLUSTER:
      if (value < 0 || value > 1024)
        return set_error(ctx, SDL_EINVAL, "SDL_OPT_CLUSTER takes 0 to 1024 (above 16: the wide form only)");
      ctx->opt_cluster = (int)value;
      return SDL_OK;
    case SDL_OPT_MOD_TILE:
      if (value != 0 && value != 16 && value != 32 && value != 64)
        return set_error(ctx, SDL_EINVAL, "SDL_OPT_MOD_TILE takes 0, 16, 32 or 64");
      ctx->opt_tile = (int)value;
      return SDL_OK;
    case SDL_OPT_AUTOTUNE:
      if (value != 0 && value != 1) return set_error(ctx, SDL_EINVAL, "SDL_OPT_AUTOTUNE takes 0 or 1");
      ctx->opt_autotune = (int)value;
      if (!value) {
        ctx->tuned.clear();
        ctx->tuned_sel.clear();
      }
      return SDL_OK;
    case SDL_OPT_SM_BLOCKS:
      if (value < 0 || value > 3) return set_error(ctx, SDL_EINVAL, "SDL_OPT_SM_BLOCKS takes 0 to 3");
      ctx->opt_sm_blocks = (int)value;
      return SDL_OK;
    case SDL_OPT_REPLACE:
      if (value < 0 || value > ((int64_t)1 << 30))
        return set_error(ctx, SDL_EINVAL, "SDL_OPT_REPLACE takes 0 to 2^30");
      ctx->opt_replace = (int)value;
      return SDL_OK;
    case SDL_OPT_OMP_FORM:
      if (value < 0 || value > 2) return set_error(ctx, SDL_EINVAL, "SDL_OPT_OMP_FORM takes 0, 1 or 2");
      ctx->opt_omp_form = (int)value;
      return SDL_OK;
    case SDL_OPT_WAIT_LIMIT:
      if (value < 1) return set_error(ctx, SDL_EINVAL, "SDL_OPT_WAIT_LIMIT takes a positive poll count");
      ctx->opt_wait_limit = (long long)value;
      return SDL_OK;
    case SDL_OPT_WAIT_TEST:
      if (value != 0 && value != 1) return set_error(ctx, SDL_EINVAL, "SDL_OPT_WAIT_TEST takes 0 or 1");
      ctx->opt_wait_test = (int)value;
      return SDL_OK;
    case SDL_OPT_A0_CHUNK_MB:
      if (value < 0 || value > 1024) return set_error(ctx, SDL_EINVAL, "SDL_OPT_A0_CHUNK_MB takes 0 to 1024");
      ctx->opt_a0_chunk_mb = (int)value;
      return SDL_OK;
    case SDL_OPT_SEL_SPW:
      if (value != 0 && value != 1 && value != 2 && value != 4)
        return set_error(ctx, SDL_EINVAL, "SDL_OPT_SEL_SPW takes 0, 1, 2 or 4");
      ctx->opt_sel_spw = (int)value;
      return SDL_OK;
    case SDL_OPT_SEL_GCACHE:
      if (value < 0 || value > 2) return set_error(ctx, SDL_EINVAL, "SDL_OPT_SEL_GCACHE takes 0, 1 or 2");
      ctx->opt_sel_gcache = (int)value;
      return SDL_OK;
    case SDL_OPT_MOD_CHECK_TOL:
      if (value < 1 || value > 1000000000)
        return set_error(ctx, SDL_EINVAL, "SDL_OPT_MOD_CHECK_TOL takes 1 to 10^9 (parts per 10^9)");
      ctx->opt_mod_check_ppb = (int)value;
      return SDL_OK;
    case SDL_OPT_MOD_MIXED:
      if (value != 0 && value != 1) return set_error(ctx, SDL_EINVAL, "SDL_OPT_MOD_MIXED takes 0 or 1");
      ctx->opt_mod_mixed = (int)value;
      return SDL_OK;
    case SDL_OPT_BF16_FORM:
      if (value < 0 || value > 3) return set_error(ctx, SDL_EINVAL, "SDL_OPT_BF16_FORM takes 0 to 3");
      ctx->opt_bf16_form = (int)value;
      return SDL_OK;
    case SDL_OPT_GRAPH:
      if (value != 0 && value != 1) return set_error(ctx, SDL_EINVAL, "SDL_OPT_GRAPH takes 0 or 1");
      ctx->opt_graph = (int)value;
      if (!value) clear_graphs(ctx);
      return SDL_OK;
    default:
      return set_error(ctx, SDL_EINVAL, "unknown option");
  }
}

}  // extern "C"
