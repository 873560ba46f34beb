// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "sdl.h"

namespace sdl {

// Upper limits of the compiled kernels.
constexpr int kMaxM = 256;      // signal length
constexpr int kMaxK = 1024;     // atoms per dictionary
constexpr int kMaxS = 32;       // sparsity (one lane per selected atom)

// Pivot floors: an OMP atom whose squared distance to span(D_S) is below this
// fraction of its squared norm is not added; a MOD normal-equation pivot below
// this fraction of its diagonal counts as a breakdown.
constexpr double kOmpPivotRelF64 = 1e-10;
constexpr float kOmpPivotRelF32 = 1e-6f;
constexpr double kModPivotRel = 1e-12;
constexpr double kModRidge = 1e-10;

// Device workspace: one cudaMalloc'd block, carved by a bump allocator that is
// reset at the start of every public call.
struct Workspace {
  char *base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  size_t want = 0;     // bytes the current call asked for (to size a regrowth)
};

// Per-kernel instrumentation: CUDA-event pairs on the context stream around
// each launcher, resolved lazily when read.
struct ProfEntry {
  std::string name;
  int64_t launches = 0;
  int64_t calls = 0;
  double ms = 0.0;
};
struct ProfPending {
  int entry;
  cudaEvent_t e0, e1;
};
struct Prof {
  bool on = false;
  std::vector<ProfEntry> entries;
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> pool;
};

}  // namespace sdl

struct sdl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  sdl::Workspace ws;
  int num_sms = 0;
  int32_t *h_status = nullptr;   // pinned host word for device status read-back
  int64_t launches = 0;          // kernels launched by this context
  sdl::Prof prof;
  int opt_mod_solve = 0;         // 0 auto, 1 DSMEM cluster, 2 block per subset, 3 tiled
  int opt_cluster = 0;           // 0 = automatic
  int opt_tile = 0;              // tiled solve: 16, 32 or 0 = automatic
  int opt_sm_blocks = 0;         // tiled solve: blocks per SM cap (0 = none) when set by hand
  std::map<int64_t, int> occ;    // cached max active clusters of the tiled solve
  int opt_autotune = 1;          // time candidate launch shapes on first use
  struct TunedSolve {
    int ts, C, cap;
    int wide;    // 1: the wide form with C blocks per subset
    int mixed;   // 1: the checked FP32 pass (tile ts, cluster C), then the FP64 solve of what it left
  };
  std::map<std::string, TunedSolve> tuned;   // shape key -> chosen tile, cluster size, blocks-per-SM cap
  int opt_graph = 0;             // replay training loops as captured CUDA graphs
  int opt_replace = 0;           // atom replacement after every MOD update: min_use (0 = off)
  int opt_omp_form = 0;          // FP32 OMP: 0 automatic, 1 fused kernel, 2 correlation GEMM + selection
  int opt_bf16_form = 0;         // BF16 OMP: 0 automatic, 1 Batch-OMP selection, 2 residual form,
                                 // 3 Batch-OMP with a half-precision Gram copy in the running update
  long long opt_wait_limit = 1ll << 24;   // polls before a barrier wait of the wide solve gives up
  int opt_wait_test = 0;         // 1: one block of each wide-solve group leaves at once
  int opt_mod_mixed = 1;         // FP32 data: 1 the checked FP32 pass of the tiled solve may run, 0 FP64 only
  int opt_mod_check_ppb = 20000; // tolerance of that check, parts per 10^9 of each atom's norm
  int opt_a0_chunk_mb = 0;       // alpha0 scratch chunk of the two-kernel coding passes, MB (0: automatic)
  int opt_sel_spw = 0;           // selection launch: signals per warp (0 automatic, 1, 2, 4)
  int opt_sel_gcache = 0;        // selection launch: G-column cache (0 automatic, 1 as fits, 2 none)
  struct TunedSelect {
    int spw, gcn;
  };
  std::map<std::string, TunedSelect> tuned_sel;   // coding-pass shape key -> selection launch shape
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
  };
  std::map<std::string, GraphEntry> graphs;   // call key -> instantiated training loop
  cudaStream_t capture_stream = nullptr;       // graphs are captured here (never the legacy stream)
  std::map<std::string, int> graph_seen;      // call keys run once eagerly
};

namespace sdl {

// --- error plumbing ------------------------------------------------------------
sdl_status set_error(sdl_ctx *ctx, sdl_status st, const std::string &msg);
sdl_status check_cuda(sdl_ctx *ctx, cudaError_t e, const char *what);

// Reserve `bytes` (256-byte aligned) from the workspace; grows it if needed.
// Returns nullptr and sets ctx->err on failure.
void *ws_alloc(sdl_ctx *ctx, size_t bytes);
void ws_reset(sdl_ctx *ctx);

// Tiles of a batched signal range: tile_start[t] = first tile of subset t.
struct TilePlan {
  std::vector<int32_t> tile_start;   // L+1 entries
  int64_t total_tiles = 0;
};
TilePlan make_tiles(const int64_t *offsets, int L, int tile);

// --- kernel launchers (templated on the data type T = float or double) ------
template <typename T>
cudaError_t launch_gram(const T *D, int m, int K, int L, T *G, cudaStream_t st);

struct OmpArgs {
  const void *D;          // [L][K][m]
  const void *G;          // [L][K][K]
  const void *Y;          // [n][m]
  const int64_t *offsets; // device [L+1]
  const int32_t *tile_start;  // device [L+1]
  int64_t total_tiles;
  int L, m, K, s;
  double eps;
  int32_t *idx;
  void *val;
  int32_t *nnz;
  void *resid2;           // may be null
  // tensor-core paths only
  int32_t *err;           // device word: bit 0 set when a bounded wait gave up
  int64_t a0_cap;         // bytes of one alpha0 scratch chunk (0: 1 GiB)
  const void *G16;        // BF16 path: half-precision copy of G for the running update (or null)
  // shape of the two-kernel selection launch (the autotuner's knobs; the
  // results do not depend on them): signals per warp (1, 2 or 4; 0: 4) and
  // the G columns cached per warp (0: as many as fit, -1: none, k: at most k)
  int sel_spw, sel_gcn;
};
template <typename T>
cudaError_t launch_omp(const OmpArgs &a, int num_sms, cudaStream_t st);
int omp_tile_signals();

// Bounds of the tensor-core kernels' mbarrier waits: limit polls each; with
// leave set the loader role leaves at once, so that the other roles' waits run
// out (a test).
struct X3Wait {
  int limit;
  int leave;
};

// BF16 tensor-core path (tcgen05 + TMEM, operands fed by bulk TMA copies).
inline int round16(int x) { return (x + 15) & ~15; }
// BF16 images of D: hi = bf16(d) and (lo_img not null) lo = bf16(d - hi).
cudaError_t launch_bf16_image(const float *D, int K, int m, int L, void *img, void *lo_img, cudaStream_t st);
// G = hi hi^T + hi lo^T + lo hi^T per dictionary on the tensor cores (FP32
// accumulation, about 2^-16 relative to the exact Gram of D).
// G16 (or null): a half-precision copy of G written beside it.
cudaError_t launch_gram_tc(const void *hi, const void *lo, int K, int m, int L, float *G, int32_t *err,
                           cudaStream_t st, void *G16 = nullptr);
// Correlations of 128-signal tiles on the tensor cores into the scratch a0c
// (omp_tc_chunk_tiles tiles of 128 x K floats at a time) by a persistent kernel
// (num_sms blocks at most) reading the slab image img of D (launch_rtc_image),
// then the selection loop from there.
cudaError_t launch_omp_tc(const OmpArgs &a, const void *img, float *a0c, int num_sms, const X3Wait &w,
                          cudaStream_t st);
int omp_tc_tile_signals(int K, int m, int s);
// Residual-form OMP on the tensor cores (same 128-signal tiles, same BF16
// images and FP32 Gram): D^T r of every step by tcgen05 into TMEM, picks,
// Cholesky rows and FP32 residuals per signal.  Shapes: s <= 16, m <= 256.
bool omp_rtc_supported(int K, int m, int s);
// The slab image of D that it and the correlation kernel read:
// [L][round64(m)/64][round256(K)][64] BF16, 256-atom x 64-entry slabs
// (rtc_image_bytes(L, K, m) bytes).
size_t rtc_image_bytes(int L, int K, int m);
cudaError_t launch_rtc_image(const float *D, int K, int m, int L, void *img, cudaStream_t st);
cudaError_t launch_omp_rtc(const OmpArgs &a, const void *img, cudaStream_t st);
// The selection kernel over 128-signal tiles tile0 .. tile0+ntile-1 whose
// alpha0 rows are in a0c (FP32 data).  exact: alpha0 came from BF16 products,
// so the coefficients are refitted from D_S^T y.
// h16: the running update reads the half copy a.G16 of the Gram.
cudaError_t launch_omp_select(const OmpArgs &a, const float *a0c, int64_t tile0, int64_t ntile, bool exact,
                              cudaStream_t st, bool h16 = false);
// FP32 OMP in two kernels: FFMA correlation GEMM of 128-signal tiles into a0c,
// then the selection kernel (same plan and scratch as the BF16 path).
cudaError_t launch_omp_split_f32(const OmpArgs &a, float *a0c, cudaStream_t st);
// G_t = D_t D_t^T with the correlation GEMM's 128 x 128 register-tiled blocks
// (used by launch_gram<float> when there are enough blocks to fill the GPU).
cudaError_t launch_gram_f32_tiles(const float *D, int m, int K, int L, float *G, cudaStream_t st);
// Tiles per chunk of the alpha0 scratch: at most cap bytes (0: 1 GiB), at least one tile.
int64_t omp_tc_chunk_tiles(int K, int64_t total_tiles, int64_t cap = 0);
// FP32-accurate tensor-core path (3 x TF32): hi = tf32(d), lo = tf32(d - hi)
// images of D [L][round32(m)/32][round128(K)][32] (x3_image_bytes each), the
// Gram and the correlations as hi hi^T + hi lo^T + lo hi^T with FP32
// accumulation, then the FP32 selection kernel from the alpha0 scratch.
// num_sms sizes the persistent grid; err as for the BF16 kernels; w bounds
// every mbarrier wait.
size_t x3_image_bytes(int L, int K, int m);
cudaError_t launch_x3_image(const float *D, int K, int m, int L, void *hi, void *lo, cudaStream_t st);
cudaError_t launch_gram_x3(const float *D, const void *hi, const void *lo, int K, int m, int L, float *G,
                           int32_t *err, int num_sms, const X3Wait &w, cudaStream_t st);
// single: the correlations from hi hi^T alone, one TF32 product (SDL_PREC_TF32;
// the Gram stays the three-product split).
cudaError_t launch_omp_x3(const OmpArgs &a, const void *hi, const void *lo, float *a0c, int num_sms,
                          const X3Wait &w, cudaStream_t st, bool single = false);
// Correlation features F = |D_t^T y| (FP32 FMA chains) of the 128-signal tiles
// tile0 .. tile0+ntile-1 of the plan; signal row r goes to row r - row_base of F.
cudaError_t launch_corr_features(const OmpArgs &a, int64_t tile0, int64_t ntile, int64_t row_base, float *F,
                                 cudaStream_t st);

struct ModArgs {
  const void *Y;          // [n][m]
  const int64_t *offsets; // device [L+1]
  const int32_t *tile_start;  // device [L+1] (tiles of kModTile signals)
  int64_t total_tiles;
  int64_t n;
  int L, m, K, s;
  const int32_t *idx;
  const void *val;
  void *D;                // [L][K][m] in/out
  int32_t *usage;         // [L][K] out (always provided internally)
  // FP64 scratch
  int32_t *cursor;        // [L][K]
  int32_t *ptr;           // [L][K+1]
  int32_t *lsig;          // [n*s]
  int32_t *lslot;         // [n*s]
  int32_t *latom;         // [n*s] atom of each CSC entry
  double *A;              // [L][K][K]
  double *Lf;             // [L][K][K]
  double *B;              // [L][K][m]
  int32_t *status;        // [L] out: 0 ok, 1 ridge used, 2 breakdown
  int32_t *status_max;    // may be null: the tiled solve folds max(status) into it
};
// MOD in four launchers: accumulation (usage count, scan, CSC fill, A/B
// accumulation: 4 kernels), FP64 Cholesky, FP64 solve, renormalisation.
template <typename T>
cudaError_t launch_mod_accum(const ModArgs &a, cudaStream_t st);
cudaError_t launch_mod_chol(const ModArgs &a, cudaStream_t st);
cudaError_t launch_mod_solve(const ModArgs &a, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t launch_mod_normalise(const ModArgs &a, cudaStream_t st);
// Cholesky + solve + renormalisation in one launch, one thread-block cluster
// of `cluster` (16 or 8) CTAs per subset; K <= 512.  Returns
// cudaErrorNotSupported when the shape or the device does not allow it.
template <typename T>
cudaError_t launch_mod_solve_cluster(const ModArgs &a, int cluster, cudaStream_t st);
int mod_tile_signals();
// Tiled FP64 factorisation + solve + renormalisation, one cluster of C (1..16)
// blocks per subset, TS x TS tiles (16 or 32); scratch in a.Lf of
// mod_tiled_scratch_doubles(L, K, m) doubles.
// cap: at most that many blocks per SM (1..3, through padded dynamic shared
// memory), 0 = as many as fit.  num_sms decides whether every block has an SM
// to itself (then the block factoring a diagonal tile takes no trailing tile).
// only_deferred: solve only the subsets whose status is 4 (left by the FP32
// pass below), the others untouched.
template <typename T>
cudaError_t launch_mod_tiled(const ModArgs &a, int ts, int C, int cap, int num_sms, cudaStream_t st,
                             bool only_deferred = false);
// The FP32 pass of the checked mixed-precision solve (FP32 data): the same
// tiled factorisation and solve in FP32 over the same scratch (laid out in
// floats), the unnormalised solution left there; status 0, or 4 where a
// squared pivot fell to 1e-3 of its diagonal (then the FP64 solve takes it).
template <typename T>
cudaError_t launch_mod_tiled32(const ModArgs &a, int ts, int C, int cap, int num_sms, cudaStream_t st);
// The check of that pass: per subset, the error of every used atom estimated
// from 8 random-sign probes of the FP64 residual D A - B mapped through the
// FP32 factor; accepted subsets (every estimated error norm at most tau of the
// atom's norm) are renormalised and written with status 0, the others get status 4.
// ts: the tile edge the FP32 pass ran with.  K <= 1024, m <= 256.
template <typename T>
cudaError_t launch_mod_check(const ModArgs &a, int ts, float tau, cudaStream_t st);
template <typename T>
int mod_tiled_max_clusters(int ts, int C, int cap, bool f32 = false);
size_t mod_tiled_scratch_doubles(int L, int K, int m);
// The wide form of the tiled solve for few subsets: the tile tasks of each
// subset spread over G blocks of a cooperative launch that meet at barriers in
// global memory.  Status 3 when a barrier wait gave up (after `spin` polls of
// 64 ns); absent >= 0 makes that rank of each group leave at once (the test of
// the bounded waits), -1 normally.
template <typename T>
cudaError_t launch_mod_wide(const ModArgs &a, int ts, int G, long long spin, int absent, cudaStream_t st);
template <typename T>
int mod_wide_max_blocks(int ts, int num_sms);

template <typename T>
cudaError_t launch_split(const T *Y, int m, int64_t N, const int64_t *perm, T *Yp, cudaStream_t st);
template <typename T>
cudaError_t launch_init_dict(const T *Y, int m, const int64_t *pick, const T *fill, int64_t count,
                             T *D, cudaStream_t st);
template <typename T>
cudaError_t launch_stack(const T *Dloc, const double *xfro, int m, int K1, int L, T *Yt,
                         cudaStream_t st);
template <typename T>
cudaError_t launch_pick_init(const T *Yt, int m, const int32_t *pick, int K, T *D, cudaStream_t st);
// Per-subset sums: rmse[t] = sqrt(sum resid2 / (m n_t)); xfro[t] = sqrt(sum val^2).
template <typename T>
cudaError_t launch_subset_stats(const T *resid2, const T *val, const int64_t *offsets, int L, int m,
                                int s, double *rmse_out, int64_t rmse_stride, double *xfro_out,
                                cudaStream_t st);
template <typename T>
cudaError_t launch_residual(const T *Y, int m, int64_t n, const T *D, const int32_t *idx,
                            const T *val, int s, double *out2, cudaStream_t st);
template <typename T>
cudaError_t launch_recovery(const T *D0, int K0, const T *D, int K, int m, double thresh,
                            int32_t *count, cudaStream_t st);
cudaError_t launch_status_max(const int32_t *status, int L, int32_t *out, cudaStream_t st);
// Atom replacement (replace.cu): atoms of subset t used by fewer than min_use
// signals become the worst-coded signals of the subset, normalised; rep[L][K]
// (may be null) receives the signal row or -1.  offsets on the device.  K <= 1024.
template <typename T>
cudaError_t launch_replace_atoms(const T *Y, int m, const int64_t *offsets, int L, const int32_t *usage,
                                 const T *resid2, int min_use, T *D, int K, int32_t *rep, cudaStream_t st);
// Denoising (denoise.cu).
template <typename T>
cudaError_t launch_extract_patches(const T *img, int H, int W, int p, T *out, cudaStream_t st);
template <typename T>
cudaError_t launch_patch_average(const T *D, int K, const int32_t *idx, const T *val, int s, int H, int W, int p,
                                 T *out, cudaStream_t st);
template <typename T>
cudaError_t launch_sq_error(const T *a, const T *b, int64_t n, double *out2, cudaStream_t st);

// Learned support proposer (proposer.cu).
int proposer_m(const sdl_proposer *p);
int proposer_K(const sdl_proposer *p);
// Scores of n signals (chunked forward passes) and their top-c atoms cand [n][c].
cudaError_t proposer_topk(sdl_proposer *p, const float *Y, int64_t n, int c, int32_t *cand, cudaStream_t st);
// OMP restricted to the candidates; flag[i] = 1 where ||r|| > eps_fb.
// offsets (device [L+1]) null: one dictionary; else signal i uses D_t(i), G_t(i).
cudaError_t launch_romp(const float *D, const float *G, int m, int K, const float *Y, int64_t n, int s, int c,
                        const int32_t *cand, float eps_fb, int32_t *idx, float *val, int32_t *nnz, float *resid2,
                        int32_t *flag, const int64_t *offsets, int L, cudaStream_t st);
// Flagged signals by subset: cnt[t] (device [L+1], cnt[L] = total), then
// list[foff[t] + k] for the k-th flagged signal of subset t (pos: device [L]).
cudaError_t launch_count_flags(const int32_t *flag, const int64_t *offsets, int L, int64_t n, int32_t *cnt,
                               cudaStream_t st);
cudaError_t launch_place_flags(const int32_t *flag, const int64_t *offsets, int L, int64_t n, const int64_t *foff,
                               int32_t *pos, int32_t *list, cudaStream_t st);
cudaError_t launch_gather_rows(const float *Y, int m, const int32_t *list, const int32_t *count, int64_t nmax,
                               float *Yf, cudaStream_t st);
cudaError_t launch_scatter_codes(const int32_t *list, const int32_t *count, int64_t nmax, int s, const int32_t *fi,
                                 const float *fv, const int32_t *fn, const float *fr, int32_t *idx, float *val,
                                 int32_t *nnz, float *resid2, cudaStream_t st);

}  // namespace sdl
