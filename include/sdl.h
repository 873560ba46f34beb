/*
 * sdl.h -- C ABI of the GB300 (sm_103a) split-and-merge dictionary-learning library.
 *
 * The library implements the data-parallel hot path of "A split-and-merge
 * dictionary learning algorithm for sparse representation" (Mukherjee and
 * Seelamantula, arXiv 1403.4781): OMP sparse coding (Sec. 1; error-constrained
 * form Sec. 3.2.2), the MOD dictionary update with column renormalisation
 * (Sec. 1, Sec. 3.1), and Algorithm 1 (split, independent local training,
 * scaled-stack merge).
 *
 * Conventions shared by every call
 *  - Matrices are column-major with one signal or one atom contiguous:
 *    Y in R^{m x n} is n*m elements, signal i at Y + i*m; D in R^{m x K} is K*m
 *    elements, atom j at D + j*m.  Sparse codes are ELL: idx[i*s + k] (atom,
 *    -1 pads, selection order), val[i*s + k], nnz[i].
 *  - "device" pointers must be addresses in the context device's memory (e.g.
 *    torch tensors); "host" pointers are ordinary CPU memory.  The caller owns
 *    every buffer it passes; the library never frees or retains them beyond the
 *    call.  Device pointers must be 16-byte aligned.
 *  - Element type: SDL_PREC_F64 uses double for D, Y, val and resid2; the other
 *    precisions use float.  Accumulators of the MOD normal equations are
 *    always FP64; their Cholesky factor and solve are FP64, or for FP32 data an
 *    FP32 pass whose error is checked against the FP64 residual per subset
 *    (SDL_OPT_MOD_MIXED).
 *  - Every call enqueues its kernels on the context's stream and returns a
 *    status.  Calls that can report a device-side condition (Cholesky breakdown)
 *    synchronise that stream before returning.  A call may grow the context's
 *    device workspace (cudaMalloc, synchronising) the first time it sees a
 *    larger shape.
 *  - Errors: SDL_EINVAL for a null pointer, a bad size or option (message via
 *    sdl_last_error); SDL_ENOTPD when the MOD normal equations of some subset
 *    are not positive definite even after the ridge retry (that subset's atoms
 *    keep their previous values); SDL_ECUDA for a CUDA runtime error;
 *    SDL_ENOMEM when the workspace cannot be allocated.  On SDL_EINVAL nothing
 *    is launched.
 */
#ifndef SDL_H
#define SDL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SDL_OK = 0,
  SDL_EINVAL = 1,
  SDL_ENOTPD = 2,
  SDL_ETIMEOUT = 3,
  SDL_ECUDA = 4,
  SDL_ENOMEM = 5,
  SDL_ERANGE = 6   /* a size exceeds the fixed limit of sdl_omp_noalloc */
} sdl_status;

typedef enum {
  /* FP64 data and FP64 arithmetic everywhere. */
  SDL_PREC_F64 = 0,
  /* FP32 data; correlations, Gram and the OMP loop in FP32 (CUDA cores);
     coefficients recomputed on the support with one refinement step. */
  SDL_PREC_F32 = 1,
  /* FP32 data; correlations from BF16 operands on the tensor cores with
     FP32 accumulation; the Gram on the tensor cores from a two-term BF16 split
     of D (about 2^-16); coefficients on the support corrected by one FP32
     refinement step (residual from D_S and y in FP32), which removes the BF16
     rounding they inherit from the correlations. */
  SDL_PREC_BF16 = 2,
  /* FP32 data; correlations and Gram on the tensor cores from a two-term TF32
     split of both operands (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)),
     hi hi^T + hi lo^T + lo hi^T with FP32 accumulation: within 3 2^-22 of each
     |x_i z_i| plus the FP32 accumulation, the accuracy of the FP32 CUDA-core
     sum; the OMP loop, refit and refinement step as for SDL_PREC_F32. */
  SDL_PREC_F32X3 = 3,
  /* FP32 data; correlations from one TF32 product on the tensor cores
     (kind::tf32, each operand rounded to 11 significant bits: within 2 2^-11
     of each |x_i z_i| plus the FP32 accumulation), the Gram from the
     three-product split as for SDL_PREC_F32X3; coefficients on the support
     corrected by one FP32 refinement step, as for SDL_PREC_BF16. */
  SDL_PREC_TF32 = 4
} sdl_precision;

typedef struct sdl_ctx sdl_ctx;

/* Create a context on CUDA device `device` that enqueues on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the handle. */
sdl_status sdl_create(sdl_ctx **ctx, int device, void *stream);
/* Free the context's workspace and the handle (NULL is accepted). */
sdl_status sdl_destroy(sdl_ctx *ctx);
/* Change the stream later calls enqueue on. */
sdl_status sdl_set_stream(sdl_ctx *ctx, void *stream);
/* Text of the last error on this context ("" if none).  Owned by the context. */
const char *sdl_last_error(const sdl_ctx *ctx);
/* Bytes of device workspace the context currently holds. */
size_t sdl_workspace_bytes(const sdl_ctx *ctx);

/* OMP sparse coding (Sec. 1; stop rule of Sec. 3.2.2).  For every signal y_i:
 * r = y_i, S = {}; while |S| < s and ||r||_2 > eps: add the unselected atom with
 * the largest |d_j^T r| (lowest index on ties) unless that value is 0 or the atom
 * lies numerically in span(D_S); x_S = argmin ||y_i - D_S x||.  Computed in the
 * Batch-OMP form (progressive Cholesky of the Gram submatrix), after which the
 * coefficients are recomputed on the support with one refinement step.
 *   D      device, K atoms of length m (unit norm expected; not checked)
 *   Y      device, n signals of length m
 *   s      1 <= s <= min(m, K, 32);  eps >= 0 (0 = pure sparsity stop)
 *   idx    device int32 [n][s] out;  val device [n][s] out;  nnz device int32 [n] out
 *   resid2 device [n] out, ||y_i - D x_i||^2, may be NULL
 * Limits: 1 <= m <= 256, 1 <= K <= 1024, n >= 0 (n = 0 launches nothing). */
sdl_status sdl_omp(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K,
                   const void *Y, int64_t n, int s, double eps, int32_t *idx, void *val,
                   int32_t *nnz, void *resid2);

/* Batched OMP (Algorithm 1 step 2's coding stage): subset t = signals
 * offsets[t] .. offsets[t+1]-1 of Y is coded against its own dictionary
 * D + t*K*m.  offsets is HOST int64 [L+1], non-decreasing, offsets[0] = 0.
 * Outputs are indexed by the global signal index as in sdl_omp. */
sdl_status sdl_omp_batched(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K,
                           const void *Y, const int64_t *offsets, int L, int s, double eps,
                           int32_t *idx, void *val, int32_t *nnz, void *resid2);

/* MOD dictionary update (Sec. 1) with renormalisation (Sec. 3.1):
 * D_U = B_U A_UU^{-1} with A = X X^T, B = Y X^T accumulated in FP64 from the ELL
 * codes, U = atoms used by at least one signal.  A_UU is factored by FP64
 * Cholesky; on breakdown (a squared pivot <= 1e-12 of its diagonal) it is
 * retried once with A_UU + lambda I, lambda = 1e-10 tr(A_UU)/|U|.  Used atoms are
 * scaled to unit norm; unused atoms and atoms whose solution is zero keep their
 * value from D.
 *   Y device [n][m];  idx/val device [n][s] (val of the data type);
 *   D device [K][m], in: previous dictionary, out: updated dictionary
 *   usage device int32 [K] out (signals per atom), may be NULL. */
sdl_status sdl_mod_update(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t n,
                          const int32_t *idx, const void *val, int s, void *D, int K,
                          int32_t *usage);

/* Batched MOD: subset t uses signals offsets[t]..offsets[t+1]-1 and updates
 * D + t*K*m.  offsets is HOST int64 [L+1].  usage device int32 [L][K] or NULL. */
sdl_status sdl_mod_update_batched(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m,
                                  const int64_t *offsets, int L, const int32_t *idx,
                                  const void *val, int s, void *D, int K, int32_t *usage);

/* Atom replacement, an alternative dictionary-update policy.  The paper has no
 * counterpart: its MOD (Sec. 1) leaves unused atoms as they are.  For every
 * subset t (signals offsets[t] .. offsets[t+1]-1, dictionary D + t*K*m), the
 * atoms j with usage[t][j] < min_use are visited in increasing j, and each
 * becomes y_i / ||y_i||.  Signal i is the one of the subset with the largest
 * resid2[i] that no earlier atom took, the lower i on ties.  Only signals with
 * resid2 > 0 qualify.  Once none is left, the remaining atoms keep their value.
 *   prec    F32 or F64 (the data type of Y, resid2 and D)
 *   Y       device [n][m];  resid2 device [n], squared residuals of the coding
 *           pass that produced the usage counts (sdl_omp's resid2)
 *   offsets HOST int64 [L+1];  usage device int32 [L][K] (sdl_mod_update's)
 *   D       device [L][K][m], updated in place
 *   rep     device int32 [L][K] out (the signal row that replaced an atom, or
 *           -1), may be NULL
 * min_use = 0 replaces nothing.  SDL_OPT_REPLACE applies the same step after
 * every MOD update of sdl_local_train and sdl_merge.  Errors:
 * SDL_EINVAL for a bad shape, precision or pointer. */
sdl_status sdl_replace_atoms(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m,
                             const int64_t *offsets, int L, const int32_t *usage,
                             const void *resid2, int min_use, void *D, int K, int32_t *rep);

/* Algorithm 1 step 1: Yp[:, i] = Y[:, perm[i]].  perm device int64 [N], a
 * permutation of 0..N-1 drawn by the caller; consecutive ranges of Yp given by
 * the caller's offsets are the random subsets. */
sdl_status sdl_split(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t N,
                     const int64_t *perm, void *Yp);

/* Initial atoms (Sec. 3.1: atoms taken from training vectors): column c of the
 * output is Y[:, pick[c]] scaled to unit norm, or, where pick[c] < 0, fill[c]
 * scaled to unit norm.  pick device int64 [count]; fill device [count][m] or
 * NULL (then every pick must be >= 0); D device [count][m] out. */
sdl_status sdl_init_dict(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t nY,
                         const int64_t *pick, const void *fill, int64_t count, void *D);

/* Algorithm 1 step 2: every subset t (signals offsets[t]..offsets[t+1]-1 of Y,
 * offsets HOST int64 [L+1], every subset non-empty) is trained independently
 * for `iters` rounds of { X = OMP(D^(t), Y^(t), s1, eps); D^(t) = MOD(Y^(t), X) }.
 *   D_local device [L][K1][m]: initial atoms in, trained atoms out
 *   xfro    device double [L] out: ||X^(t)||_F of the last coding pass
 *   rmse    device double [L][iters] out, ||Y^(t) - D^(t) X^(t)||_F / sqrt(m n_t)
 *           of each coding pass; may be NULL. */
sdl_status sdl_local_train(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m,
                           const int64_t *offsets, int L, int K1, int s1, double eps, int iters,
                           void *D_local, double *xfro, double *rmse);

/* Algorithm 1 step 3: Ytilde = [ xfro[0] D^(0) ... xfro[L-1] D^(L-1) ] (m x K1 L);
 * D starts from the unit-normalised columns Ytilde[:, pick[j]] and is trained on
 * Ytilde for `iters` rounds with sparsity s2.
 *   D_local device [L][K1][m];  xfro device double [L]
 *   pick device int32 [K], or NULL: then D's contents on entry are the initial
 *        atoms (any fixed initial dictionary, e.g. the overcomplete DCT the
 *        paper's image experiments start from, Sec. 3.2.1)
 *   D device [K][m] out (in as well when pick is NULL);  rmse device double
 *   [iters] out or NULL. */
sdl_status sdl_merge(sdl_ctx *ctx, sdl_precision prec, const void *D_local, const double *xfro,
                     int m, int K1, int L, const int32_t *pick, int K, int s2, double eps,
                     int iters, void *D, double *rmse);

/* Table 1's MSE_train ingredients: out2 device double [2] receives
 * ||Y - D X||_F^2 and ||Y||_F^2 for ELL codes X (s entries per signal, -1
 * pads).  m <= 256, s <= 32, as for sdl_omp; SDL_EINVAL otherwise. */
sdl_status sdl_residual(sdl_ctx *ctx, sdl_precision prec, const void *Y, int m, int64_t n,
                        const void *D, int K, const int32_t *idx, const void *val, int s,
                        double *out2);

/* Gram matrices G_t = D_t D_t^T of L dictionaries, the products the
 * Batch-OMP update uses (Sec. 1).  D device [L][K][m] (the data type), G device
 * [L][K][K] (the data type; FP32 for BF16).  F64 and F32: FMA chains over the
 * m entries on the CUDA cores.  BF16: FP32 data split as d = hi + lo + r with
 * hi = bf16(d), lo = bf16(d - hi), and G = hi hi^T + hi lo^T + lo hi^T on the
 * tensor cores with FP32 accumulation, about 2^-16 of |d_i||d_j| from the
 * exact Gram.  F32X3: the same three products from a two-term TF32 split
 * (kind::tf32), within 3 2^-22 of |d_i||d_j| plus the FP32 accumulation; TF32
 * forms the same three-product Gram.  BF16, F32X3 and TF32 synchronise to read
 * the tensor-core kernels' error word.
 * Errors: SDL_EINVAL for a bad shape or pointer, SDL_ETIMEOUT when a bounded
 * wait of the tensor-core kernel gave up. */
sdl_status sdl_gram(sdl_ctx *ctx, sdl_precision prec, const void *D, int m, int K, int L, void *G);

/* Atom recovery (Sec. 3.1): count device int32 [1] receives the number of atoms
 * of D0 (K0 x m) for which some atom of D (K x m) has |d0_i^T d_j| >= thresh. */
sdl_status sdl_recovery(sdl_ctx *ctx, sdl_precision prec, const void *D0, int K0, const void *D,
                        int K, int m, double thresh, int32_t *count);

/* ---- Image denoising with the learned dictionary (Sec. 3.2.2).  Every p x p
 * patch of an H x W image (row-major pixels, one patch per position (r, c) with
 * r < H-p+1, c < W-p+1; patch index r (W-p+1) + c; entry (u, v) at u p + v) is
 * coded with the error-constrained sdl_omp (eps = 8.5 sigma in the paper), its
 * estimate is D x, and the denoised image holds at every pixel the mean of the
 * estimates of the patches covering it.  prec F64 or F32 (BF16: FP32 data).
 *
 * sdl_extract_patches: img device [H][W]; patches device [(H-p+1)(W-p+1)][p p]
 *   out.  1 <= p <= 16, p <= H, p <= W.
 * sdl_patch_average: D device [K][p p]; idx/val device ELL codes
 *   [(H-p+1)(W-p+1)][s] (-1 pads at the end of a row); out device [H][W].
 * sdl_sq_error: out2 device double [2] receives sum (a - b)^2 and sum b^2 over
 *   n entries (PSNR = 10 log10(peak^2 n / out2[0])).
 * All return SDL_EINVAL on a bad size or a NULL / unaligned pointer. */
sdl_status sdl_extract_patches(sdl_ctx *ctx, sdl_precision prec, const void *img, int H, int W, int p,
                               void *patches);
sdl_status sdl_patch_average(sdl_ctx *ctx, sdl_precision prec, const void *D, int K, const int32_t *idx,
                             const void *val, int s, int H, int W, int p, void *out);
sdl_status sdl_sq_error(sdl_ctx *ctx, sdl_precision prec, const void *a, const void *b, int64_t n,
                        double *out2);

/* ---- Learned support proposer (an extension beyond the paper: it accelerates
 * the OMP stage of Sec. 1 by proposing candidate atoms).  An MLP
 * m -> h1 -> h2 -> K with GELU hidden layers scores every atom for a signal;
 * its products run on the tensor cores in BF16 with FP32 accumulation; master
 * weights, Adam moments and the loss are FP32.  Parameters are one packed FP32
 * array: W1 [h1][m], b1 [h1], W2 [h2][h1], b2 [h2], W3 [K][h2], b3 [K].
 * The proposer owns its device memory (allocated at creation and grown to the
 * largest batch seen); it is tied to the context's device. */
typedef struct sdl_proposer sdl_proposer;

/* Create a proposer with initial parameters `params` (device, packed as above).
 * m is the input size: the signal length for a proposer that reads signals,
 * the atom count K for one that reads correlation features |D^T y| (see
 * sdl_corr_features).  h1, h2, K multiples of 8; 1 <= m <= 1024; K <= 1024.
 * Synchronises. */
sdl_status sdl_proposer_create(sdl_ctx *ctx, int m, int h1, int h2, int K, const float *params,
                               sdl_proposer **out);
sdl_status sdl_proposer_destroy(sdl_proposer *p);
/* Copy the FP32 master parameters into `params` (device, packed). */
sdl_status sdl_proposer_get_params(sdl_ctx *ctx, const sdl_proposer *p, float *params);
/* Binary cross-entropy of the logits against support labels, averaged over the
 * batch: (1/B) sum_b sum_j [max(z,0) - z t + log(1 + exp(-|z|))], t_bj = 1 iff atom
 * j is in idx[b] (device int32 [B][s], -1 pads).  loss: device float [1] or NULL;
 * grad: device float [nparams] packed like the parameters, or NULL.  B must be a
 * positive multiple of 8. */
sdl_status sdl_proposer_loss_grad(sdl_ctx *ctx, sdl_proposer *p, const float *Y, const int32_t *idx, int s,
                                  int64_t B, float *loss, float *grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the batch. */
sdl_status sdl_proposer_train_step(sdl_ctx *ctx, sdl_proposer *p, const float *Y, const int32_t *idx, int s,
                                   int64_t B, float lr, float *loss);
/* Logits Z (device float [n][K]) of n signals. */
sdl_status sdl_proposer_scores(sdl_ctx *ctx, sdl_proposer *p, const float *Y, int64_t n, float *Z);
/* Proposer-assisted OMP (FP32 data): for each signal, the top `ncand` atoms by
 * score (s <= ncand <= 32) are the candidates; OMP (Sec. 1 greedy rule, lowest
 * atom index on ties) runs over them, the coefficients are refitted on the
 * support; every signal whose residual norm exceeds eps_fb is recoded by the
 * full OMP of sdl_omp (the fallback).  Outputs as sdl_omp; *n_fallback (host)
 * receives the number of recoded signals.  Synchronises once. */
sdl_status sdl_omp_proposed(sdl_ctx *ctx, sdl_proposer *p, const float *D, int m, int K, const float *Y,
                            int64_t n, int s, int ncand, double eps_fb, int32_t *idx, float *val,
                            int32_t *nnz, float *resid2, int64_t *n_fallback);

/* Correlation features (the input of a dictionary-conditioned proposer, which
 * reads |D_t^T y| instead of y so that one network serves every dictionary of a
 * batch): F[i][j] = |<d_(t(i), j), y_i>| for signal i of subset t(i), each an
 * ordered chain of FP32 FMAs over the m entries (the correlation of OMP's first
 * step, Sec. 1, before the argmax).
 *   D        device float [L][K][m] (row-major, atoms as rows), 16-byte aligned
 *   Y        device float [n][m], n = offsets[L]; offsets host int64 [L+1] as in
 *            sdl_omp_batched (empty subsets allowed)
 *   F        device float [n][K] out, 16-byte aligned
 * 1 <= m <= 256, 1 <= K <= 1024.  Errors: SDL_EINVAL on bad sizes, offsets or
 * pointers (nothing is written).  Does not synchronise beyond the upload of the
 * offsets. */
sdl_status sdl_corr_features(sdl_ctx *ctx, const float *D, int m, int K, const float *Y, const int64_t *offsets,
                             int L, float *F);

/* Proposer input for sdl_omp_proposed_batched. */
#define SDL_FEATURES_SIGNAL 0   /* the proposer reads y (m inputs) */
#define SDL_FEATURES_CORR 1     /* the proposer reads |D_t^T y| (K inputs) */

/* Proposer-assisted OMP over L subsets, each coded against its own dictionary
 * D_t (FP32 data): candidates are the top `ncand` atoms of the proposer's scores
 * of y (SDL_FEATURES_SIGNAL) or of |D_t^T y| (SDL_FEATURES_CORR; one network
 * for every dictionary), OMP runs over them with D_t's Gram and refits on the
 * support, and each signal whose residual norm exceeds eps_fb is recoded by the
 * full OMP of sdl_omp_batched against its own D_t.  D, m, K, Y, offsets, L, s
 * and the outputs as sdl_omp_batched (eps = 0); ncand, eps_fb, *n_fallback as
 * sdl_omp_proposed.  The proposer must have K outputs and m (signal) or K
 * (correlation) inputs.  Synchronises once. */
sdl_status sdl_omp_proposed_batched(sdl_ctx *ctx, sdl_proposer *p, int features, const float *D, int m, int K,
                                    const float *Y, const int64_t *offsets, int L, int s, int ncand, double eps_fb,
                                    int32_t *idx, float *val, int32_t *nnz, float *resid2, int64_t *n_fallback);

/* OMP without any allocation (the paper has no counterpart: this is a service
 * entry point).  For callers that cannot call cudaMalloc where they code signals:
 * processes whose device memory is entirely owned by another allocator, or loops
 * that must not take the implicit synchronisation of an allocation.  It runs the
 * fused FP32 OMP kernel, the form sdl_omp runs for SDL_PREC_F32 under
 * SDL_OPT_OMP_FORM = 1, and returns the same codes bit for bit; sdl_omp's
 * default two-kernel form forms every correlation as the same ordered chain of
 * FP32 FMAs and gives the same codes too.  It keeps its scratch -- the K x K
 * Gram matrix and a small launch plan -- in a fixed array of 1 MiB + 256 bytes
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no context workspace.
 *   stream  cudaStream_t on the calling thread's current device (NULL = legacy)
 *   D, Y, idx, val, nnz, resid2: as sdl_omp with float data; resid2 may be NULL
 * Limits: K <= 512 and m <= 256, else SDL_ERANGE (nothing launched); other bad
 * arguments give SDL_EINVAL.  The first call on a device looks up the array's
 * device address (once per device, with that device current); make that first
 * call before any stream capture.  Every call on a device shares the one array
 * and overwrites all of it that it reads, so calls that overlap on the GPU
 * (concurrent streams, or several host threads) race and must be serialised by
 * the caller. */
sdl_status sdl_omp_noalloc(void *stream, const float *D, int m, int K, const float *Y, int64_t n,
                           int s, double eps, int32_t *idx, float *val, int32_t *nnz,
                           float *resid2);

/* Execution options (the paper has no counterpart; all but SDL_OPT_REPLACE
 * select between implementations that compute the same result, which enables
 * an alternative dictionary-update policy):
 *   SDL_OPT_MOD_SOLVE: 0 = automatic (default: the tiled solve with an
 *     automatic tile and cluster size), 1 = one thread-block cluster per subset
 *     holding the factor in distributed shared memory (K <= 512), 2 = one
 *     thread block per subset for the factorisation, then a separate solve,
 *     3 = the tiled solve with the tile and cluster size set below, 4 = the
 *     wide form of the tiled solve: each subset's tile tasks spread over
 *     SDL_OPT_CLUSTER blocks (0: the SM count over the number of subsets) of a
 *     cooperative launch anywhere on the GPU, meeting at barriers in global
 *     memory whose waits are bounded (SDL_ETIMEOUT when one gives up).  The
 *     automatic choice also times the wide form for fewer subsets than SMs / 16
 *     and, for FP32 data, the checked mixed-precision solve (SDL_OPT_MOD_MIXED).
 *   SDL_OPT_MOD_MIXED: FP32 data only.  1 (default) = under SDL_OPT_MOD_SOLVE
 *     0 the tiled factorisation and solve may run in FP32, followed by a check
 *     of every subset's solution: 8 random-sign probes of the FP64 residual
 *     D A - B, mapped through the FP32 factor, estimate each used atom's error
 *     (Hutchinson); a subset whose estimated error norms are all within 2e-5
 *     of the atom's norm (SDL_OPT_MOD_CHECK_TOL) is renormalised and kept, every other subset (and one whose FP32
 *     squared pivot fell to 1e-3 of its diagonal) is solved again in FP64 as
 *     it would have been alone, ridge retry included.  Chosen when the
 *     autotuner times it faster than the FP64 candidates.  0 = FP64 only.
 *   SDL_OPT_A0_CHUNK_MB: the two-kernel coding passes (FP32, BF16, F32X3)
 *     write the correlations alpha0 of 128-signal tiles to a workspace scratch
 *     and run the selection from there, chunk by chunk: the chunk's size in
 *     MB, 1 to 1024, or 0 (default) for the automatic size.
 *   SDL_OPT_MOD_CHECK_TOL: the tolerance of that check in parts per 10^9 of
 *     each atom's norm, 1 to 10^9, default 20000 (2e-5).  A smaller value sends
 *     more subsets to the FP64 solve; 1 sends every one.
 *     The result then differs from the FP64 solve's by the FP32 solve's
 *     error, about 2e-5 of each atom's norm at most (the FP32 atom
 *     tolerance).
 *   SDL_OPT_CLUSTER: cluster size, 0 = automatic (default); 4, 8 or 16 for
 *     option 1, 1 to 16 for option 3; blocks per subset for option 4.
 *   SDL_OPT_MOD_TILE: tile edge of the tiled solve: 0 = automatic (default),
 *     16, 32 or 64 (64: the FP32 pass of the checked solve, with 4 x 4
 *     register micro-tiles; an FP64 solve then takes 32).
 *   SDL_OPT_SM_BLOCKS: with the tile or cluster size set by hand, at most this
 *     many blocks of the tiled solve per SM (1 to 3; 0 = as many as fit, the
 *     default).  The autotuner also tries a cap of 2.
 *   SDL_OPT_AUTOTUNE: 1 (default) = where tile and cluster size are automatic,
 *     the first call for a shape (element type, number of subsets, K, m) times
 *     every candidate on the call's own inputs with CUDA events (this
 *     synchronises the stream once) and keeps the fastest for the context;
 *     calls made while the stream is being captured use a rule on the shape
 *     instead.  The same holds for the selection launch of the two-kernel
 *     coding passes (FP32 form 2, BF16 form 1 or 3, F32X3) where
 *     SDL_OPT_SEL_SPW and SDL_OPT_SEL_GCACHE are both 0 and the call has at
 *     least two 128-signal tiles per SM: the first call for a shape
 *     (precision, number of subsets, K, m, s, tiles rounded down to a power of
 *     two) runs the whole pass once per selection shape and keeps the fastest.
 *     0 = always use that rule (and forget tuned shapes).
 *   SDL_OPT_GRAPH: 1 = the training loops of sdl_local_train and sdl_merge run
 *     as CUDA graphs: the first call with a given set of buffers, sizes and
 *     options runs eagerly, the second captures the iterations and launches
 *     the graph, later ones relaunch it (the per-call plans and the status
 *     read-back stay outside the graph).  While instrumentation is on, calls
 *     run eagerly.  Graphs refer to the caller's buffers: do not free a buffer
 *     that a cached graph uses while the option is on (turning it off, or a
 *     workspace reallocation, drops the cache).  0 (default) = always eager.
 *   SDL_OPT_OMP_FORM: FP32 OMP kernels.  0 = automatic (default): form 2.
 *     1 = one fused kernel per pass, the correlations of 32-signal tiles in
 *     shared memory.  2 = a correlation GEMM of 128-signal tiles into a
 *     workspace scratch, then the selection kernel.  Both compute the same
 *     correlations (FMAs over the signal entries in order).
 *   SDL_OPT_BF16_FORM: BF16 OMP kernels.  0 = automatic (default): form 1.
 *     1 = Batch-OMP form: alpha0 =
 *     D^T y of 128-signal tiles on the tensor cores into a workspace scratch,
 *     then the selection kernel's running correlations through the FP32 Gram.
 *     3 = the same with the running update's K-wide Gram columns read from a
 *     half-precision copy (2^-11 of each entry, below the correlations' own
 *     BF16 rounding; the Cholesky entries stay FP32): half the bytes of those
 *     reads.  2 = residual form: one kernel recomputes D^T r of a
 *     128-signal tile at every step on the tensor cores (accumulators in tensor
 *     memory) and forms the residuals and right-hand sides in FP32 (s <= 16 and
 *     m <= 256; other shapes run form 1).  All correct the coefficients on the
 *     chosen support in FP32 with one refinement step; they may choose
 *     differently among atoms whose correlations tie to within BF16 rounding.
 *   SDL_OPT_SEL_SPW: signals per warp of the selection launch of the
 *     two-kernel coding passes: 1, 2 or 4, or 0 (default) for automatic (the
 *     autotuner's choice, else 4).
 *   SDL_OPT_SEL_GCACHE: the Gram columns of the support that each warp of
 *     that launch caches in shared memory: 1 = as many as fit, 2 = none, 0
 *     (default) = automatic (the autotuner's choice, else as many as fit).
 *     Neither option changes the result.
 *   SDL_OPT_WAIT_LIMIT: polls (64 ns apart) before a barrier wait of the wide
 *     solve gives up, default 2^24; the call then returns SDL_ETIMEOUT with the
 *     atoms unchanged and the context usable.  The same number, capped at
 *     2^22, bounds the mbarrier waits of the persistent tensor-core
 *     correlation and Gram kernels (SDL_PREC_BF16 correlations,
 *     SDL_PREC_F32X3, SDL_PREC_TF32).
 *   SDL_OPT_WAIT_TEST: 1 makes one block of every wide-solve group leave at
 *     once, so that the others' first barrier wait runs out, and the loader
 *     role of the persistent tensor-core kernels leave before its first copy,
 *     so that the MMA issuer's first wait runs out: the tests of the bounded
 *     waits (default 0).
 *   SDL_OPT_REPLACE: min_use of the atom replacement (sdl_replace_atoms) run
 *     after every MOD update of the training loops.  0 (default) = off, the
 *     paper's reading: unused atoms keep their value.  This option changes the
 *     result; the others above do not.
 * Returns SDL_EINVAL for an unknown option or value. */
typedef enum {
  SDL_OPT_MOD_SOLVE = 1,
  SDL_OPT_CLUSTER = 2,
  SDL_OPT_MOD_TILE = 3,
  SDL_OPT_AUTOTUNE = 4,
  SDL_OPT_GRAPH = 5,
  SDL_OPT_SM_BLOCKS = 6,
  SDL_OPT_REPLACE = 7,
  SDL_OPT_OMP_FORM = 8,
  SDL_OPT_BF16_FORM = 9,
  SDL_OPT_WAIT_LIMIT = 10,
  SDL_OPT_WAIT_TEST = 11,
  SDL_OPT_MOD_MIXED = 12,
  SDL_OPT_MOD_CHECK_TOL = 13,
  SDL_OPT_A0_CHUNK_MB = 14,
  SDL_OPT_SEL_SPW = 15,
  SDL_OPT_SEL_GCACHE = 16
} sdl_option;
sdl_status sdl_set_option(sdl_ctx *ctx, int option, int64_t value);

/* Instrumentation (the paper has no counterpart; it serves the roofline
 * measurements): while enabled, every kernel launcher the context runs is
 * bracketed by a pair of CUDA events recorded on the context's stream and
 * accumulated per kernel name ("omp", "gram", "mod_accum", "chol_fp64",
 * "solve_fp64", "normalise", ...).  Reading resolves the events, which
 * synchronises on them.  Entry names are owned by the context and stay valid
 * until the next sdl_profile_reset or sdl_destroy. */
sdl_status sdl_profile_enable(sdl_ctx *ctx, int on);
/* Drop the accumulated entries (pending events are resolved first). */
sdl_status sdl_profile_reset(sdl_ctx *ctx);
/* Number of distinct entries; -1 for a NULL context. */
int sdl_profile_count(sdl_ctx *ctx);
/* Entry i: kernel name, kernels launched, launcher calls, total milliseconds. */
sdl_status sdl_profile_entry(sdl_ctx *ctx, int i, const char **name, int64_t *launches,
                             int64_t *calls, double *total_ms);
/* Kernels this context has launched since creation (profiling on or off). */
int64_t sdl_launch_count(const sdl_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SDL_H */
