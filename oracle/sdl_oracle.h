/*
 * sdl_oracle.h -- plain FP64 CPU oracle for split-and-merge dictionary learning.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.  The
 * product path (the CUDA library under paper_1403_4781_gb300/) never links,
 * imports or calls it, and this code shares nothing with that path.
 *
 * Notation follows the paper (Mukherjee & Seelamantula, "A split-and-merge
 * dictionary learning algorithm for sparse representation", arXiv 1403.4781):
 *   Y  in R^{m x N}  training signals, one signal per column      (Sec. 2)
 *   D  in R^{m x K}  dictionary with unit-norm atoms d_j           (Def. 1, Sec. 2)
 *   X  in R^{K x N}  s-sparse coefficient columns                  (Sec. 2)
 * Storage: every matrix is column-major with the m entries of one signal or
 * one atom contiguous (Y[i*m + r], D[j*m + r]).  Sparse coefficient columns are
 * stored in ELL form: idx[i*s + k] (atom index, -1 pads), val[i*s + k].
 *
 * Every function is a direct transcription of a definition; none is blocked,
 * fused or reordered.  Return value: 0 ok, 1 invalid argument, 2 Cholesky
 * breakdown after the ridge retry.
 */
#ifndef SDL_ORACLE_H
#define SDL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Orthogonal matching pursuit (Sec. 1 and the error-constrained form of
 * Sec. 3.2.2), one signal at a time:
 *   r = y, S = {}; while |S| < s and ||r||_2 > eps:
 *     j* = argmax_{j not in S} |d_j^T r|  (lowest index wins a tie);
 *     stop if that maximum is 0 or d_j* is numerically inside span(D_S);
 *     S = S u {j*};  x_S = argmin ||y - D_S x||_2;  r = y - D_S x_S.
 * Outputs per signal i: idx/val [s] in selection order, nnz, resid2 = ||r||^2,
 * gap[s] = top-two gap of |d_j^T r| among unselected atoms at each step
 * (+inf where no step was taken).  resid2 and gap may be NULL. */
int orc_omp(const double *D, int m, int K, const double *Y, int64_t n, int s,
            double eps, int32_t *idx, double *val, int32_t *nnz,
            double *resid2, double *gap, int nthreads);

/* Method of optimal directions (Sec. 1): D = Y X^T (X X^T)^{-1} over the used
 * atoms U (atoms with at least one signal); atoms outside U keep Dprev.  If the
 * Cholesky factor of A_UU = (X X^T)_UU breaks down it is retried once with
 * A_UU + lambda I, lambda = 1e-10 tr(A_UU)/|U|.  normalise != 0 then scales
 * every column to unit norm (Sec. 3.1), keeping Dprev for a zero column.
 * usage[K] (may be NULL) receives the number of signals using each atom;
 * ridge (may be NULL) receives 1 when the ridge retry was taken. */
int orc_mod(const double *Y, int m, int64_t n, const int32_t *idx,
            const double *val, int s, const double *Dprev, int K, int normalise,
            double *Dout, int32_t *usage, int *ridge);

/* Atom replacement, an alternative dictionary-update policy (not in the paper,
 * whose reading keeps unused atoms): atoms are visited in increasing index and
 * atom j with usage[j] < min_use becomes y_i / ||y_i|| for the signal i with the
 * largest resid2[i] not yet taken (lower i on ties; only resid2 > 0 qualifies;
 * when none is left the remaining atoms keep their value).  rep[K] (may be
 * NULL) receives i or -1 per atom, nrep (may be NULL) the number replaced. */
int orc_replace_atoms(const double *Y, int m, int64_t n, const int32_t *usage,
                      const double *resid2, int min_use, double *D, int K, int32_t *rep,
                      int *nrep);

/* Alternating minimisation (Sec. 1, "standard approach"): for it in 0..iters-1
 * { X = OMP(D, Y, s, eps); rmse[it] = ||Y - D X||_F / sqrt(m n); D = MOD(Y, X) }.
 * With min_use > 0 every MOD update is followed by orc_replace_atoms with the
 * usage counts of X and the squared residuals of that coding pass.
 * D is the initial dictionary on entry and the trained one on exit.
 * xfro receives ||X||_F of the last coding pass.  idx/val/nnz (may be NULL)
 * receive that last coding.  rmse may be NULL. */
int orc_train(const double *Y, int m, int64_t n, double *D, int K, int s,
              double eps, int iters, int min_use, double *rmse, double *xfro,
              int32_t *idx, double *val, int32_t *nnz, int nthreads);

/* Algorithm 1 step 1: Yp[:, i] = Y[:, perm[i]] (the random partition is the
 * permutation followed by contiguous subsets given by offsets). */
int orc_split(const double *Y, int m, int64_t N, const int64_t *perm, double *Yp);

/* Algorithm 1 step 2: subset t = columns offsets[t] .. offsets[t+1]-1 of Y is
 * trained independently with K1 atoms and sparsity s1.  Dloc is [L][K1][m]
 * (init on entry, trained on exit); xfro[L]; rmse [L][iters] (may be NULL). */
int orc_local_train(const double *Y, int m, const int64_t *offsets, int L,
                    double *Dloc, int K1, int s1, double eps, int iters, int min_use,
                    double *xfro, double *rmse, int nthreads);

/* Algorithm 1 step 3: Ytilde = [ xfro[0] D^(0) ... xfro[L-1] D^(L-1) ]
 * (m x K1 L); D is initialised with the normalised columns Ytilde[:, pick[j]]
 * and trained on Ytilde with K atoms and sparsity s2.  D is [K][m] out.
 * Ytilde_out [K1 L][m] may be NULL. */
int orc_merge(const double *Dloc, const double *xfro, int m, int K1, int L,
              const int32_t *pick, int K, int s2, double eps, int iters, int min_use,
              double *D, double *rmse, double *Ytilde_out, int nthreads);

/* ||Y - D X||_F^2 and ||Y||_F^2 with X in ELL form (Table 1's MSE_train is
 * 20 log10 of the square root of their ratio). */
int orc_residual(const double *Y, int m, int64_t n, const double *D, int K,
                 const int32_t *idx, const double *val, int s,
                 double *res2, double *y2);

/* Atom recovery (Sec. 3.1): number of atoms d_i of D0 with some atom of D
 * such that |d_i^T dhat_j| >= thresh. */
int orc_recovery(const double *D0, int K0, const double *D, int K, int m,
                 double thresh, int *count);

/* Input of a dictionary-conditioned support proposer (an extension beyond the
 * paper): F[i][j] = |d_(t,j)^T y_i| for every signal i of subset t (rows
 * offsets[t] .. offsets[t+1]-1 of Y), D [L][K][m].  These are the magnitudes
 * OMP's first greedy step ranks (Sec. 1), written out as plain dot products. */
int orc_corr_features(const double *D, int m, int K, const double *Y, const int64_t *offsets, int L,
                      double *F);

#ifdef __cplusplus
}
#endif
#endif

#ifdef __cplusplus
extern "C" {
#endif
/* Learned support proposer (an extension beyond the paper: a small MLP that
 * scores atoms for a signal).  Parameters are packed in one array:
 *   W1 [h1][m], b1 [h1], W2 [h2][h1], b2 [h2], W3 [K][h2], b3 [K].
 * Forward: a1 = W1 y + b1, h1 = gelu(a1), a2 = W2 h1 + b2, h2 = gelu(a2),
 * z = W3 h2 + b3 with gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
 * Loss over a batch of B signals with supports idx [B][s] (-1 pads):
 *   (1/B) sum_b sum_j [ max(z,0) - z t + log(1 + exp(-|z|)) ], t_bj = 1 iff j in
 *   the support of signal b (binary cross-entropy on the logits).
 * orc_mlp_loss_grad returns the loss and (grad != NULL) its gradient with
 * respect to every packed parameter, by backpropagation; orc_mlp_forward
 * returns the logits z [B][K]. */
int orc_mlp_forward(const double *params, int m, int h1, int h2, int K, const double *Y, int64_t B,
                    double *Z);
int orc_mlp_loss_grad(const double *params, int m, int h1, int h2, int K, const double *Y,
                      const int32_t *idx, int s, int64_t B, double *loss, double *grad);

/* One Adam step (Kingma & Ba 2015, Algorithm 1) of the proposer's optimiser:
 * theta, m, v updated in place; t >= 1 is the step number (bias correction). */
int orc_adam_step(double *theta, const double *g, double *m, double *v, int64_t n, int t, double alpha,
                  double beta1, double beta2, double eps);
#ifdef __cplusplus
}
#endif

#ifdef __cplusplus
extern "C" {
#endif
/* Image denoising with the learned dictionary (Sec. 3.2.2): every p x p patch
 * of an H x W image (row-major, one patch per position (r, c), r < H-p+1,
 * c < W-p+1, patch index r (W-p+1) + c, entry (u, v) at u p + v) is coded
 * with the error-constrained OMP, its estimate is D x, and the denoised image
 * is, at every pixel, the mean of the estimates of the patches covering it.
 *   orc_extract_patches: out [(H-p+1)(W-p+1)][p p].
 *   orc_patch_average:   D [K][p p]; codes idx/val [(H-p+1)(W-p+1)][s]
 *                        (-1 pads); out [H][W]. */
int orc_extract_patches(const double *img, int H, int W, int p, double *out);
int orc_patch_average(const double *D, int K, const int32_t *idx, const double *val, int s, int H, int W,
                      int p, double *out);
#ifdef __cplusplus
}
#endif
