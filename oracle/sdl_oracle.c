/*
 * sdl_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline legs use
 * this file.  It shares no code, header or constant with the CUDA library.
 * Each routine writes out the definition it cites in the simplest loops; the
 * least-squares sub-problems are solved by a textbook Cholesky factorisation
 * recomputed from scratch, never updated in place.
 */
#include "sdl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Relative pivot floor of the OMP Gram factor: a new atom whose squared
 * distance to span(D_S) is below this fraction of ||d_j||^2 is not added. */
#define ORC_OMP_PIVOT_REL 1e-10
/* Relative pivot floor of the MOD normal-equation factor. */
#define ORC_MOD_PIVOT_REL 1e-12
/* Ridge of the single retry: lambda = ORC_RIDGE * tr(A_UU) / |U|. */
#define ORC_RIDGE 1e-10

static double dot(const double *a, const double *b, int len) {
  double acc = 0.0;
  for (int r = 0; r < len; ++r) acc += a[r] * b[r];
  return acc;
}

/* In-place lower Cholesky of the p x p matrix G (row-major, lower triangle
 * used).  Returns 0 when every squared pivot exceeds rel * (original diagonal),
 * else 1. */
static int cholesky(double *G, int p, double rel) {
  for (int j = 0; j < p; ++j) {
    double diag0 = G[j * p + j];
    double d = diag0;
    for (int k = 0; k < j; ++k) d -= G[j * p + k] * G[j * p + k];
    if (!(d > rel * diag0) || !(d > 0.0)) return 1;
    double ljj = sqrt(d);
    G[j * p + j] = ljj;
    for (int i = j + 1; i < p; ++i) {
      double v = G[i * p + j];
      for (int k = 0; k < j; ++k) v -= G[i * p + k] * G[j * p + k];
      G[i * p + j] = v / ljj;
    }
  }
  return 0;
}

/* Solve L L^T x = b given the lower factor L (row-major p x p); x may alias b. */
static void cholesky_solve(const double *L, int p, const double *b, double *x) {
  double *z = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
  for (int i = 0; i < p; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i * p + k] * z[k];
    z[i] = v / L[i * p + i];
  }
  for (int i = p - 1; i >= 0; --i) {
    double v = z[i];
    for (int k = i + 1; k < p; ++k) v -= L[k * p + i] * x[k];
    x[i] = v / L[i * p + i];
  }
  free(z);
}

/* ---------------------------------------------------------------- OMP --- */

static void omp_one(const double *D, int m, int K, const double *y, int s,
                    double eps, int32_t *idx, double *val, int32_t *nnz,
                    double *resid2, double *gap) {
  double *r = (double *)malloc(sizeof(double) * (size_t)m);
  double *G = (double *)malloc(sizeof(double) * (size_t)(s * s + 1));
  double *rhs = (double *)malloc(sizeof(double) * (size_t)(s + 1));
  double *x = (double *)malloc(sizeof(double) * (size_t)(s + 1));
  int *S = (int *)malloc(sizeof(int) * (size_t)(s + 1));
  char *in_S = (char *)calloc((size_t)K, 1);
  memcpy(r, y, sizeof(double) * (size_t)m);
  for (int k = 0; k < s; ++k) {
    idx[k] = -1;
    val[k] = 0.0;
    if (gap) gap[k] = INFINITY;
  }
  int k = 0;
  while (k < s) {
    if (sqrt(dot(r, r, m)) <= eps) break;
    /* greedy selection: largest |d_j^T r| over unselected atoms */
    int best = -1;
    double bestv = -1.0, second = -1.0;
    for (int j = 0; j < K; ++j) {
      if (in_S[j]) continue;
      double a = fabs(dot(D + (size_t)j * m, r, m));
      if (a > bestv) {
        second = bestv;
        bestv = a;
        best = j;
      } else if (a > second) {
        second = a;
      }
    }
    if (best < 0 || !(bestv > 0.0)) break;
    /* least squares on S u {best}: normal equations by a fresh Cholesky */
    S[k] = best;
    int p = k + 1;
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b)
        G[a * p + b] = dot(D + (size_t)S[a] * m, D + (size_t)S[b] * m, m);
    if (cholesky(G, p, ORC_OMP_PIVOT_REL)) break; /* atom inside span(D_S) */
    for (int a = 0; a < p; ++a) rhs[a] = dot(D + (size_t)S[a] * m, y, m);
    cholesky_solve(G, p, rhs, x);
    for (int r0 = 0; r0 < m; ++r0) {
      double v = y[r0];
      for (int a = 0; a < p; ++a) v -= D[(size_t)S[a] * m + r0] * x[a];
      r[r0] = v;
    }
    if (gap) gap[k] = bestv - (second < 0.0 ? 0.0 : second);
    in_S[best] = 1;
    k = p;
  }
  for (int a = 0; a < k; ++a) {
    idx[a] = S[a];
    val[a] = x[a];
  }
  *nnz = k;
  if (resid2) *resid2 = dot(r, r, m);
  free(r);
  free(G);
  free(rhs);
  free(x);
  free(S);
  free(in_S);
}

int orc_omp(const double *D, int m, int K, const double *Y, int64_t n, int s,
            double eps, int32_t *idx, double *val, int32_t *nnz,
            double *resid2, double *gap, int nthreads) {
  if (m <= 0 || K <= 0 || n < 0 || s <= 0 || !D || (n > 0 && (!Y || !idx || !val || !nnz)))
    return 1;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t i = 0; i < n; ++i)
    omp_one(D, m, K, Y + (size_t)i * m, s, eps, idx + (size_t)i * s,
            val + (size_t)i * s, nnz + i, resid2 ? resid2 + i : NULL,
            gap ? gap + (size_t)i * s : NULL);
  return 0;
}

/* ---------------------------------------------------------------- MOD --- */

int orc_mod(const double *Y, int m, int64_t n, const int32_t *idx,
            const double *val, int s, const double *Dprev, int K, int normalise,
            double *Dout, int32_t *usage, int *ridge) {
  if (m <= 0 || K <= 0 || n < 0 || s <= 0 || !Dprev || !Dout) return 1;
  /* A = X X^T (K x K), B = Y X^T (m x K, stored [K][m]), usage counts */
  double *A = (double *)calloc((size_t)K * K, sizeof(double));
  double *B = (double *)calloc((size_t)K * m, sizeof(double));
  int32_t *cnt = (int32_t *)calloc((size_t)K, sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *ii = idx + (size_t)i * s;
    const double *vi = val + (size_t)i * s;
    for (int a = 0; a < s; ++a) {
      if (ii[a] < 0) continue;
      cnt[ii[a]] += 1;
      for (int b = 0; b < s; ++b) {
        if (ii[b] < 0) continue;
        A[(size_t)ii[a] * K + ii[b]] += vi[a] * vi[b];
      }
      for (int r = 0; r < m; ++r)
        B[(size_t)ii[a] * m + r] += Y[(size_t)i * m + r] * vi[a];
    }
  }
  int nu = 0;
  int *U = (int *)malloc(sizeof(int) * (size_t)K);
  for (int j = 0; j < K; ++j)
    if (cnt[j] > 0) U[nu++] = j;
  int status = 0, used_ridge = 0;
  memcpy(Dout, Dprev, sizeof(double) * (size_t)K * m);
  if (nu > 0) {
    double *AU = (double *)malloc(sizeof(double) * (size_t)nu * nu);
    for (int a = 0; a < nu; ++a)
      for (int b = 0; b < nu; ++b) AU[a * nu + b] = A[(size_t)U[a] * K + U[b]];
    if (cholesky(AU, nu, ORC_MOD_PIVOT_REL)) {
      double tr = 0.0;
      for (int a = 0; a < nu; ++a) tr += A[(size_t)U[a] * K + U[a]];
      double lambda = ORC_RIDGE * tr / nu;
      for (int a = 0; a < nu; ++a)
        for (int b = 0; b < nu; ++b)
          AU[a * nu + b] = A[(size_t)U[a] * K + U[b]] + (a == b ? lambda : 0.0);
      used_ridge = 1;
      if (cholesky(AU, nu, ORC_MOD_PIVOT_REL)) status = 2;
    }
    if (status == 0) {
      /* row r of D_U solves A_UU d = (row r of B_U) since A_UU is symmetric */
      double *b = (double *)malloc(sizeof(double) * (size_t)nu);
      for (int r = 0; r < m; ++r) {
        for (int a = 0; a < nu; ++a) b[a] = B[(size_t)U[a] * m + r];
        cholesky_solve(AU, nu, b, b);
        for (int a = 0; a < nu; ++a) Dout[(size_t)U[a] * m + r] = b[a];
      }
      free(b);
    }
    free(AU);
  }
  if (status == 0 && normalise) {
    for (int j = 0; j < K; ++j) {
      if (cnt[j] == 0) continue; /* unused atoms keep their previous value */
      double nrm = sqrt(dot(Dout + (size_t)j * m, Dout + (size_t)j * m, m));
      if (nrm > 0.0 && isfinite(nrm)) {
        for (int r = 0; r < m; ++r) Dout[(size_t)j * m + r] /= nrm;
      } else {
        memcpy(Dout + (size_t)j * m, Dprev + (size_t)j * m, sizeof(double) * (size_t)m);
      }
    }
  }
  if (status != 0) memcpy(Dout, Dprev, sizeof(double) * (size_t)K * m);
  if (usage) memcpy(usage, cnt, sizeof(int32_t) * (size_t)K);
  if (ridge) *ridge = used_ridge;
  free(A);
  free(B);
  free(cnt);
  free(U);
  return status;
}

/* -------------------------------------------------------------- train --- */

/* Atom replacement (not in the paper, which keeps unused atoms).  Atoms are
   visited in increasing index; atom j with usage[j] < min_use becomes the unit
   vector along the training signal with the largest squared residual resid2[i]
   among those not yet taken, ties to the lower signal index.  Only signals with
   resid2 > 0 qualify (such a signal is nonzero); once none is left, the
   remaining atoms keep their value.  rep[j] = i for a replaced atom, else -1. */
int orc_replace_atoms(const double *Y, int m, int64_t n, const int32_t *usage,
                      const double *resid2, int min_use, double *D, int K, int32_t *rep,
                      int *nrep) {
  if (m <= 0 || K <= 0 || n < 0 || !usage || !D || (n > 0 && (!Y || !resid2))) return 1;
  unsigned char *taken = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
  int count = 0;
  for (int j = 0; j < K; ++j) {
    if (rep) rep[j] = -1;
    if (usage[j] >= min_use) continue;
    int64_t best = -1;
    for (int64_t i = 0; i < n; ++i) {
      if (taken[i] || !(resid2[i] > 0.0)) continue;
      if (best < 0 || resid2[i] > resid2[best]) best = i;
    }
    if (best < 0) continue;
    taken[best] = 1;
    const double *y = Y + (size_t)best * m;
    const double nrm = sqrt(dot(y, y, m));
    for (int r = 0; r < m; ++r) D[(size_t)j * m + r] = y[r] / nrm;
    if (rep) rep[j] = (int32_t)best;
    ++count;
  }
  free(taken);
  if (nrep) *nrep = count;
  return 0;
}

int orc_train(const double *Y, int m, int64_t n, double *D, int K, int s,
              double eps, int iters, int min_use, double *rmse, double *xfro,
              int32_t *idx, double *val, int32_t *nnz, int nthreads) {
  if (m <= 0 || K <= 0 || n <= 0 || s <= 0 || iters < 0 || !Y || !D) return 1;
  int32_t *ix = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * s);
  double *vx = (double *)malloc(sizeof(double) * (size_t)n * s);
  int32_t *nz = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *r2 = (double *)malloc(sizeof(double) * (size_t)n);
  double *Dn = (double *)malloc(sizeof(double) * (size_t)K * m);
  int32_t *use = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
  int status = 0;
  double fro2 = 0.0;
  for (int it = 0; it < iters; ++it) {
    orc_omp(D, m, K, Y, n, s, eps, ix, vx, nz, r2, NULL, nthreads);
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += r2[i];
    if (rmse) rmse[it] = sqrt(acc / ((double)m * (double)n));
    fro2 = 0.0;
    for (int64_t e = 0; e < n * s; ++e) fro2 += vx[e] * vx[e];
    int st = orc_mod(Y, m, n, ix, vx, s, D, K, 1, Dn, use, NULL);
    if (st) status = st;
    if (min_use > 0) orc_replace_atoms(Y, m, n, use, r2, min_use, Dn, K, NULL, NULL);
    memcpy(D, Dn, sizeof(double) * (size_t)K * m);
  }
  if (xfro) *xfro = sqrt(fro2);
  if (iters > 0) {
    if (idx) memcpy(idx, ix, sizeof(int32_t) * (size_t)n * s);
    if (val) memcpy(val, vx, sizeof(double) * (size_t)n * s);
    if (nnz) memcpy(nnz, nz, sizeof(int32_t) * (size_t)n);
  }
  free(ix);
  free(vx);
  free(nz);
  free(r2);
  free(Dn);
  free(use);
  return status;
}

/* ---------------------------------------------------- Algorithm 1 steps --- */

int orc_split(const double *Y, int m, int64_t N, const int64_t *perm, double *Yp) {
  if (m <= 0 || N < 0 || (N > 0 && (!Y || !perm || !Yp))) return 1;
  for (int64_t i = 0; i < N; ++i) {
    if (perm[i] < 0 || perm[i] >= N) return 1;
    memcpy(Yp + (size_t)i * m, Y + (size_t)perm[i] * m, sizeof(double) * (size_t)m);
  }
  return 0;
}

int orc_local_train(const double *Y, int m, const int64_t *offsets, int L,
                    double *Dloc, int K1, int s1, double eps, int iters, int min_use,
                    double *xfro, double *rmse, int nthreads) {
  if (m <= 0 || L <= 0 || K1 <= 0 || s1 <= 0 || !offsets || !Dloc || !xfro) return 1;
  for (int t = 0; t < L; ++t)
    if (offsets[t + 1] <= offsets[t]) return 1;
  if (nthreads < 1) nthreads = 1;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int t = 0; t < L; ++t) {
    int st = orc_train(Y + (size_t)offsets[t] * m, m, offsets[t + 1] - offsets[t],
                       Dloc + (size_t)t * K1 * m, K1, s1, eps, iters, min_use,
                       rmse ? rmse + (size_t)t * iters : NULL, xfro + t, NULL, NULL,
                       NULL, 1);
    if (st) {
#pragma omp critical
      status = st;
    }
  }
  return status;
}

int orc_merge(const double *Dloc, const double *xfro, int m, int K1, int L,
              const int32_t *pick, int K, int s2, double eps, int iters, int min_use,
              double *D, double *rmse, double *Ytilde_out, int nthreads) {
  if (m <= 0 || K1 <= 0 || L <= 0 || K <= 0 || s2 <= 0 || !Dloc || !xfro || !pick || !D)
    return 1;
  int64_t nt = (int64_t)K1 * L;
  double *Yt = (double *)malloc(sizeof(double) * (size_t)nt * m);
  for (int t = 0; t < L; ++t)
    for (int j = 0; j < K1; ++j)
      for (int r = 0; r < m; ++r)
        Yt[((size_t)t * K1 + j) * m + r] = xfro[t] * Dloc[((size_t)t * K1 + j) * m + r];
  for (int j = 0; j < K; ++j) {
    if (pick[j] < 0 || pick[j] >= nt) {
      free(Yt);
      return 1;
    }
    const double *c = Yt + (size_t)pick[j] * m;
    double nrm = sqrt(dot(c, c, m));
    for (int r = 0; r < m; ++r) D[(size_t)j * m + r] = nrm > 0.0 ? c[r] / nrm : 0.0;
  }
  double xf;
  int st = orc_train(Yt, m, nt, D, K, s2, eps, iters, min_use, rmse, &xf, NULL, NULL, NULL,
                     nthreads);
  if (Ytilde_out) memcpy(Ytilde_out, Yt, sizeof(double) * (size_t)nt * m);
  free(Yt);
  return st;
}

/* ------------------------------------------------------------ metrics --- */

int orc_residual(const double *Y, int m, int64_t n, const double *D, int K,
                 const int32_t *idx, const double *val, int s,
                 double *res2, double *y2) {
  if (m <= 0 || K <= 0 || n < 0 || s <= 0 || !res2 || !y2) return 1;
  double acc = 0.0, accy = 0.0;
  double *r = (double *)malloc(sizeof(double) * (size_t)m);
  for (int64_t i = 0; i < n; ++i) {
    for (int q = 0; q < m; ++q) r[q] = Y[(size_t)i * m + q];
    for (int a = 0; a < s; ++a) {
      int j = idx[(size_t)i * s + a];
      if (j < 0) continue;
      if (j >= K) {
        free(r);
        return 1;
      }
      for (int q = 0; q < m; ++q) r[q] -= D[(size_t)j * m + q] * val[(size_t)i * s + a];
    }
    acc += dot(r, r, m);
    accy += dot(Y + (size_t)i * m, Y + (size_t)i * m, m);
  }
  free(r);
  *res2 = acc;
  *y2 = accy;
  return 0;
}

int orc_recovery(const double *D0, int K0, const double *D, int K, int m,
                 double thresh, int *count) {
  if (K0 <= 0 || K <= 0 || m <= 0 || !D0 || !D || !count) return 1;
  int c = 0;
  for (int i = 0; i < K0; ++i) {
    int hit = 0;
    for (int j = 0; j < K && !hit; ++j)
      if (fabs(dot(D0 + (size_t)i * m, D + (size_t)j * m, m)) >= thresh) hit = 1;
    c += hit;
  }
  *count = c;
  return 0;
}

int orc_corr_features(const double *D, int m, int K, const double *Y, const int64_t *offsets, int L,
                      double *F) {
  if (m <= 0 || K <= 0 || L <= 0 || !D || !offsets || (offsets[L] > 0 && (!Y || !F))) return 1;
  for (int t = 0; t < L; ++t) {
    if (offsets[t + 1] < offsets[t]) return 1;
    const double *Dt = D + (size_t)t * K * m;
    for (int64_t i = offsets[t]; i < offsets[t + 1]; ++i)
      for (int j = 0; j < K; ++j) F[(size_t)i * K + j] = fabs(dot(Dt + (size_t)j * m, Y + (size_t)i * m, m));
  }
  return 0;
}

/* ------------------------------------------------------- MLP proposer --- */

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_prime(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) * 0.39894228040143267794; /* 1/sqrt(2 pi) */
}

int orc_mlp_forward(const double *params, int m, int h1, int h2, int K, const double *Y, int64_t B,
                    double *Z) {
  if (m <= 0 || h1 <= 0 || h2 <= 0 || K <= 0 || B < 0 || !params || !Z) return 1;
  const double *W1 = params, *b1 = W1 + (size_t)h1 * m, *W2 = b1 + h1, *b2 = W2 + (size_t)h2 * h1;
  const double *W3 = b2 + h2, *b3 = W3 + (size_t)K * h2;
  double *x1 = (double *)malloc(sizeof(double) * (size_t)h1);
  double *x2 = (double *)malloc(sizeof(double) * (size_t)h2);
  for (int64_t b = 0; b < B; ++b) {
    const double *y = Y + (size_t)b * m;
    for (int i = 0; i < h1; ++i) x1[i] = gelu(dot(W1 + (size_t)i * m, y, m) + b1[i]);
    for (int i = 0; i < h2; ++i) x2[i] = gelu(dot(W2 + (size_t)i * h1, x1, h1) + b2[i]);
    for (int j = 0; j < K; ++j) Z[(size_t)b * K + j] = dot(W3 + (size_t)j * h2, x2, h2) + b3[j];
  }
  free(x1);
  free(x2);
  return 0;
}

int orc_mlp_loss_grad(const double *params, int m, int h1, int h2, int K, const double *Y,
                      const int32_t *idx, int s, int64_t B, double *loss, double *grad) {
  if (m <= 0 || h1 <= 0 || h2 <= 0 || K <= 0 || B <= 0 || s <= 0 || !params || !loss) return 1;
  const size_t nW1 = (size_t)h1 * m, nW2 = (size_t)h2 * h1, nW3 = (size_t)K * h2;
  const size_t np = nW1 + h1 + nW2 + h2 + nW3 + K;
  const double *W1 = params, *b1 = W1 + nW1, *W2 = b1 + h1, *b2 = W2 + nW2, *W3 = b2 + h2, *b3 = W3 + nW3;
  double *gW1 = NULL, *gb1 = NULL, *gW2 = NULL, *gb2 = NULL, *gW3 = NULL, *gb3 = NULL;
  if (grad) {
    memset(grad, 0, sizeof(double) * np);
    gW1 = grad; gb1 = gW1 + nW1; gW2 = gb1 + h1; gb2 = gW2 + nW2; gW3 = gb2 + h2; gb3 = gW3 + nW3;
  }
  double *a1 = (double *)malloc(sizeof(double) * (size_t)h1), *x1 = (double *)malloc(sizeof(double) * (size_t)h1);
  double *a2 = (double *)malloc(sizeof(double) * (size_t)h2), *x2 = (double *)malloc(sizeof(double) * (size_t)h2);
  double *z = (double *)malloc(sizeof(double) * (size_t)K), *dz = (double *)malloc(sizeof(double) * (size_t)K);
  double *d2 = (double *)malloc(sizeof(double) * (size_t)h2), *d1 = (double *)malloc(sizeof(double) * (size_t)h1);
  char *t = (char *)malloc((size_t)K);
  double total = 0.0;
  for (int64_t b = 0; b < B; ++b) {
    const double *y = Y + (size_t)b * m;
    for (int i = 0; i < h1; ++i) { a1[i] = dot(W1 + (size_t)i * m, y, m) + b1[i]; x1[i] = gelu(a1[i]); }
    for (int i = 0; i < h2; ++i) { a2[i] = dot(W2 + (size_t)i * h1, x1, h1) + b2[i]; x2[i] = gelu(a2[i]); }
    memset(t, 0, (size_t)K);
    for (int k = 0; k < s; ++k) {
      int j = idx[(size_t)b * s + k];
      if (j >= 0 && j < K) t[j] = 1;
    }
    for (int j = 0; j < K; ++j) {
      z[j] = dot(W3 + (size_t)j * h2, x2, h2) + b3[j];
      total += (z[j] > 0 ? z[j] : 0.0) - z[j] * t[j] + log1p(exp(-fabs(z[j])));
      dz[j] = (1.0 / (1.0 + exp(-z[j])) - t[j]) / (double)B;
    }
    if (!grad) continue;
    for (int j = 0; j < K; ++j) {
      gb3[j] += dz[j];
      for (int i = 0; i < h2; ++i) gW3[(size_t)j * h2 + i] += dz[j] * x2[i];
    }
    for (int i = 0; i < h2; ++i) {
      double v = 0.0;
      for (int j = 0; j < K; ++j) v += W3[(size_t)j * h2 + i] * dz[j];
      d2[i] = v * gelu_prime(a2[i]);
      gb2[i] += d2[i];
      for (int q = 0; q < h1; ++q) gW2[(size_t)i * h1 + q] += d2[i] * x1[q];
    }
    for (int q = 0; q < h1; ++q) {
      double v = 0.0;
      for (int i = 0; i < h2; ++i) v += W2[(size_t)i * h1 + q] * d2[i];
      d1[q] = v * gelu_prime(a1[q]);
      gb1[q] += d1[q];
      for (int r = 0; r < m; ++r) gW1[(size_t)q * m + r] += d1[q] * y[r];
    }
  }
  *loss = total / (double)B;
  free(a1); free(x1); free(a2); free(x2); free(z); free(dz); free(d2); free(d1); free(t);
  return 0;
}

/* Adam (Kingma & Ba 2015, Algorithm 1), the optimiser the proposer trains
 * with (the paper has no learned part): step t >= 1 on n parameters theta with
 * gradient g.  The first and second moment estimates are exponential moving
 * averages of g and g^2 (rates beta1, beta2) held in m and v; their initial
 * bias towards zero is removed by dividing by 1 - beta^t; theta moves by
 * alpha * mhat / (sqrt(vhat) + eps). */
int orc_adam_step(double *theta, const double *g, double *m, double *v, int64_t n, int t, double alpha,
                  double beta1, double beta2, double eps) {
  if (n < 0 || t < 1 || (n > 0 && (!theta || !g || !m || !v))) return 1;
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mhat = m[i] / c1, vhat = v[i] / c2;
    theta[i] -= alpha * mhat / (sqrt(vhat) + eps);
  }
  return 0;
}

/* ------------------------------------------------- image denoising --- */

int orc_extract_patches(const double *img, int H, int W, int p, double *out) {
  if (!img || !out || p <= 0 || H < p || W < p) return 1;
  const int nr = H - p + 1, nc = W - p + 1;
  for (int r = 0; r < nr; ++r)
    for (int c = 0; c < nc; ++c) {
      double *dst = out + ((size_t)r * nc + c) * (size_t)p * p;
      for (int u = 0; u < p; ++u)
        for (int v = 0; v < p; ++v) dst[u * p + v] = img[(size_t)(r + u) * W + (c + v)];
    }
  return 0;
}

int orc_patch_average(const double *D, int K, const int32_t *idx, const double *val, int s, int H, int W,
                      int p, double *out) {
  if (!D || !idx || !val || !out || p <= 0 || H < p || W < p || s <= 0 || K <= 0) return 1;
  const int nr = H - p + 1, nc = W - p + 1, m = p * p;
  double *acc = (double *)calloc((size_t)H * W, sizeof(double));
  int *cnt = (int *)calloc((size_t)H * W, sizeof(int));
  double *rec = (double *)malloc(sizeof(double) * (size_t)m);
  for (int r = 0; r < nr; ++r)
    for (int c = 0; c < nc; ++c) {
      const size_t i = (size_t)r * nc + c;
      for (int e = 0; e < m; ++e) rec[e] = 0.0;
      for (int k = 0; k < s; ++k) {
        const int j = idx[i * s + k];
        if (j < 0 || j >= K) continue;
        for (int e = 0; e < m; ++e) rec[e] += val[i * s + k] * D[(size_t)j * m + e];
      }
      for (int u = 0; u < p; ++u)
        for (int v = 0; v < p; ++v) {
          acc[(size_t)(r + u) * W + (c + v)] += rec[u * p + v];
          cnt[(size_t)(r + u) * W + (c + v)] += 1;
        }
    }
  for (size_t q = 0; q < (size_t)H * W; ++q) out[q] = acc[q] / (double)cnt[q];
  free(acc);
  free(cnt);
  free(rec);
  return 0;
}
