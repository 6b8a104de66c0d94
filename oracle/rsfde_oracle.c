/*
 * rsfde_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the volume-penalized 2D Riesz
 * space-fractional diffusion scheme and of its sine-transform (tau)
 * preconditioned GMRES solve (Huang & Sun, "A preconditioner based on sine
 * transform for two-dimensional Riesz space fractional diffusion equations in
 * convex domains", arXiv 2102.11576).
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline may call this code.  The GPU library never links it and shares no
 * code, header, table or constant with it.  Everything here is written from
 * the paper's definitions in the paper's order: dense sums instead of FFTs,
 * an O(n^2) sine transform, textbook GMRES.  Compiled with -O2
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Layout: a grid function u is stored x-fastest, u[j*n1 + i] with
 * i = 0..n1-1 standing for the paper's x-index 1..n1 and j for the y-index
 * 1..n2 (the ordering of u^k in Section 2, before Eq. 2.14).
 *
 * Parity status: every function below is pinned by a test in
 * tests/test_oracle_pins.py against a closed form, a textbook or library
 * routine, a theorem of the paper or the paper's printed tables.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------- */
/* Section 1: c_alpha = -1 / (2 cos(alpha pi / 2)), positive for 1<alpha<2. */
double or_c_alpha(double alpha) { return -1.0 / (2.0 * cos(alpha * M_PI / 2.0)); }

/* Eq. 2.6: shifted Grunwald-Letnikov weights g_0 = 1,
 * g_l = (1 - (alpha+1)/l) g_{l-1};  writes g_0 .. g_{count-1}. */
void or_gl_weights(double alpha, int count, double* g) {
  if (count <= 0) return;
  g[0] = 1.0;
  for (int l = 1; l < count; ++l) g[l] = (1.0 - (alpha + 1.0) / (double)l) * g[l - 1];
}

/* Section 2 (definition of c_x, c_y after Eq. 2.10):
 * c = dt * k * c_alpha / h^alpha. */
double or_diffusion_scale(double dt, double k, double alpha, double h) {
  return dt * k * or_c_alpha(alpha) / pow(h, alpha);
}

/* Eq. 2.16: first column of the symmetric Toeplitz G_n^(alpha) times `scale`:
 * t_0 = 2 g_1, t_1 = g_0 + g_2, t_k = g_{k+1} for k >= 2. */
void or_toeplitz_column(double alpha, double scale, int n, double* t) {
  double* g = (double*)malloc(sizeof(double) * (size_t)(n + 2));
  or_gl_weights(alpha, n + 2, g);
  for (int k = 0; k < n; ++k) {
    double v;
    if (k == 0) v = 2.0 * g[1];
    else if (k == 1) v = g[0] + g[2];
    else v = g[k + 1];
    t[k] = scale * v;
  }
  free(g);
}

/* Section 4.1: the orthonormal sine-transform matrix
 * [S_n]_{ij} = sqrt(2/(n+1)) sin(pi i j / (n+1)), 1 <= i,j <= n,
 * applied naively in O(n^2).  The product i*j is reduced modulo 2(n+1)
 * (the period of the sine in that argument) before the sine is taken, so the
 * argument is exact; `sin_tab` may be NULL or hold sin(pi m/(n+1)) for
 * m = 0 .. 2n+1.  in/out are strided so rows and columns of a grid can be
 * transformed in place of a copy. */
static void dst1_strided(int n, const double* in, long in_stride, double* out, long out_stride,
                         const double* sin_tab) {
  const double scale = sqrt(2.0 / (double)(n + 1));
  const long period = 2L * (n + 1);
  for (int k = 1; k <= n; ++k) {
    double acc = 0.0;
    for (int j = 1; j <= n; ++j) {
      long m = ((long)j * (long)k) % period;
      double s = sin_tab ? sin_tab[m] : sin(M_PI * (double)m / (double)(n + 1));
      acc += s * in[(long)(j - 1) * in_stride];
    }
    out[(long)(k - 1) * out_stride] = scale * acc;
  }
}

void or_dst1(int n, const double* v, double* out) {
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  dst1_strided(n, v, 1, tmp, 1, NULL);
  memcpy(out, tmp, sizeof(double) * (size_t)n);
  free(tmp);
}

/* Section 4.1: eigenvalues of the tau matrix tau(T_n) = T_n - H_n, where H_n
 * is the Hankel matrix whose 2n-1 antidiagonals are
 * [t_2, ..., t_{n-1}, 0, 0, 0, t_{n-1}, ..., t_2].  Since tau(T_n) = S L S
 * with S symmetric orthogonal, S tau(T_n) e_1 = L S e_1, so
 * lambda_k = (S tau(T_n) e_1)_k / (S e_1)_k.  The first column of tau(T_n)
 * is t_i - h_i, with h_s the s-th antidiagonal of H_n. */
static double hankel_antidiag(const double* t, int n, int s) {
  if (s + 2 <= n - 1) return t[s + 2];
  if (s >= n + 1 && 2 * n - s >= 2) return t[2 * n - s];
  return 0.0;
}

void or_tau_first_column(int n, const double* t, double* col) {
  for (int i = 0; i < n; ++i) col[i] = t[i] - hankel_antidiag(t, n, i);
}

void or_tau_matrix(int n, const double* t, double* tau /* n*n row-major */) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) tau[(long)i * n + j] = t[abs(i - j)] - hankel_antidiag(t, n, i + j);
}

void or_tau_eigenvalues(int n, const double* t, double* lam) {
  double* col = (double*)malloc(sizeof(double) * (size_t)n);
  double* e1 = (double*)calloc((size_t)n, sizeof(double));
  double* s_col = (double*)malloc(sizeof(double) * (size_t)n);
  double* s_e1 = (double*)malloc(sizeof(double) * (size_t)n);
  or_tau_first_column(n, t, col);
  e1[0] = 1.0;
  dst1_strided(n, col, 1, s_col, 1, NULL);
  dst1_strided(n, e1, 1, s_e1, 1, NULL);
  for (int k = 0; k < n; ++k) lam[k] = s_col[k] / s_e1[k];
  free(col);
  free(e1);
  free(s_col);
  free(s_e1);
}

/* ---------------------------------------------------------------------- */
/* Problem context: the data of one linear system M = I - A + D of Eq. 2.17. */
typedef struct {
  int n1, n2;
  double hx, hy;
  double alpha1, alpha2, kx, ky, dt, eta;
  double cx, cy, pen; /* pen = dt/eta, the penalty entry d_ij outside Omega (Section 2) */
  double *tx, *ty;     /* scaled Toeplitz first columns of A_x = c_x G_{n1}, A_y = c_y G_{n2} */
  double *lamx, *lamy; /* eigenvalues of tau(A_x), tau(A_y) */
  uint8_t* phi;        /* Section 4.1: phi_ij = 1 outside Omega, 0 inside */
  double *sinx, *siny; /* sin(pi m/(n+1)), m = 0..2n+1 */
} or_ctx;

or_ctx* or_setup(int n1, int n2, double ax, double bx, double ay, double by,
                 const uint8_t* in_omega, double alpha1, double alpha2, double kx, double ky,
                 double dt, double eta) {
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->n1 = n1;
  c->n2 = n2;
  c->hx = (bx - ax) / (double)(n1 + 1); /* Section 2: h_x = (b-a)/(n1+1) */
  c->hy = (by - ay) / (double)(n2 + 1);
  c->alpha1 = alpha1;
  c->alpha2 = alpha2;
  c->kx = kx;
  c->ky = ky;
  c->dt = dt;
  c->eta = eta;
  c->cx = or_diffusion_scale(dt, kx, alpha1, c->hx);
  c->cy = or_diffusion_scale(dt, ky, alpha2, c->hy);
  c->pen = dt / eta;
  c->tx = (double*)malloc(sizeof(double) * (size_t)n1);
  c->ty = (double*)malloc(sizeof(double) * (size_t)n2);
  or_toeplitz_column(alpha1, c->cx, n1, c->tx);
  or_toeplitz_column(alpha2, c->cy, n2, c->ty);
  c->lamx = (double*)malloc(sizeof(double) * (size_t)n1);
  c->lamy = (double*)malloc(sizeof(double) * (size_t)n2);
  or_tau_eigenvalues(n1, c->tx, c->lamx);
  or_tau_eigenvalues(n2, c->ty, c->lamy);
  long N = (long)n1 * n2;
  c->phi = (uint8_t*)malloc((size_t)N);
  for (long p = 0; p < N; ++p) c->phi[p] = in_omega[p] ? 0 : 1;
  c->sinx = (double*)malloc(sizeof(double) * (size_t)(2 * n1 + 2));
  c->siny = (double*)malloc(sizeof(double) * (size_t)(2 * n2 + 2));
  for (int m = 0; m < 2 * n1 + 2; ++m) c->sinx[m] = sin(M_PI * (double)m / (double)(n1 + 1));
  for (int m = 0; m < 2 * n2 + 2; ++m) c->siny[m] = sin(M_PI * (double)m / (double)(n2 + 1));
  return c;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->tx);
  free(c->ty);
  free(c->lamx);
  free(c->lamy);
  free(c->phi);
  free(c->sinx);
  free(c->siny);
  free(c);
}

void or_get_params(const or_ctx* c, double* out /* hx hy cx cy pen */) {
  out[0] = c->hx;
  out[1] = c->hy;
  out[2] = c->cx;
  out[3] = c->cy;
  out[4] = c->pen;
}
void or_get_toeplitz(const or_ctx* c, double* tx, double* ty) {
  memcpy(tx, c->tx, sizeof(double) * (size_t)c->n1);
  memcpy(ty, c->ty, sizeof(double) * (size_t)c->n2);
}
void or_get_tau_eigs(const or_ctx* c, double* lx, double* ly) {
  memcpy(lx, c->lamx, sizeof(double) * (size_t)c->n1);
  memcpy(ly, c->lamy, sizeof(double) * (size_t)c->n2);
}

/* Eq. 2.14-2.17: w = M z = z - (I (x) A_x) z - (A_y (x) I) z + D z, with the
 * Toeplitz sums written out entry by entry and D = (dt/eta) Phi. */
void or_apply_M(const or_ctx* c, const double* z, double* w) {
  const int n1 = c->n1, n2 = c->n2;
  for (int j = 0; j < n2; ++j) {
    for (int i = 0; i < n1; ++i) {
      double ax = 0.0, ay = 0.0;
      for (int l = 0; l < n1; ++l) ax += c->tx[abs(i - l)] * z[(long)j * n1 + l];
      for (int l = 0; l < n2; ++l) ay += c->ty[abs(j - l)] * z[(long)l * n1 + i];
      long p = (long)j * n1 + i;
      double d = c->phi[p] ? c->pen : 0.0;
      w[p] = z[p] - ax - ay + d * z[p];
    }
  }
}

/* (M z) at the flat grid indices idx[0..npts-1] only: the same sums as
 * or_apply_M, for spot checks of grids too large for a full product. */
void or_apply_M_points(const or_ctx* c, const double* z, long npts, const long* idx, double* out) {
  const int n1 = c->n1, n2 = c->n2;
  for (long q = 0; q < npts; ++q) {
    long p = idx[q];
    int j = (int)(p / n1), i = (int)(p % n1);
    double ax = 0.0, ay = 0.0;
    for (int l = 0; l < n1; ++l) ax += c->tx[abs(i - l)] * z[(long)j * n1 + l];
    for (int l = 0; l < n2; ++l) ay += c->ty[abs(j - l)] * z[(long)l * n1 + i];
    double d = c->phi[p] ? c->pen : 0.0;
    out[q] = z[p] - ax - ay + d * z[p];
  }
}

/* (S_{n2} (x) S_{n1}) v: sine transform of every row (x), then every column (y). */
void or_dst2(const or_ctx* c, const double* v, double* out) {
  const int n1 = c->n1, n2 = c->n2;
  long N = (long)n1 * n2;
  double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
  for (int j = 0; j < n2; ++j) dst1_strided(n1, v + (long)j * n1, 1, tmp + (long)j * n1, 1, c->sinx);
  for (int i = 0; i < n1; ++i) dst1_strided(n2, tmp + i, n1, out + i, n1, c->siny);
  free(tmp);
}

/* The first `count` row (x) or column (y) sine transforms that or_dst2 performs,
 * with the same table-driven routine; used to time a bounded sample of the
 * oracle's transform work on grids too large to transform whole. */
void or_dst2_rows_sample(const or_ctx* c, const double* v, int count, double* out) {
  for (int j = 0; j < count && j < c->n2; ++j)
    dst1_strided(c->n1, v + (long)j * c->n1, 1, out + (long)j * c->n1, 1, c->sinx);
}
void or_dst2_cols_sample(const or_ctx* c, const double* v, int count, double* out) {
  for (int i = 0; i < count && i < c->n1; ++i) dst1_strided(c->n2, v + i, c->n1, out + i, c->n1, c->siny);
}

/* Eq. 4.6: z = P^-1 v = (I - Phi)(I - tau_1(A))^-1 v + Phi((1 + dt/eta) I - tau_1(A))^-1 v,
 * with I - tau_1(A) = (S (x) S)(I - I (x) L_x - L_y (x) I)(S (x) S) (proof of Lemma 4.2). */
void or_apply_precond(const or_ctx* c, const double* v, double* z) {
  const int n1 = c->n1, n2 = c->n2;
  long N = (long)n1 * n2;
  double* W = (double*)malloc(sizeof(double) * (size_t)N);
  double* W1 = (double*)malloc(sizeof(double) * (size_t)N);
  double* W2 = (double*)malloc(sizeof(double) * (size_t)N);
  or_dst2(c, v, W);
  for (int j = 0; j < n2; ++j)
    for (int i = 0; i < n1; ++i) {
      long p = (long)j * n1 + i;
      W1[p] = W[p] / (1.0 - c->lamx[i] - c->lamy[j]);
      W2[p] = W[p] / (1.0 + c->pen - c->lamx[i] - c->lamy[j]);
    }
  double* z1 = W;   /* reuse */
  double* z2 = (double*)malloc(sizeof(double) * (size_t)N);
  or_dst2(c, W1, z1);
  or_dst2(c, W2, z2);
  for (long p = 0; p < N; ++p) z[p] = c->phi[p] ? z2[p] : z1[p];
  free(W);
  free(W1);
  free(W2);
  free(z2);
}

/* ---------------------------------------------------------------------- */
/* Textbook Krylov solvers (Section 5: GMRES with restart and the tau preconditioner). */
static double dot(long N, const double* a, const double* b) {
  double s = 0.0;
  for (long p = 0; p < N; ++p) s += a[p] * b[p];
  return s;
}
static double nrm2(long N, const double* a) { return sqrt(dot(N, a, a)); }

/* Givens rotation zeroing b in (a, b). */
static void givens(double a, double b, double* cs, double* sn) {
  if (b == 0.0) {
    *cs = 1.0;
    *sn = 0.0;
    return;
  }
  double r = hypot(a, b);
  *cs = a / r;
  *sn = b / r;
}

/* Right-preconditioned flexible GMRES(m) (Saad's FGMRES) with modified
 * Gram-Schmidt and Givens rotations.  Stops when the true residual satisfies
 * ||b - M x||_2 <= tol ||b||_2 (checked explicitly at the end of each cycle;
 * a cycle ends early when the Givens estimate |g_{j+1}| <= tol ||b||).
 * use_precond = 0 replaces P^-1 by the identity.
 * Returns 0 on convergence, 1 if max_iter inner iterations were used first.
 * out_stats: [iterations, restarts, final true relative residual]. */
int or_fgmres(const or_ctx* c, const double* b, double* x, int m, double tol, int max_iter,
              int use_precond, double* out_stats) {
  const long N = (long)c->n1 * c->n2;
  double* V = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(m + 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)N * (size_t)m);
  double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m + j] */
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)m);
  double* r = (double*)malloc(sizeof(double) * (size_t)N);
  int iters = 0, restarts = 0, status = 1;
  const double bnorm = nrm2(N, b);
  double beta;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)N);
    status = 0;
    beta = 0.0;
    goto done;
  }
  or_apply_M(c, x, r);
  for (long p = 0; p < N; ++p) r[p] = b[p] - r[p];
  beta = nrm2(N, r);
  while (1) {
    if (beta <= tol * bnorm) {
      status = 0;
      break;
    }
    if (iters >= max_iter) break;
    for (long p = 0; p < N; ++p) V[p] = r[p] / beta;
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    g[0] = beta;
    int jlast = 0;
    for (int j = 0; j < m && iters < max_iter; ++j) {
      double* vj = V + (long)j * N;
      double* zj = Z + (long)j * N;
      double* w = V + (long)(j + 1) * N;
      if (use_precond) or_apply_precond(c, vj, zj);
      else memcpy(zj, vj, sizeof(double) * (size_t)N);
      or_apply_M(c, zj, w);
      for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
        double h = dot(N, w, V + (long)i * N);
        H[(long)i * m + j] = h;
        for (long p = 0; p < N; ++p) w[p] -= h * V[(long)i * N + p];
      }
      double hn = nrm2(N, w);
      H[(long)(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (long p = 0; p < N; ++p) w[p] /= hn;
      for (int i = 0; i < j; ++i) { /* apply the stored rotations to column j */
        double a = H[(long)i * m + j], bb = H[(long)(i + 1) * m + j];
        H[(long)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(long)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      givens(H[(long)j * m + j], H[(long)(j + 1) * m + j], &cs[j], &sn[j]);
      H[(long)j * m + j] = cs[j] * H[(long)j * m + j] + sn[j] * H[(long)(j + 1) * m + j];
      H[(long)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      jlast = j + 1;
      if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = jlast - 1; i >= 0; --i) { /* back substitution H y = g */
      double s = g[i];
      for (int k = i + 1; k < jlast; ++k) s -= H[(long)i * m + k] * y[k];
      y[i] = s / H[(long)i * m + i];
    }
    for (int i = 0; i < jlast; ++i)
      for (long p = 0; p < N; ++p) x[p] += y[i] * Z[(long)i * N + p];
    or_apply_M(c, x, r);
    for (long p = 0; p < N; ++p) r[p] = b[p] - r[p];
    beta = nrm2(N, r);
    if (beta <= tol * bnorm) {
      status = 0;
      break;
    }
    ++restarts;
  }
done:
  if (out_stats) {
    out_stats[0] = iters;
    out_stats[1] = restarts;
    out_stats[2] = bnorm == 0.0 ? 0.0 : beta / bnorm;
  }
  free(V);
  free(Z);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(y);
  free(r);
  return status;
}

/* Left-preconditioned GMRES(m) as the experiments of Section 5 run it: the
 * system P^-1 M x = P^-1 b, stopped when ||P^-1 (b - M x)||_2 / ||P^-1 b||_2 < tol
 * (the Givens estimate ends a cycle; the preconditioned residual is then
 * recomputed and tested).  use_precond = 0 gives plain GMRES.  Returns 0 on
 * convergence.  out_stats: [iterations, restarts, final preconditioned relres]. */
int or_gmres_left(const or_ctx* c, const double* b, double* x, int m, double tol, int max_iter,
                  int use_precond, double* out_stats) {
  const long N = (long)c->n1 * c->n2;
  double* V = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)m);
  double* r = (double*)malloc(sizeof(double) * (size_t)N);
  double* t = (double*)malloc(sizeof(double) * (size_t)N);
  int iters = 0, restarts = 0, status = 1;
  double pbnorm, beta;
#define PREC(in, out)                                                   \
  do {                                                                  \
    if (use_precond) or_apply_precond(c, in, out);                      \
    else memcpy(out, in, sizeof(double) * (size_t)N);                   \
  } while (0)
  PREC(b, t);
  pbnorm = nrm2(N, t);
  if (pbnorm == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)N);
    status = 0;
    beta = 0.0;
    goto done;
  }
  or_apply_M(c, x, t);
  for (long p = 0; p < N; ++p) t[p] = b[p] - t[p];
  PREC(t, r);
  beta = nrm2(N, r);
  while (1) {
    if (beta / pbnorm < tol) {
      status = 0;
      break;
    }
    if (iters >= max_iter) break;
    for (long p = 0; p < N; ++p) V[p] = r[p] / beta;
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    g[0] = beta;
    int jlast = 0;
    for (int j = 0; j < m && iters < max_iter; ++j) {
      double* w = V + (long)(j + 1) * N;
      or_apply_M(c, V + (long)j * N, t);
      PREC(t, w);
      for (int i = 0; i <= j; ++i) {
        double h = dot(N, w, V + (long)i * N);
        H[(long)i * m + j] = h;
        for (long p = 0; p < N; ++p) w[p] -= h * V[(long)i * N + p];
      }
      double hn = nrm2(N, w);
      H[(long)(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (long p = 0; p < N; ++p) w[p] /= hn;
      for (int i = 0; i < j; ++i) {
        double a = H[(long)i * m + j], bb = H[(long)(i + 1) * m + j];
        H[(long)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(long)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      givens(H[(long)j * m + j], H[(long)(j + 1) * m + j], &cs[j], &sn[j]);
      H[(long)j * m + j] = cs[j] * H[(long)j * m + j] + sn[j] * H[(long)(j + 1) * m + j];
      H[(long)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      jlast = j + 1;
      if (fabs(g[j + 1]) / pbnorm < tol || hn == 0.0) break;
    }
    for (int i = jlast - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jlast; ++k) s -= H[(long)i * m + k] * y[k];
      y[i] = s / H[(long)i * m + i];
    }
    for (int i = 0; i < jlast; ++i)
      for (long p = 0; p < N; ++p) x[p] += y[i] * V[(long)i * N + p];
    or_apply_M(c, x, t);
    for (long p = 0; p < N; ++p) t[p] = b[p] - t[p];
    PREC(t, r);
    beta = nrm2(N, r);
    if (beta / pbnorm < tol) {
      status = 0;
      break;
    }
    ++restarts;
  }
#undef PREC
done:
  if (out_stats) {
    out_stats[0] = iters;
    out_stats[1] = restarts;
    out_stats[2] = pbnorm == 0.0 ? 0.0 : beta / pbnorm;
  }
  free(V);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(y);
  free(r);
  free(t);
  return status;
}

/* ---------------------------------------------------------------------- */
/* Time march, Eq. 2.17 with the built-in source f(u) = u - u^3 (+ s), zero
 * outside Omega (Section 2, zero extension of f):
 *   b = u^{k-1} + dt (1 - phi) (u^{k-1} - (u^{k-1})^3 + s). */
void or_rhs(const or_ctx* c, const double* u_prev, const double* src, double* b) {
  const long N = (long)c->n1 * c->n2;
  for (long p = 0; p < N; ++p) {
    double u = u_prev[p];
    double f = u - u * u * u + (src ? src[p] : 0.0);
    b[p] = u + (c->phi[p] ? 0.0 : c->dt * f);
  }
}

/* Section 5 initial guess: u^{k-1} for the first step, else 2 u^{k-1} - u^{k-2}. */
void or_initial_guess(long N, const double* u_prev, const double* u_prevprev, double* x0) {
  for (long p = 0; p < N; ++p) x0[p] = u_prevprev ? 2.0 * u_prev[p] - u_prevprev[p] : u_prev[p];
}

/* One implicit step: b from or_rhs, x_0 from or_initial_guess, FGMRES(m). */
int or_step(const or_ctx* c, const double* u_prev, const double* u_prevprev, const double* src,
            double* u_next, int m, double tol, int max_iter, double* out_stats) {
  const long N = (long)c->n1 * c->n2;
  double* b = (double*)malloc(sizeof(double) * (size_t)N);
  or_rhs(c, u_prev, src, b);
  or_initial_guess(N, u_prev, u_prevprev, u_next);
  int st = or_fgmres(c, b, u_next, m, tol, max_iter, 1, out_stats);
  free(b);
  return st;
}

/* ---------------------------------------------------------------------- */
/* Discrete adjoint of the march (the paper has no gradient; this is the
 * exact derivative of the scheme of Eq. 2.17 with f(u) = u - u^3 + s):
 * L = sum_cells (u^m - target)^2.  With lambda^m = 2 (u^m - target), for
 * k = m..1:  M mu^k = lambda^k  (M symmetric, Lemma 2.3),
 *            lambda^{k-1} = mu^k + dt (1 - phi)(1 - 3 (u^{k-1})^2) mu^k,
 *            dL/ds += dt (1 - phi) mu^k,
 *            dL/dk_x += <mu^k, (I (x) A_x) u^k> / k_x   (A_x is linear in k_x),
 *            dL/dk_y += <mu^k, (A_y (x) I) u^k> / k_y,
 * and dL/du0 = lambda^0.  All states are kept (small grids only).
 * Returns the loss; g_k = [dL/dk_x, dL/dk_y]. */
static void apply_Ax(const or_ctx* c, const double* z, double* w) {
  for (int j = 0; j < c->n2; ++j)
    for (int i = 0; i < c->n1; ++i) {
      double a = 0.0;
      for (int l = 0; l < c->n1; ++l) a += c->tx[abs(i - l)] * z[(long)j * c->n1 + l];
      w[(long)j * c->n1 + i] = a;
    }
}
static void apply_Ay(const or_ctx* c, const double* z, double* w) {
  for (int j = 0; j < c->n2; ++j)
    for (int i = 0; i < c->n1; ++i) {
      double a = 0.0;
      for (int l = 0; l < c->n2; ++l) a += c->ty[abs(j - l)] * z[(long)l * c->n1 + i];
      w[(long)j * c->n1 + i] = a;
    }
}

double or_adjoint_march(const or_ctx* c, const double* u0, const double* src, int steps, const double* target,
                        int m, double tol, double* u_final, double* g_u0, double* g_src, double* g_k) {
  const long N = (long)c->n1 * c->n2;
  double* U = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(steps + 1));
  double* lam = (double*)malloc(sizeof(double) * (size_t)N);
  double* mu = (double*)malloc(sizeof(double) * (size_t)N);
  double* t = (double*)malloc(sizeof(double) * (size_t)N);
  memcpy(U, u0, sizeof(double) * (size_t)N);
  for (int k = 1; k <= steps; ++k)
    or_step(c, U + (long)(k - 1) * N, k >= 2 ? U + (long)(k - 2) * N : NULL, src, U + (long)k * N, m, tol,
            100000, NULL);
  const double* um = U + (long)steps * N;
  double loss = 0.0;
  for (long p = 0; p < N; ++p) {
    double d = um[p] - target[p];
    loss += d * d;
    lam[p] = 2.0 * d;
  }
  if (u_final) memcpy(u_final, um, sizeof(double) * (size_t)N);
  if (g_src) memset(g_src, 0, sizeof(double) * (size_t)N);
  g_k[0] = g_k[1] = 0.0;
  for (int k = steps; k >= 1; --k) {
    const double* uk = U + (long)k * N;
    const double* ukm1 = U + (long)(k - 1) * N;
    memset(mu, 0, sizeof(double) * (size_t)N);
    or_fgmres(c, lam, mu, m, tol, 100000, 1, NULL);
    apply_Ax(c, uk, t);
    double sx = 0.0, sy = 0.0;
    for (long p = 0; p < N; ++p) sx += mu[p] * t[p];
    apply_Ay(c, uk, t);
    for (long p = 0; p < N; ++p) sy += mu[p] * t[p];
    g_k[0] += sx / c->kx;
    g_k[1] += sy / c->ky;
    for (long p = 0; p < N; ++p) {
      double out = c->phi[p] ? 0.0 : 1.0;
      if (g_src) g_src[p] += c->dt * out * mu[p];
      lam[p] = mu[p] + c->dt * out * (1.0 - 3.0 * ukm1[p] * ukm1[p]) * mu[p];
    }
  }
  if (g_u0) memcpy(g_u0, lam, sizeof(double) * (size_t)N);
  free(U);
  free(lam);
  free(mu);
  free(t);
  return loss;
}

/* ---------------------------------------------------------------------- */
/* Dense path for tiny grids: M assembled column by column from Eq. 2.17
 * (M e_q), then textbook LU with partial pivoting. */
void or_assemble_dense(const or_ctx* c, double* Md /* N*N row-major */) {
  const long N = (long)c->n1 * c->n2;
  double* e = (double*)calloc((size_t)N, sizeof(double));
  double* col = (double*)malloc(sizeof(double) * (size_t)N);
  for (long q = 0; q < N; ++q) {
    e[q] = 1.0;
    or_apply_M(c, e, col);
    for (long p = 0; p < N; ++p) Md[p * N + q] = col[p];
    e[q] = 0.0;
  }
  free(e);
  free(col);
}

/* Solves A x = b in place (A overwritten by its LU factors, b by x).
 * Returns 0, or 1 if a zero pivot is met. */
int or_lu_solve(long N, double* A, double* b) {
  for (long k = 0; k < N; ++k) {
    long piv = k;
    double best = fabs(A[k * N + k]);
    for (long i = k + 1; i < N; ++i)
      if (fabs(A[i * N + k]) > best) {
        best = fabs(A[i * N + k]);
        piv = i;
      }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (long j = 0; j < N; ++j) {
        double tmp = A[k * N + j];
        A[k * N + j] = A[piv * N + j];
        A[piv * N + j] = tmp;
      }
      double tmp = b[k];
      b[k] = b[piv];
      b[piv] = tmp;
    }
    for (long i = k + 1; i < N; ++i) {
      double l = A[i * N + k] / A[k * N + k];
      A[i * N + k] = l;
      for (long j = k + 1; j < N; ++j) A[i * N + j] -= l * A[k * N + j];
      b[i] -= l * b[k];
    }
  }
  for (long i = N - 1; i >= 0; --i) {
    double s = b[i];
    for (long j = i + 1; j < N; ++j) s -= A[i * N + j] * b[j];
    b[i] = s / A[i * N + i];
  }
  return 0;
}
