/*
 * FP64 CPU oracle for the spectrahedron boundary oracle and the random walks
 * built on it (arXiv 2010.03817, "Efficient Sampling from Feasible Sets of
 * SDPs and Volume Approximation").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  It shares no code, header, table or
 * constant with the CUDA path.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product never does.
 *
 * Everything works on full m x m row-major matrices, in double precision,
 * one obvious step at a time:
 *
 *   F(x) = A_0 + sum_i x_i A_i                        (Eq. 1, the LMI)
 *   membership: Cholesky of F(x) succeeds             (Sec. 2.2, Alg. 1; F > 0)
 *   intersection: t+ = smallest positive, t- = largest negative root of
 *       det(F(p) + t V), V = sum_i v_i A_i            (Sec. 2.3, Alg. 2,
 *       Lemma "PEP and S cap C": a degree-1 PEP for a line)
 *     computed as t = 1/mu over the eigenvalues mu of M = -L^{-1} V L^{-T},
 *     F(p) = L L^T, by a cyclic Jacobi eigensolver (Sec. 4: the paper solves
 *     the pencil by a largest-eigenvalue routine after a transformation).
 *   normal: w_j = u^T A_j u, u in ker F(p + t+ v)     (Lemma "Gradient of
 *       det F", Sec. 2.4)
 *   reflection: s = v - 2 <v, w^> w^, w^ = w/|w|      (Eq. "reflection", Alg. 3)
 *   Hit-and-Run step                                   (Sec. 3.1, Alg. 4)
 *   Coordinate-direction Hit-and-Run step              (Sec. 3.1, CDHR)
 *   Billiard step                                      (Sec. 3.2, Alg. 5)
 *
 * Accuracy steps (not in the paper, which leaves precision open, Sec. 4):
 *   - after Jacobi, t+ is re-evaluated as the pencil Rayleigh quotient
 *     t = -(u^T F u)/(u^T V u), which is stationary at the eigenvector, with
 *     compensated dot products (Ogita, Rump, Oishi 2005, "Accurate sum and dot
 *     product", Dot2);
 *   - u is polished by two steps of inverse iteration on F + t V (Wilkinson),
 *     solved by Gaussian elimination with partial pivoting.
 *   The difference between the Jacobi value and the refined value is returned
 *   as the oracle's own error bar.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011,
 * "Parallel random numbers: as easy as 1, 2, 3"), written from its published
 * definition; uniforms on (0,1) from 52 random bits; Gaussians by Box-Muller.
 * Counter layout: (chain, step, stream, index), key = (seed low, seed high).
 *   stream 0: direction (index i gives Gaussians 2i, 2i+1)
 *   stream 1: eta (Billiard length, Hit-and-Run chord position)
 *   stream 2: coordinate index (CDHR)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_PD 1
#define ORC_UNBOUNDED 2
#define ORC_NOCONV 3
#define ORC_RHO 4
#define ORC_DEGENERATE 5
#define ORC_EINVAL 6

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  /* round multipliers and Weyl key increments of Philox4x32 (Salmon et al.) */
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c0, &hi0, &lo0);
    mulhilo32(M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 52 random bits -> (2k+1) 2^-53, exactly representable, strictly in (0,1) */
double orc_u01(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return (double)(2 * k + 1) * 0x1p-53;
}

static void philox_draw(uint64_t seed, uint32_t chain, uint32_t step, uint32_t stream,
                        uint32_t index, uint32_t out[4]) {
  uint32_t ctr[4] = {chain, step, stream, index};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* uniform on (0,1) for (chain, step, stream) */
double orc_uniform(uint64_t seed, uint32_t chain, uint32_t step, uint32_t stream) {
  uint32_t r[4];
  philox_draw(seed, chain, step, stream, 0, r);
  return orc_u01(r[0], r[1]);
}

/* standard normal vector g[0..n-1] by Box-Muller */
void orc_gaussians(int n, uint64_t seed, uint32_t chain, uint32_t step, double* g) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; 2 * i < n; ++i) {
    uint32_t r[4];
    philox_draw(seed, chain, step, 0, (uint32_t)i, r);
    double u1 = orc_u01(r[0], r[1]);
    double u2 = orc_u01(r[2], r[3]);
    double rad = sqrt(-2.0 * log(u1));
    double th = two_pi * u2;
    g[2 * i] = rad * cos(th);
    if (2 * i + 1 < n) g[2 * i + 1] = rad * sin(th);
  }
}

/* v ~ U(unit sphere) as a normalised Gaussian (Alg. 4 and Alg. 5) */
void orc_direction(int n, uint64_t seed, uint32_t chain, uint32_t step, double* v) {
  orc_gaussians(n, seed, chain, step, v);
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += v[i] * v[i];
  s = sqrt(s);
  for (int i = 0; i < n; ++i) v[i] /= s;
}

/* ------------------------------------------------------------------------ */
/* Compensated arithmetic (Ogita-Rump-Oishi, TwoSum / TwoProduct / Dot2)    */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static void two_sum(double a, double b, double* s, double* e) {
  *s = a + b;
  double z = *s - a;
  *e = (a - (*s - z)) + (b - z);
}

static void dd_add_prod(dd* acc, double a, double b) {
  double p = a * b;
  double pe = fma(a, b, -p);
  double s, e;
  two_sum(acc->hi, p, &s, &e);
  acc->hi = s;
  acc->lo += e + pe;
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra, row-major m x m                                     */
/* ------------------------------------------------------------------------ */
#define IDX(i, j, m) ((size_t)(i) * (size_t)(m) + (size_t)(j))

/* out = c0 * A_0 + sum_{i=1..n} c[i-1] * A_i   (Eq. 1) */
void orc_lmi(int n, int m, const double* A, double c0, const double* c, double* out) {
  size_t mm = (size_t)m * m;
  for (size_t e = 0; e < mm; ++e) out[e] = c0 * A[e];
  for (int i = 1; i <= n; ++i) {
    double ci = c[i - 1];
    if (ci == 0.0) continue;
    const double* Ai = A + (size_t)i * mm;
    for (size_t e = 0; e < mm; ++e) out[e] += ci * Ai[e];
  }
}

/* textbook Cholesky F = L L^T; returns 0, or k+1 if the pivot of column k is
 * not positive (F is not positive definite) */
int orc_cholesky(int m, const double* F, double* L) {
  memset(L, 0, sizeof(double) * (size_t)m * m);
  for (int j = 0; j < m; ++j) {
    double d = F[IDX(j, j, m)];
    for (int k = 0; k < j; ++k) d -= L[IDX(j, k, m)] * L[IDX(j, k, m)];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    L[IDX(j, j, m)] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double s = F[IDX(i, j, m)];
      for (int k = 0; k < j; ++k) s -= L[IDX(i, k, m)] * L[IDX(j, k, m)];
      L[IDX(i, j, m)] = s / ljj;
    }
  }
  return 0;
}

/* membership test in the strict sense: F(x) > 0 (Alg. 1 with the interior
 * read as positive definite) */
int orc_membership(int n, int m, const double* A, const double* x) {
  double* F = (double*)malloc(sizeof(double) * (size_t)m * m);
  double* L = (double*)malloc(sizeof(double) * (size_t)m * m);
  orc_lmi(n, m, A, 1.0, x, F);
  int r = orc_cholesky(m, F, L);
  free(F);
  free(L);
  return r == 0;
}

/* cyclic Jacobi eigensolver for a symmetric matrix (Golub & Van Loan,
 * "Matrix Computations", symmetric Schur decomposition and cyclic Jacobi).
 * S is overwritten; evals[k] and column k of Q (row-major, Q[i*m+k]) are the
 * eigenpairs.  Returns the number of sweeps, or -1 if not converged. */
int orc_jacobi(int m, double* S, double* evals, double* Q, int max_sweeps) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Q[IDX(i, j, m)] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (size_t e = 0; e < (size_t)m * m; ++e) fro += S[e] * S[e];
  fro = sqrt(fro);
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += 2.0 * S[IDX(p, q, m)] * S[IDX(p, q, m)];
    if (sqrt(off) <= 1e-17 * fro || fro == 0.0) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        double apq = S[IDX(p, q, m)];
        if (apq == 0.0) continue;
        double app = S[IDX(p, p, m)], aqq = S[IDX(q, q, m)];
        /* rotation that zeroes S[p][q] */
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* S <- J^T S J with J the rotation in the (p,q) plane */
        for (int k = 0; k < m; ++k) {
          double skp = S[IDX(k, p, m)], skq = S[IDX(k, q, m)];
          S[IDX(k, p, m)] = c * skp - s * skq;
          S[IDX(k, q, m)] = s * skp + c * skq;
        }
        for (int k = 0; k < m; ++k) {
          double spk = S[IDX(p, k, m)], sqk = S[IDX(q, k, m)];
          S[IDX(p, k, m)] = c * spk - s * sqk;
          S[IDX(q, k, m)] = s * spk + c * sqk;
        }
        S[IDX(p, q, m)] = 0.0;
        S[IDX(q, p, m)] = 0.0;
        for (int k = 0; k < m; ++k) {
          double qkp = Q[IDX(k, p, m)], qkq = Q[IDX(k, q, m)];
          Q[IDX(k, p, m)] = c * qkp - s * qkq;
          Q[IDX(k, q, m)] = s * qkp + c * qkq;
        }
      }
    }
  }
  for (int k = 0; k < m; ++k) evals[k] = S[IDX(k, k, m)];
  return sweep < max_sweeps ? sweep : -1;
}

/* solve L y = b (L lower triangular, row-major) */
static void fwd_subst(int m, const double* L, const double* b, double* y) {
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[IDX(i, k, m)] * y[k];
    y[i] = s / L[IDX(i, i, m)];
  }
}

/* solve L^T y = b */
static void back_subst_t(int m, const double* L, const double* b, double* y) {
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < m; ++k) s -= L[IDX(k, i, m)] * y[k];
    y[i] = s / L[IDX(i, i, m)];
  }
}

/* M = -L^{-1} V L^{-T}, symmetrised */
static void pencil_matrix(int m, const double* L, const double* V, double* M) {
  double* X = (double*)malloc(sizeof(double) * (size_t)m * m); /* X = L^{-1} V, column by column */
  double* col = (double*)malloc(sizeof(double) * m);
  double* res = (double*)malloc(sizeof(double) * m);
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) col[i] = V[IDX(i, j, m)];
    fwd_subst(m, L, col, res);
    for (int i = 0; i < m; ++i) X[IDX(i, j, m)] = res[i];
  }
  /* (L^{-1} V L^{-T})^T = L^{-1} X^T: column j of it is L^{-1} (row j of X) */
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) col[i] = X[IDX(j, i, m)];
    fwd_subst(m, L, col, res);
    for (int i = 0; i < m; ++i) M[IDX(j, i, m)] = -res[i]; /* transpose back */
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      double a = 0.5 * (M[IDX(i, j, m)] + M[IDX(j, i, m)]);
      M[IDX(i, j, m)] = a;
      M[IDX(j, i, m)] = a;
    }
  free(X);
  free(col);
  free(res);
}

/* w_j = u^T A_j u for j = 0..n, each in compensated (double-double) form */
static void quad_forms_dd(int n, int m, const double* A, const double* u, dd* w) {
  size_t mm = (size_t)m * m;
  for (int j = 0; j <= n; ++j) {
    const double* Aj = A + (size_t)j * mm;
    dd acc = {0.0, 0.0};
    for (int a = 0; a < m; ++a) {
      dd z = {0.0, 0.0};
      for (int b = 0; b < m; ++b) dd_add_prod(&z, Aj[IDX(a, b, m)], u[b]);
      dd_add_prod(&acc, u[a], z.hi);
      dd_add_prod(&acc, u[a], z.lo);
    }
    w[j] = acc;
  }
}

/* pencil Rayleigh quotient t = -(u^T F(p) u)/(u^T V u) from the quadratic
 * forms w_j: u^T F(p) u = w_0 + sum p_j w_j, u^T V u = sum v_j w_j */
static double rayleigh_t(int n, const dd* w, const double* p, const double* v) {
  dd num = {0.0, 0.0}, den = {0.0, 0.0};
  dd_add_prod(&num, 1.0, w[0].hi);
  dd_add_prod(&num, 1.0, w[0].lo);
  for (int j = 1; j <= n; ++j) {
    dd_add_prod(&num, p[j - 1], w[j].hi);
    dd_add_prod(&num, p[j - 1], w[j].lo);
    dd_add_prod(&den, v[j - 1], w[j].hi);
    dd_add_prod(&den, v[j - 1], w[j].lo);
  }
  return -(num.hi + num.lo) / (den.hi + den.lo);
}

/* inverse iteration step: z = G^{-1} u by Gaussian elimination with partial
 * pivoting; pivots below eps*|G| are replaced by eps*|G| (G is singular to
 * working precision by construction).  u <- z/|z|. */
static void inverse_iteration(int m, const double* G_in, double* u) {
  double* G = (double*)malloc(sizeof(double) * (size_t)m * m);
  double* b = (double*)malloc(sizeof(double) * m);
  memcpy(G, G_in, sizeof(double) * (size_t)m * m);
  memcpy(b, u, sizeof(double) * m);
  double gmax = 0.0;
  for (size_t e = 0; e < (size_t)m * m; ++e) gmax = fmax(gmax, fabs(G[e]));
  double tiny = 2.220446049250313e-16 * gmax * m;
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(G[IDX(i, k, m)]) > fabs(G[IDX(piv, k, m)])) piv = i;
    if (piv != k) {
      for (int j = 0; j < m; ++j) {
        double t = G[IDX(k, j, m)];
        G[IDX(k, j, m)] = G[IDX(piv, j, m)];
        G[IDX(piv, j, m)] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    if (fabs(G[IDX(k, k, m)]) < tiny) G[IDX(k, k, m)] = (G[IDX(k, k, m)] < 0.0 ? -tiny : tiny);
    for (int i = k + 1; i < m; ++i) {
      double f = G[IDX(i, k, m)] / G[IDX(k, k, m)];
      if (f == 0.0) continue;
      for (int j = k; j < m; ++j) G[IDX(i, j, m)] -= f * G[IDX(k, j, m)];
      b[i] -= f * b[k];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < m; ++j) s -= G[IDX(i, j, m)] * u[j];
    u[i] = s / G[IDX(i, i, m)];
  }
  double nrm = 0.0;
  for (int i = 0; i < m; ++i) nrm += u[i] * u[i];
  nrm = sqrt(nrm);
  for (int i = 0; i < m; ++i) u[i] /= nrm;
  free(G);
  free(b);
}

/* sign convention for returned null vectors: unit length, largest-magnitude
 * entry positive (the null vector is defined up to sign and scale) */
static void normalise_sign(int m, double* u) {
  double nrm = 0.0;
  int big = 0;
  for (int i = 0; i < m; ++i) {
    nrm += u[i] * u[i];
    if (fabs(u[i]) > fabs(u[big])) big = i;
  }
  nrm = sqrt(nrm);
  double s = (u[big] < 0.0 ? -1.0 : 1.0) / nrm;
  for (int i = 0; i < m; ++i) u[i] *= s;
}

/* Refine one end of the chord: Rayleigh quotient, two inverse-iteration
 * polishes of u on F + tV, Rayleigh quotient again.  On return u is the unit
 * null vector and w[0..n] its quadratic forms. */
static double refine_end(int n, int m, const double* A, const double* p, const double* v,
                         const double* F, const double* V, double t, double* u, dd* w) {
  double* G = (double*)malloc(sizeof(double) * (size_t)m * m);
  quad_forms_dd(n, m, A, u, w);
  t = rayleigh_t(n, w, p, v);
  for (int it = 0; it < 2; ++it) {
    for (size_t e = 0; e < (size_t)m * m; ++e) G[e] = F[e] + t * V[e];
    inverse_iteration(m, G, u);
    quad_forms_dd(n, m, A, u, w);
    t = rayleigh_t(n, w, p, v);
  }
  normalise_sign(m, u);
  quad_forms_dd(n, m, A, u, w);
  free(G);
  return t;
}

/*
 * INTERSECTION (Alg. 2) for the line p + t v.
 *   out: t_minus (-INF if none), t_plus (+INF if none), u_plus[m] and
 *        u_minus[m] (unit null vectors, may be NULL), w_plus[n+1] (u+^T A_j u+,
 *        j = 0..n, may be NULL), info[4] (may be NULL):
 *        info[0] = |t+ (Jacobi) - t+ (refined)| / |t+|   (oracle error bar)
 *        info[1] = relative eigengap (mu_max - mu_2)/|mu_max|
 *        info[2] = Jacobi sweeps
 *        info[3] = |t- (Jacobi) - t- (refined)| / |t-|
 *   returns ORC_OK, ORC_NOT_PD (p not interior), ORC_NOCONV.
 *   t_plus = +INF (ORC_OK) means the ray is unbounded: S is assumed bounded,
 *   so callers treat it as an error.
 */
int orc_intersect(int n, int m, const double* A, const double* p, const double* v,
                  double* t_minus, double* t_plus, double* u_plus, double* u_minus,
                  double* w_plus, double* info) {
  size_t mm = (size_t)m * m;
  double* F = (double*)malloc(sizeof(double) * mm);
  double* V = (double*)malloc(sizeof(double) * mm);
  double* L = (double*)malloc(sizeof(double) * mm);
  double* M = (double*)malloc(sizeof(double) * mm);
  double* Q = (double*)malloc(sizeof(double) * mm);
  double* ev = (double*)malloc(sizeof(double) * m);
  double* y = (double*)malloc(sizeof(double) * m);
  double* up = (double*)malloc(sizeof(double) * m);
  double* um = (double*)malloc(sizeof(double) * m);
  dd* w = (dd*)malloc(sizeof(dd) * (n + 1));
  int status = ORC_OK;

  orc_lmi(n, m, A, 1.0, p, F);
  orc_lmi(n, m, A, 0.0, v, V);
  if (orc_cholesky(m, F, L) != 0) {
    status = ORC_NOT_PD;
    goto done;
  }
  pencil_matrix(m, L, V, M);
  int sweeps = orc_jacobi(m, M, ev, Q, 100);
  if (sweeps < 0) {
    status = ORC_NOCONV;
    goto done;
  }
  int kmax = 0, kmin = 0;
  for (int k = 1; k < m; ++k) {
    if (ev[k] > ev[kmax]) kmax = k;
    if (ev[k] < ev[kmin]) kmin = k;
  }
  double mu2 = -INFINITY;
  for (int k = 0; k < m; ++k)
    if (k != kmax && ev[k] > mu2) mu2 = ev[k];
  double tp = INFINITY, tm = -INFINITY;
  double errp = 0.0, errm = 0.0;
  if (ev[kmax] > 0.0) {
    for (int i = 0; i < m; ++i) y[i] = Q[IDX(i, kmax, m)];
    back_subst_t(m, L, y, up);
    double tj = 1.0 / ev[kmax];
    tp = refine_end(n, m, A, p, v, F, V, tj, up, w);
    errp = fabs(tj - tp) / fabs(tp);
    if (w_plus)
      for (int j = 0; j <= n; ++j) w_plus[j] = w[j].hi + w[j].lo;
    if (u_plus) memcpy(u_plus, up, sizeof(double) * m);
  }
  if (ev[kmin] < 0.0) {
    for (int i = 0; i < m; ++i) y[i] = Q[IDX(i, kmin, m)];
    back_subst_t(m, L, y, um);
    double tj = 1.0 / ev[kmin];
    tm = refine_end(n, m, A, p, v, F, V, tj, um, w);
    errm = fabs(tj - tm) / fabs(tm);
    if (u_minus) memcpy(u_minus, um, sizeof(double) * m);
  }
  *t_plus = tp;
  *t_minus = tm;
  if (info) {
    info[0] = errp;
    info[1] = (m > 1 && ev[kmax] > 0.0) ? (ev[kmax] - mu2) / fabs(ev[kmax]) : 1.0;
    info[2] = sweeps;
    info[3] = errm;
  }
done:
  free(F); free(V); free(L); free(M); free(Q); free(ev); free(y); free(up); free(um); free(w);
  return status;
}

/*
 * REFLECTION (Alg. 3, Eq. "reflection", Lemma "Gradient of det F").
 *   out: t_plus, w_hat[n] = w/|w| with w_j = u^T A_j u (j = 1..n),
 *        s[n] = v - 2 <v, w_hat> w_hat, info[4] as in orc_intersect.
 *   returns ORC_OK, ORC_NOT_PD, ORC_UNBOUNDED, ORC_NOCONV, ORC_DEGENERATE
 *   (|w| = 0: F(p + t+ v) has rank <= m-2 and the normal is undefined).
 */
int orc_reflect(int n, int m, const double* A, const double* p, const double* v,
                double* t_plus, double* w_hat, double* s, double* info) {
  double tm, tp;
  double* wf = (double*)malloc(sizeof(double) * (n + 1));
  int st = orc_intersect(n, m, A, p, v, &tm, &tp, NULL, NULL, wf, info);
  if (st != ORC_OK) goto out;
  if (!isfinite(tp)) {
    st = ORC_UNBOUNDED;
    goto out;
  }
  *t_plus = tp;
  double nw = 0.0;
  for (int j = 1; j <= n; ++j) nw += wf[j] * wf[j];
  nw = sqrt(nw);
  if (!(nw > 0.0)) {
    st = ORC_DEGENERATE;
    goto out;
  }
  double vw = 0.0;
  for (int j = 1; j <= n; ++j) {
    w_hat[j - 1] = wf[j] / nw;
    vw += v[j - 1] * w_hat[j - 1];
  }
  for (int j = 0; j < n; ++j) s[j] = v[j] - 2.0 * vw * w_hat[j];
out:
  free(wf);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Random walks                                                              */
/* ------------------------------------------------------------------------ */

/*
 * One Billiard step (Alg. 5) for chain `chain`, step number `step`.
 *   l = -tau ln eta, v ~ U(sphere); repeat REFLECTION until l is used up.
 *   Readings where the paper is silent:
 *   - reflect iff t+ < l; on a tie move l and stop;
 *   - after a hit the point is p + (1 - kappa) t+ v (kappa keeps F(p) > 0),
 *     and l decreases by t+;
 *   - the reflection count increments at each reflection; once it exceeds
 *     rho the step ends and x is left unchanged (status ORC_RHO).
 *   x[n] is updated in place on success.  nrefl / nseg report the reflections
 *   and the boundary-oracle calls (segments) used.
 */
/* The Billiard step of Alg. 5 with an optional trace: when rec_p / rec_v are
 * given, the line (p, v) of each of the first max_rec segments (the start
 * point and direction that the boundary oracle is called on) is appended to
 * them (max_rec x n each). */
static int billiard_step_traced(int n, int m, const double* A, double* x, double tau, int rho,
                                double kappa, uint64_t seed, uint32_t chain, uint32_t step,
                                int* nrefl, int* nseg, double* rec_p, double* rec_v,
                                int max_rec) {
  double* v = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* wh = (double*)malloc(sizeof(double) * n);
  double* s = (double*)malloc(sizeof(double) * n);
  double eta = orc_uniform(seed, chain, step, 1);
  double ell = -tau * log(eta);
  orc_direction(n, seed, chain, step, v);
  memcpy(p, x, sizeof(double) * n);
  int refl = 0, seg = 0, st = ORC_OK;
  for (;;) {
    double tp;
    if (rec_p && seg < max_rec) {
      memcpy(rec_p + (size_t)seg * n, p, sizeof(double) * n);
      memcpy(rec_v + (size_t)seg * n, v, sizeof(double) * n);
    }
    st = orc_reflect(n, m, A, p, v, &tp, wh, s, NULL);
    ++seg;
    if (st != ORC_OK) break;
    if (tp < ell) {
      for (int i = 0; i < n; ++i) p[i] += (1.0 - kappa) * tp * v[i];
      ell -= tp;
      memcpy(v, s, sizeof(double) * n);
      ++refl;
      if (refl > rho) {
        st = ORC_RHO;
        break;
      }
    } else {
      for (int i = 0; i < n; ++i) p[i] += ell * v[i];
      memcpy(x, p, sizeof(double) * n);
      break;
    }
  }
  if (nrefl) *nrefl = refl;
  if (nseg) *nseg = seg;
  free(v); free(p); free(wh); free(s);
  return st;
}

int orc_billiard_step(int n, int m, const double* A, double* x, double tau, int rho,
                      double kappa, uint64_t seed, uint32_t chain, uint32_t step,
                      int* nrefl, int* nseg) {
  return billiard_step_traced(n, m, A, x, tau, rho, kappa, seed, chain, step, nrefl, nseg, NULL,
                              NULL, 0);
}

/*
 * The lines the boundary oracle meets during one Billiard step (Alg. 5) of
 * each of C chains: chain c (Philox chain index chain0 + c, step number
 * `step`) starts at X[c] (updated in place, as orc_billiard_step) and appends
 * the (p, v) of its first max_per_chain segments to rec_p / rec_v at rows
 * c * max_per_chain + k (C * max_per_chain x n each); nseg[c] receives its
 * number of segments (all of them, recorded or not) and status[c] the step's
 * status.  Chains run in parallel (OpenMP) when built with it.
 */
void orc_billiard_trace(int n, int m, const double* A, int C, double* X, uint32_t step,
                        uint32_t chain0, double tau, int rho, double kappa, uint64_t seed,
                        int max_per_chain, double* rec_p, double* rec_v, int* nseg,
                        int* status) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < C; ++c) {
    int nr = 0, ns = 0;
    status[c] = billiard_step_traced(n, m, A, X + (size_t)c * n, tau, rho, kappa, seed,
                                     chain0 + (uint32_t)c, step, &nr, &ns,
                                     rec_p + (size_t)c * max_per_chain * n,
                                     rec_v + (size_t)c * max_per_chain * n, max_per_chain);
    nseg[c] = ns;
  }
}

/*
 * orc_intersect on `count` independent lines (rows of P and V, count x n):
 * t_minus[c], t_plus[c], status[c] (in parallel with OpenMP).
 */
void orc_intersect_batch(int n, int m, const double* A, int count, const double* P,
                         const double* V, double* t_minus, double* t_plus, int* status) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < count; ++c) {
    t_minus[c] = 0.0;
    t_plus[c] = 0.0;
    status[c] = orc_intersect(n, m, A, P + (size_t)c * n, V + (size_t)c * n, t_minus + c,
                              t_plus + c, NULL, NULL, NULL, NULL);
  }
}

/*
 * orc_reflect on `count` independent lines (p_c, v_c) (rows of P and V,
 * count x n): t_plus[c], w_hat (count x n), status[c] and info (count x 4, the
 * per-line info of orc_intersect).  Lines run in parallel (OpenMP).
 */
void orc_reflect_batch(int n, int m, const double* A, int count, const double* P,
                       const double* V, double* t_plus, double* w_hat, double* s, int* status,
                       double* info) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < count; ++c) {
    t_plus[c] = 0.0;
    status[c] = orc_reflect(n, m, A, P + (size_t)c * n, V + (size_t)c * n, t_plus + c,
                            w_hat + (size_t)c * n, s + (size_t)c * n, info + (size_t)c * 4);
  }
}

/* One Hit-and-Run step (Alg. 4) with pi_l uniform on the chord:
 * x <- x + (t- + eta (t+ - t-)) v. */
int orc_hnr_step(int n, int m, const double* A, double* x, uint64_t seed, uint32_t chain,
                 uint32_t step) {
  double* v = (double*)malloc(sizeof(double) * n);
  orc_direction(n, seed, chain, step, v);
  double tm, tp;
  int st = orc_intersect(n, m, A, x, v, &tm, &tp, NULL, NULL, NULL, NULL);
  if (st == ORC_OK && (!isfinite(tp) || !isfinite(tm))) st = ORC_UNBOUNDED;
  if (st == ORC_OK) {
    double eta = orc_uniform(seed, chain, step, 1);
    double t = tm + eta * (tp - tm);
    for (int i = 0; i < n; ++i) x[i] += t * v[i];
  }
  free(v);
  return st;
}

/* coordinate index of a CDHR step: floor(u n) from stream 2 */
int orc_cdhr_coord(int n, uint64_t seed, uint32_t chain, uint32_t step) {
  double u = orc_uniform(seed, chain, step, 2);
  int j = (int)(u * n);
  return j < n ? j : n - 1;
}

/* One coordinate-direction Hit-and-Run step (Sec. 3.1): direction e_j. */
int orc_cdhr_step(int n, int m, const double* A, double* x, uint64_t seed, uint32_t chain,
                  uint32_t step) {
  double* v = (double*)calloc(n, sizeof(double));
  int j = orc_cdhr_coord(n, seed, chain, step);
  v[j] = 1.0;
  double tm, tp;
  int st = orc_intersect(n, m, A, x, v, &tm, &tp, NULL, NULL, NULL, NULL);
  if (st == ORC_OK && (!isfinite(tp) || !isfinite(tm))) st = ORC_UNBOUNDED;
  if (st == ORC_OK) {
    double eta = orc_uniform(seed, chain, step, 1);
    x[j] += tm + eta * (tp - tm);
  }
  free(v);
  return st;
}

/*
 * Run `steps` steps of a walk on C chains (chain c uses Philox chain index
 * chain0 + c and step numbers step0 .. step0+steps-1).  kind: 0 Billiard,
 * 1 Hit-and-Run, 2 CDHR.  X is C x n row-major, updated in place.  Chains
 * run in parallel (OpenMP) when built with it.
 *   counts[0] = segments (boundary-oracle calls), counts[1] = reflections,
 *   counts[2] = steps that ended with a non-OK status (x kept).
 *   Returns the number of chains that met an error other than ORC_RHO.
 */
int orc_walk(int kind, int n, int m, const double* A, int C, double* X, int steps,
             uint32_t step0, uint32_t chain0, double tau, int rho, double kappa, uint64_t seed,
             long long* counts) {
  long long seg_total = 0, refl_total = 0, bad_steps = 0;
  int errors = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : seg_total, refl_total, bad_steps, errors)
  for (int c = 0; c < C; ++c) {
    double* x = X + (size_t)c * n;
    int chain_err = 0;
    for (int k = 0; k < steps; ++k) {
      uint32_t st_no = step0 + (uint32_t)k;
      int st;
      if (kind == 0) {
        int nr = 0, ns = 0;
        st = orc_billiard_step(n, m, A, x, tau, rho, kappa, seed, chain0 + (uint32_t)c, st_no,
                               &nr, &ns);
        seg_total += ns;
        refl_total += nr;
      } else if (kind == 1) {
        st = orc_hnr_step(n, m, A, x, seed, chain0 + (uint32_t)c, st_no);
        seg_total += 1;
      } else {
        st = orc_cdhr_step(n, m, A, x, seed, chain0 + (uint32_t)c, st_no);
        seg_total += 1;
      }
      if (st != ORC_OK) {
        ++bad_steps;
        if (st != ORC_RHO) chain_err = 1;
      }
    }
    errors += chain_err;
  }
  if (counts) {
    counts[0] = seg_total;
    counts[1] = refl_total;
    counts[2] = bad_steps;
  }
  return errors;
}

/* number of OpenMP threads the walk would use (1 without OpenMP) */
int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
