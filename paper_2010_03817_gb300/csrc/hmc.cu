// Hamiltonian Monte Carlo with reflections (Sec. 3.3, Alg. 6) for the
// Boltzmann density pi(x) ~ exp(-c.x / T) on S, FP64 path.
//
// For f(x) = c.x / T the Hamiltonian ODE (Eq. ode_ham) has the exact
// degree-2 solution Phi(t) = p + v t - (c / (2T)) t^2, so along it
//   F(Phi(t)) = F(p) + t V + t^2 C,   V = sum v_j A_j,  C = -(1/(2T)) sum c_j A_j,
// a quadratic eigenvalue problem (Sec. 2.1).  Its first positive root t+ is
// where the trajectory meets the boundary; unlike a line, a parabola can
// leave S and come back, so t+ is taken from all the roots: with F(p) = L L^T,
// B = L^{-1} V L^{-T} and K = L^{-1} C L^{-T}, the roots are t = 1/mu for the
// eigenvalues mu of the companion linearisation G = [[0, I], [-K, -B]]
// (size 2m, Sec. 2.1), and t+ = 1/mu for the largest real positive mu.
// One CTA per item:
//   F (packed, shared), Cholesky;  G (dense, shared) from triangular solves;
//   Householder reduction of G to Hessenberg form (all warps);
//   Francis double-shift QR for all its eigenvalues (one warp);
//   the null vector u of F(Phi(t+)) by inverse iteration on F(Phi(sigma)),
//   sigma just below t+ (a factorisation that succeeds there also certifies
//   the point interior), then two corrections toward the null vector of
//   F(Phi(t)) itself; t refined on the scalar quadratic u^T F(Phi(t)) u = 0
//   (stationary at u; no root of it lies below t+, since F(Phi(t)) is
//   positive definite before t+; the refinement is kept within 1e-7 of t);
//   the normal w_j = u^T A_j u at Phi(t+) (Lemma "Gradient of det F") and the
//   reflection of the velocity Phi'(t+) = v - (c/T) t+ (Sec. 2.4).
#include <math.h>

#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"

extern "C" int spg_set_error(int code, const char* msg);

namespace spg {
namespace {

constexpr double kCurveRefineWindow = 1e-7;

__host__ __device__ inline int curve_ld(int m) { return 2 * m + 1; }  // odd: no bank conflicts

struct CurveSmem {
  double* L;    // P: packed factor
  double* G;    // N x ld (N = 2m), row-major
  double* p;    // n: point
  double* v;    // n: velocity
  double* c;    // n
  double* x0;   // n: start of the step (walk)
  double* w;    // n + 1: quadratic forms u^T A_j u
  double* wh;   // n: unit normal (also the point Phi(sigma))
  double* u;    // m
  double* wr;   // N: eigenvalues (real parts)
  double* wi;   // N: (imaginary parts)
  double* hv;   // N: Householder vector
  double* hw;   // N: its products
  double* col;  // cholesky scratch
  double* red;  // SPG_WARPS
  double* bc;   // 16
  int* ib;      // 16
};

__host__ __device__ inline size_t curve_doubles(int n, int m) {
  const size_t P = (size_t)m * (m + 1) / 2, N = 2 * (size_t)m;
  return P + N * curve_ld(m) + 6 * (size_t)n + 1 + (size_t)m + 4 * N + cholesky_scratch(m) +
         SPG_WARPS + 16;
}

__device__ CurveSmem curve_carve(double* base, int n, int m) {
  CurveSmem s;
  const size_t P = (size_t)m * (m + 1) / 2, N = 2 * (size_t)m;
  double* q = base;
  s.L = q; q += P;
  s.G = q; q += N * curve_ld(m);
  s.p = q; q += n;
  s.v = q; q += n;
  s.c = q; q += n;
  s.x0 = q; q += n;
  s.w = q; q += n + 1;
  s.wh = q; q += n;
  s.u = q; q += m;
  s.wr = q; q += N;
  s.wi = q; q += N;
  s.hv = q; q += N;
  s.hw = q; q += N;
  s.col = q; q += cholesky_scratch(m);
  s.red = q; q += SPG_WARPS;
  s.bc = q; q += 16;
  s.ib = reinterpret_cast<int*>(q);
  return s;
}

// packed F at the point q (CTA-wide): A_0 + sum q_j A_j
__device__ void form_at(const DevSpec& sp, const double* q, double* Lp) {
  const int n = sp.n;
  const long long P = sp.P;
  for (long long e = threadIdx.x; e < P; e += SPG_THREADS) {
    const double* Ae = sp.A + e;
    double f0 = 0.0, f1 = 0.0;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      f0 += q[j] * Ae[(size_t)(j + 1) * P];
      f1 += q[j + 1] * Ae[(size_t)(j + 2) * P];
    }
    if (j < n) f0 += q[j] * Ae[(size_t)(j + 1) * P];
    Lp[e] = Ae[0] + (f0 + f1);
  }
  __syncthreads();
}

// Householder reduction of the N x N matrix G (leading dimension ld, shared)
// to upper Hessenberg form, CTA-wide: for column k the reflector
// I - beta h h^T with h = x - alpha e_1, x = G[k+1.., k], applied from the
// left and from the right
__device__ void hessenberg(double* G, int N, int ld, CurveSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k + 2 < N; ++k) {
    const int len = N - k - 1;
    double a = 0.0;
    for (int i = tid; i < len; i += SPG_THREADS) {
      const double x = G[(size_t)(k + 1 + i) * ld + k];
      a += x * x;
    }
    const double nrm2 = block_sum(a, sm.red);
    const double x0 = G[(size_t)(k + 1) * ld + k];
    const double tail = nrm2 - x0 * x0;
    if (!(tail > 0.0)) continue;  // the column is already reduced (CTA-uniform)
    const double alpha = x0 >= 0.0 ? -sqrt(nrm2) : sqrt(nrm2);
    for (int i = tid; i < len; i += SPG_THREADS)
      sm.hv[i] = G[(size_t)(k + 1 + i) * ld + k] - (i == 0 ? alpha : 0.0);
    __syncthreads();
    const double h0 = x0 - alpha;
    const double beta = 2.0 / (tail + h0 * h0);
    // left, rows k+1.., columns k..:  G -= h (beta h^T G)
    for (int j = k + tid; j < N; j += SPG_THREADS) {
      double s = 0.0;
      for (int i = 0; i < len; ++i) s += sm.hv[i] * G[(size_t)(k + 1 + i) * ld + j];
      sm.hw[j] = beta * s;
    }
    __syncthreads();
    for (int q = tid; q < len * (N - k); q += SPG_THREADS) {
      const int i = q / (N - k), j = k + q % (N - k);
      G[(size_t)(k + 1 + i) * ld + j] -= sm.hv[i] * sm.hw[j];
    }
    __syncthreads();
    // right, all rows, columns k+1..:  G -= (beta G h) h^T (a warp per row)
    for (int i = wid; i < N; i += SPG_WARPS) {
      double s = 0.0;
      for (int j = lane; j < len; j += 32) s += G[(size_t)i * ld + k + 1 + j] * sm.hv[j];
      s = warp_sum(s);
      if (lane == 0) sm.hw[i] = beta * s;
    }
    __syncthreads();
    for (int q = tid; q < N * len; q += SPG_THREADS) {
      const int i = q / len, j = q % len;
      G[(size_t)i * ld + k + 1 + j] -= sm.hw[i] * sm.hv[j];
    }
    __syncthreads();
    for (int i = tid; i < len; i += SPG_THREADS)
      G[(size_t)(k + 1 + i) * ld + k] = i == 0 ? alpha : 0.0;
    __syncthreads();
  }
}

// the reflector I - beta h h^T that maps (x, y, z) to a multiple of e_1
__device__ __forceinline__ void house3(double x, double y, double z, double* h, double& beta) {
  const double a = sqrt(x * x + y * y + z * z);
  if (!(a > 0.0)) {
    h[0] = 1.0;
    h[1] = h[2] = 0.0;
    beta = 0.0;
    return;
  }
  h[0] = x + (x >= 0.0 ? a : -a);
  h[1] = y;
  h[2] = z;
  beta = 2.0 / (h[0] * h[0] + y * y + z * z);
}

// All eigenvalues of the upper Hessenberg H (N x N, leading dimension ld,
// shared) by the Francis double-shift QR iteration with deflation: one warp,
// the active block only, no Schur vectors.  After 10 and 20 iterations
// without a deflation the shifts are the exceptional ones of LAPACK's
// DLAHQR (from the trailing subdiagonal magnitudes).  Returns false when the
// iteration budget (60 N sweeps) runs out.
__device__ bool hessenberg_eig(double* H, int N, int ld, double* wr, double* wi) {
  const int lane = threadIdx.x & 31;
  const double eps = 2.220446049250313e-16;
  auto at = [&](int i, int j) -> double& { return H[(size_t)i * ld + j]; };
  int hi = N - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      const double sub = fabs(at(l, l - 1));
      const double dia = fabs(at(l - 1, l - 1)) + fabs(at(l, l));
      if (sub <= eps * (dia > 0.0 ? dia : 1.0)) break;
      --l;
    }
    __syncwarp();
    if (lane == 0 && l > 0) at(l, l - 1) = 0.0;
    __syncwarp();
    if (l == hi) {  // a 1 x 1 block
      if (lane == 0) {
        wr[hi] = at(hi, hi);
        wi[hi] = 0.0;
      }
      --hi;
      iter = 0;
      __syncwarp();
      continue;
    }
    if (l == hi - 1) {  // a 2 x 2 block: its two eigenvalues
      const double a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
      const double p = 0.5 * (a - d), bc = b * c, disc = p * p + bc;
      if (lane == 0) {
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          const double z = p >= 0.0 ? p + sq : p - sq;
          wr[hi - 1] = d + z;
          wr[hi] = z != 0.0 ? d - bc / z : d;
          wi[hi - 1] = wi[hi] = 0.0;
        } else {
          const double sq = sqrt(-disc);
          wr[hi - 1] = wr[hi] = d + p;
          wi[hi - 1] = sq;
          wi[hi] = -sq;
        }
      }
      hi -= 2;
      iter = 0;
      __syncwarp();
      continue;
    }
    if (++total > 60 * N) return false;
    ++iter;
    // s, t: the sum and product of the two shifts
    double s, t;
    if (iter == 10 || iter == 20) {
      const double e = fabs(at(hi, hi - 1)) + fabs(at(hi - 1, hi - 2));
      const double h11 = 0.75 * e + at(hi, hi);
      s = 2.0 * h11;
      t = h11 * h11 + 0.4375 * e * e;
    } else {
      s = at(hi - 1, hi - 1) + at(hi, hi);
      t = at(hi - 1, hi - 1) * at(hi, hi) - at(hi - 1, hi) * at(hi, hi - 1);
    }
    // first column of (H - s1)(H - s2), then the bulge chased down
    double x = at(l, l) * at(l, l) + at(l, l + 1) * at(l + 1, l) - s * at(l, l) + t;
    double y = at(l + 1, l) * (at(l, l) + at(l + 1, l + 1) - s);
    double z = at(l + 1, l) * at(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      double h[3], beta;
      house3(x, y, z, h, beta);
      const int q0 = k > l ? k - 1 : l;
      for (int j = q0 + lane; j <= hi; j += 32) {  // rows k..k+2
        const double sd = beta * (h[0] * at(k, j) + h[1] * at(k + 1, j) + h[2] * at(k + 2, j));
        at(k, j) -= h[0] * sd;
        at(k + 1, j) -= h[1] * sd;
        at(k + 2, j) -= h[2] * sd;
      }
      __syncwarp();
      const int r = k + 3 < hi ? k + 3 : hi;
      for (int i = l + lane; i <= r; i += 32) {  // columns k..k+2
        const double sd = beta * (at(i, k) * h[0] + at(i, k + 1) * h[1] + at(i, k + 2) * h[2]);
        at(i, k) -= sd * h[0];
        at(i, k + 1) -= sd * h[1];
        at(i, k + 2) -= sd * h[2];
      }
      __syncwarp();
      x = at(k + 1, k);
      y = at(k + 2, k);
      z = k < hi - 2 ? at(k + 3, k) : 0.0;
      __syncwarp();
    }
    {
      double h[3], beta;
      house3(x, y, 0.0, h, beta);
      for (int j = hi - 2 + lane; j <= hi; j += 32) {
        const double sd = beta * (h[0] * at(hi - 1, j) + h[1] * at(hi, j));
        at(hi - 1, j) -= h[0] * sd;
        at(hi, j) -= h[1] * sd;
      }
      __syncwarp();
      for (int i = l + lane; i <= hi; i += 32) {
        const double sd = beta * (at(i, hi - 1) * h[0] + at(i, hi) * h[1]);
        at(i, hi - 1) -= sd * h[0];
        at(i, hi) -= sd * h[1];
      }
      __syncwarp();
    }
  }
  return true;
}

// L^{-1} b for the packed lower factor L, one thread, b at stride st (in place)
__device__ void fwd_solve(const double* L, double* b, int m, int st) {
  for (int i = 0; i < m; ++i) {
    double s = b[(size_t)i * st];
    const double* row = L + tri(i, 0);
    for (int k = 0; k < i; ++k) s -= row[k] * b[(size_t)k * st];
    b[(size_t)i * st] = s / row[i];
  }
}

// u <- L^{-T} L^{-1} u, one warp, m <= 64 (lane holds u[lane], u[lane + 32])
__device__ void warp_llt_solve(const double* L, double* u, int m) {
  const int lane = threadIdx.x & 31;
  double r0 = lane < m ? u[lane] : 0.0, r1 = lane + 32 < m ? u[lane + 32] : 0.0;
  for (int i = 0; i < m; ++i) {  // L y = u, column by column
    const double ui = __shfl_sync(0xffffffffu, i < 32 ? r0 : r1, i & 31) / L[tri(i, i)];
    if (lane == (i & 31)) {
      if (i < 32) r0 = ui; else r1 = ui;
    }
    if (lane > i && lane < m) r0 -= L[tri(lane, i)] * ui;
    if (lane + 32 > i && lane + 32 < m) r1 -= L[tri(lane + 32, i)] * ui;
  }
  for (int i = m - 1; i >= 0; --i) {  // L^T u = y, row by row of L
    const double ui = __shfl_sync(0xffffffffu, i < 32 ? r0 : r1, i & 31) / L[tri(i, i)];
    if (lane == (i & 31)) {
      if (i < 32) r0 = ui; else r1 = ui;
    }
    if (lane < i) r0 -= L[tri(i, lane)] * ui;
    if (lane + 32 < i) r1 -= L[tri(i, lane + 32)] * ui;
  }
  if (lane < m) u[lane] = r0;
  if (lane + 32 < m) u[lane + 32] = r1;
}

struct CurveResult {
  double t_plus;
  int status;
};

// The boundary oracle of the trajectory Phi(t) = p + v t - (c/(2T)) t^2
// (sm.p, sm.v, sm.c).  On kOk: t_plus, the unit normal in sm.wh.
// sigma0 >= 0: the expansion point (below; 0 at a step start).
__device__ __noinline__ CurveResult curve_segment(const DevSpec& sp, const CurveParams& cp,
                                                  CurveSmem& sm, double* __restrict__ Vp,
                                                  double sigma0) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = sp.n, m = sp.m, N = 2 * m, ld = curve_ld(m);
  const long long P = sp.P;
  CurveResult res;
  res.t_plus = 0.0;
  // ---- the pencil at the expansion point s0 ---------------------------------
  // After a reflection the walker sits kappa-close to the boundary it left:
  // F(p) is then nearly singular, L^{-1} huge and the companion matrix badly
  // scaled (its Francis iteration converges slowly or not at all).  As the
  // line walks do, the expansion moves a little along the curve:
  // F(Phi(s0 + s)) = F(Phi(s0)) + s (V + 2 s0 C) + s^2 C, the same quadratic
  // eigenvalue problem from the point Phi(s0) with velocity Phi'(s0); its
  // roots s give t = s0 + s (the boundary left behind: t < 0).  s0 backs off
  // x0.2 (then 0) while F(Phi(s0)) does not factor.
  double s0 = sigma0 > 0.0 ? sigma0 : 0.0;
  for (int attempt = 0;; ++attempt) {
    for (int j = tid; j < n; j += SPG_THREADS) {
      sm.wh[j] = sm.p[j] + sm.v[j] * s0 - sm.c[j] / (2.0 * cp.T) * s0 * s0;
      sm.w[j] = sm.v[j] - sm.c[j] / cp.T * s0;
    }
    __syncthreads();
    form_at(sp, sm.wh, sm.L);
    for (long long e = tid; e < P; e += SPG_THREADS) {
      const double* Ae = sp.A + e;
      double g = 0.0;
      for (int j = 0; j < n; ++j) g += sm.w[j] * Ae[(size_t)(j + 1) * P];
      Vp[e] = g;
    }
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    if (factor_cholesky<double>(sm.L, m, sm.col, &sm.ib[0])) break;
    if (s0 == 0.0) {
      res.status = kNotPD;
      return res;
    }
    s0 = attempt < 2 ? 0.2 * s0 : 0.0;
  }
  // ---- the companion G = [[0, I], [-K, -B]] ---------------------------------
  // S -> L^{-1} S (columns, in the upper-right block), its transpose into the
  // target block, L^{-1} again: L^{-1} S L^{-T}, negated; S = V into the
  // lower-right block, then S = C into the lower-left one
  double* G = sm.G;
  for (int pass = 0; pass < 2; ++pass) {
    const double* S = pass == 0 ? Vp : cp.Cp;
    for (int q = tid; q < m * m; q += SPG_THREADS) {
      const int i = q / m, j = q % m;
      G[(size_t)i * ld + m + j] = S[i >= j ? tri(i, j) : tri(j, i)];
    }
    __syncthreads();
    for (int j = tid; j < m; j += SPG_THREADS) fwd_solve(sm.L, G + m + j, m, ld);
    __syncthreads();
    const int c0 = pass == 0 ? m : 0;
    for (int q = tid; q < m * m; q += SPG_THREADS) {
      const int i = q / m, j = q % m;
      G[(size_t)(m + i) * ld + c0 + j] = G[(size_t)j * ld + m + i];
    }
    __syncthreads();
    for (int j = tid; j < m; j += SPG_THREADS) fwd_solve(sm.L, G + (size_t)m * ld + c0 + j, m, ld);
    __syncthreads();
    for (int q = tid; q < m * m; q += SPG_THREADS) {
      const int i = q / m, j = q % m;
      G[(size_t)(m + i) * ld + c0 + j] = -G[(size_t)(m + i) * ld + c0 + j];
    }
    __syncthreads();
  }
  for (int q = tid; q < m * N; q += SPG_THREADS) {
    const int i = q / N, j = q % N;
    G[(size_t)i * ld + j] = (j == m + i) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- its eigenvalues: Hessenberg form, then the Francis iteration -------
  hessenberg(G, N, ld, sm);
  if (wid == 0) {
    const bool ok = hessenberg_eig(G, N, ld, sm.wr, sm.wi);
    if (lane == 0) sm.ib[1] = ok ? 1 : 0;
  }
  __syncthreads();
  if (!sm.ib[1]) {
    res.status = kNoConv;
    return res;
  }
  if (tid == 0) {
    // the first root ahead: the smallest t = s0 + 1/mu > 0 over the real
    // eigenvalues (mu = 0: a root at infinity)
    double best = INFINITY;
    for (int i = 0; i < N; ++i) {
      const double mu = sm.wr[i];
      if (mu != 0.0 && fabs(sm.wi[i]) <= 1e-10 * fabs(mu)) {
        const double tk = s0 + 1.0 / mu;
        if (tk > 0.0 && tk < best) best = tk;
      }
    }
    sm.bc[0] = best;
  }
  __syncthreads();
  double t = sm.bc[0];
  if (!(t < INFINITY)) {
    res.status = kUnbounded;
    res.t_plus = INFINITY;
    return res;
  }
  // ---- the null vector at the hit point; t refined --------------------------
  // F(Phi(sigma)) is positive definite for sigma below t+; inverse iteration
  // on it gives u0, its eigenvector of the smallest eigenvalue, which is the
  // null vector of F(Phi(t)) up to O((t - sigma) |F'| / lambda_2).  Two
  // corrections u <- u - F(Phi(sigma))^{-1} F(Phi(t)) u remove that error:
  // the iteration's fixed points are the null vectors of F(Phi(t)), and it
  // contracts the rest by about (t - sigma) |F'| / lambda_2 per step.
  bool ok = false;
  int used = 0;
  for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
    used = attempt;
    const double sig = t * (1.0 - (attempt == 0 ? 1e-5 : (attempt == 1 ? 1e-3 : 1e-1)));
    for (int j = tid; j < n; j += SPG_THREADS)
      sm.wh[j] = sm.p[j] + sm.v[j] * sig - sm.c[j] / (2.0 * cp.T) * sig * sig;
    __syncthreads();
    form_at(sp, sm.wh, sm.L);
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    ok = factor_cholesky<double>(sm.L, m, sm.col, &sm.ib[0]);
  }
  if (!ok) {
    res.status = kNotPD;
    return res;
  }
  for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = 1.0 + 0.5 * sin(0.9 * i + 0.3);
  __syncthreads();
  // (the corrections only from the closest shift, where they contract)
  const int iters = used == 0 ? 6 : 4;
  for (int it = 0; it < iters; ++it) {
    double* r = sm.hv;
    if (it >= 4) {
      // r = F(Phi(t)) u, with F(Phi(t)) formed into the global scratch
      for (int j = tid; j < n; j += SPG_THREADS)
        sm.wh[j] = sm.p[j] + sm.v[j] * t - sm.c[j] / (2.0 * cp.T) * t * t;
      __syncthreads();
      form_at(sp, sm.wh, Vp);
      for (int i = tid; i < m; i += SPG_THREADS) {
        double a = 0.0;
        for (int k = 0; k < m; ++k) a += Vp[i >= k ? tri(i, k) : tri(k, i)] * sm.u[k];
        r[i] = a;
      }
    } else {
      for (int i = tid; i < m; i += SPG_THREADS) r[i] = sm.u[i];
    }
    __syncthreads();
    if (wid == 0) warp_llt_solve(sm.L, r, m);
    __syncthreads();
    double a = 0.0;
    for (int i = tid; i < m; i += SPG_THREADS) {
      const double ui = it >= 4 ? sm.u[i] - r[i] : r[i];
      sm.u[i] = ui;
      a += ui * ui;
    }
    const double rn = 1.0 / sqrt(block_sum(a, sm.red));
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] *= rn;
    __syncthreads();
  }
  // w_j = u^T A_j u, j = 0..n (packed: off-diagonal entries twice)
  for (int j = wid; j <= n; j += SPG_WARPS) {
    const double* Aj = sp.A + (size_t)j * P;
    double a0 = 0.0;
    for (long long e = lane; e < P; e += 32) {
      const uint32_t ik = sp.pidx[e];
      const int i = ik >> 16, k = ik & 0xffff;
      a0 += Aj[e] * (i == k ? 1.0 : 2.0) * sm.u[i] * sm.u[k];
    }
    a0 = warp_sum(a0);
    if (lane == 0) sm.w[j] = a0;
  }
  __syncthreads();
  if (tid == 0) {
    // u^T F(Phi(t)) u = a + b t + c2 t^2 with a = w_0 + p.w, b = v.w,
    // c2 = -(c.w) / (2T): its root nearest t
    double a = sm.w[0], b = 0.0, c2 = 0.0;
    for (int j = 0; j < n; ++j) {
      a += sm.p[j] * sm.w[j + 1];
      b += sm.v[j] * sm.w[j + 1];
      c2 -= sm.c[j] * sm.w[j + 1] / (2.0 * cp.T);
    }
    double tr = t;
    if (c2 != 0.0) {
      const double disc = b * b - 4.0 * a * c2;
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        const double q = -0.5 * (b + (b >= 0.0 ? sq : -sq));
        const double r1 = q / c2, r2 = q != 0.0 ? a / q : r1;
        tr = fabs(r1 - t) < fabs(r2 - t) ? r1 : r2;
      }
    } else if (b != 0.0) {
      tr = -a / b;
    }
    sm.bc[1] = (tr > 0.0 && fabs(tr - t) <= kCurveRefineWindow * t) ? tr : t;
  }
  __syncthreads();
  t = sm.bc[1];
  double a = 0.0;
  for (int j = tid; j < n; j += SPG_THREADS) a += sm.w[j + 1] * sm.w[j + 1];
  const double nw = sqrt(block_sum(a, sm.red));
  if (!(nw > 0.0)) {
    res.status = kDegenerate;
    res.t_plus = t;
    return res;
  }
  for (int j = tid; j < n; j += SPG_THREADS) sm.wh[j] = sm.w[j + 1] / nw;
  __syncthreads();
  res.t_plus = t;
  res.status = kOk;
  return res;
}

// <Phi'(t), w^> for the velocity at t (CTA-wide)
__device__ double velocity_dot_normal(const CurveSmem& sm, int n, double T, double t) {
  double a = 0.0;
  for (int j = threadIdx.x; j < n; j += SPG_THREADS) a += (sm.v[j] - sm.c[j] / T * t) * sm.wh[j];
  return block_sum(a, sm.red);
}

__global__ void __launch_bounds__(SPG_THREADS, 1) curve_kernel(DevSpec sp, CurveParams cp,
                                                                double* Vwork) {
  extern __shared__ double smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n;
  CurveSmem sm = curve_carve(smem_raw, n, sp.m);
  double* Vp = Vwork + (size_t)blockIdx.x * sp.P;
  for (int j = tid; j < n; j += SPG_THREADS) sm.c[j] = cp.c[j];
  __syncthreads();
  for (int item = blockIdx.x; item < cp.count; item += gridDim.x) {
    if (cp.op == 0) {
      // REFLECTION of one trajectory
      for (int j = tid; j < n; j += SPG_THREADS) {
        sm.p[j] = cp.x[(size_t)item * n + j];
        sm.v[j] = cp.v[(size_t)item * n + j];
      }
      __syncthreads();
      const CurveResult r = curve_segment(sp, cp, sm, Vp, 0.0);
      if (r.status == kOk) {
        const double vw = velocity_dot_normal(sm, n, cp.T, r.t_plus);
        for (int j = tid; j < n; j += SPG_THREADS) {
          const double vel = sm.v[j] - sm.c[j] / cp.T * r.t_plus;
          cp.w_hat[(size_t)item * n + j] = sm.wh[j];
          cp.s[(size_t)item * n + j] = vel - 2.0 * vw * sm.wh[j];
        }
      } else {
        for (int j = tid; j < n; j += SPG_THREADS) {
          cp.w_hat[(size_t)item * n + j] = 0.0;
          cp.s[(size_t)item * n + j] = 0.0;
        }
      }
      if (tid == 0) {
        cp.t_plus[item] = r.t_plus;
        cp.status[item] = r.status;
      }
      __syncthreads();
      continue;
    }
    // ---- the walk (Alg. 6) on chain `item` ----------------------------------
    const uint32_t chain = cp.chain0 + (uint32_t)item;
    double* xc = cp.X + (size_t)item * n;
    long long segs = 0, refl_total = 0, bad = 0;
    int last = kOk;
    for (int j = tid; j < n; j += SPG_THREADS) sm.x0[j] = xc[j];
    __syncthreads();
    for (int k = 0; k < cp.steps; ++k) {
      const uint32_t step = cp.step0 + (uint32_t)k;
      // the momentum v ~ N(0, I_n) (not normalised); the length l = tau eta
      for (int i = tid; 2 * i < n; i += SPG_THREADS) {
        double g0, g1;
        rng_gauss_pair(cp.seed, chain, step, (uint32_t)i, &g0, &g1);
        sm.v[2 * i] = g0;
        if (2 * i + 1 < n) sm.v[2 * i + 1] = g1;
      }
      for (int j = tid; j < n; j += SPG_THREADS) sm.p[j] = sm.x0[j];
      double ell = cp.tau * rng_uniform(cp.seed, chain, step, kStreamEta);
      __syncthreads();
      int refl = 0, status = kOk;
      double tprev = 0.0;  // the last hit's t+ within this step (0 at its start)
      for (;;) {
        const CurveResult r = curve_segment(sp, cp, sm, Vp, 0.1 * tprev);
        ++segs;
        if (r.status != kOk) {
          status = r.status;
          break;
        }
        if (r.t_plus < ell) {
          // on to Phi((1 - kappa) t+) with Phi'(t+) reflected on the normal
          const double tp = r.t_plus, tb = (1.0 - cp.kappa) * tp;
          const double vw = velocity_dot_normal(sm, n, cp.T, tp);
          for (int j = tid; j < n; j += SPG_THREADS) {
            sm.p[j] += sm.v[j] * tb - sm.c[j] / (2.0 * cp.T) * tb * tb;
            const double vel = sm.v[j] - sm.c[j] / cp.T * tp;
            sm.v[j] = vel - 2.0 * vw * sm.wh[j];
          }
          __syncthreads();
          ell -= tp;
          tprev = tp;
          if (++refl > cp.rho) {
            status = kRho;
            break;
          }
        } else {
          for (int j = tid; j < n; j += SPG_THREADS)
            sm.x0[j] = sm.p[j] + sm.v[j] * ell - sm.c[j] / (2.0 * cp.T) * ell * ell;
          __syncthreads();
          break;
        }
      }
      refl_total += refl;
      if (status != kOk) {
        ++bad;
        last = status;
      }
      __syncthreads();
    }
    for (int j = tid; j < n; j += SPG_THREADS) xc[j] = sm.x0[j];
    if (tid == 0) {
      long long* st = cp.stats + (size_t)item * kNumStats;
      st[kStatSegments] += segs;
      st[kStatReflections] += refl_total;
      st[kStatBadSteps] += bad;
      cp.status[item] = last;
    }
    __syncthreads();
  }
}

// packed C = -(1/(2T)) sum_j c_j A_j
__global__ void curve_c_kernel(DevSpec sp, const double* c, double T, double* Cp) {
  const long long P = sp.P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P;
       e += (long long)gridDim.x * blockDim.x) {
    double g = 0.0;
    for (int j = 0; j < sp.n; ++j) g += c[j] * sp.A[(size_t)(j + 1) * P + e];
    Cp[e] = -g / (2.0 * T);
  }
}

}  // namespace

size_t curve_smem_bytes(int n, int m) { return curve_doubles(n, m) * 8 + 16 * sizeof(int); }

cudaError_t launch_curve(const DevSpec& sp, const CurveParams& cp, int ctas, cudaStream_t st) {
  if (cp.count <= 0) return cudaSuccess;
  const size_t smem = curve_smem_bytes(sp.n, sp.m);
  cudaError_t e = cudaFuncSetAttribute(curve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = cp.count < ctas ? cp.count : ctas;
  double* Vwork = nullptr;
  e = cudaMallocAsync(&Vwork, sizeof(double) * (size_t)grid * sp.P, st);
  if (e != cudaSuccess) return e;
  curve_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, cp, Vwork);
  e = cudaGetLastError();
  cudaFreeAsync(Vwork, st);
  return e;
}

}  // namespace spg

namespace {

bool on_device(const void* p) {
  cudaPointerAttributes at;
  const bool dev = cudaPointerGetAttributes(&at, p) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  return dev;
}

// c (host or device) to the device, and the packed C of the trajectory
int curve_setup(const spg::DevSpec& sp, const double* c, double T, cudaStream_t st, double** dc,
                double** Cp, const char* too_big) {
  *dc = *Cp = nullptr;
  if (sp.m > spg::kCurveMaxM) return spg_set_error(SP_EINVAL, too_big);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (spg::curve_smem_bytes(sp.n, sp.m) > (size_t)optin)
    return spg_set_error(SP_EINVAL, "curve: n too large for the shared-memory layout");
  if (cudaMallocAsync(dc, sizeof(double) * sp.n, st) != cudaSuccess ||
      cudaMallocAsync(Cp, sizeof(double) * sp.P, st) != cudaSuccess) {
    cudaGetLastError();
    if (*dc) cudaFreeAsync(*dc, st);
    *dc = nullptr;
    return spg_set_error(SP_ENOMEM, "curve: allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(*dc, c, sizeof(double) * sp.n,
                                  on_device(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  st);
  if (e == cudaSuccess) {
    int blocks = (int)((sp.P + 255) / 256);
    blocks = blocks < 1024 ? blocks : 1024;
    spg::curve_c_kernel<<<blocks, 256, 0, st>>>(sp, *dc, T, *Cp);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(*dc, st);
    cudaFreeAsync(*Cp, st);
    return spg_set_error(SP_ECUDA, cudaGetErrorString(e));
  }
  return SP_OK;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

extern "C" int sp_curve_reflect(sp_spec* s, int count, const double* x, const double* v,
                                const double* c, double T, double* t_plus, double* w_hat,
                                double* s_out, int* status, void* stream) {
  if (!s || !c || (count > 0 && (!x || !v || !t_plus || !w_hat || !s_out || !status)))
    return spg_set_error(SP_EINVAL, "sp_curve_reflect: null argument");
  if (count < 0 || !(T > 0.0))
    return spg_set_error(SP_EINVAL, "sp_curve_reflect: need count >= 0 and T > 0");
  if (count == 0) return SP_OK;
  const spg::DevSpec sp = spg::spec_dev(s);
  cudaStream_t st = (cudaStream_t)stream;
  double *dc = nullptr, *Cp = nullptr;
  if (int r = curve_setup(sp, c, T, st, &dc, &Cp, "sp_curve_reflect: m above 64")) return r;
  spg::CurveParams cp{};
  cp.op = 0;
  cp.count = count;
  cp.x = x;
  cp.v = v;
  cp.c = dc;
  cp.Cp = Cp;
  cp.T = T;
  cp.t_plus = t_plus;
  cp.w_hat = w_hat;
  cp.s = s_out;
  cp.status = status;
  cudaError_t e = spg::launch_curve(sp, cp, sm_count(), st);
  cudaFreeAsync(dc, st);
  cudaFreeAsync(Cp, st);
  if (e != cudaSuccess) return spg_set_error(SP_ECUDA, cudaGetErrorString(e));
  return SP_OK;
}

extern "C" int sp_step_hmc(sp_chains* ch, int steps, const double* c, double T, double tau,
                           int rho, double kappa, void* stream) {
  if (!ch || !c) return spg_set_error(SP_EINVAL, "sp_step_hmc: null argument");
  if (steps < 0 || !(T > 0.0) || !(tau > 0.0) || rho < 0 || !(kappa >= 0.0 && kappa < 1.0))
    return spg_set_error(SP_EINVAL,
                         "sp_step_hmc: need steps >= 0, T > 0, tau > 0, rho >= 0, 0 <= kappa < 1");
  if (steps == 0) return SP_OK;
  const spg::ChainState cs = spg::chain_state(ch);
  const spg::DevSpec sp = spg::spec_dev(cs.spec);
  cudaStream_t st = (cudaStream_t)stream;
  double *dc = nullptr, *Cp = nullptr;
  if (int r = curve_setup(sp, c, T, st, &dc, &Cp, "sp_step_hmc: m above 64")) return r;
  spg::CurveParams cp{};
  cp.op = 1;
  cp.count = cs.C;
  cp.c = dc;
  cp.Cp = Cp;
  cp.T = T;
  cp.status = cs.status;
  cp.X = cs.X;
  cp.stats = cs.stats;
  cp.steps = steps;
  cp.step0 = cs.step;
  cp.chain0 = cs.chain0;
  cp.seed = cs.seed;
  cp.tau = tau;
  cp.kappa = kappa;
  cp.rho = rho;
  cudaError_t e = spg::launch_curve(sp, cp, sm_count(), st);
  cudaFreeAsync(dc, st);
  cudaFreeAsync(Cp, st);
  if (e != cudaSuccess) return spg_set_error(SP_ECUDA, cudaGetErrorString(e));
  spg::chain_advance(ch, (uint32_t)steps);
  return SP_OK;
}
