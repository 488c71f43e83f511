// Extreme eigenpairs of the shifted pencil operator
//   M_sigma = -L^{-1} V L^{-T},   F(x) + sigma V = L L^T,
// by Lanczos with full reorthogonalisation (two classical Gram-Schmidt
// passes per step).  Eigenvalues mu of M_sigma give the roots of
// det(F(x) + t V) as t = sigma + 1/mu: the largest mu gives t+ (Sec. 2.3,
// Lemma "PEP and S cap C"), the smallest gives t-.
//
// The small tridiagonal matrix T_K is analysed by multisection on Sturm
// counts (one warp) and inverse iteration (one thread), both in FP64.
#pragma once
#include "common.cuh"
#include "dense.cuh"

namespace spg {

constexpr int kMaxLanczos = 128;

// scalar workspace of the Lanczos run (in shared memory)
struct LanczosScalars {
  double alpha[kMaxLanczos];
  double beta[kMaxLanczos + 1];  // beta[i] couples i-1 and i; beta[K] = residual norm
  double s_max[kMaxLanczos];     // Ritz coefficient vectors
  double s_min[kMaxLanczos];
  double cwork[kMaxLanczos];
  double h[kMaxLanczos];
  double red[SPG_WARPS];
  double theta_max, theta_min, res_max, res_min;
  int K, done, flag;
};

// Sturm count: number of eigenvalues of T below x
__device__ __forceinline__ int sturm_count(const double* a, const double* b, int K, double x) {
  const double tiny = 1e-300;
  double d = a[0] - x;
  int c = d < 0.0;
  for (int i = 1; i < K; ++i) {
    if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
    d = (a[i] - x) - b[i] * (b[i] / d);
    c += d < 0.0;
  }
  return c;
}

// warp 0: the largest (want_max) or smallest eigenvalue of T_K by 33-way
// multisection on Sturm counts, to a relative width of ~1e-15
__device__ double tri_extreme(const double* a, const double* b, int K, bool want_max) {
  const int lane = threadIdx.x & 31;
  double lo = 1.0e308, hi = -1.0e308;
  for (int i = lane; i < K; i += 32) {
    double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < K ? fabs(b[i + 1]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  double span = fmax(hi - lo, 1e-300);
  lo -= 1e-3 * span;
  hi += 1e-3 * span;
  // invariant: max -> count(lo) <= K-1, count(hi) == K ; min -> count(lo) == 0, count(hi) >= 1
  for (int round = 0; round < 40; ++round) {
    const double w = hi - lo;
    if (!(w > 8.0 * 2.2e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + (double)(lane + 1) * (w / 33.0);
    const int c = sturm_count(a, b, K, x);
    const bool below = want_max ? (c <= K - 1) : (c == 0);
    unsigned mb = __ballot_sync(0xffffffffu, below);
    unsigned ma = ~mb;
    int lb = mb ? 31 - __clz(mb) : -1;  // highest lane still below
    int la = ma ? __ffs(ma) - 1 : 32;   // lowest lane above
    double nlo = lb >= 0 ? __shfl_sync(0xffffffffu, x, lb) : lo;
    double nhi = la < 32 ? __shfl_sync(0xffffffffu, x, la) : hi;
    if (!(nlo < nhi)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// thread 0: inverse iteration on (T - theta I) for the eigenvector s (two
// passes, Thomas algorithm with guarded pivots).  Returns the Rayleigh
// quotient s^T T s / s^T s and writes the normalised s.
template <typename R>
__device__ R tri_eigvec(const double* a, const double* b, int K, R theta, R* s, R* cw) {
  const R tiny = (sizeof(R) == 8) ? R(1e-300) : R(1e-30);
  const R eps = (sizeof(R) == 8) ? R(2.2e-16) : R(1.2e-7);
  R scale = R(0);
  for (int i = 0; i < K; ++i) scale = fmax(scale, fabs((R)a[i] - theta) + fabs((R)b[i]));
  const R guard = fmax(eps * scale, tiny);
  for (int i = 0; i < K; ++i) s[i] = R(1);
  for (int pass = 0; pass < 2; ++pass) {
    R den = (R)a[0] - theta;
    if (fabs(den) < guard) den = den < R(0) ? -guard : guard;
    cw[0] = (K > 1 ? (R)b[1] : R(0)) / den;
    s[0] = s[0] / den;
    for (int i = 1; i < K; ++i) {
      den = ((R)a[i] - theta) - (R)b[i] * cw[i - 1];
      if (fabs(den) < guard) den = den < R(0) ? -guard : guard;
      cw[i] = (i + 1 < K ? (R)b[i + 1] : R(0)) / den;
      s[i] = (s[i] - (R)b[i] * s[i - 1]) / den;
    }
    for (int i = K - 2; i >= 0; --i) s[i] -= cw[i] * s[i + 1];
    // scale by the largest entry first (the solve may produce huge values)
    R mx = R(0);
    for (int i = 0; i < K; ++i) mx = fmax(mx, fabs(s[i]));
    if (!(mx > R(0)) || !isfinite(mx)) {
      for (int i = 0; i < K; ++i) s[i] = (i == K - 1) ? R(1) : R(0);
      mx = R(1);
    }
    for (int i = 0; i < K; ++i) s[i] /= mx;
    R nrm = R(0);
    for (int i = 0; i < K; ++i) nrm += s[i] * s[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < K; ++i) s[i] /= nrm;
  }
  R rq = R(0);
  for (int i = 0; i < K; ++i) {
    R ts = (R)a[i] * s[i];
    if (i > 0) ts += (R)b[i] * s[i - 1];
    if (i + 1 < K) ts += (R)b[i + 1] * s[i + 1];
    rq += s[i] * ts;
  }
  return rq;
}

// The operator M_sigma = -L^{-1} V L^{-T}: L packed with inverted diagonal
// blocks; V either full row-major (packed = false) or a packed lower
// triangle (packed = true, `part` is the symv scratch of SPG_WARPS * m).
template <typename T>
struct PencilOp {
  const T* L;
  const T* V;
  bool packed;
  T* part;
};

// r <- M_sigma q.  z: scratch vector (m), s: scratch (>= 288)
template <typename T>
__device__ void apply_pencil(const PencilOp<T>& op, const T* q, T* r, T* z, int m, T* s) {
  for (int i = threadIdx.x; i < m; i += SPG_THREADS) z[i] = q[i];
  __syncthreads();
  solve_upper(op.L, z, m, s);
  if (op.packed)
    symv_packed(op.V, z, r, m, T(-1), op.part);
  else
    gemv_full(op.V, z, r, m, T(-1));
  solve_lower(op.L, r, m, s);
}

struct LanczosOut {
  double theta_max, theta_min;  // extreme Ritz values (FP64 Rayleigh quotients)
  int iters;
  bool converged;
};

// Lanczos with full reorthogonalisation.
//   q0 (m, smem): start vector (overwritten); Q (kmax x m, global): basis;
//   ymax / ymin (m, smem): Ritz vectors of the extreme eigenvalues (ymin only
//   if want_min); r, z (m, smem) and s (>= 288, smem): scratch.
//   tol: relative residual target |M y - theta y| <= tol |theta|.
template <typename T>
__device__ LanczosOut lanczos_extreme(const PencilOp<T>& op, T* __restrict__ Q, T* q, T* r, T* z,
                                      T* s, T* ymax, T* ymin, int m, int kmax, bool want_min,
                                      double tol, LanczosScalars* sc) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  kmax = min(min(kmax, kMaxLanczos), m);
  // normalise q
  {
    T p = T(0);
    for (int i = tid; i < m; i += SPG_THREADS) p += q[i] * q[i];
    double nrm = sqrt((double)block_sum(p, (T*)sc->red));
    for (int i = tid; i < m; i += SPG_THREADS) q[i] = (T)(q[i] / nrm);
    if (tid == 0) {
      sc->done = 0;
      sc->beta[0] = 0.0;
    }
    __syncthreads();
  }
  int K = 0;
  for (int k = 0; k < kmax; ++k) {
    T* Qk = Q + (size_t)k * m;
    for (int i = tid; i < m; i += SPG_THREADS) Qk[i] = q[i];
    apply_pencil(op, q, r, z, m, s);
    // two passes of classical Gram-Schmidt against Q[0..k]
    double alpha = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = wid; j <= k; j += SPG_WARPS) {
        const T* Qj = Q + (size_t)j * m;
        T acc = T(0);
        for (int i = lane; i < m; i += 32) acc += Qj[i] * r[i];
        acc = warp_sum(acc);
        if (lane == 0) sc->h[j] = (double)acc;
      }
      __syncthreads();
      for (int i = tid; i < m; i += SPG_THREADS) {
        T acc = T(0);
        for (int j = 0; j <= k; ++j) acc += (T)sc->h[j] * Q[(size_t)j * m + i];
        r[i] -= acc;
      }
      alpha += sc->h[k];
      __syncthreads();
    }
    T p = T(0);
    for (int i = tid; i < m; i += SPG_THREADS) p += r[i] * r[i];
    const double beta = sqrt((double)block_sum(p, (T*)sc->red));
    K = k + 1;
    if (tid == 0) {
      sc->alpha[k] = alpha;
      sc->beta[K] = beta;
    }
    __syncthreads();
    // convergence test every few steps (and on breakdown / last step)
    const bool breakdown = !(beta > 1e-300) ||
                           beta <= 1e-15 * fabs(alpha) + 1e-300;
    const bool check = breakdown || K == kmax || (K >= 6 && (K % 4 == 0));
    if (check) {
      if (wid == 0) {
        double tmax = tri_extreme(sc->alpha, sc->beta, K, true);
        double tmin = want_min ? tri_extreme(sc->alpha, sc->beta, K, false) : 0.0;
        if (lane == 0) {
          double th = tri_eigvec<double>(sc->alpha, sc->beta, K, tmax, sc->s_max, sc->cwork);
          double resmax = fabs(beta * sc->s_max[K - 1]);
          double thn = 0.0, resmin = 0.0;
          if (want_min) {
            thn = tri_eigvec<double>(sc->alpha, sc->beta, K, tmin, sc->s_min, sc->cwork);
            resmin = fabs(beta * sc->s_min[K - 1]);
          }
          const double big = fmax(fabs(th), fabs(thn));
          // attainable accuracy: the operator is applied with relative error ~ eps |T|
          const double floor_ = 64.0 * (sizeof(T) == 8 ? 2.2e-16 : 1.2e-7) * big;
          bool ok = resmax <= fmax(tol * fabs(th), floor_);
          if (want_min) ok = ok && resmin <= fmax(tol * fabs(thn), floor_);
          sc->theta_max = th;
          sc->theta_min = thn;
          sc->res_max = resmax;
          sc->res_min = resmin;
          sc->done = (ok || breakdown) ? 2 : (K == kmax ? 1 : 0);
        }
      }
      __syncthreads();
      if (sc->done) break;
    }
    for (int i = tid; i < m; i += SPG_THREADS) q[i] = (T)(r[i] / beta);
    __syncthreads();
  }
  // the last check left the FP64 Ritz coefficients in s_max / s_min
  if (tid == 0) sc->K = K;
  __syncthreads();
  for (int i = tid; i < m; i += SPG_THREADS) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < K; ++j) {
      const double qv = (double)Q[(size_t)j * m + i];
      a += sc->s_max[j] * qv;
      if (want_min) b += sc->s_min[j] * qv;
    }
    ymax[i] = (T)a;
    if (want_min) ymin[i] = (T)b;
  }
  __syncthreads();
  LanczosOut o;
  o.theta_max = sc->theta_max;
  o.theta_min = want_min ? sc->theta_min : 0.0;
  o.iters = K;
  o.converged = sc->done == 2;
  return o;
}

}  // namespace spg
