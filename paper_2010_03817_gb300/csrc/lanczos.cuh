// Extreme eigenpairs of the shifted pencil operator
//   M_sigma = -L^{-1} V L^{-T},   F(x) + sigma V = L L^T,
// by Lanczos with full reorthogonalisation (two classical Gram-Schmidt
// passes per step).  Eigenvalues mu of M_sigma give the roots of
// det(F(x) + t V) as t = sigma + 1/mu: the largest mu gives t+ (Sec. 2.3,
// Lemma "PEP and S cap C"), the smallest gives t-.
//
// The small tridiagonal matrix T_K is analysed in FP32 (multisection on
// Sturm counts by one warp, inverse iteration by one thread) for the
// convergence tests; FP64 inverse iteration, shifted by its own Rayleigh
// quotient, gives the final Ritz pairs (and the tests of the FP64 solve once
// the FP32 residual estimate reaches its floor).
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
  float af[kMaxLanczos];         // FP32 copies of alpha, beta and beta^2 (cheap analysis)
  float bf[kMaxLanczos + 1];
  float b2f[kMaxLanczos + 1];
  float sf[2 * kMaxLanczos];     // FP32 Ritz coefficients + Thomas scratch
  double theta_max, theta_min, res_max, res_min;
  long long* prof;               // optional clock64 sums per sub-stage (4 slots) or null
  int K, done, flag, precise;
};

// add the cycles since t0 to sub-stage slot s of the profile (thread 0)
__device__ __forceinline__ void lz_mark(LanczosScalars* sc, int s, long long& t0) {
  if (sc->prof && threadIdx.x == 0) {
    const long long t1 = clock64();
    atomicAdd(reinterpret_cast<unsigned long long*>(sc->prof + s), (unsigned long long)(t1 - t0));
    t0 = t1;
  }
}

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

// FP32 Sturm count (cheap: FP32 pipe)
__device__ __forceinline__ int sturm_count_f(const float* a, const float* b2, int K, float x) {
  const float tiny = 1e-30f;
  float d = a[0] - x;
  int c = d < 0.f;
  for (int i = 1; i < K; ++i) {
    if (fabsf(d) < tiny) d = d < 0.f ? -tiny : tiny;
    d = (a[i] - x) - b2[i] / d;
    c += d < 0.f;
  }
  return c;
}

// warp 0: FP32 estimate (relative width ~1e-6) of the largest (want_max) or
// smallest eigenvalue of T_K; af / b2f hold the FP32 diagonal and squared
// off-diagonal
__device__ inline float tri_extreme_f(const float* af, const float* b2f, int K, bool want_max) {
  const int lane = threadIdx.x & 31;
  float lo = 3.0e38f, hi = -3.0e38f;
  for (int i = lane; i < K; i += 32) {
    const float r = (i > 0 ? sqrtf(b2f[i]) : 0.f) + (i + 1 < K ? sqrtf(b2f[i + 1]) : 0.f);
    lo = fminf(lo, af[i] - r);
    hi = fmaxf(hi, af[i] + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const float span = fmaxf(hi - lo, 1e-30f);
  lo -= 1e-3f * span;
  hi += 1e-3f * span;
  for (int round = 0; round < 12; ++round) {
    const float w = hi - lo;
    if (!(w > 4e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
    const float x = lo + (float)(lane + 1) * (w / 33.f);
    const int c = sturm_count_f(af, b2f, K, x);
    const bool below = want_max ? (c <= K - 1) : (c == 0);
    const unsigned mb = __ballot_sync(0xffffffffu, below);
    const unsigned ma = ~mb;
    const int lb = mb ? 31 - __clz(mb) : -1;
    const int la = ma ? __ffs(ma) - 1 : 32;
    const float nlo = lb >= 0 ? __shfl_sync(0xffffffffu, x, lb) : lo;
    const float nhi = la < 32 ? __shfl_sync(0xffffffffu, x, la) : hi;
    if (!(nlo < nhi)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5f * (lo + hi);
}

// warp 0: the largest (want_max) or smallest eigenvalue of T_K by 33-way
// multisection on Sturm counts, to a relative width of ~1e-15
__device__ inline double tri_extreme(const double* a, const double* b, int K, bool want_max) {
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

// 1/x in FP64 from an FP32 seed and two Newton steps (quadratic convergence:
// 2^-23 -> 2^-46 -> below 2^-53); x is never 0 here (pivots are guarded)
__device__ __forceinline__ double recip64(double x) {
  double r = (double)(1.0f / (float)x);
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
}
__device__ __forceinline__ float recip_any(float x) { return 1.0f / x; }
__device__ __forceinline__ double recip_any(double x) { return recip64(x); }

// thread 0: inverse iteration on (T - theta I) for the eigenvector s (two
// passes, Thomas algorithm with guarded pivots).  Returns the Rayleigh
// quotient s^T T s / s^T s and writes the normalised s.
template <typename R>
__device__ R tri_eigvec(const double* a, const double* b, int K, R theta, R* s, R* cw) {
  const R tiny = (sizeof(R) == 8) ? R(1e-300) : R(1e-30);
  const R eps = (sizeof(R) == 8) ? R(2.2e-16) : R(1.2e-7);
  R scale = R(0);
  for (int i = 0; i < K; ++i) scale = fmax(scale, fabs((R)a[i] - theta) + fabs((R)b[i]));
  // the FP32 seed of recip64 needs a guard inside the FP32 range
  const R guard = fmax(eps * scale, (sizeof(R) == 8) ? R(1e-30) : tiny);
  for (int i = 0; i < K; ++i) s[i] = R(1);
  for (int pass = 0; pass < 2; ++pass) {
    R den = (R)a[0] - theta;
    if (fabs(den) < guard) den = den < R(0) ? -guard : guard;
    R rd = recip_any(den);
    cw[0] = (K > 1 ? (R)b[1] : R(0)) * rd;
    s[0] = s[0] * rd;
    for (int i = 1; i < K; ++i) {
      den = ((R)a[i] - theta) - (R)b[i] * cw[i - 1];
      if (fabs(den) < guard) den = den < R(0) ? -guard : guard;
      rd = recip_any(den);
      cw[i] = (i + 1 < K ? (R)b[i + 1] : R(0)) * rd;
      s[i] = (s[i] - (R)b[i] * s[i - 1]) * rd;
    }
    for (int i = K - 2; i >= 0; --i) s[i] -= cw[i] * s[i + 1];
    // scale by the largest entry first (the solve may produce huge values)
    R mx = R(0);
    for (int i = 0; i < K; ++i) mx = fmax(mx, fabs(s[i]));
    if (!(mx > R(0)) || !isfinite(mx)) {
      for (int i = 0; i < K; ++i) s[i] = (i == K - 1) ? R(1) : R(0);
      mx = R(1);
    }
    const R rmx = R(1) / mx;
    R nrm = R(0);
    for (int i = 0; i < K; ++i) {
      s[i] *= rmx;
      nrm += s[i] * s[i];
    }
    const R rn = R(1) / sqrt(nrm);
    for (int i = 0; i < K; ++i) s[i] *= rn;
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

// eigenpair of T_K near theta to full FP64 accuracy: inverse iteration at the
// estimate, then again at the Rayleigh quotient it returns
__device__ inline double tri_eigpair64(const double* a, const double* b, int K, double theta,
                                       double* s, double* cw) {
  const double rq = tri_eigvec<double>(a, b, K, theta, s, cw);
  return tri_eigvec<double>(a, b, K, rq, s, cw);
}

// warp 0 (all lanes): the extreme eigenpair of T_K (largest if want_max, else
// smallest) to FP64 accuracy.  Inverse iteration converges to the eigenvalue
// nearest to its shift, which for a shift from an FP32 analysis need not be
// the extreme one when two eigenvalues lie within the FP32 resolution of the
// spectrum; an FP64 Sturm count certifies that no eigenvalue lies beyond the
// result, else an FP64 multisection finds the extreme eigenvalue and the
// inverse iteration restarts there.  s, cw: K-vectors (s receives the
// normalised eigenvector).
__device__ inline double tri_extreme_pair64(const double* a, const double* b, int K, double est,
                                            bool want_max, double* s, double* cw) {
  const int lane = threadIdx.x & 31;
  double th = 0.0;
  int beyond = 0;
  if (lane == 0) {
    th = tri_eigpair64(a, b, K, est, s, cw);
    double nt = 0.0;
    for (int i = 0; i < K; ++i)
      nt = fmax(nt, fabs(a[i]) + (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < K ? fabs(b[i + 1]) : 0.0));
    const double d = 1e-13 * fabs(th) + 8.0 * K * 2.2e-16 * nt;
    beyond = !isfinite(th) ||
             (want_max ? sturm_count(a, b, K, th + d) < K : sturm_count(a, b, K, th - d) > 0);
  }
  beyond = __shfl_sync(0xffffffffu, beyond, 0);
  th = __shfl_sync(0xffffffffu, th, 0);
  if (beyond) {
    const double xe = tri_extreme(a, b, K, want_max);
    if (lane == 0) th = tri_eigpair64(a, b, K, xe, s, cw);
    th = __shfl_sync(0xffffffffu, th, 0);
  }
  __syncwarp();
  return th;
}

// FP32 inverse iteration on the FP32 copies (a, b): same scheme as tri_eigvec
__device__ inline float tri_eigvec_f(const float* a, const float* b, int K, float theta, float* s,
                                     float* cw) {
  float scale = 0.f;
  for (int i = 0; i < K; ++i) scale = fmaxf(scale, fabsf(a[i] - theta) + fabsf(b[i]));
  const float guard = fmaxf(1.2e-7f * scale, 1e-30f);
  for (int i = 0; i < K; ++i) s[i] = 1.f;
  for (int pass = 0; pass < 2; ++pass) {
    float den = a[0] - theta;
    if (fabsf(den) < guard) den = den < 0.f ? -guard : guard;
    cw[0] = (K > 1 ? b[1] : 0.f) / den;
    s[0] = s[0] / den;
    for (int i = 1; i < K; ++i) {
      den = (a[i] - theta) - b[i] * cw[i - 1];
      if (fabsf(den) < guard) den = den < 0.f ? -guard : guard;
      cw[i] = (i + 1 < K ? b[i + 1] : 0.f) / den;
      s[i] = (s[i] - b[i] * s[i - 1]) / den;
    }
    for (int i = K - 2; i >= 0; --i) s[i] -= cw[i] * s[i + 1];
    float mx = 0.f;
    for (int i = 0; i < K; ++i) mx = fmaxf(mx, fabsf(s[i]));
    if (!(mx > 0.f) || !isfinite(mx)) {
      for (int i = 0; i < K; ++i) s[i] = (i == K - 1) ? 1.f : 0.f;
      mx = 1.f;
    }
    float nrm = 0.f;
    for (int i = 0; i < K; ++i) {
      s[i] /= mx;
      nrm += s[i] * s[i];
    }
    nrm = sqrtf(nrm);
    for (int i = 0; i < K; ++i) s[i] /= nrm;
  }
  float rq = 0.f;
  for (int i = 0; i < K; ++i) {
    float ts = a[i] * s[i];
    if (i > 0) ts += b[i] * s[i - 1];
    if (i + 1 < K) ts += b[i + 1] * s[i + 1];
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

// r <- M_sigma q.  z: scratch vector (m), s: scratch (>= SPG_SCR)
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
//   if want_min); r, z (m, smem) and s (>= SPG_SCR, smem): scratch.
//   tol: relative residual target |M y - theta y| <= tol |theta|.
template <typename T>
__device__ LanczosOut lanczos_extreme(const PencilOp<T>& op, T* __restrict__ Q, T* q, T* r, T* z,
                                      T* s, T* ymax, T* ymin, int m, int kmax, bool want_min,
                                      double tol, LanczosScalars* sc, int check_from = 6,
                                      int check_every = 4) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  kmax = min(min(kmax, kMaxLanczos), m);
  // normalise q
  {
    T p = T(0);
    for (int i = tid; i < m; i += SPG_THREADS) p += q[i] * q[i];
    const T rn = T(1) / sqrt(block_sum(p, (T*)sc->red));
    for (int i = tid; i < m; i += SPG_THREADS) q[i] *= rn;
    if (tid == 0) {
      sc->done = 0;
      sc->precise = 0;
      sc->beta[0] = 0.0;
      sc->bf[0] = 0.f;
      sc->b2f[0] = 0.f;
    }
    __syncthreads();
  }
  int K = 0;
  long long tz = clock64();
  for (int k = 0; k < kmax; ++k) {
    T* Qk = Q + (size_t)k * m;
    for (int i = tid; i < m; i += SPG_THREADS) Qk[i] = q[i];
    apply_pencil(op, q, r, z, m, s);
    lz_mark(sc, 0, tz);
    // two passes of classical Gram-Schmidt against Q[0..k]; the coefficients
    // are kept in T (a double -> float conversion runs on the FP64 pipe)
    T* hT = reinterpret_cast<T*>(sc->h);
    double alpha = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = wid; j <= k; j += SPG_WARPS) {
        const T* Qj = Q + (size_t)j * m;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int i = lane;
        for (; i + 96 < m; i += 128) {
          a0 += Qj[i] * r[i];
          a1 += Qj[i + 32] * r[i + 32];
          a2 += Qj[i + 64] * r[i + 64];
          a3 += Qj[i + 96] * r[i + 96];
        }
        for (; i < m; i += 32) a0 += Qj[i] * r[i];
        const T acc = warp_sum((a0 + a1) + (a2 + a3));
        if (lane == 0) hT[j] = acc;
      }
      __syncthreads();
      for (int i = tid; i < m; i += SPG_THREADS) {
        // four independent loads in flight per step
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int j = 0;
        for (; j + 3 <= k; j += 4) {
          a0 += hT[j] * Q[(size_t)j * m + i];
          a1 += hT[j + 1] * Q[(size_t)(j + 1) * m + i];
          a2 += hT[j + 2] * Q[(size_t)(j + 2) * m + i];
          a3 += hT[j + 3] * Q[(size_t)(j + 3) * m + i];
        }
        for (; j <= k; ++j) a0 += hT[j] * Q[(size_t)j * m + i];
        r[i] -= (a0 + a1) + (a2 + a3);
      }
      alpha += (double)hT[k];
      __syncthreads();
    }
    T p = T(0);
    for (int i = tid; i < m; i += SPG_THREADS) p += r[i] * r[i];
    const T beta_t = sqrt(block_sum(p, (T*)sc->red));
    const double beta = (double)beta_t;
    K = k + 1;
    if (tid == 0) {
      sc->alpha[k] = alpha;
      sc->beta[K] = beta;
      sc->af[k] = (float)alpha;
      sc->bf[K] = (float)beta;
      sc->b2f[K] = (float)(beta * beta);
    }
    __syncthreads();
    lz_mark(sc, 1, tz);
    // convergence test every few steps (and on breakdown / last step)
    const bool breakdown = !(beta > 1e-300) ||
                           beta <= 1e-15 * fabs(alpha) + 1e-300;
    const bool check =
        breakdown || K == kmax || (K >= check_from && ((K - check_from) % check_every == 0));
    if (check) {
      if (wid == 0) {
        // FP32 analysis first; the FP64 analysis (certified extreme eigenpair
        // of T_K) only once the FP32 residual estimate has reached its floor
        // (or on breakdown / at the last step)
        const float tmaxf = tri_extreme_f(sc->af, sc->b2f, K, true);
        const float tminf = want_min ? tri_extreme_f(sc->af, sc->b2f, K, false) : 0.f;
        const double eps_t = sizeof(T) == 8 ? 2.2e-16 : 1.2e-7;
        int ok = 0, precise = 0;
        float thf = 0.f, thnf = 0.f;
        if (lane == 0) {
          float* sfv = sc->sf;
          float* cwf = sc->sf + kMaxLanczos;
          thf = tri_eigvec_f(sc->af, sc->bf, K, tmaxf, sfv, cwf);
          const float rmf = fabsf((float)beta * sfv[K - 1]);
          float rnf = 0.f;
          if (want_min) {
            thnf = tri_eigvec_f(sc->af, sc->bf, K, tminf, sfv, cwf);
            rnf = fabsf((float)beta * sfv[K - 1]);
          }
          const float bigf = fmaxf(fabsf(thf), fabsf(thnf));
          const float floor32 = 64.f * 1.2e-7f * bigf;
          const float floorT = (float)(64.0 * eps_t) * bigf;
          bool ok32 = rmf <= fmaxf((float)tol * fabsf(thf), floorT);
          if (want_min) ok32 = ok32 && rnf <= fmaxf((float)tol * fabsf(thnf), floorT);
          const bool at_floor = rmf <= 4.f * floor32 && (!want_min || rnf <= 4.f * floor32);
          if (sizeof(T) == 4 || (double)tol >= 1e-6)
            ok = ok32;
          else
            precise = at_floor || breakdown || K == kmax;
        }
        precise = __shfl_sync(0xffffffffu, precise, 0);
        if (precise) {
          const double th = tri_extreme_pair64(sc->alpha, sc->beta, K, (double)tmaxf, true,
                                               sc->s_max, sc->cwork);
          double thn = 0.0;
          if (want_min)
            thn = tri_extreme_pair64(sc->alpha, sc->beta, K, (double)tminf, false, sc->s_min,
                                     sc->cwork);
          if (lane == 0) {
            sc->precise = 1;
            const double rm = fabs(beta * sc->s_max[K - 1]);
            const double rn = want_min ? fabs(beta * sc->s_min[K - 1]) : 0.0;
            const double big = fmax(fabs(th), fabs(thn));
            const double floor_ = 64.0 * eps_t * big;
            ok = rm <= fmax(tol * fabs(th), floor_);
            if (want_min) ok = ok && rn <= fmax(tol * fabs(thn), floor_);
            sc->theta_max = th;
            sc->theta_min = thn;
          }
        }
        if (lane == 0) {
          if (!precise) {
            sc->theta_max = thf;
            sc->theta_min = thnf;
          }
          sc->done = (ok || breakdown) ? 2 : (K == kmax ? 1 : 0);
        }
      }
      __syncthreads();
      lz_mark(sc, 2, tz);
      if (sc->done) break;
    }
    {
      const T rb = T(1) / beta_t;
      for (int i = tid; i < m; i += SPG_THREADS) q[i] = r[i] * rb;
    }
    __syncthreads();
  }
  // final Ritz pairs: for an FP64 run, FP64 inverse iteration at the last
  // estimate, certified extreme by a Sturm count (also the FP64 Rayleigh
  // quotient of T_K); for an FP32 run, the FP32 analysis
  if (wid == 0) {
    if (sizeof(T) == 4) {
      // an FP32 run: the FP32 analysis suffices (the multisection on Sturm
      // counts returns the extreme eigenvalue itself; a later refinement
      // certifies the result)
      const float tmaxf = tri_extreme_f(sc->af, sc->b2f, K, true);
      const float tminf = want_min ? tri_extreme_f(sc->af, sc->b2f, K, false) : 0.f;
      if (lane == 0) {
        float* sfv = sc->sf;
        float* cwf = sc->sf + kMaxLanczos;
        sc->theta_max = tri_eigvec_f(sc->af, sc->bf, K, tmaxf, sfv, cwf);
        for (int j = 0; j < K; ++j) sc->s_max[j] = sfv[j];
        if (want_min) {
          sc->theta_min = tri_eigvec_f(sc->af, sc->bf, K, tminf, sfv, cwf);
          for (int j = 0; j < K; ++j) sc->s_min[j] = sfv[j];
        }
        sc->K = K;
      }
    } else {
      const double th = tri_extreme_pair64(sc->alpha, sc->beta, K, sc->theta_max, true,
                                           sc->s_max, sc->cwork);
      double thn = 0.0;
      if (want_min)
        thn = tri_extreme_pair64(sc->alpha, sc->beta, K, sc->theta_min, false, sc->s_min,
                                 sc->cwork);
      if (lane == 0) {
        sc->theta_max = th;
        if (want_min) sc->theta_min = thn;
        sc->K = K;
      }
    }
  }
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
  lz_mark(sc, 3, tz);
  LanczosOut o;
  o.theta_max = sc->theta_max;
  o.theta_min = want_min ? sc->theta_min : 0.0;
  o.iters = K;
  o.converged = sc->done == 2;
  return o;
}

}  // namespace spg
