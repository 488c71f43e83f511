// Plain FP64 path: one CTA runs the whole boundary oracle for one chain at a
// time (persistent over chains).  Per segment:
//   form F(p) = A_0 + sum p_j A_j and V = sum v_j A_j      (Eq. 1; Lemma
//       "PEP and S cap C": the pencil B_0 + t B_1 of a line)
//   Cholesky of F + sigma V (shared memory)                (Alg. 1 as the
//       interior certificate)
//   Lanczos on M_sigma = -L^{-1} V L^{-T}: t = sigma + 1/mu (Alg. 2)
//   w_j = u^T A_j u, u = L^{-T} y                          (Lemma "Gradient
//       of det F")
//   t+ (and t-) refined by the pencil Rayleigh correction
//       t <- t - u^T (F + t V) u / (u^T V u) on the exact F and V
//   reflection s = v - 2 <v, w^> w^                        (Eq. "reflection")
// and the walk drivers of Alg. 4 (Hit-and-Run), CDHR and Alg. 5 (Billiard).
#include <math.h>

#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"
#include "lanczos.cuh"

namespace spg {

namespace {

struct Smem {
  double* L;     // packed factor (shared or global)
  double* p;     // n: current point
  double* v;     // n: direction
  double* x0;    // n: start of the step
  double* w;     // n+1: quadratic forms u^T A_j u
  double* wh;    // n: unit normal
  double* q;     // m
  double* r;     // m
  double* z;     // m
  double* ymax;  // m
  double* ymin;  // m
  double* u;     // m
  double* col;   // cholesky_scratch(m) (Cholesky panel)
  double* scr;   // SPG_SCR (triangular-solve partial sums)
  LanczosScalars* sc;
  double* bc;    // small broadcast area (16 doubles)
  int* ib;       // small int broadcast area (16 ints)
};

__host__ __device__ inline size_t align8(size_t b) { return (b + 7) & ~size_t(7); }

// carve the dynamic shared memory
__device__ Smem carve(double* base, int n, int m, bool l_in_smem, double* Lg, int pw = kPanel) {
  Smem s;
  double* q = base;
  const long long P = (long long)m * (m + 1) / 2;
  if (l_in_smem) {
    s.L = q;
    q += P;
  } else {
    s.L = Lg;
  }
  s.p = q; q += n;
  s.v = q; q += n;
  s.x0 = q; q += n;
  s.w = q; q += n + 1;
  s.wh = q; q += n;
  s.q = q; q += m;
  s.r = q; q += m;
  s.z = q; q += m;
  s.ymax = q; q += m;
  s.ymin = q; q += m;
  s.u = q; q += m;
  s.col = q; q += cholesky_scratch(m, pw);
  s.scr = q; q += SPG_SCR;
  s.bc = q; q += 16;
  s.sc = reinterpret_cast<LanczosScalars*>(q);
  if (threadIdx.x == 0) s.sc->prof = nullptr;
  q += (sizeof(LanczosScalars) + 7) / 8;
  s.ib = reinterpret_cast<int*>(q);
  return s;
}

// The FP64 factorisation with a run-time panel width (one compiled copy per
// width, called, so that the walk itself is compiled once)
template <int PW>
__device__ __noinline__ bool factor64_w(double* G, int m, double* pan, int* flag) {
  return factor_cholesky<double, PW>(G, m, pan, flag);
}
__device__ __forceinline__ bool factor64(int pw, double* G, int m, double* pan, int* flag) {
  if (pw == 4) return factor64_w<4>(G, m, pan, flag);
  if (pw == 16) return factor64_w<16>(G, m, pan, flag);
  return factor64_w<8>(G, m, pan, flag);
}

constexpr int kCdhrRefresh = 64;  // CDHR: steps between re-formations of F(p)
constexpr double kRedoRatio = 100.0;  // |mu_min| / mu_max above which the solve is redone
constexpr double kCorrectWindow = 1e-7;  // largest relative pencil correction kept

struct SegResult {
  double t_plus, t_minus, t_raw;
  int status;
  int iters;
  int retried;
  int flags;  // kSegFlag* of the segment record
};

// One boundary-oracle evaluation for the line p + t v (CTA-wide).
// vcol >= 0: v is the coordinate direction e_vcol (CDHR), so V = A_{vcol+1}
// is read from the stack instead of formed.
__device__ __noinline__ SegResult segment_fp64(const DevSpec& sp, const DevWork& wk, Smem& sm,
                                  double* __restrict__ Vfull, double* __restrict__ Fg,
                                  double* __restrict__ Q, double sigma, bool want_min,
                                  bool want_w, bool form_f, int vcol = -1, int PW = kPanel) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = sp.n, m = sp.m;
  const long long P = sp.P;
  SegResult res;
  res.retried = 0;
  res.flags = 0;
  // ---- form V (and F(p) when form_f; otherwise F is carried in Fg) ---------
  if (vcol >= 0) {
    // CDHR (Sec. 3.1): V = A_j is a slice of the stack; F(p) carried or formed
    const double* Aj = sp.A + (size_t)(vcol + 1) * P;
    for (long long e = tid; e < P; e += SPG_THREADS) {
      double f;
      if (form_f) {
        const double* Ae = sp.A + e;
        double f0 = 0.0, f1 = 0.0;
        int j = 0;
        for (; j + 1 < n; j += 2) {
          f0 += sm.p[j] * Ae[(size_t)(j + 1) * P];
          f1 += sm.p[j + 1] * Ae[(size_t)(j + 2) * P];
        }
        if (j < n) f0 += sm.p[j] * Ae[(size_t)(j + 1) * P];
        f = f0 + f1;
        Fg[e] = f;
      } else {
        f = Fg[e];
      }
      const double g = Aj[e];
      sm.L[e] = fma(sigma, g, sp.A[e] + f);
      const uint32_t ik = sp.pidx[e];
      const int i = ik >> 16, k = ik & 0xffff;
      Vfull[(size_t)i * m + k] = g;
      Vfull[(size_t)k * m + i] = g;
    }
  } else if (form_f) {
    for (long long e = tid; e < P; e += SPG_THREADS) {
      const double* Ae = sp.A + e;
      double f0 = 0.0, f1 = 0.0, g0 = 0.0, g1 = 0.0;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < n; j += 2) {
        const double a0 = Ae[(size_t)(j + 1) * P], a1 = Ae[(size_t)(j + 2) * P];
        f0 += sm.p[j] * a0;
        g0 += sm.v[j] * a0;
        f1 += sm.p[j + 1] * a1;
        g1 += sm.v[j + 1] * a1;
      }
      if (j < n) {
        const double a0 = Ae[(size_t)(j + 1) * P];
        f0 += sm.p[j] * a0;
        g0 += sm.v[j] * a0;
      }
      const double f = f0 + f1, g = g0 + g1;
      Fg[e] = f;
      sm.L[e] = fma(sigma, g, Ae[0] + f);
      const uint32_t ik = sp.pidx[e];
      const int i = ik >> 16, k = ik & 0xffff;
      Vfull[(size_t)i * m + k] = g;
      Vfull[(size_t)k * m + i] = g;
    }
  } else {
    for (long long e = tid; e < P; e += SPG_THREADS) {
      const double* Ae = sp.A + e;
      double g0 = 0.0, g1 = 0.0;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < n; j += 2) {
        g0 += sm.v[j] * Ae[(size_t)(j + 1) * P];
        g1 += sm.v[j + 1] * Ae[(size_t)(j + 2) * P];
      }
      if (j < n) g0 += sm.v[j] * Ae[(size_t)(j + 1) * P];
      const double g = g0 + g1;
      sm.L[e] = fma(sigma, g, Ae[0] + Fg[e]);
      const uint32_t ik = sp.pidx[e];
      const int i = ik >> 16, k = ik & 0xffff;
      Vfull[(size_t)i * m + k] = g;
      Vfull[(size_t)k * m + i] = g;
    }
  }
  __syncthreads();
  // ---- Cholesky of F + sigma V; a smaller shift if it overshot -------------
  // (x 0.2 per retry, then 0: the shift keeps the root just behind the point
  // -- the boundary it left -- from dominating M_sigma, whose rounding would
  // otherwise swamp the wanted eigenvector; unshifted, next to the boundary,
  // |M| / mu+ reaches 1 / kappa)
  for (int attempt = 0;; ++attempt) {
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    bool ok = factor64(PW, sm.L, m, sm.col, &sm.ib[0]);
    if (ok) break;
    if (sigma != 0.0) {
      sigma = attempt < 3 ? 0.2 * sigma : 0.0;
      res.retried = 1;
      res.flags |= kSegShiftRetry;
      for (long long e = tid; e < P; e += SPG_THREADS) {
        const uint32_t ik = sp.pidx[e];
        sm.L[e] = fma(sigma, Vfull[(size_t)(ik >> 16) * m + (ik & 0xffff)], sp.A[e] + Fg[e]);
      }
      __syncthreads();
      continue;
    }
    res.status = kNotPD;
    res.t_plus = res.t_minus = res.t_raw = 0.0;
    res.iters = 0;
    return res;
  }
  invert_diag_blocks(sm.L, m);
  // ---- Lanczos ------------------------------------------------------------
  for (int i = tid; i < m; i += SPG_THREADS) sm.q[i] = 1.0 + 0.5 * sin(0.7 * i + 0.1);
  __syncthreads();
  PencilOp<double> op{sm.L, Vfull, false, nullptr};
  LanczosOut lo = lanczos_extreme<double>(op, Q, sm.q, sm.r, sm.z, sm.scr, sm.ymax, sm.ymin, m,
                                          wk.kmax, want_min, wk.tol, sm.sc);
  int iters = lo.iters;
  // A root just behind the point (the boundary it sits next to) dominates
  // M_sigma when |mu_min| >> mu_max; the rounding of M, about eps |mu_min|,
  // then swamps the wanted eigenvector.  Redo the solve at a shift halfway to
  // the estimated root, where both ends weigh alike.
  {
    double th_lo = lo.theta_min;
    if (!want_min) {
      if (wid == 0) {
        const double x = tri_extreme(sm.sc->alpha, sm.sc->beta, lo.iters, false);
        if (lane == 0) sm.bc[1] = x;
      }
      __syncthreads();
      th_lo = sm.bc[1];
      __syncthreads();
    }
    if (lo.theta_max > 0.0 && -th_lo > kRedoRatio * lo.theta_max) {
      const double s2 = sigma + 0.5 / lo.theta_max;
      for (long long e = tid; e < P; e += SPG_THREADS) {
        const uint32_t ik = sp.pidx[e];
        sm.L[e] = fma(s2, Vfull[(size_t)(ik >> 16) * m + (ik & 0xffff)], sp.A[e] + Fg[e]);
      }
      if (tid == 0) sm.ib[0] = 0;
      __syncthreads();
      const bool ok2 = factor64(PW, sm.L, m, sm.col, &sm.ib[0]);
      if (ok2) {
        sigma = s2;
        res.flags |= kSegRefined;
      } else {
        // (the estimate overshot: back to the first factor)
        for (long long e = tid; e < P; e += SPG_THREADS) {
          const uint32_t ik = sp.pidx[e];
          sm.L[e] = fma(sigma, Vfull[(size_t)(ik >> 16) * m + (ik & 0xffff)], sp.A[e] + Fg[e]);
        }
        if (tid == 0) sm.ib[0] = 0;
        __syncthreads();
        factor64(PW, sm.L, m, sm.col, &sm.ib[0]);
      }
      invert_diag_blocks(sm.L, m);
      if (ok2) {
        for (int i = tid; i < m; i += SPG_THREADS) sm.q[i] = 1.0 + 0.5 * sin(0.7 * i + 0.1);
        __syncthreads();
        lo = lanczos_extreme<double>(op, Q, sm.q, sm.r, sm.z, sm.scr, sm.ymax, sm.ymin, m,
                                     wk.kmax, want_min, wk.tol, sm.sc);
        iters += lo.iters;
      }
    }
  }
  res.iters = iters;
  res.status = lo.converged ? kOk : kNoConv;
  if (!lo.converged) res.flags |= kSegNoConv;
  res.t_plus = lo.theta_max > 0.0 ? sigma + 1.0 / lo.theta_max : INFINITY;
  res.t_minus = (want_min && lo.theta_min < 0.0) ? sigma + 1.0 / lo.theta_min : -INFINITY;
  res.t_raw = res.t_plus;
  if (!(lo.theta_max > 0.0)) {
    if (res.status == kOk) res.status = kUnbounded;
    return res;
  }
  // ---- null vector u = L^{-T} y and the forms w_j = u^T A_j u --------------
  for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = sm.ymax[i];
  __syncthreads();
  solve_upper(sm.L, sm.u, m, sm.scr);
  {  // unit length, largest-magnitude entry positive
    double a = 0.0;
    for (int i = tid; i < m; i += SPG_THREADS) a += sm.u[i] * sm.u[i];
    const double nrm = sqrt(block_sum(a, sm.sc->red));
    if (tid == 0) {
      int big = 0;
      for (int i = 1; i < m; ++i)
        if (fabs(sm.u[i]) > fabs(sm.u[big])) big = i;
      sm.bc[0] = (sm.u[big] < 0.0 ? -1.0 : 1.0) / nrm;
    }
    __syncthreads();
    const double sc = sm.bc[0];
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] *= sc;
    __syncthreads();
  }
  // both ends of a converged solve refined by the pencil Rayleigh correction
  // on the exact F = A_0 + Y and V (the A stack, Fg, Vfull).  The quotient
  // never lies below the root (F + t+ V is semidefinite), so a correction is
  // kept only while it stays within kCorrectWindow of the Ritz value, well
  // inside the walk's backoff kappa: a larger one means an inaccurate u.
  if (res.status == kOk) {
    const double tr = pencil_correct_split(sp.A, Fg, Vfull, true, m, P, sp.pidx, sm.u,
                                           res.t_plus, sm.scr);
    if (tr > 0.0 && fabs(tr - res.t_plus) <= kCorrectWindow * res.t_plus) res.t_plus = tr;
  }
  if (res.status == kOk && want_min && isfinite(res.t_minus)) {
    for (int i = tid; i < m; i += SPG_THREADS) sm.z[i] = sm.ymin[i];
    __syncthreads();
    solve_upper(sm.L, sm.z, m, sm.scr);
    const double tr = pencil_correct_split(sp.A, Fg, Vfull, true, m, P, sp.pidx, sm.z,
                                           res.t_minus, sm.scr);
    if (tr < 0.0 && fabs(tr - res.t_minus) <= kCorrectWindow * fabs(res.t_minus))
      res.t_minus = tr;
  }
  __syncthreads();
  if (!want_w) return res;
  // U_e = u_i u_k (x2 off the diagonal) overwrites the factor
  double* U = sm.L;
  for (long long e = tid; e < P; e += SPG_THREADS) {
    const uint32_t ik = sp.pidx[e];
    const int i = ik >> 16, k = ik & 0xffff;
    U[e] = (i == k ? 1.0 : 2.0) * sm.u[i] * sm.u[k];
  }
  __syncthreads();
  for (int j = wid; j <= n; j += SPG_WARPS) {
    const double* Aj = sp.A + (size_t)j * P;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long e = lane;
    for (; e + 96 < P; e += 128) {
      a0 += Aj[e] * U[e];
      a1 += Aj[e + 32] * U[e + 32];
      a2 += Aj[e + 64] * U[e + 64];
      a3 += Aj[e + 96] * U[e + 96];
    }
    for (; e < P; e += 32) a0 += Aj[e] * U[e];
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) sm.w[j] = acc;
  }
  __syncthreads();
  return res;
}

// unit normal w^ = w_{1..n}/|w| into dst; returns |w|
__device__ double unit_normal(const Smem& sm, int n, double* dst) {
  double a = 0.0;
  for (int j = threadIdx.x; j < n; j += SPG_THREADS) a += sm.w[j + 1] * sm.w[j + 1];
  const double nw = sqrt(block_sum(a, sm.sc->red));
  if (nw > 0.0)
    for (int j = threadIdx.x; j < n; j += SPG_THREADS) dst[j] = sm.w[j + 1] / nw;
  __syncthreads();
  return nw;
}

// Every step of the walk `wp` for chain c (CTA-wide): wp.X, wp.status and
// wp.stats are indexed by c, the Philox chain index is wp.chain0 + c; the
// factor, V, F and the Lanczos basis live in sm / Vfull, Fg, Q.
__device__ __noinline__ void walk_chain(const DevSpec& sp, const DevWork& wk,
                                        const WalkParams& wp, Smem& sm, double* Vfull,
                                        double* Fg, double* Q, int c, int PW = kPanel) {
  const int tid = threadIdx.x;
  const int n = sp.n;
  {
    double* xc = wp.X + (size_t)c * n;
    long long* st = wp.stats + (size_t)c * kNumStats;
    long long segs = 0, refl = 0, bad = 0, iters = 0, retries = 0, noconv = 0;
    int last_status = kOk;
    const uint32_t chain = wp.chain0 + (uint32_t)c;
    for (int j = tid; j < n; j += SPG_THREADS) sm.x0[j] = xc[j];
    __syncthreads();
    for (int k = 0; k < wp.steps; ++k) {
      const uint32_t step = wp.step0 + (uint32_t)k;
      for (int j = tid; j < n; j += SPG_THREADS) sm.p[j] = sm.x0[j];
      // ---- direction ----------------------------------------------------
      if (wp.kind == 2) {
        const double uc = rng_uniform(wp.seed, chain, step, kStreamCoord);
        int jc = (int)(uc * n);
        jc = jc < n ? jc : n - 1;
        for (int j = tid; j < n; j += SPG_THREADS) sm.v[j] = (j == jc) ? 1.0 : 0.0;
        __syncthreads();
      } else {
        for (int i = tid; 2 * i < n; i += SPG_THREADS) {
          double g0, g1;
          rng_gauss_pair(wp.seed, chain, step, (uint32_t)i, &g0, &g1);
          sm.v[2 * i] = g0;
          if (2 * i + 1 < n) sm.v[2 * i + 1] = g1;
        }
        __syncthreads();
        double a = 0.0;
        for (int j = tid; j < n; j += SPG_THREADS) a += sm.v[j] * sm.v[j];
        const double nv = sqrt(block_sum(a, sm.sc->red));
        for (int j = tid; j < n; j += SPG_THREADS) sm.v[j] /= nv;
        __syncthreads();
      }
      const double eta = rng_uniform(wp.seed, chain, step, kStreamEta);
      int status = kOk;
      if (wp.kind == 0) {
        // ---- Billiard (Alg. 5) -------------------------------------------
        double ell = -wp.tau * log(eta);
        int nrefl = 0;
        double sigma = 0.0;
        for (;;) {
          // F(p) is formed afresh with V on every segment (the formation loop
          // reads the A stack once for both), as A_0 + Y with Y = sum p_j A_j
          // kept apart: an F carried through a long run of reflections
          // accumulates the rounding of every update, which short chords next
          // to the boundary amplify by |F| / |u^T V u|
          SegResult r = segment_fp64(sp, wk, sm, Vfull, Fg, Q, sigma, false, true, true, -1, PW);
          ++segs;
          iters += r.iters;
          retries += r.retried;
          if (r.status == kNoConv) {
            ++noconv;
            r.status = kOk;  // the Ritz value is still the best estimate
          }
          if (r.status != kOk) {
            const int slot = seglog_slot(wp.seg, &sm.ib[3]);
            if (slot >= 0)
              seglog_write(wp.seg, slot, n, sm.p, sm.v, nullptr, r.t_plus, -INFINITY, r.status, 0,
                           chain, step, nrefl, r.flags);
            status = r.status;
            break;
          }
          if (r.t_plus < ell) {
            // hit the boundary: move to (1 - kappa) t+ and reflect
            const double tp = r.t_plus;
            double* wh = sm.wh;
            const double nw = unit_normal(sm, n, wh);
            {
              const int slot = seglog_slot(wp.seg, &sm.ib[3]);
              if (slot >= 0)
                seglog_write(wp.seg, slot, n, sm.p, sm.v, nw > 0.0 ? wh : nullptr, tp, -INFINITY,
                             nw > 0.0 ? kOk : kDegenerate, 1, chain, step, nrefl, r.flags);
            }
            if (!(nw > 0.0)) {
              status = kDegenerate;
              break;
            }
            double a = 0.0;
            for (int j = tid; j < n; j += SPG_THREADS) a += sm.v[j] * wh[j];
            const double vw = block_sum(a, sm.sc->red);
            const double step_len = (1.0 - wp.kappa) * tp;
            for (int j = tid; j < n; j += SPG_THREADS) {
              sm.p[j] += step_len * sm.v[j];
              sm.v[j] -= 2.0 * vw * wh[j];
            }
            __syncthreads();
            ell -= tp;
            ++nrefl;
            if (nrefl > wp.rho) {
              status = kRho;
              break;
            }
            sigma = wp.sigma_frac * tp;
          } else {
            const int slot = seglog_slot(wp.seg, &sm.ib[3]);
            if (slot >= 0)
              seglog_write(wp.seg, slot, n, sm.p, sm.v, nullptr, r.t_plus, -INFINITY, kOk, 0,
                           chain, step, nrefl, r.flags);
            for (int j = tid; j < n; j += SPG_THREADS) sm.x0[j] = sm.p[j] + ell * sm.v[j];
            __syncthreads();
            break;
          }
        }
        refl += nrefl;
      } else {
        // ---- Hit-and-Run (Alg. 4) / CDHR: uniform point on the chord ------
        // CDHR reads V = A_j from the stack and carries F from step to step,
        // F(p + t e_j) = F(p) + t A_j (Sec. 3.1), re-forming it every
        // kCdhrRefresh steps so that the rounding of the updates stays below
        // ~sqrt(kCdhrRefresh) ulp of F
        const bool cd = wp.kind == 2;
        int jc = -1;
        if (cd)
          for (int j = 0; j < n; ++j)
            if (sm.v[j] != 0.0) jc = j;
        const bool form = !cd || k % kCdhrRefresh == 0;
        SegResult r = segment_fp64(sp, wk, sm, Vfull, Fg, Q, 0.0, true, false, form, jc, PW);
        ++segs;
        iters += r.iters;
        if (r.status == kNoConv) {
          ++noconv;
          r.status = kOk;
        }
        if (r.status == kOk && !(isfinite(r.t_plus) && isfinite(r.t_minus))) r.status = kUnbounded;
        {
          const int slot = seglog_slot(wp.seg, &sm.ib[3]);
          if (slot >= 0)
            seglog_write(wp.seg, slot, n, sm.p, sm.v, nullptr, r.t_plus, r.t_minus, r.status, 0,
                         chain, step, 0, r.flags);
        }
        if (r.status == kOk) {
          const double t = r.t_minus + eta * (r.t_plus - r.t_minus);
          for (int j = tid; j < n; j += SPG_THREADS) sm.x0[j] = sm.p[j] + t * sm.v[j];
          if (cd) {
            const double* Aj = sp.A + (size_t)(jc + 1) * sp.P;
            for (long long e = tid; e < sp.P; e += SPG_THREADS) Fg[e] += t * Aj[e];
          }
          __syncthreads();
        } else {
          status = r.status;
        }
      }
      if (status != kOk) {
        ++bad;
        last_status = status;
      }
      __syncthreads();
    }
    for (int j = tid; j < n; j += SPG_THREADS) xc[j] = sm.x0[j];
    if (tid == 0) {
      st[kStatSegments] += segs;
      st[kStatReflections] += refl;
      st[kStatBadSteps] += bad;
      st[kStatLanczos] += iters;
      st[kStatShiftRetry] += retries;
      st[kStatNoConv] += noconv;
      wp.status[c] = last_status;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SPG_THREADS, 1)
    walk_fp64_kernel(DevSpec sp, DevWork wk, WalkParams wp) {
  extern __shared__ double smem_raw[];
  const int m = sp.m;
  const size_t cta = blockIdx.x;
  double* Vfull = wk.Vfull + cta * (size_t)m * m;
  double* Fg = wk.Fg + cta * (size_t)sp.P;
  double* Q = wk.Q + cta * (size_t)wk.kmax * m;
  double* Lg = wk.l_in_smem ? nullptr : wk.Lg + cta * (size_t)sp.P;
  Smem sm = carve(smem_raw, sp.n, m, wk.l_in_smem, Lg);
  for (int c = blockIdx.x; c < wp.C; c += gridDim.x)
    walk_chain(sp, wk, wp, sm, Vfull, Fg, Q, c);
}

__global__ void __launch_bounds__(SPG_THREADS, 1)
    prim_fp64_kernel(DevSpec sp, DevWork wk, PrimParams pp, int PW) {
  extern __shared__ double smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n, m = sp.m;
  const size_t cta = blockIdx.x;
  double* Vfull = wk.Vfull + cta * (size_t)m * m;
  double* Fg = wk.Fg + cta * (size_t)sp.P;
  double* Q = wk.Q + cta * (size_t)wk.kmax * m;
  double* Lg = wk.l_in_smem ? nullptr : wk.Lg + cta * (size_t)sp.P;
  Smem sm = carve(smem_raw, n, m, wk.l_in_smem, Lg, PW);
  for (int c = blockIdx.x; c < pp.count; c += gridDim.x) {
    double bad = 0.0;
    for (int j = tid; j < n; j += SPG_THREADS) {
      sm.p[j] = pp.x[(size_t)c * n + j];
      sm.v[j] = pp.op == 2 ? 0.0 : pp.v[(size_t)c * n + j];
      if (!isfinite(sm.p[j]) || !isfinite(sm.v[j])) bad = 1.0;
    }
    if (block_sum(bad, sm.sc->red) > 0.0) {
      // a non-finite point or direction: nothing to compute
      if (tid == 0) {
        if (pp.op == 2) {
          pp.inside[c] = 0;
        } else {
          pp.status[c] = kInvalid;
          pp.t_plus[c] = NAN;
          if (pp.op == 0) pp.t_minus[c] = NAN;
        }
      }
      __syncthreads();
      continue;
    }
    if (pp.op == 2) {
      // membership: Cholesky of F(x) succeeds
      const long long P = sp.P;
      for (long long e = tid; e < P; e += SPG_THREADS) {
        const double* Ae = sp.A + e;
        double f = Ae[0];
        for (int j = 0; j < n; ++j) f += sm.p[j] * Ae[(size_t)(j + 1) * P];
        sm.L[e] = f;
      }
      if (tid == 0) sm.ib[0] = 0;
      __syncthreads();
      bool ok = factor64(PW, sm.L, m, sm.col, &sm.ib[0]);
      if (tid == 0) pp.inside[c] = ok ? 1 : 0;
      __syncthreads();
      continue;
    }
    SegResult r = segment_fp64(sp, wk, sm, Vfull, Fg, Q, 0.0, pp.op == 0, true, true, -1, PW);
    int status = r.status;
    if (pp.op == 0) {
      if (tid == 0) {
        pp.t_plus[c] = r.t_plus;
        pp.t_minus[c] = r.t_minus;
        pp.status[c] = status;
      }
      if (pp.u && (status == kOk || status == kNoConv))
        for (int i = tid; i < m; i += SPG_THREADS) pp.u[(size_t)c * m + i] = sm.u[i];
    } else {
      double* wh = sm.wh;
      double nw = 0.0;
      if (status == kOk || status == kNoConv) {
        nw = unit_normal(sm, n, wh);
        if (!(nw > 0.0)) status = kDegenerate;
      }
      if (status == kOk || status == kNoConv) {
        double a = 0.0;
        for (int j = tid; j < n; j += SPG_THREADS) a += sm.v[j] * wh[j];
        const double vw = block_sum(a, sm.sc->red);
        for (int j = tid; j < n; j += SPG_THREADS) {
          pp.w_hat[(size_t)c * n + j] = wh[j];
          pp.s[(size_t)c * n + j] = sm.v[j] - 2.0 * vw * wh[j];
        }
      }
      if (tid == 0) {
        pp.t_plus[c] = r.t_plus;
        pp.status[c] = status;
      }
    }
    __syncthreads();
  }
}

// The walks of a batch of spectrahedra of uneven n and m in one persistent
// launch: every block takes the next (body, chain) item from the queue (items
// in decreasing order of estimated cost, so the longest ones start first and
// the tail is short), carves its shared memory for that body's n and m, and
// runs all the steps of that chain with the body's Cholesky panel width.
__global__ void __launch_bounds__(SPG_THREADS, 1) batch_fp64_kernel(BatchParams bp) {
  extern __shared__ double smem_raw[];
  __shared__ int ticket;
  const size_t cta = blockIdx.x;
  for (;;) {
    if (threadIdx.x == 0) ticket = atomicAdd(bp.next, 1);
    __syncthreads();
    const int it = ticket;
    __syncthreads();
    if (it >= bp.total) break;
    const int2 item = bp.items[it];
    const BatchBody B = bp.bodies[item.x];
    DevWork wk;
    wk.Vfull = bp.Vfull + cta * (size_t)bp.max_mm;
    wk.Fg = bp.Fg + cta * (size_t)bp.max_P;
    wk.Q = bp.Q + cta * (size_t)bp.kmax * bp.max_m;
    wk.Lg = B.l_in_smem ? nullptr : bp.Lg + cta * (size_t)bp.max_P;
    wk.kmax = bp.kmax;
    wk.tol = bp.tol;
    wk.l_in_smem = B.l_in_smem;
    wk.ctas = gridDim.x;
    Smem sm = carve(smem_raw, B.sp.n, B.sp.m, B.l_in_smem, wk.Lg, kMaxPanel);
    WalkParams wp{};
    wp.kind = 0;
    wp.C = B.C;
    wp.steps = bp.steps;
    wp.step0 = bp.step0;
    wp.chain0 = (uint32_t)B.c0;
    wp.seed = bp.seed;
    wp.tau = B.tau;
    wp.kappa = bp.kappa;
    wp.sigma_frac = bp.sigma_frac;
    wp.rho = bp.rho;
    wp.X = bp.X + B.xoff;
    wp.status = bp.status + B.c0;
    wp.stats = bp.stats + (size_t)B.c0 * kNumStats;
    wp.seg = SegLog{nullptr, 0, 1, nullptr};
    __syncthreads();
    walk_chain(B.sp, wk, wp, sm, wk.Vfull, wk.Fg, wk.Q, item.y, B.panel);
    __syncthreads();
  }
}

}  // namespace

size_t batch_smem_bytes(int n, int m, bool l_in_smem) {
  const size_t P = (size_t)m * (m + 1) / 2;
  size_t d = (l_in_smem ? P : 0) + 4 * (size_t)n + (n + 1) + 6 * (size_t)m +
             cholesky_scratch(m, kMaxPanel) + SPG_SCR + 16;
  return d * 8 + align8(sizeof(LanczosScalars)) + 16 * sizeof(int);
}

cudaError_t launch_batch_fp64(const BatchParams& bp, int ctas, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(batch_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ctas <= 0 || bp.total <= 0) return cudaSuccess;
  batch_fp64_kernel<<<ctas, SPG_THREADS, smem, st>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_prim_fp64_panel(const DevSpec& sp, const DevWork& wk, const PrimParams& pp,
                                   int panel, cudaStream_t st) {
  const int pw = panel == 4 ? 4 : (panel == 16 ? 16 : 8);
  // the default kernel's shared memory with the scratch of this panel width
  const size_t smem = fp64_smem_bytes(sp.n, sp.m, wk.l_in_smem) + 8 * cholesky_scratch(sp.m, pw) -
                      8 * cholesky_scratch(sp.m);
  cudaError_t e = cudaFuncSetAttribute(prim_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = pp.count < wk.ctas ? pp.count : wk.ctas;
  if (grid <= 0) return cudaSuccess;
  prim_fp64_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, wk, pp, pw);
  return cudaGetLastError();
}

size_t fp64_smem_bytes(int n, int m, bool l_in_smem) {
  const size_t P = (size_t)m * (m + 1) / 2;
  size_t d = (l_in_smem ? P : 0) + 4 * (size_t)n + (n + 1) + 6 * (size_t)m +
             cholesky_scratch(m) + SPG_SCR + 16;
  size_t b = d * 8 + align8(sizeof(LanczosScalars)) + 16 * sizeof(int);
  return b;
}

cudaError_t launch_walk_fp64(const DevSpec& sp, const DevWork& wk, const WalkParams& wp,
                             cudaStream_t st) {
  const size_t smem = fp64_smem_bytes(sp.n, sp.m, wk.l_in_smem);
  cudaError_t e = cudaFuncSetAttribute(walk_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = wp.C < wk.ctas ? wp.C : wk.ctas;
  if (grid <= 0) return cudaSuccess;
  walk_fp64_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, wk, wp);
  return cudaGetLastError();
}

cudaError_t launch_prim_fp64(const DevSpec& sp, const DevWork& wk, const PrimParams& pp,
                             cudaStream_t st) {
  const size_t smem = fp64_smem_bytes(sp.n, sp.m, wk.l_in_smem);
  cudaError_t e = cudaFuncSetAttribute(prim_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = pp.count < wk.ctas ? pp.count : wk.ctas;
  if (grid <= 0) return cudaSuccess;
  prim_fp64_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, wk, pp, kPanel);
  return cudaGetLastError();
}

}  // namespace spg
