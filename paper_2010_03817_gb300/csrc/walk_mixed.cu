// Mixed-precision path of the boundary oracle.  Per segment (line p + t v):
//   V = sum v_j A_j arrives from the tensor-core formation (FP64 quality);
//   F(p) is carried in FP64 from segment to segment (F <- F + t V).
//   Stage 1 (FP32): Cholesky of F + sigma0 V and Lanczos on
//     M = -L^{-1} V L^{-T} give an estimate t~ of t+ (Alg. 2) and u0.
//   Stage 2 (double-float, FP64 as the fallback): Cholesky of F + sigma1 V
//     with sigma1 just below t~ -- the near-singular factorisation next to
//     the boundary needs more than FP32 -- then a few power iterations on
//     M_sigma1, whose dominant eigenvalue 1/(t+ - sigma1) is separated by
//     orders of magnitude, give t+ and the null vector u.  Success of that
//     factorisation certifies that F + sV > 0 on [0, sigma1], so the root
//     found is the smallest positive one (Lemma "PEP and S cap C").
//   Stage 3: normal w_j = u^T A_j u (Lemma "Gradient of det F") on the
//     tensor cores for a whole wave (ozaki.cu), or in-kernel by a
//     double-float contraction; reflection (Eq. "reflection").
// t- (Hit-and-Run / intersection) comes from stage 1 refined by the pencil
// Rayleigh quotient -(u^T F u)/(u^T V u) with the exact F and V
// (double-float) and stage 2 on the negative side.
#include <math.h>

#include "common.cuh"
#include "dense.cuh"
#include "df.cuh"
#include "kernels.h"
#include "lanczos.cuh"

namespace spg {
namespace {

constexpr int kStage2Panel = 8;  // panel width of the double-float factorisation

struct MixSmem {
  uint8_t* R;     // region: stage 1 (G32, V32), stage 2 (G64), stage 3 (U hi, lo)
  double* p;      // n
  double* v;      // n
  double* w;      // n + 1
  double* wh;     // n
  double* y;      // m
  double* r;      // m
  double* z;      // m
  double* u;      // m
  double* um;     // m (null vector at t-)
  double* part;   // SPG_WARPS * m + 128 (>= cholesky_scratch_la(m, 8) for any m)
  double* scr;    // SPG_SCR
  double* bc;     // 16
  float* q32;     // m
  float* r32;     // m
  float* z32;     // m
  float* y32;     // m
  float* ym32;    // m
  float* pad32;   // m: keeps the number of m-float arrays even (alignment)
  float* duh;     // m: u as an FP32 pair (stage 2)
  float* dul;     // m
  float* dfh;     // m: F u (pair)
  float* dfl;     // m
  float* dgh;     // m: V u (pair)
  float* dgl;     // m
  LanczosScalars* sc;
  int* ib;        // 16
};

__device__ MixSmem mix_carve(uint8_t* base, int n, int m, uint8_t* region_global,
                             size_t region_bytes) {
  MixSmem s;
  uint8_t* q = base;
  if (region_global) {
    s.R = region_global;
  } else {
    s.R = q;
    q += (region_bytes + 15) & ~size_t(15);
  }
  double* d = reinterpret_cast<double*>(q);
  s.p = d; d += n;
  s.v = d; d += n;
  s.w = d; d += n + 1;
  s.wh = d; d += n;
  s.y = d; d += m;
  s.r = d; d += m;
  s.z = d; d += m;
  s.u = d; d += m;
  s.um = d; d += m;
  s.part = d; d += (size_t)SPG_WARPS * m + 128;  // also the two look-ahead panel copies
  s.scr = d; d += SPG_SCR;
  s.bc = d; d += 16;
  float* f = reinterpret_cast<float*>(d);
  s.q32 = f; f += m;
  s.r32 = f; f += m;
  s.z32 = f; f += m;
  s.y32 = f; f += m;
  s.ym32 = f; f += m;
  s.pad32 = f; f += m;
  s.duh = f; f += m;
  s.dul = f; f += m;
  s.dfh = f; f += m;
  s.dfl = f; f += m;
  s.dgh = f; f += m;
  s.dgl = f; f += m;
  // 12 m floats: the next address stays 8-byte aligned
  s.sc = reinterpret_cast<LanczosScalars*>(f);
  if (threadIdx.x == 0) s.sc->prof = nullptr;
  s.ib = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(s.sc) + sizeof(LanczosScalars));
  return s;
}

struct MixResult {
  double t_plus, t_minus;
  int status, iters, retries, fallback, power;
  int learned;  // 1: warm start accepted, -1: rejected, 0: not used
  int refined;  // a shift-invert refinement next to the boundary ran
};

// unit length, largest-magnitude entry positive (CTA-wide, FP64)
__device__ void normalise_vec(double* u, int m, MixSmem& sm) {
  double a = 0.0;
  for (int i = threadIdx.x; i < m; i += SPG_THREADS) a += u[i] * u[i];
  const double nrm = sqrt(block_sum(a, sm.sc->red));
  if (threadIdx.x == 0) {
    int big = 0;
    for (int i = 1; i < m; ++i)
      if (fabs(u[i]) > fabs(u[big])) big = i;
    sm.bc[0] = (u[big] < 0.0 ? -1.0 : 1.0) / nrm;
  }
  __syncthreads();
  const double sc = sm.bc[0];
  for (int i = threadIdx.x; i < m; i += SPG_THREADS) u[i] *= sc;
  __syncthreads();
}

__device__ __forceinline__ void stage_mark(const MixWork& mw, int stage, long long& t0) {
  if (mw.prof && threadIdx.x == 0) {
    const long long t1 = clock64();
    atomicAdd(reinterpret_cast<unsigned long long*>(&mw.prof[blockIdx.x * kProfSlots + stage]),
              (unsigned long long)(t1 - t0));
    t0 = t1;
  }
}

// CTA-wide double-float sum (result on every thread); red: 2 * SPG_WARPS floats
__device__ __forceinline__ void block_sum_df(float& h, float& l, float* red) {
  warp_sum_df(h, l);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[2 * wid] = h;
    red[2 * wid + 1] = l;
  }
  __syncthreads();
  h = 0.f;
  l = 0.f;
#pragma unroll
  for (int w = 0; w < SPG_WARPS; ++w) df_add(h, l, red[2 * w], red[2 * w + 1]);
  df_norm(h, l);
}

constexpr int kDfColBlocks = 8;  // column blocks of 32 per pass of symv_df2

// f = F u and g = V u in double-float: F, V packed FP64 (global), u as an FP32
// pair (uh, ul), results as pairs.  Passes over groups of 8 column blocks of
// 32; in each, warp w takes the rows r = w, w + 8, ... that reach the group,
// its lanes the group's columns k <= r of row r: entry (r, k) adds F_rk u_k to
// the row sum of r and, for k < r, F_rk u_r to the column sum of k (kept per
// lane in registers, then reduced over the warps through scr:
// 4 SPG_WARPS 256 floats).  A row's partial sums are added by the warp that
// owns it, and every entry belongs to the pass of its column, so the passes
// need no further ordering.
__device__ void symv_df2(const double* __restrict__ F, const double* __restrict__ V,
                         const float* uh, const float* ul, int m, float* fh, float* fl, float* gh,
                         float* gl, float* scr) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kW = 32 * kDfColBlocks;
  float* s0 = scr;
  float* s1 = scr + SPG_WARPS * kW;
  float* s2 = scr + 2 * SPG_WARPS * kW;
  float* s3 = scr + 3 * SPG_WARPS * kW;
  for (int k0 = 0; k0 < m; k0 += kW) {
    float cfh[kDfColBlocks], cfl[kDfColBlocks], cgh[kDfColBlocks], cgl[kDfColBlocks];
#pragma unroll
    for (int b = 0; b < kDfColBlocks; ++b) cfh[b] = cfl[b] = cgh[b] = cgl[b] = 0.f;
    for (int r = k0 + ((wid - k0 % SPG_WARPS + SPG_WARPS) % SPG_WARPS); r < m; r += SPG_WARPS) {
      const size_t base = tri(r, 0);
      double fv[kDfColBlocks], vv[kDfColBlocks];
#pragma unroll
      for (int b = 0; b < kDfColBlocks; ++b) {
        const int k = k0 + lane + 32 * b;
        fv[b] = k <= r ? F[base + k] : 0.0;
        vv[b] = k <= r ? V[base + k] : 0.0;
      }
      const float urh = uh[r], url = ul[r];
      float rfh = 0.f, rfl = 0.f, rgh = 0.f, rgl = 0.f;
#pragma unroll
      for (int b = 0; b < kDfColBlocks; ++b) {
        const int k = k0 + lane + 32 * b;
        if (k <= r) {
          const float2 a = split_df(fv[b]);
          const float2 c = split_df(vv[b]);
          const float xh = uh[k], xl = ul[k];
          df_mac(rfh, rfl, a.x, a.y, xh, xl);
          df_mac(rgh, rgl, c.x, c.y, xh, xl);
          if (k < r) {
            df_mac(cfh[b], cfl[b], a.x, a.y, urh, url);
            df_mac(cgh[b], cgl[b], c.x, c.y, urh, url);
          }
        }
      }
      warp_sum_df(rfh, rfl);
      warp_sum_df(rgh, rgl);
      if (lane == 0) {
        if (k0 > 0) {
          df_add(rfh, rfl, fh[r], fl[r]);
          df_add(rgh, rgl, gh[r], gl[r]);
        }
        fh[r] = rfh;
        fl[r] = rfl;
        gh[r] = rgh;
        gl[r] = rgl;
      }
    }
#pragma unroll
    for (int b = 0; b < kDfColBlocks; ++b) {
      const int q = lane + 32 * b;
      s0[wid * kW + q] = cfh[b];
      s1[wid * kW + q] = cfl[b];
      s2[wid * kW + q] = cgh[b];
      s3[wid * kW + q] = cgl[b];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kW && k0 + q < m; q += SPG_THREADS) {
      const int k = k0 + q;
      float h = fh[k], l = fl[k], h2 = gh[k], l2 = gl[k];
#pragma unroll
      for (int w = 0; w < SPG_WARPS; ++w) {
        df_add(h, l, s0[w * kW + q], s1[w * kW + q]);
        df_add(h2, l2, s2[w * kW + q], s3[w * kW + q]);
      }
      df_norm(h, l);
      df_norm(h2, l2);
      fh[k] = h;
      fl[k] = l;
      gh[k] = h2;
      gl[k] = l2;
    }
    __syncthreads();
  }
}

// pencil Rayleigh quotient t = -(u^T F u)/(u^T V u) with the exact F, V
// (packed FP64, global) in double-float; stationary at the null vector, so
// an FP32-accurate u gives t to about FP32 precision squared.  scr: the
// region after the FP32 factor (4 SPG_WARPS 256 floats).
__device__ __noinline__ double pencil_rq(const double* Fg, const double* Vg, const double* u, int m,
                            MixSmem& sm, float* scr) {
  for (int i = threadIdx.x; i < m; i += SPG_THREADS) {
    const float2 s = split_df(u[i]);
    sm.duh[i] = s.x;
    sm.dul[i] = s.y;
  }
  __syncthreads();
  symv_df2(Fg, Vg, sm.duh, sm.dul, m, sm.dfh, sm.dfl, sm.dgh, sm.dgl, scr);
  float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
  for (int i = threadIdx.x; i < m; i += SPG_THREADS) {
    df_mac(ah, al, sm.duh[i], sm.dul[i], sm.dfh[i], sm.dfl[i]);
    df_mac(bh, bl, sm.duh[i], sm.dul[i], sm.dgh[i], sm.dgl[i]);
  }
  float* red = reinterpret_cast<float*>(sm.sc->red);
  block_sum_df(ah, al, red);
  block_sum_df(bh, bl, red);
  return -df_to_double(ah, al) / df_to_double(bh, bl);
}

// the two look-ahead factorisations, not inlined: each gets the full
// register budget instead of sharing it with its caller's live values
__device__ __noinline__ bool factor_df_la(dfloat* G, int m, dfloat* pan, int* flag) {
  return factor_cholesky_la<dfloat, kStage2Panel>(G, m, pan, flag);
}
__device__ __noinline__ bool factor_f32_la(float* G, int m, float* pan, int* flag) {
  return factor_cholesky_la<float>(G, m, pan, flag);
}

// Stage 2 in double-float for one end of the chord (the FP32 pipe; on this
// GPU the FP64 pipe runs at about 1/58 of its rate).  The factorisation next
// to the boundary needs more than FP32: F + sigma1 V is within delta of
// singular, and the LMI's own condition number (10^4 for the Dabbene
// generator's A_0) would make FP32's backward error exceed its smallest
// eigenvalue.  Double-float (about 48 bits) leaves a wide margin:
//   Cholesky of F + sigma1 V, sigma1 = sigma0 + (t_est - sigma0)(1 - delta)
//   (retries with delta x 8), power iteration on M_sigma1 = -L^{-1} V L^{-T}
//   from y = L^T u0 (u0 slightly perturbed), certificate as in the FP64
//   refinement.  u0 (FP64) in sm.u, left untouched unless the result is
//   kOk: then t and the unit null vector (sm.u).
__device__ __noinline__ int refine_end_dd(const DevSpec& sp, const MixWork& mw, MixSmem& sm,
                             const double* __restrict__ Fg, const double* __restrict__ Vg,
                             double sigma0, double t_est, double* t, MixResult* res, bool plus,
                             double delta0, int attempts, int iters) {
  using T = dfloat;
  const int tid = threadIdx.x;
  const int m = sp.m;
  const long long P = sp.P;
  T* G = reinterpret_cast<T*>(sm.R);
  T* y = reinterpret_cast<T*>(sm.y);
  T* r = reinterpret_cast<T*>(sm.r);
  T* z = reinterpret_cast<T*>(sm.z);
  T* part = reinterpret_cast<T*>(sm.part);
  T* scr = reinterpret_cast<T*>(sm.scr);
  T* red = reinterpret_cast<T*>(sm.sc->red);
  // V as pairs, split once for all power iterations (global, per block)
  T* Vd = reinterpret_cast<T*>(mw.vdf) + (size_t)blockIdx.x * P;
  long long tmark = clock64();
  double sigma1 = sigma0;
  bool ok = false;
  double delta = delta0;
  for (int attempt = 0; attempt < attempts && !ok; ++attempt) {
    sigma1 = sigma0 + (t_est - sigma0) * (1.0 - delta);
    const T s1(sigma1);
    for (long long e = tid; e < P; e += SPG_THREADS) {
      const T ve(Vg[e]);
      Vd[e] = ve;
      G[e] = T(Fg[e]) + s1 * ve;
    }
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    // the factorisation that dominates the segment: look-ahead of one panel
    ok = factor_df_la(G, m, part, &sm.ib[0]);
    if (!ok) {
      ++res->retries;
      delta *= 8.0;
    }
  }
  stage_mark(mw, 2, tmark);  // double-float fill + Cholesky
  if (!ok) return kNotPD;
  // start vector u0 + a small deterministic perturbation (every eigenvector
  // gets a component: a start on the wrong root cannot pass the residual
  // test by an absent component), then y = L^T u
  {
    double a = 0.0;
    for (int i = tid; i < m; i += SPG_THREADS) a += sm.u[i] * sm.u[i];
    const double nu = sqrt(block_sum(a, sm.sc->red));
    const double pert = 1e-6 * nu / sqrt((double)m);
    for (int i = tid; i < m; i += SPG_THREADS) z[i] = T(sm.u[i] + pert * sin(1.3 * i + 0.7));
    __syncthreads();
  }
  mul_upper<T>(G, z, y, m, part);
  invert_diag_blocks<T>(G, m);
  bool converged = false;
  double mu = 0.0;
  for (int it = 0; it < iters; ++it) {
    T a(0);
    for (int i = tid; i < m; i += SPG_THREADS) a += y[i] * y[i];
    const T rn = rsqrt_t(block_sum(a, red));
    for (int i = tid; i < m; i += SPG_THREADS) {
      y[i] *= rn;
      z[i] = y[i];
    }
    __syncthreads();
    long long ts = clock64();
    // r = M y = -L^{-1} V L^{-T} y
    solve_upper<T>(G, z, m, scr);
    stage_mark(mw, 12, ts);
    symv_packed<T>(Vd, z, r, m, T(-1), part);
    stage_mark(mw, 13, ts);
    solve_lower<T>(G, r, m, scr);
    stage_mark(mw, 14, ts);
    T b(0);
    for (int i = tid; i < m; i += SPG_THREADS) b += y[i] * r[i];
    const T mut = block_sum(b, red);
    T c(0);
    for (int i = tid; i < m; i += SPG_THREADS) {
      const T d = r[i] - mut * y[i];
      c += d * d;
    }
    const double res2 = to_double(block_sum(c, red));
    mu = to_double(mut);
    for (int i = tid; i < m; i += SPG_THREADS) y[i] = r[i];
    __syncthreads();
    stage_mark(mw, 15, ts);  // reductions and vector updates
    ++res->power;
    if (res2 <= mw.tol64 * mw.tol64 * mu * mu) {
      converged = true;
      break;
    }
  }
  // certificate: the dominant eigenvalue belongs to this end and its root
  // lies closer to sigma1 than 0 does (no root of the other side dominates)
  if (plus ? !(mu > 0.0 && 1.0 / mu < sigma1) : !(mu < 0.0 && -1.0 / mu < -sigma1))
    converged = false;
  if (converged) {
    *t = sigma1 + 1.0 / mu;
    // u = L^{-T} y
    for (int i = tid; i < m; i += SPG_THREADS) z[i] = y[i];
    __syncthreads();
    solve_upper<T>(G, z, m, scr);
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = to_double(z[i]);
    __syncthreads();
    normalise_vec(sm.u, m, sm);
  }
  stage_mark(mw, 3, tmark);  // double-float power iterations
  return converged ? kOk : kNoConv;
}

// Stage 2 for one end of the chord: FP64 Cholesky of F + sigma1 V with
// sigma1 = sigma0 + (t_est - sigma0)(1 - delta) just inside that end, power
// iteration on M_sigma1 from u0 (in sm.u), FP64 Lanczos fallback.  On return
// sm.u holds the unit null vector and *t the root.  plus: t+ end (else t-).
// cold: no usable estimate (factor at sigma0 and go straight to Lanczos).
__device__ __noinline__ int refine_end_fp64(const DevSpec& sp, const MixWork& mw, MixSmem& sm,
                               const double* __restrict__ Fg, const double* __restrict__ Vg,
                               double* __restrict__ Q64, double sigma0, double t_est, bool cold,
                               double* t, MixResult* res, bool plus = true) {
  const int tid = threadIdx.x;
  const int m = sp.m;
  const long long P = sp.P;
  double* G64 = reinterpret_cast<double*>(sm.R);
  long long tmark = clock64();
  double sigma1 = sigma0;
  bool ok = false;
  if (!cold) {
    double delta = mw.delta1;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
      sigma1 = sigma0 + (t_est - sigma0) * (1.0 - delta);
      for (long long e = tid; e < P; e += SPG_THREADS) G64[e] = Fg[e] + sigma1 * Vg[e];
      if (tid == 0) sm.ib[0] = 0;
      __syncthreads();
      ok = factor_cholesky<double>(G64, m, sm.part, &sm.ib[0]);
      if (!ok) {
        ++res->retries;
        delta *= 8.0;
      }
    }
  }
  const bool power = ok;
  // fall back to a factorisation at sigma0, then at the point itself (sigma =
  // 0: interior by construction); only if that fails is the point outside S
  for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
    sigma1 = attempt == 0 ? sigma0 : 0.0;
    if (attempt == 1 && sigma0 == 0.0) break;
    for (long long e = tid; e < P; e += SPG_THREADS) G64[e] = Fg[e] + sigma1 * Vg[e];
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    ok = factor_cholesky<double>(G64, m, sm.part, &sm.ib[0]);
  }
  if (!ok) {
    *t = 0.0;
    return kNotPD;
  }
  stage_mark(mw, 2, tmark);  // FP64 fill + Cholesky
  double mu = 0.0;
  bool converged = false;
  if (power) {
    // y = L^T u0, then power iteration on M_sigma1: its dominant eigenvalue is
    // 1/(t - sigma1) for the root t at this end.  A small deterministic
    // perturbation of u0 gives every eigenvector a component, so that an
    // estimate of the wrong root (two nearly equal roots) cannot pass the
    // residual test by an absent component: it converges to the right root
    // or fails over to the Lanczos solve.
    {
      double a = 0.0;
      for (int i = tid; i < m; i += SPG_THREADS) a += sm.u[i] * sm.u[i];
      const double nu = sqrt(block_sum(a, sm.sc->red));
      for (int i = tid; i < m; i += SPG_THREADS)
        sm.u[i] += 1e-4 * nu * sin(1.3 * i + 0.7) / sqrt((double)m);
      __syncthreads();
    }
    mul_upper<double>(G64, sm.u, sm.y, m, sm.part);
    invert_diag_blocks<double>(G64, m);
    PencilOp<double> op{G64, Vg, true, sm.part};
    for (int it = 0; it < mw.power_iters; ++it) {
      double a = 0.0;
      for (int i = tid; i < m; i += SPG_THREADS) a += sm.y[i] * sm.y[i];
      const double ny = sqrt(block_sum(a, sm.sc->red));
      for (int i = tid; i < m; i += SPG_THREADS) sm.y[i] /= ny;
      __syncthreads();
      apply_pencil<double>(op, sm.y, sm.r, sm.z, m, sm.scr);
      double b = 0.0;
      for (int i = tid; i < m; i += SPG_THREADS) b += sm.y[i] * sm.r[i];
      mu = block_sum(b, sm.sc->red);
      double c = 0.0;
      for (int i = tid; i < m; i += SPG_THREADS) {
        const double d = sm.r[i] - mu * sm.y[i];
        c += d * d;
      }
      const double resid = sqrt(block_sum(c, sm.sc->red));
      for (int i = tid; i < m; i += SPG_THREADS) sm.y[i] = sm.r[i];
      __syncthreads();
      ++res->power;
      if (resid <= mw.tol64 * fabs(mu)) {
        converged = true;
        break;
      }
    }
    // certificate: the dominant eigenvalue belongs to this end and its root
    // lies closer to sigma1 than 0 does (then no root of the other side can
    // dominate); sign: mu > 0 for t+, mu < 0 for t-
    if (plus ? !(mu > 0.0 && 1.0 / mu < sigma1) : !(mu < 0.0 && -1.0 / mu < -sigma1))
      converged = false;
  } else {
    invert_diag_blocks<double>(G64, m);
  }
  stage_mark(mw, 3, tmark);  // FP64 power iterations (fallback)
  if (!converged) {
    res->fallback = 1;
    // robust fallback: FP64 Lanczos for the extreme eigenvalue of this end
    PencilOp<double> op{G64, Vg, true, sm.part};
    for (int i = tid; i < m; i += SPG_THREADS) sm.z[i] = 1.0 + 0.5 * sin(0.7 * i + 0.1);
    __syncthreads();
    // (cold start on the t+ side: also the t- end, for the Hit-and-Run chord)
    const bool both = !plus || cold;
    LanczosOut lo = lanczos_extreme<double>(op, Q64, sm.z, sm.r, sm.u, sm.scr, sm.y,
                                            plus ? sm.um : sm.y, m, mw.kmax64, both, mw.tol64,
                                            sm.sc);
    res->iters += lo.iters;
    mu = plus ? lo.theta_max : lo.theta_min;
    if (plus && cold) {
      res->t_minus = lo.theta_min < 0.0 ? sigma1 + 1.0 / lo.theta_min : -INFINITY;
      if (lo.theta_min < 0.0) {
        solve_upper<double>(G64, sm.um, m, sm.scr);
        normalise_vec(sm.um, m, sm);
      }
    }
    converged = lo.converged;
    if (plus ? !(mu > 0.0) : !(mu < 0.0)) {
      *t = plus ? INFINITY : -INFINITY;
      stage_mark(mw, 4, tmark);
      return kUnbounded;
    }
  }
  stage_mark(mw, 4, tmark);  // FP64 Lanczos fallback
  *t = sigma1 + 1.0 / mu;
  // u = L^{-T} y
  for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = sm.y[i];
  __syncthreads();
  solve_upper<double>(G64, sm.u, m, sm.scr);
  normalise_vec(sm.u, m, sm);
  return converged ? kOk : kNoConv;
}

// Stage 2 for one end: the double-float refinement, the FP64 one when it
// does not converge (or without an estimate: cold).  u0 in sm.u.
__device__ __noinline__ int refine_end(const DevSpec& sp, const MixWork& mw, MixSmem& sm,
                          const double* __restrict__ Fg, const double* __restrict__ Vg,
                          double* __restrict__ Q64, double sigma0, double t_est, bool cold,
                          double* t, MixResult* res, bool plus) {
  int st;
  if (!cold &&
      refine_end_dd(sp, mw, sm, Fg, Vg, sigma0, t_est, t, res, plus, mw.delta1, 3,
                    mw.power_iters) == kOk) {
    st = kOk;
  } else {
    res->fallback = 1;
    st = refine_end_fp64(sp, mw, sm, Fg, Vg, Q64, sigma0, t_est, cold, t, res, plus);
    if (cold && (st == kOk || st == kNoConv) && isfinite(*t)) {
      // a cold start factors at sigma0 or at the point itself, where a root
      // just behind it can dominate the Lanczos operator and blur u: refine
      // once more by shift-invert next to the root just found
      double t2 = *t;
      const int st2 =
          refine_end_fp64(sp, mw, sm, Fg, Vg, Q64, sigma0, *t, false, &t2, res, plus);
      if (st2 == kOk) {
        *t = t2;
        st = kOk;
        res->refined = 1;
      }
    }
  }
  if (st == kOk) {
    // the pencil Rayleigh correction on the exact F and V, summed without
    // rounding error: removes the factorisation's backward error (about
    // m eps |F|) from t.  The quotient never lies below the root (F + t+ V is
    // semidefinite), so a correction is kept only within 1e-7 of t, well
    // inside the walk's backoff kappa.
    const double tr = pencil_correct_dot2(Fg, Vg, sp.m, sp.P, sp.pidx, sm.u, *t, sm.scr);
    if ((plus ? tr > 0.0 : tr < 0.0) && fabs(tr - *t) <= 1e-7 * fabs(*t)) *t = tr;
  }
  return st;
}

// One boundary-oracle evaluation in mixed precision (CTA-wide).
//   Fg, Vg: packed FP64 F(p) and V (global).  sigma0: stage-1 shift.
//   pred (learned warm start): the network's (log(t+/t_scale), u) for this
//   line; the shift sigma1 = (1 - margin) t^ replaces stage 1.
__device__ __noinline__ MixResult segment_mixed(const DevSpec& sp, const MixWork& mw, MixSmem& sm,
                                   const double* __restrict__ Fg, const double* __restrict__ Vg,
                                   float* __restrict__ Q32, double* __restrict__ Q64,
                                   double sigma0, bool want_min, bool stage2,
                                   const float* __restrict__ pred = nullptr,
                                   double t_scale = 0.0, double margin = 0.0) {
  const int tid = threadIdx.x;
  const int m = sp.m;
  const long long P = sp.P;
  MixResult res;
  res.retries = 0;
  res.iters = 0;
  res.fallback = 0;
  res.power = 0;
  res.learned = 0;
  res.refined = 0;
  res.t_minus = -INFINITY;
  float* G32 = reinterpret_cast<float*>(sm.R);
  float* V32 = G32 + P;
  long long tmark = clock64();
  // F and V are read by both fills and by every product with V of stage 2:
  // bring them into the L2 once, all lines at a time
  prefetch_l2(Fg, sizeof(double) * (size_t)P);
  prefetch_l2(Vg, sizeof(double) * (size_t)P);

  // ---------------- stage 1 with the learned warm start ---------------------
  // The network predicts t+ and the null vector u.  Stage 1 factors at
  // sigma0 = (1 - margin) t^ instead (a failed factorisation, t^ too large,
  // falls back to the plain stage 1) and starts the Lanczos from L^T u^: next
  // to the boundary the wanted eigenvalue 1/(t+ - sigma0) of M_sigma0
  // stands apart from the rest, so fewer iterations reach the tolerance
  // (checked every second step).  Stage 2 certifies and refines as usual.
  double t1 = 0.0, t1m = -INFINITY;
  bool have_t1 = false;
  if (pred && !want_min) {
    const double that = t_scale * exp((double)pred[0]);
    const double sig = that * (1.0 - margin);
    bool okl = false;
    if (isfinite(sig) && sig > 0.0) {
      const float sf = (float)sig;
      for (long long e = tid; e < P; e += SPG_THREADS) {
        const float vh = trunc_f32(Vg[e]);
        G32[e] = fmaf(sf, vh, trunc_f32(Fg[e]));
        V32[e] = vh;
      }
      if (tid == 0) sm.ib[0] = 0;
      __syncthreads();
      okl = factor_f32_la(G32, m, reinterpret_cast<float*>(sm.part), &sm.ib[0]);
      if (!okl) ++res.retries;
    }
    stage_mark(mw, 0, tmark);
    if (okl) {
      for (int i = tid; i < m; i += SPG_THREADS) sm.z32[i] = pred[1 + i];
      __syncthreads();
      mul_upper<float>(G32, sm.z32, sm.q32, m, reinterpret_cast<float*>(sm.part));
      invert_diag_blocks<float>(G32, m);
      PencilOp<float> op{G32, V32, true, reinterpret_cast<float*>(sm.part)};
      LanczosOut lo = lanczos_extreme<float>(op, Q32, sm.q32, sm.r32, sm.z32,
                                             reinterpret_cast<float*>(sm.scr), sm.y32, sm.ym32,
                                             m, mw.kmax32, false, mw.tol32, sm.sc, 4, 2);
      res.iters += lo.iters;
      if (lo.converged && lo.theta_max > 0.0) {
        sigma0 = sig;
        t1 = sig + 1.0 / lo.theta_max;
        have_t1 = true;
        solve_upper<float>(G32, sm.y32, m, reinterpret_cast<float*>(sm.scr));
        for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = (double)sm.y32[i];
        __syncthreads();
      }
    }
    res.learned = have_t1 ? 1 : -1;
    stage_mark(mw, 1, tmark);
  }

  // ---------------- stage 1: FP32 estimate ---------------------------------
  bool ok = have_t1;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
    const float s0f = (float)sigma0;
    for (long long e = tid; e < P; e += SPG_THREADS) {
      const float vh = trunc_f32(Vg[e]);
      G32[e] = fmaf(s0f, vh, trunc_f32(Fg[e]));
      V32[e] = vh;
    }
    if (tid == 0) sm.ib[0] = 0;
    __syncthreads();
    ok = factor_f32_la(G32, m, reinterpret_cast<float*>(sm.part), &sm.ib[0]);
    if (!ok) {
      ++res.retries;
      sigma0 *= 0.2;  // back off toward the point itself
    }
  }
  stage_mark(mw, 0, tmark);  // stage 1 fill + FP32 Cholesky
  const int fp64_fallback = !ok;
  if (ok && !have_t1) {
    invert_diag_blocks<float>(G32, m);
    for (int i = tid; i < m; i += SPG_THREADS) sm.q32[i] = 1.0f + 0.5f * __sinf(0.7f * i + 0.1f);
    __syncthreads();
    PencilOp<float> op{G32, V32, true, reinterpret_cast<float*>(sm.part)};
    LanczosOut lo = lanczos_extreme<float>(op, Q32, sm.q32, sm.r32, sm.z32,
                                           reinterpret_cast<float*>(sm.scr), sm.y32, sm.ym32, m,
                                           mw.kmax32, want_min, mw.tol32, sm.sc);
    res.iters += lo.iters;
    if (!(lo.theta_max > 0.0)) {
      res.status = kUnbounded;
      res.t_plus = INFINITY;
      return res;
    }
    t1 = sigma0 + 1.0 / lo.theta_max;
    // u0 = L^{-T} y (FP32), kept as the start vector of stage 2
    solve_upper<float>(G32, sm.y32, m, reinterpret_cast<float*>(sm.scr));
    if (want_min) {
      if (lo.theta_min < 0.0) {
        t1m = sigma0 + 1.0 / lo.theta_min;
        solve_upper<float>(G32, sm.ym32, m, reinterpret_cast<float*>(sm.scr));
        for (int i = tid; i < m; i += SPG_THREADS) sm.um[i] = (double)sm.ym32[i];
        __syncthreads();
      }
    }
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = (double)sm.y32[i];
    __syncthreads();
  }
  stage_mark(mw, 1, tmark);  // FP32 Lanczos
  if (want_min && isfinite(t1m)) {
    // t- from the FP64 pencil Rayleigh quotient (stationary at the eigenvector)
    res.t_minus = pencil_rq(Fg, Vg, sm.um, m, sm, V32);
    normalise_vec(sm.um, m, sm);
  }

  if (!stage2 && !fp64_fallback) {
    // t+ from the FP64 pencil Rayleigh quotient of the stage-1 vector
    res.t_plus = pencil_rq(Fg, Vg, sm.u, m, sm, V32);
    normalise_vec(sm.u, m, sm);
    res.status = kOk;
    return res;
  }
  // ---------------- stage 2: refinement at each end ------------------------
  if (fp64_fallback) t1 = 0.0;
  if (want_min && isfinite(t1m) && !fp64_fallback) {
    // t- end first (its u0 is in um); the t+ start vector waits in y32
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = sm.um[i];
    __syncthreads();
    double tm;
    const int st = refine_end(sp, mw, sm, Fg, Vg, Q64, sigma0, t1m, false, &tm, &res, false);
    if (st == kOk) {
      res.t_minus = tm;
      for (int i = tid; i < m; i += SPG_THREADS) sm.um[i] = sm.u[i];
      __syncthreads();
    }
    for (int i = tid; i < m; i += SPG_THREADS) sm.u[i] = (double)sm.y32[i];
    __syncthreads();
  }
  if (!fp64_fallback) {
    // the stage-1 estimate sharpened before stage 2 places its shift: the
    // pencil Rayleigh quotient of the stage-1 vector on the exact F and V is,
    // like the Ritz estimate, never below t+ (F + t+ V is semidefinite), but
    // its error is quadratic in the vector's instead of linear: on short
    // chords at grazing incidence, where FP32's backward error makes the
    // Ritz estimate overshoot by 10^-3 - 10^-2 relative and the double-float
    // factorisation at sigma1 fail, the quotient is within about 10^-4
    const double rq = pencil_rq(Fg, Vg, sm.u, m, sm, V32);
    if (isfinite(rq) && rq > sigma0 && rq < t1) t1 = rq;
  }
  double tp;
  res.status = refine_end(sp, mw, sm, Fg, Vg, Q64, sigma0, t1, fp64_fallback, &tp, &res, true);
  res.t_plus = tp;
  return res;
}

// w_j = u^T A_j u, j = 0..n (Lemma "Gradient of det F"), by a double-float
// contraction over the packed entries: A_j = hi + lo (FP32 pair,
// precomputed), U = u_i u_k (x2 off the diagonal) as an FP32 pair, formed
// once in the work region; each product is split exactly with an FMA and the
// high parts are summed with TwoSum, the rounding errors of both kept in a
// separate accumulator (Ogita, Rump, Oishi: Sum2 / Dot2).  Error ~ n eps^2 of
// sum |terms| (eps = 2^-24).  Warp w takes the matrices j = w, w + 8, ...
__device__ __noinline__ void contract_forms(const DevSpec& sp, const float2* __restrict__ Ahl, MixSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = sp.n, m = sp.m;
  const long long P = sp.P;
  float* Uh = reinterpret_cast<float*>(sm.R);
  float* Ul = Uh + P;
  float* uh = sm.duh;
  float* ul = sm.dul;
  for (int i = tid; i < m; i += SPG_THREADS) {
    const float2 s = split_df(sm.u[i]);
    uh[i] = s.x;
    ul[i] = s.y;
  }
  __syncthreads();
  for (long long e = tid; e < P; e += SPG_THREADS) {
    const uint32_t ik = sp.pidx[e];
    const int i = ik >> 16, k = ik & 0xffff;
    const float a = uh[i], b = uh[k];
    const float p = a * b;
    float q = fmaf(a, b, -p);
    q = fmaf(a, ul[k], fmaf(ul[i], b, q));
    const float s = p + q;  // |q| << |p|: fast two-sum
    const float t = q - (s - p);
    const float f = (i == k) ? 1.0f : 2.0f;
    Uh[e] = f * s;
    Ul[e] = f * t;
  }
  __syncthreads();
  for (int j = wid; j <= n; j += SPG_WARPS) {
    const float2* Aj = Ahl + (size_t)j * P;
    float acc = 0.f, lo = 0.f;
    for (long long e = lane; e < P; e += 32) {
      const float2 a = Aj[e];
      df_mac(acc, lo, a.x, a.y, Uh[e], Ul[e]);
    }
    warp_sum_df(acc, lo);
    if (lane == 0) sm.w[j] = (double)acc + (double)lo;
  }
  __syncthreads();
}

__device__ double mix_unit_normal(MixSmem& sm, int n) {
  double a = 0.0;
  for (int j = threadIdx.x; j < n; j += SPG_THREADS) a += sm.w[j + 1] * sm.w[j + 1];
  const double nw = sqrt(block_sum(a, sm.sc->red));
  if (nw > 0.0)
    for (int j = threadIdx.x; j < n; j += SPG_THREADS) sm.wh[j] = sm.w[j + 1] / nw;
  __syncthreads();
  return nw;
}

__device__ void draw_direction(uint64_t seed, uint32_t chain, uint32_t step, double* v, int n,
                               MixSmem& sm) {
  for (int i = threadIdx.x; 2 * i < n; i += SPG_THREADS) {
    double g0, g1;
    rng_gauss_pair(seed, chain, step, (uint32_t)i, &g0, &g1);
    v[2 * i] = g0;
    if (2 * i + 1 < n) v[2 * i + 1] = g1;
  }
  __syncthreads();
  double a = 0.0;
  for (int j = threadIdx.x; j < n; j += SPG_THREADS) a += v[j] * v[j];
  const double nv = sqrt(block_sum(a, sm.sc->red));
  for (int j = threadIdx.x; j < n; j += SPG_THREADS) v[j] /= nv;
  __syncthreads();
}

// Completes the segment of chain c (slot r of this wave) from the oracle's
// result: the Billiard move or reflection (Alg. 5, Eq. "reflection"; sm.w
// holds w_j = u^T A_j u, j = 0..n, when t+ < ell), the Hit-and-Run move
// (Alg. 4), a rejected step (back to its start, F re-formed), the carried F,
// the end of a step (next direction and length) and the queue of the next
// wave.  sm.p, sm.v: the chain's point and direction.
__device__ __noinline__ void complete_segment(const DevSpec& sp, const MixWork& mw, const MixWave& wv,
                                 MixSmem& sm, int r, int c, int status, double t_plus,
                                 double t_minus, double ell, int nrefl, double* __restrict__ Fc,
                                 const double* __restrict__ Vr, long long* st, int flags) {
  const int tid = threadIdx.x;
  const int n = sp.n;
  const long long P = sp.P;
  const uint32_t chain = wv.chain0 + (uint32_t)c;
  (void)r;
  bool step_done = false, rejected = false;
  double move = 0.0;
  // the unit normal of a reflection, then the sampled segment record (the
  // line as the oracle met it, before the move)
  if (wv.kind != 0 && status == kOk && !(isfinite(t_plus) && isfinite(t_minus)))
    status = kUnbounded;
  const bool hit = wv.kind == 0 && status == kOk && t_plus < ell;
  if (hit && !(mix_unit_normal(sm, n) > 0.0)) status = kDegenerate;
  {
    const int slot = seglog_slot(wv.seg, &sm.ib[3]);
    if (slot >= 0)
      seglog_write(wv.seg, slot, n, sm.p, sm.v, (hit && status == kOk) ? sm.wh : nullptr, t_plus,
                   wv.kind == 0 ? -INFINITY : t_minus, status, hit ? 1 : 0, chain,
                   wv.step0 + (uint32_t)wv.done[c], wv.kind == 0 ? nrefl : 0, flags);
  }
  if (wv.kind == 0) {
    if (hit) {
      if (status != kOk) {
        // degenerate normal: the step is rejected below
      } else {
        double a = 0.0;
        for (int j = tid; j < n; j += SPG_THREADS) a += sm.v[j] * sm.wh[j];
        const double vw = block_sum(a, sm.sc->red);
        move = (1.0 - wv.kappa) * t_plus;
        for (int j = tid; j < n; j += SPG_THREADS) {
          sm.p[j] += move * sm.v[j];
          sm.v[j] -= 2.0 * vw * sm.wh[j];
        }
        ell -= t_plus;
        ++nrefl;
        if (tid == 0) st[kStatReflections] += 1;
        if (nrefl > wv.rho) {
          status = kRho;
        }
      }
    } else if (status == kOk) {
      move = ell;
      for (int j = tid; j < n; j += SPG_THREADS) sm.p[j] += ell * sm.v[j];
      step_done = true;
    }
  } else {
    if (status == kOk && !(isfinite(t_plus) && isfinite(t_minus))) status = kUnbounded;
    if (status == kOk) {
      const double eta = rng_uniform(wv.seed, chain, wv.step0 + wv.done[c], kStreamEta);
      move = t_minus + eta * (t_plus - t_minus);
      for (int j = tid; j < n; j += SPG_THREADS) sm.p[j] += move * sm.v[j];
      step_done = true;
    }
  }
  __syncthreads();
  long long tu0 = clock64();
  int fage = wv.fage[c];
  if (status != kOk) {
    // the step is rejected: back to its start point; F(x) is formed afresh
    // (listed for the next wave's formation, below)
    rejected = true;
    step_done = true;
    for (int j = tid; j < n; j += SPG_THREADS) sm.p[j] = wv.Xstart[(size_t)c * n + j];
    fage = 1 << 20;
    if (tid == 0) {
      st[kStatBadSteps] += 1;
      wv.status[c] = status;
    }
  } else if (move != 0.0) {
    // carried F: F(p + move v) = F(p) + move V
    for (long long e = tid; e < P; e += SPG_THREADS) Fc[e] += move * Vr[e];
    ++fage;
  }
  __syncthreads();
  int done = wv.done[c];
  if (step_done) {
    ++done;
    nrefl = 0;
    ell = 0.0;
    for (int j = tid; j < n; j += SPG_THREADS) wv.Xstart[(size_t)c * n + j] = sm.p[j];
    if (done < wv.steps) {
      const uint32_t stp = wv.step0 + (uint32_t)done;
      if (wv.kind == 2) {
        const double uc = rng_uniform(wv.seed, chain, stp, kStreamCoord);
        int jc = (int)(uc * n);
        jc = jc < n ? jc : n - 1;
        for (int j = tid; j < n; j += SPG_THREADS) sm.v[j] = (j == jc) ? 1.0 : 0.0;
        __syncthreads();
      } else {
        draw_direction(wv.seed, chain, stp, sm.v, n, sm);
      }
      if (wv.kind == 0) ell = -wv.tau * log(rng_uniform(wv.seed, chain, stp, kStreamEta));
    }
  }
  for (int j = tid; j < n; j += SPG_THREADS) wv.X[(size_t)c * n + j] = sm.p[j];
  if (done < wv.steps) {
    // still active: queue the chain (and its direction) for the next wave,
    // and for a fresh formation of F when its carried F is old: every update
    // adds a rounding, which short chords next to the boundary amplify by
    // |F| / |u^T V u|
    if (tid == 0) {
      sm.ib[1] = atomicAdd(wv.count_next, 1);
      if (fage >= (wv.kind == 2 ? kFRefreshCdhr : kFRefresh)) {
        wv.ref_ids[atomicAdd(wv.ref_count, 1)] = c;
        fage = 0;
      }
    }
    __syncthreads();
    const int slot = sm.ib[1];
    for (int j = tid; j < n; j += SPG_THREADS) wv.dir_next[(size_t)slot * n + j] = sm.v[j];
    if (tid == 0) wv.id_next[slot] = c;
  }
  if (tid == 0) wv.fage[c] = fage;
  stage_mark(mw, 6, tu0);  // F update, next direction, queueing
  if (tid == 0) {
    wv.done[c] = done;
    wv.ell[c] = ell;
    wv.nrefl[c] = nrefl;
    wv.tprev[c] = (rejected || step_done) ? 0.0 : t_plus;
  }
}

// ---------------------------------------------------------------------------
// walk: one segment per active chain per launch (wave)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SPG_THREADS, 1)
    mixed_wave_kernel(DevSpec sp, MixWork mw, MixWave wv) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n, m = sp.m;
  const long long P = sp.P;
  const size_t cta = blockIdx.x;
  uint8_t* rg = mw.region_global ? mw.region_global + cta * mw.region_bytes : nullptr;
  MixSmem sm = mix_carve(smem_raw, n, m, rg, mw.region_bytes);
  if (tid == 0 && mw.prof) sm.sc->prof = mw.prof + blockIdx.x * kProfSlots + 8;
  float* Q32 = mw.Q32 + cta * (size_t)mw.kmax32 * m;
  double* Q64 = mw.Q64 + cta * (size_t)mw.kmax64 * m;
  const int count = *wv.count_cur;
  for (;;) {
    // the next line from the wave's counter: a CTA that drew expensive lines
    // (long eigen-solves, FP64 fallbacks) takes fewer, so the wave ends
    // within about one segment of its mean load
    if (tid == 0) sm.ib[5] = atomicAdd(wv.ticket, 1);
    __syncthreads();
    const int r = sm.ib[5];
    __syncthreads();
    if (r >= count) break;
    const int c = wv.id_cur[r];
    double* Fc = wv.F + (size_t)c * P;
    for (int j = tid; j < n; j += SPG_THREADS) {
      sm.p[j] = wv.X[(size_t)c * n + j];
      sm.v[j] = wv.dir_cur[(size_t)r * n + j];
      if (wv.kind == 2 && sm.v[j] != 0.0) sm.ib[4] = j;
    }
    __syncthreads();
    // CDHR (Sec. 3.1): V = A_j, a slice of the stack (no formation); the
    // carried F moves by t A_j
    const double* Vr = wv.kind == 2 ? sp.A + (size_t)(sm.ib[4] + 1) * P : wv.Vrows + (size_t)r * P;
    double ell = wv.ell[c];
    int nrefl = wv.nrefl[c];
    const double tprev = wv.tprev[c];
    long long* st = wv.stats + (size_t)c * kNumStats;
    __syncthreads();
    const double sigma0 = (wv.kind == 0 && nrefl > 0) ? mw.sigma_frac * tprev : 0.0;
    const float* prow =
        (wv.pred && wv.kind == 0) ? wv.pred + (size_t)r * wv.ld_pred : nullptr;
    // every walk refines its roots next to the boundary (stage 2): the chord
    // walks both ends, since a uniform point of a chord whose end is off by
    // the FP32 estimate's error can leave S
    MixResult res = segment_mixed(sp, mw, sm, Fc, Vr, Q32, Q64, sigma0, wv.kind != 0, true,
                                  prow, wv.t_scale, wv.margin);
    if (wv.rec_x && wv.kind == 0 && res.status == kOk && isfinite(res.t_plus)) {
      // training tuple: (x * x_scale, v) -> (log(t+ / t_scale), u)
      if (tid == 0) sm.ib[2] = atomicAdd(wv.rec_count, 1);
      __syncthreads();
      const int slot = sm.ib[2];
      if (slot < wv.rec_cap) {
        float* fx = wv.rec_x + (size_t)slot * 2 * n;
        float* fy = wv.rec_y + (size_t)slot * (1 + m);
        for (int j = tid; j < n; j += SPG_THREADS) {
          fx[j] = (float)(sm.p[j] * wv.x_scale);
          fx[n + j] = (float)sm.v[j];
        }
        for (int i = tid; i < m; i += SPG_THREADS) fy[1 + i] = (float)sm.u[i];
        if (tid == 0) fy[0] = (float)log(res.t_plus / wv.t_scale);
      }
      __syncthreads();
    }
    if (tid == 0) {
      st[kStatSegments] += 1;
      st[kStatLanczos] += res.iters;
      st[kStatShiftRetry] += res.retries;
      st[kStatFallback] += res.fallback;
      st[kStatPower] += res.power;
      if (res.learned > 0) st[kStatLearnedOk] += 1;
      if (res.learned < 0) st[kStatLearnedMiss] += 1;
      if (res.status == kNoConv) st[kStatNoConv] += 1;
    }
    const int flags = (res.retries > 0 ? kSegShiftRetry : 0) | (res.fallback ? kSegFallback : 0) |
                      (res.learned > 0 ? kSegLearnedOk : 0) |
                      (res.learned < 0 ? kSegLearnedMiss : 0) |
                      (res.status == kNoConv ? kSegNoConv : 0) | (res.refined ? kSegRefined : 0);
    if (res.status == kNoConv) res.status = kOk;
    const bool reflect = wv.kind == 0 && res.status == kOk && res.t_plus < ell;
    if (wv.pend) {
      // the wave's normals come from the tensor-core contraction; the
      // reflection completes in the finish kernel
      double* ub = wv.Ubuf + (size_t)r * m;
      for (int i = tid; i < m; i += SPG_THREADS) ub[i] = reflect ? sm.u[i] : 0.0;
      if (tid == 0) {
        wv.pend[r] = reflect ? 1 | (flags << 1) : 0;  // pending, and the record's flags
        wv.Tbuf[r] = res.t_plus;
      }
      __syncthreads();
      if (reflect) continue;
    } else if (reflect) {
      long long tc0 = clock64();
      contract_forms(sp, mw.Ahl, sm);
      stage_mark(mw, 5, tc0);  // normal contraction
    }
    complete_segment(sp, mw, wv, sm, r, c, res.status, res.t_plus, res.t_minus, ell, nrefl, Fc,
                     Vr, st, flags);
    __syncthreads();
  }
}

// Finish of the deferred reflections of a wave: w_j from the contraction's
// partial sums (fixed order), then the reflection and the rest of the
// segment (complete_segment).  One block per pending slot.
__global__ void __launch_bounds__(SPG_THREADS)
    mixed_reflect_kernel(DevSpec sp, MixWork mw, MixWave wv, int count) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n;
  const long long P = sp.P;
  MixSmem sm;
  double* d = reinterpret_cast<double*>(smem_raw);
  sm.p = d; d += n;
  sm.v = d; d += n;
  sm.w = d; d += n + 1;
  sm.wh = d; d += n;
  sm.bc = d; d += 16;
  sm.sc = reinterpret_cast<LanczosScalars*>(d);
  sm.ib = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(sm.sc) + sizeof(LanczosScalars));
  mw.prof = nullptr;
  for (int r = blockIdx.x; r < count; r += gridDim.x) {
    if (!wv.pend[r]) continue;
    const int c = wv.id_cur[r];
    for (int j = tid; j < n; j += SPG_THREADS) {
      sm.p[j] = wv.X[(size_t)c * n + j];
      sm.v[j] = wv.dir_cur[(size_t)r * n + j];
    }
    for (int j = tid; j <= n; j += SPG_THREADS) {
      const double* wp = wv.Wpart + ((size_t)r * (n + 1) + j) * wv.wtiles;
      double a = 0.0;
      for (int t = 0; t < wv.wtiles; ++t) a += wp[t];
      sm.w[j] = a;
    }
    __syncthreads();
    complete_segment(sp, mw, wv, sm, r, c, kOk, wv.Tbuf[r], -INFINITY, wv.ell[c], wv.nrefl[c],
                     wv.F + (size_t)c * P, wv.Vrows + (size_t)r * P,
                     wv.stats + (size_t)c * kNumStats, wv.pend[r] >> 1);
    __syncthreads();
  }
}

// first wave of a walk call: directions and lengths of the first step
__global__ void mixed_begin_kernel(DevSpec sp, MixWave wv) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int n = sp.n;
  MixSmem sm;
  double* d = reinterpret_cast<double*>(smem_raw);
  sm.v = d;
  sm.sc = reinterpret_cast<LanczosScalars*>(d + n + 1);
  for (int c = blockIdx.x; c < wv.C; c += gridDim.x) {
    const uint32_t chain = wv.chain0 + (uint32_t)c;
    if (wv.kind == 2) {
      const double uc = rng_uniform(wv.seed, chain, wv.step0, kStreamCoord);
      int jc = (int)(uc * n);
      jc = jc < n ? jc : n - 1;
      for (int j = threadIdx.x; j < n; j += SPG_THREADS) sm.v[j] = (j == jc) ? 1.0 : 0.0;
      __syncthreads();
    } else {
      draw_direction(wv.seed, chain, wv.step0, sm.v, n, sm);
    }
    for (int j = threadIdx.x; j < n; j += SPG_THREADS) {
      wv.dir_cur[(size_t)c * n + j] = sm.v[j];
      wv.Xstart[(size_t)c * n + j] = wv.X[(size_t)c * n + j];
    }
    if (threadIdx.x == 0) {
      wv.id_cur[c] = c;
      wv.done[c] = 0;
      wv.nrefl[c] = 0;
      wv.tprev[c] = 0.0;
      wv.ell[c] = wv.kind == 0
                      ? -wv.tau * log(rng_uniform(wv.seed, chain, wv.step0, kStreamEta))
                      : 0.0;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *wv.count_cur = wv.C;
}

// ---------------------------------------------------------------------------
// primitives (intersection / reflection) in mixed precision
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SPG_THREADS, 1)
    prim_mixed_kernel(DevSpec sp, MixWork mw, PrimParams pp, const double* Frows,
                      const double* Vrows) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n, m = sp.m;
  const long long P = sp.P;
  const size_t cta = blockIdx.x;
  uint8_t* rg = mw.region_global ? mw.region_global + cta * mw.region_bytes : nullptr;
  MixSmem sm = mix_carve(smem_raw, n, m, rg, mw.region_bytes);
  if (tid == 0 && mw.prof) sm.sc->prof = mw.prof + blockIdx.x * kProfSlots + 8;
  float* Q32 = mw.Q32 + cta * (size_t)mw.kmax32 * m;
  double* Q64 = mw.Q64 + cta * (size_t)mw.kmax64 * m;
  for (int c = blockIdx.x; c < pp.count; c += gridDim.x) {
    double bad = 0.0;
    for (int j = tid; j < n; j += SPG_THREADS) {
      sm.v[j] = pp.v[(size_t)c * n + j];
      if (!isfinite(sm.v[j]) || !isfinite(pp.x[(size_t)c * n + j])) bad = 1.0;
    }
    if (block_sum(bad, sm.sc->red) > 0.0) {
      // a non-finite point or direction: nothing to compute (its formed rows
      // are garbage and stay unused)
      if (tid == 0) {
        pp.status[c] = kInvalid;
        pp.t_plus[c] = NAN;
        if (pp.op == 0) pp.t_minus[c] = NAN;
      }
      if (pp.Ubuf)
        for (int i = tid; i < m; i += SPG_THREADS) pp.Ubuf[(size_t)c * m + i] = 0.0;
      __syncthreads();
      continue;
    }
    const float* prow = (pp.pred && pp.op == 1) ? pp.pred + (size_t)c * pp.ld_pred : nullptr;
    MixResult res = segment_mixed(sp, mw, sm, Frows + (size_t)c * P, Vrows + (size_t)c * P, Q32,
                                  Q64, 0.0, pp.op == 0, true, prow, pp.t_scale, pp.margin);
    if (tid == 0 && pp.learned_ok && res.learned != 0)
      atomicAdd(res.learned > 0 ? &pp.learned_ok[0] : &pp.learned_ok[1], 1);
    int status = res.status == kNoConv ? kOk : res.status;
    if (pp.op == 0) {
      if (tid == 0) {
        pp.t_plus[c] = res.t_plus;
        pp.t_minus[c] = res.t_minus;
        pp.status[c] = res.status;
      }
      if (pp.u && status == kOk)
        for (int i = tid; i < m; i += SPG_THREADS) pp.u[(size_t)c * m + i] = sm.u[i];
    } else if (pp.Ubuf) {
      // normals of all lines at once on the tensor cores (finish kernel)
      for (int i = tid; i < m; i += SPG_THREADS)
        pp.Ubuf[(size_t)c * m + i] = status == kOk ? sm.u[i] : 0.0;
      if (tid == 0) {
        pp.t_plus[c] = res.t_plus;
        pp.status[c] = status == kOk ? res.status : status;
      }
    } else {
      if (status == kOk) {
        contract_forms(sp, mw.Ahl, sm);
        const double nw = mix_unit_normal(sm, n);
        if (!(nw > 0.0)) status = kDegenerate;
      }
      if (status == kOk) {
        double a = 0.0;
        for (int j = tid; j < n; j += SPG_THREADS) a += sm.v[j] * sm.wh[j];
        const double vw = block_sum(a, sm.sc->red);
        for (int j = tid; j < n; j += SPG_THREADS) {
          pp.w_hat[(size_t)c * n + j] = sm.wh[j];
          pp.s[(size_t)c * n + j] = sm.v[j] - 2.0 * vw * sm.wh[j];
        }
      }
      if (tid == 0) {
        pp.t_plus[c] = res.t_plus;
        pp.status[c] = status == kOk ? res.status : status;
      }
    }
    __syncthreads();
  }
}

// reflect, second half: w_j from the contraction's partial sums, unit normal
// and reflected direction (Eq. "reflection") for every line whose oracle
// call succeeded
__global__ void __launch_bounds__(SPG_THREADS) prim_reflect_finish_kernel(DevSpec sp, PrimParams pp) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int tid = threadIdx.x;
  const int n = sp.n;
  MixSmem sm;
  double* d = reinterpret_cast<double*>(smem_raw);
  sm.w = d; d += n + 1;
  sm.wh = d; d += n;
  sm.sc = reinterpret_cast<LanczosScalars*>(d);
  for (int c = blockIdx.x; c < pp.count; c += gridDim.x) {
    const int st0 = pp.status[c];
    if (!(st0 == kOk || st0 == kNoConv)) continue;
    for (int j = tid; j <= n; j += SPG_THREADS) {
      const double* wp = pp.Wpart + ((size_t)c * (n + 1) + j) * pp.wtiles;
      double a = 0.0;
      for (int t = 0; t < pp.wtiles; ++t) a += wp[t];
      sm.w[j] = a;
    }
    __syncthreads();
    const double nw = mix_unit_normal(sm, n);
    if (!(nw > 0.0)) {
      if (tid == 0) pp.status[c] = kDegenerate;
    } else {
      const double* v = pp.v + (size_t)c * n;
      double a = 0.0;
      for (int j = tid; j < n; j += SPG_THREADS) a += v[j] * sm.wh[j];
      const double vw = block_sum(a, sm.sc->red);
      for (int j = tid; j < n; j += SPG_THREADS) {
        pp.w_hat[(size_t)c * n + j] = sm.wh[j];
        pp.s[(size_t)c * n + j] = v[j] - 2.0 * vw * sm.wh[j];
      }
    }
    __syncthreads();
  }
}

// features of the listed chains for the warm-start network: (x * x_scale, v)
__global__ void learned_features_kernel(const double* __restrict__ X,
                                        const double* __restrict__ dir, const int* __restrict__ id,
                                        int count, int n, double x_scale,
                                        float* __restrict__ feats) {
  const long long total = (long long)count * n;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), j = (int)(q % n);
    const size_t row = id ? (size_t)id[r] : (size_t)r;  // no id list: row r is line r
    feats[(size_t)r * 2 * n + j] = (float)(X[row * n + j] * x_scale);
    feats[(size_t)r * 2 * n + n + j] = (float)dir[(size_t)r * n + j];
  }
}

}  // namespace

cudaError_t launch_learned_features(const double* X, const double* dir, const int* id, int count,
                                    int n, double x_scale, float* feats, cudaStream_t st) {
  const long long total = (long long)count * n;
  long long g = (total + 255) / 256;
  learned_features_kernel<<<(int)(g < 4096 ? (g > 0 ? g : 1) : 4096), 256, 0, st>>>(
      X, dir, id, count, n, x_scale, feats);
  return cudaGetLastError();
}

size_t mixed_region_bytes(int n, int m) {
  (void)n;
  const size_t P = (size_t)m * (m + 1) / 2;
  // max of 2 P floats (stage 1, contraction), P doubles or double-floats
  // (stage 2) and the FP32 factor plus the column partials of the
  // double-float products (pencil Rayleigh quotient)
  const size_t df = (P + 4 * (size_t)SPG_WARPS * 256) * 4;
  return ((P * 8 > df ? P * 8 : df) + 15) & ~size_t(15);
}

size_t mixed_smem_bytes(int n, int m, bool region_in_smem) {
  size_t b = region_in_smem ? ((mixed_region_bytes(n, m) + 15) & ~size_t(15)) : 0;
  b += 8 * ((size_t)4 * n + 1 + 5 * (size_t)m + (size_t)SPG_WARPS * m + 128 + SPG_SCR + 16);
  b += 4 * (size_t)12 * m;
  b += sizeof(LanczosScalars) + 16 * sizeof(int);
  return b;
}

cudaError_t launch_mixed_wave(const DevSpec& sp, const MixWork& mw, const MixWave& wv,
                              cudaStream_t st) {
  const size_t smem = mixed_smem_bytes(sp.n, sp.m, mw.region_global == nullptr);
  cudaError_t e = cudaFuncSetAttribute(mixed_wave_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mixed_wave_kernel<<<mw.ctas, SPG_THREADS, smem, st>>>(sp, mw, wv);
  return cudaGetLastError();
}

cudaError_t launch_prim_reflect_finish(const DevSpec& sp, const PrimParams& pp, int ctas,
                                       cudaStream_t st) {
  if (pp.count <= 0) return cudaSuccess;
  const size_t smem = 8 * ((size_t)2 * sp.n + 1) + sizeof(LanczosScalars);
  const int grid = pp.count < ctas ? pp.count : ctas;
  prim_reflect_finish_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, pp);
  return cudaGetLastError();
}

cudaError_t launch_mixed_reflect(const DevSpec& sp, const MixWave& wv, int count, int ctas,
                                 cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = 8 * ((size_t)4 * sp.n + 1 + 16) + sizeof(LanczosScalars) + 16 * sizeof(int);
  MixWork mw{};
  const int grid = count < ctas ? count : ctas;
  mixed_reflect_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, mw, wv, count);
  return cudaGetLastError();
}

cudaError_t launch_mixed_begin(const DevSpec& sp, const MixWave& wv, cudaStream_t st) {
  const size_t smem = 8 * ((size_t)sp.n + 1) + sizeof(LanczosScalars);
  const int grid = wv.C < 1024 ? wv.C : 1024;
  mixed_begin_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, wv);
  return cudaGetLastError();
}

cudaError_t launch_prim_mixed(const DevSpec& sp, const MixWork& mw, const PrimParams& pp,
                              const double* Frows, const double* Vrows, cudaStream_t st) {
  const size_t smem = mixed_smem_bytes(sp.n, sp.m, mw.region_global == nullptr);
  cudaError_t e = cudaFuncSetAttribute(prim_mixed_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = pp.count < mw.ctas ? pp.count : mw.ctas;
  if (grid <= 0) return cudaSuccess;
  prim_mixed_kernel<<<grid, SPG_THREADS, smem, st>>>(sp, mw, pp, Frows, Vrows);
  return cudaGetLastError();
}

}  // namespace spg
