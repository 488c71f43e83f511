// C ABI of libspectra_gb: handle management, argument checks and launches.
// Declarations and the contract of every entry point: include/spectra_gb.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "kernels.h"

using namespace spg;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, const char* a = "") {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, a);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  g_err = msg;
  return SP_ECUDA;
}

#define SP_CUDA(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// per-CTA workspace of the FP64 kernels
struct Workspace {
  int ctas = 0, kmax = 0, m = 0;
  long long P = 0;
  double* Vfull = nullptr;
  double* Fg = nullptr;
  double* Q = nullptr;
  double* Lg = nullptr;
  bool l_in_smem = true;

  void release() {
    cudaFree(Vfull);
    cudaFree(Fg);
    cudaFree(Q);
    cudaFree(Lg);
    Vfull = Fg = Q = Lg = nullptr;
    ctas = 0;
  }
  int ensure(int n, int m_, int kmax_, int ctas_) {
    if (ctas >= ctas_ && kmax >= kmax_ && m == m_) return SP_OK;
    release();
    m = m_;
    P = (long long)m * (m + 1) / 2;
    kmax = kmax_;
    ctas = ctas_;
    l_in_smem = fp64_smem_bytes(n, m, true) <= (size_t)max_smem_optin();
    if (cudaMalloc(&Vfull, sizeof(double) * (size_t)m * m * ctas) != cudaSuccess ||
        cudaMalloc(&Fg, sizeof(double) * (size_t)P * ctas) != cudaSuccess ||
        cudaMalloc(&Q, sizeof(double) * (size_t)kmax * m * ctas) != cudaSuccess ||
        (!l_in_smem && cudaMalloc(&Lg, sizeof(double) * (size_t)P * ctas) != cudaSuccess)) {
      cudaGetLastError();
      release();
      return fail(SP_ENOMEM, "workspace allocation failed%s");
    }
    return SP_OK;
  }
  DevWork dev(double tol) const {
    DevWork w;
    w.Vfull = Vfull;
    w.Fg = Fg;
    w.Q = Q;
    w.Lg = Lg;
    w.kmax = kmax;
    w.tol = tol;
    w.l_in_smem = l_in_smem ? 1 : 0;
    w.ctas = ctas;
    return w;
  }
};

}  // namespace

struct sp_spec {
  int n = 0, m = 0;
  long long P = 0;
  double* A = nullptr;      // (n+1) x P packed
  uint32_t* pidx = nullptr;  // P
  int kmax = 96;
  double tol = 1e-13;
  double sigma_frac = 0.1;
  Workspace ws;  // for the primitive entry points
  DevSpec dev() const {
    DevSpec d;
    d.n = n;
    d.m = m;
    d.P = P;
    d.A = A;
    d.pidx = pidx;
    return d;
  }
};

struct sp_chains {
  sp_spec* spec = nullptr;
  int C = 0;
  uint64_t seed = 0;
  uint32_t chain0 = 0;
  uint32_t step = 0;
  double* X = nullptr;
  int* status = nullptr;
  long long* stats = nullptr;
  Workspace ws;
};

extern "C" {

const char* sp_last_error(void) { return g_err.c_str(); }

// error reporting for entry points defined in other translation units
int sp_noalloc_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

const char* sp_version(void) { return "spectra_gb 0.1 (sm_103a)"; }

int sp_create_spectrahedron(int n, int m, const double* A, uint32_t flags, sp_spec** out) {
  (void)flags;
  if (!out || !A) return fail(SP_EINVAL, "sp_create_spectrahedron: null pointer%s");
  if (n < 1 || m < 1 || n > 4096 || m > 4096)
    return fail(SP_EINVAL, "sp_create_spectrahedron: n, m must be in [1, 4096]%s");
  const size_t mm = (size_t)m * m;
  const long long P = (long long)m * (m + 1) / 2;
  std::vector<double> packed((size_t)(n + 1) * P);
  std::vector<uint32_t> pidx(P);
  for (int j = 0; j <= n; ++j) {
    const double* Aj = A + (size_t)j * mm;
    double amax = 0.0;
    for (size_t e = 0; e < mm; ++e) amax = std::max(amax, fabs(Aj[e]));
    for (int i = 0; i < m; ++i)
      for (int k = 0; k <= i; ++k) {
        const double a = Aj[(size_t)i * m + k], b = Aj[(size_t)k * m + i];
        if (fabs(a - b) > 1e-12 * amax) {
          char buf[64];
          snprintf(buf, sizeof(buf), "%d", j);
          return fail(SP_EINVAL, "sp_create_spectrahedron: A_%s is not symmetric", buf);
        }
        packed[(size_t)j * P + tri(i, k)] = 0.5 * (a + b);
      }
  }
  for (int i = 0; i < m; ++i)
    for (int k = 0; k <= i; ++k) pidx[tri(i, k)] = ((uint32_t)i << 16) | (uint32_t)k;
  sp_spec* s = new sp_spec();
  s->n = n;
  s->m = m;
  s->P = P;
  if (cudaMalloc(&s->A, sizeof(double) * packed.size()) != cudaSuccess ||
      cudaMalloc(&s->pidx, sizeof(uint32_t) * pidx.size()) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->A);
    cudaFree(s->pidx);
    delete s;
    return fail(SP_ENOMEM, "sp_create_spectrahedron: device allocation failed%s");
  }
  cudaError_t e1 = cudaMemcpy(s->A, packed.data(), sizeof(double) * packed.size(),
                              cudaMemcpyHostToDevice);
  cudaError_t e2 = cudaMemcpy(s->pidx, pidx.data(), sizeof(uint32_t) * pidx.size(),
                              cudaMemcpyHostToDevice);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaFree(s->A);
    cudaFree(s->pidx);
    delete s;
    return cuda_fail(e1 != cudaSuccess ? e1 : e2, "sp_create_spectrahedron: upload");
  }
  *out = s;
  return SP_OK;
}

int sp_destroy_spectrahedron(sp_spec* s) {
  if (!s) return fail(SP_EINVAL, "sp_destroy_spectrahedron: null handle%s");
  cudaFree(s->A);
  cudaFree(s->pidx);
  s->ws.release();
  delete s;
  return SP_OK;
}

int sp_spec_dims(const sp_spec* s, int* n, int* m) {
  if (!s) return fail(SP_EINVAL, "sp_spec_dims: null handle%s");
  if (n) *n = s->n;
  if (m) *m = s->m;
  return SP_OK;
}

int sp_set_solver(sp_spec* s, int kmax, double tol, double sigma_frac) {
  if (!s) return fail(SP_EINVAL, "sp_set_solver: null handle%s");
  if (kmax < 1 || kmax > 128 || !(tol > 0.0) || !(sigma_frac >= 0.0 && sigma_frac < 1.0))
    return fail(SP_EINVAL, "sp_set_solver: kmax in [1,128], tol > 0, sigma_frac in [0,1)%s");
  s->kmax = kmax;
  s->tol = tol;
  s->sigma_frac = sigma_frac;
  return SP_OK;
}

static int check_mode(int mode, const char* fn) {
  if (mode != SP_MODE_FP64) return fail(SP_EINVAL, "%s: unknown mode", fn);
  return SP_OK;
}

static int run_prim(sp_spec* s, PrimParams& pp, void* stream) {
  const int ctas = std::min(pp.count, device_sms());
  int r = s->ws.ensure(s->n, s->m, s->kmax, std::max(ctas, 1));
  if (r) return r;
  DevWork wk = s->ws.dev(s->tol);
  cudaError_t e = launch_prim_fp64(s->dev(), wk, pp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "boundary-oracle kernel launch");
  return SP_OK;
}

int sp_membership(sp_spec* s, int count, const double* x, int* inside, void* stream) {
  if (!s || (count > 0 && (!x || !inside)))
    return fail(SP_EINVAL, "sp_membership: null argument%s");
  if (count < 0) return fail(SP_EINVAL, "sp_membership: count < 0%s");
  if (count == 0) return SP_OK;
  PrimParams pp{};
  pp.op = 2;
  pp.count = count;
  pp.x = x;
  pp.inside = inside;
  return run_prim(s, pp, stream);
}

int sp_intersect(sp_spec* s, int count, const double* x, const double* v, double* t_minus,
                 double* t_plus, double* u, int* status, int mode, void* stream) {
  if (!s || (count > 0 && (!x || !v || !t_minus || !t_plus || !status)))
    return fail(SP_EINVAL, "sp_intersect: null argument%s");
  if (count < 0) return fail(SP_EINVAL, "sp_intersect: count < 0%s");
  if (int r = check_mode(mode, "sp_intersect")) return r;
  if (count == 0) return SP_OK;
  PrimParams pp{};
  pp.op = 0;
  pp.count = count;
  pp.x = x;
  pp.v = v;
  pp.t_minus = t_minus;
  pp.t_plus = t_plus;
  pp.u = u;
  pp.status = status;
  return run_prim(s, pp, stream);
}

int sp_reflect(sp_spec* s, int count, const double* x, const double* v, double* t_plus,
               double* w_hat, double* s_out, int* status, int mode, void* stream) {
  if (!s || (count > 0 && (!x || !v || !t_plus || !w_hat || !s_out || !status)))
    return fail(SP_EINVAL, "sp_reflect: null argument%s");
  if (count < 0) return fail(SP_EINVAL, "sp_reflect: count < 0%s");
  if (int r = check_mode(mode, "sp_reflect")) return r;
  if (count == 0) return SP_OK;
  PrimParams pp{};
  pp.op = 1;
  pp.count = count;
  pp.x = x;
  pp.v = v;
  pp.t_plus = t_plus;
  pp.w_hat = w_hat;
  pp.s = s_out;
  pp.status = status;
  return run_prim(s, pp, stream);
}

int sp_init_chains(sp_spec* s, int C, const double* x0, uint64_t seed, uint32_t chain0,
                   sp_chains** out, void* stream) {
  if (!s || !out) return fail(SP_EINVAL, "sp_init_chains: null argument%s");
  if (C < 1) return fail(SP_EINVAL, "sp_init_chains: C must be >= 1%s");
  cudaStream_t st = (cudaStream_t)stream;
  sp_chains* ch = new sp_chains();
  ch->spec = s;
  ch->C = C;
  ch->seed = seed;
  ch->chain0 = chain0;
  const size_t xb = sizeof(double) * (size_t)C * s->n;
  if (cudaMalloc(&ch->X, xb) != cudaSuccess ||
      cudaMalloc(&ch->status, sizeof(int) * C) != cudaSuccess ||
      cudaMalloc(&ch->stats, sizeof(long long) * (size_t)C * kNumStats) != cudaSuccess) {
    cudaGetLastError();
    sp_destroy_chains(ch);
    return fail(SP_ENOMEM, "sp_init_chains: device allocation failed%s");
  }
  cudaError_t e;
  if (!x0)
    e = cudaMemsetAsync(ch->X, 0, xb, st);
  else
    e = cudaMemcpyAsync(ch->X, x0, xb, is_device_ptr(x0) ? cudaMemcpyDeviceToDevice
                                                          : cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ch->status, 0, sizeof(int) * C, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ch->stats, 0, sizeof(long long) * (size_t)C * kNumStats, st);
  if (e != cudaSuccess) {
    sp_destroy_chains(ch);
    return cuda_fail(e, "sp_init_chains: upload");
  }
  // every start point must be interior
  int* inside = nullptr;
  if (cudaMalloc(&inside, sizeof(int) * C) != cudaSuccess) {
    cudaGetLastError();
    sp_destroy_chains(ch);
    return fail(SP_ENOMEM, "sp_init_chains: device allocation failed%s");
  }
  int r = sp_membership(s, C, ch->X, inside, stream);
  std::vector<int> h(C);
  if (r == SP_OK) {
    e = cudaMemcpyAsync(h.data(), inside, sizeof(int) * C, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "sp_init_chains: membership");
  }
  cudaFree(inside);
  if (r != SP_OK) {
    sp_destroy_chains(ch);
    return r;
  }
  for (int c = 0; c < C; ++c)
    if (!h[c]) {
      sp_destroy_chains(ch);
      char buf[32];
      snprintf(buf, sizeof(buf), "%d", c);
      return fail(SP_ENOTPD, "sp_init_chains: start point %s is not interior", buf);
    }
  *out = ch;
  return SP_OK;
}

int sp_destroy_chains(sp_chains* ch) {
  if (!ch) return fail(SP_EINVAL, "sp_destroy_chains: null handle%s");
  cudaFree(ch->X);
  cudaFree(ch->status);
  cudaFree(ch->stats);
  ch->ws.release();
  delete ch;
  return SP_OK;
}

static int run_walk(sp_chains* ch, int kind, int steps, double tau, int rho, double kappa,
                    int mode, void* stream, const char* fn) {
  if (!ch) return fail(SP_EINVAL, "%s: null handle", fn);
  if (steps < 0) return fail(SP_EINVAL, "%s: steps < 0", fn);
  if (int r = check_mode(mode, fn)) return r;
  if (steps == 0) return SP_OK;
  sp_spec* s = ch->spec;
  const int ctas = std::min(ch->C, device_sms());
  int r = ch->ws.ensure(s->n, s->m, s->kmax, ctas);
  if (r) return r;
  WalkParams wp{};
  wp.kind = kind;
  wp.C = ch->C;
  wp.steps = steps;
  wp.step0 = ch->step;
  wp.chain0 = ch->chain0;
  wp.seed = ch->seed;
  wp.tau = tau;
  wp.kappa = kappa;
  wp.sigma_frac = s->sigma_frac;
  wp.rho = rho;
  wp.X = ch->X;
  wp.status = ch->status;
  wp.stats = ch->stats;
  cudaError_t e = launch_walk_fp64(s->dev(), ch->ws.dev(s->tol), wp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
  ch->step += (uint32_t)steps;
  return SP_OK;
}

int sp_step_billiard(sp_chains* ch, int steps, double tau, int rho, double kappa, int mode,
                     void* stream) {
  if (!(tau > 0.0) || rho < 0 || !(kappa >= 0.0 && kappa < 1.0))
    return fail(SP_EINVAL, "sp_step_billiard: need tau > 0, rho >= 0, 0 <= kappa < 1%s");
  return run_walk(ch, 0, steps, tau, rho, kappa, mode, stream, "sp_step_billiard");
}

int sp_step_hnr(sp_chains* ch, int steps, int mode, void* stream) {
  return run_walk(ch, 1, steps, 1.0, 0, 0.0, mode, stream, "sp_step_hnr");
}

int sp_step_cdhr(sp_chains* ch, int steps, int mode, void* stream) {
  return run_walk(ch, 2, steps, 1.0, 0, 0.0, mode, stream, "sp_step_cdhr");
}

int sp_get_state(sp_chains* ch, double* x_out, uint32_t* step_out, void* stream) {
  if (!ch) return fail(SP_EINVAL, "sp_get_state: null handle%s");
  cudaStream_t st = (cudaStream_t)stream;
  if (x_out) {
    const size_t xb = sizeof(double) * (size_t)ch->C * ch->spec->n;
    const bool dev = is_device_ptr(x_out);
    SP_CUDA(cudaMemcpyAsync(x_out, ch->X, xb,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!dev) SP_CUDA(cudaStreamSynchronize(st));
  }
  if (step_out) *step_out = ch->step;
  return SP_OK;
}

int sp_set_state(sp_chains* ch, const double* x, uint32_t step, void* stream) {
  if (!ch || !x) return fail(SP_EINVAL, "sp_set_state: null argument%s");
  const size_t xb = sizeof(double) * (size_t)ch->C * ch->spec->n;
  SP_CUDA(cudaMemcpyAsync(ch->X, x, xb,
                          is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          (cudaStream_t)stream));
  if (!is_device_ptr(x)) SP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  ch->step = step;
  return SP_OK;
}

int sp_chain_status(sp_chains* ch, int* status, long long* stats, void* stream) {
  if (!ch) return fail(SP_EINVAL, "sp_chain_status: null handle%s");
  cudaStream_t st = (cudaStream_t)stream;
  if (status)
    SP_CUDA(cudaMemcpyAsync(status, ch->status, sizeof(int) * ch->C, cudaMemcpyDeviceToDevice,
                            st));
  if (stats) {
    std::vector<long long> h((size_t)ch->C * kNumStats);
    SP_CUDA(cudaMemcpyAsync(h.data(), ch->stats, sizeof(long long) * h.size(),
                            cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < SP_NUM_STATS; ++k) stats[k] = 0;
    for (int c = 0; c < ch->C; ++c)
      for (int k = 0; k < kNumStats; ++k) stats[k] += h[(size_t)c * kNumStats + k];
  }
  return SP_OK;
}

}  // extern "C"
