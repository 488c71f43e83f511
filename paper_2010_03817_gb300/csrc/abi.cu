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

// work space of the mixed path (per CTA) plus its row buffers
struct MixSpace {
  int ctas = 0, rows = 0, m = 0, n = 0;
  float* Q32 = nullptr;
  double* Q64 = nullptr;
  uint8_t* region = nullptr;  // only when the region does not fit in shared memory
  size_t region_bytes = 0;
  void* digits = nullptr;     // 7 x rows x Kp BF16 digits of coefficient rows
  int* erow = nullptr;        // rows
  double* Frows = nullptr;    // rows x P
  double* Vrows = nullptr;    // rows x P
  int* err = nullptr;
  float2* vdf = nullptr;      // ctas x P: V as double-float pairs for stage 2
  float* feats = nullptr;     // rows x 2n: warm-start features of the lines (learned reflect)
  int* learned = nullptr;     // 2: warm starts accepted / rejected by the last learned call
  // deferred normals of a wave (tensor-core contraction)
  double* Ubuf = nullptr;     // rows x m
  double* Tbuf = nullptr;     // rows
  int* pend = nullptr;        // rows
  double* Wpart = nullptr;    // rows x (n+1) x wtiles
  void* udig = nullptr;       // 7 x rows x Kp(m) BF16 digits of the null vectors
  int* uerow = nullptr;       // rows
  int wtiles = 0;
  void release() {
    cudaFree(Q32); cudaFree(Q64); cudaFree(region); cudaFree(digits); cudaFree(erow);
    cudaFree(Frows); cudaFree(Vrows); cudaFree(err); cudaFree(vdf);
    cudaFree(feats); cudaFree(learned);
    vdf = nullptr;
    feats = nullptr;
    learned = nullptr;
    cudaFree(Ubuf); cudaFree(Tbuf); cudaFree(pend); cudaFree(Wpart); cudaFree(udig);
    cudaFree(uerow);
    Q32 = nullptr; Q64 = nullptr; region = nullptr; digits = nullptr; erow = nullptr;
    Frows = Vrows = nullptr; err = nullptr;
    Ubuf = Tbuf = Wpart = nullptr; pend = nullptr; udig = nullptr; uerow = nullptr;
    ctas = rows = 0;
  }
  int ensure_contract(int rows_) {
    if (Ubuf) return SP_OK;
    wtiles = ozaki_mpad(m) / 32;
    bool ok = cudaMalloc(&Ubuf, sizeof(double) * (size_t)rows_ * m) == cudaSuccess &&
              cudaMalloc(&Tbuf, sizeof(double) * rows_) == cudaSuccess &&
              cudaMalloc(&pend, sizeof(int) * rows_) == cudaSuccess &&
              cudaMalloc(&Wpart, sizeof(double) * (size_t)rows_ * (n + 1) * wtiles) ==
                  cudaSuccess &&
              cudaMalloc(&udig, ozaki_row_bytes(rows_, m)) == cudaSuccess &&
              cudaMalloc(&uerow, sizeof(int) * rows_) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaFree(Ubuf); cudaFree(Tbuf); cudaFree(pend); cudaFree(Wpart); cudaFree(udig);
      cudaFree(uerow);
      Ubuf = Tbuf = Wpart = nullptr; pend = nullptr; udig = nullptr; uerow = nullptr;
      return fail(SP_ENOMEM, "normal contraction work space allocation failed%s");
    }
    return SP_OK;
  }
  int ensure(int n_, int m_, int ctas_, int rows_, int kmax32, int kmax64, bool with_f) {
    if (ctas >= ctas_ && rows >= rows_ && m == m_ && n == n_ && (!with_f || Frows)) return SP_OK;
    release();
    n = n_;
    m = m_;
    ctas = ctas_;
    rows = rows_;
    const size_t P = (size_t)m * (m + 1) / 2;
    region_bytes = mixed_region_bytes(n, m);
    const bool in_smem = mixed_smem_bytes(n, m, true) <= (size_t)max_smem_optin();
    bool ok = cudaMalloc(&Q32, sizeof(float) * (size_t)kmax32 * m * ctas) == cudaSuccess &&
              cudaMalloc(&Q64, sizeof(double) * (size_t)kmax64 * m * ctas) == cudaSuccess &&
              (in_smem || cudaMalloc(&region, region_bytes * ctas) == cudaSuccess) &&
              cudaMalloc(&digits, ozaki_row_bytes(rows, n)) == cudaSuccess &&
              cudaMalloc(&erow, sizeof(int) * rows) == cudaSuccess &&
              cudaMalloc(&Vrows, sizeof(double) * P * rows) == cudaSuccess &&
              (!with_f || cudaMalloc(&Frows, sizeof(double) * P * rows) == cudaSuccess) &&
              cudaMalloc(&vdf, sizeof(float2) * P * ctas) == cudaSuccess &&
              cudaMalloc(&err, sizeof(int)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release();
      return fail(SP_ENOMEM, "mixed-path work space allocation failed%s");
    }
    cudaMemset(err, 0, sizeof(int));
    return SP_OK;
  }
};

struct sp_spec {
  int n = 0, m = 0;
  long long P = 0;
  double* A = nullptr;      // (n+1) x P packed
  uint32_t* pidx = nullptr;  // P
  int kmax = 96;
  double tol = 1e-13;
  double sigma_frac = 0.1;
  Workspace ws;  // for the primitive entry points
  // mixed path: digits of the A stack (tensor-core formation) and FP32 pairs
  bool mixed_ok = false;
  uint16_t* Bsl = nullptr;
  int* ecol = nullptr;
  float2* Ahl = nullptr;
  uint16_t* Bc = nullptr;  // digits of the rows (j, i) of A_j: tensor-core normals
  int* ecolc = nullptr;
  int kmax32 = 96, kmax64 = 96, power_iters = 8;
  double tol32 = 1e-4, tol64 = 1e-10, delta1 = 2e-4;
  long long* prof = nullptr;  // optional stage timers (device, ctas x kProfSlots)
  int learned_iters = 12;
  // learned warm start
  sp_mlp* mlp = nullptr;
  double x_scale = 1.0, t_scale = 1.0, margin = 0.05;
  MixSpace ms;  // for the primitive entry points
  MixWork mixwork(const MixSpace& sp_) const {
    MixWork w;
    w.Ahl = Ahl;
    w.Q32 = sp_.Q32;
    w.Q64 = sp_.Q64;
    w.region_global = sp_.region;
    w.region_bytes = sp_.region_bytes;
    w.vdf = sp_.vdf;
    w.kmax32 = kmax32;
    w.kmax64 = kmax64;
    w.power_iters = power_iters;
    w.learned_iters = learned_iters;
    w.tol32 = tol32;
    w.tol64 = tol64;
    w.delta1 = delta1;
    w.sigma_frac = sigma_frac;
    w.ctas = sp_.ctas;
    w.prof = prof;
    return w;
  }
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
  // mixed path state
  MixSpace ms;
  double* F = nullptr;       // C x P carried F(x)
  bool F_valid = false;
  double* Xstart = nullptr;  // C x n
  double* ell = nullptr;
  double* tprev = nullptr;
  int* nrefl = nullptr;
  int* done = nullptr;
  int* ids[2] = {nullptr, nullptr};
  double* dirs[2] = {nullptr, nullptr};
  int* counts = nullptr;     // 4: the two wave lists, the F refresh list, the wave ticket
  int* h_count = nullptr;    // pinned host mirror
  int* fage = nullptr;       // C: updates of each chain's carried F since its formation
  int* ref_ids = nullptr;    // C: chains listed for a fresh formation of F
  float* feats = nullptr;    // C x 2n features of the learned path
  // optional per-kernel timing of walk calls (CUDA events on the walk's stream)
  bool timing = false;
  double t_form_ms = 0.0, t_wave_ms = 0.0, t_mlp_ms = 0.0, t_fp64_ms = 0.0;
  double t_contract_ms = 0.0, t_finish_ms = 0.0;
  long long n_form = 0, n_wave = 0, n_mlp = 0, n_fp64 = 0, n_other = 0;
  long long n_contract = 0, n_finish = 0;
  // sampled segment record (caller buffers, sp_record_segments)
  SegLog seg{nullptr, 0, 1, nullptr};
  // tuple recording (caller buffers)
  float* rec_x = nullptr;
  float* rec_y = nullptr;
  int* rec_count = nullptr;
  int rec_cap = 0;
  void release_mixed() {
    ms.release();
    cudaFree(F); cudaFree(Xstart); cudaFree(ell); cudaFree(tprev); cudaFree(nrefl);
    cudaFree(done); cudaFree(ids[0]); cudaFree(ids[1]); cudaFree(dirs[0]); cudaFree(dirs[1]);
    cudaFree(counts);
    cudaFree(feats);
    cudaFree(fage);
    cudaFree(ref_ids);
    feats = nullptr;
    fage = ref_ids = nullptr;
    if (h_count) cudaFreeHost(h_count);
    F = Xstart = ell = tprev = nullptr;
    nrefl = done = counts = h_count = nullptr;
    ids[0] = ids[1] = nullptr;
    dirs[0] = dirs[1] = nullptr;
    F_valid = false;
  }
};

namespace spg {
int spec_copy_stack(const sp_spec* s, double* packed_host) {
  const size_t bytes = sizeof(double) * (size_t)(s->n + 1) * s->P;
  if (cudaMemcpy(packed_host, s->A, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "LMI stack copy");
  return SP_OK;
}
DevSpec spec_dev(const sp_spec* s) { return s->dev(); }
ChainState chain_state(sp_chains* ch) {
  ChainState c;
  c.X = ch->X;
  c.status = ch->status;
  c.stats = ch->stats;
  c.C = ch->C;
  c.seed = ch->seed;
  c.chain0 = ch->chain0;
  c.step = ch->step;
  c.spec = ch->spec;
  return c;
}
void chain_advance(sp_chains* ch, uint32_t steps) {
  ch->step += steps;
  ch->F_valid = false;
}
const double* chain_points(const sp_chains* ch) { return ch->X; }
const double* chain_points(const sp_chains* ch, int* C, int* n) {
  *C = ch->C;
  *n = ch->spec->n;
  return ch->X;
}
}  // namespace spg

extern "C" {

const char* sp_last_error(void) { return g_err.c_str(); }

// error reporting for entry points defined in other translation units
int spg_set_error(int code, const char* msg) {
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
  // mixed path: BF16 digits of A_1..A_n (n <= kOzakiMaxK) and FP32 pairs
  if (n <= kOzakiMaxK && !(flags & 1u)) {
    const size_t nb = ozaki_b_bytes(P, n);
    std::vector<uint16_t> bsl(nb / 2);
    std::vector<int> ecol(P);
    ozaki_slice_stack(packed.data(), n, P, bsl.data(), ecol.data());
    std::vector<float2> ahl(packed.size());
    for (size_t e = 0; e < packed.size(); ++e) {
      const float h = (float)packed[e];
      ahl[e] = make_float2(h, (float)(packed[e] - (double)h));
    }
    bool ok = cudaMalloc(&s->Bsl, nb) == cudaSuccess &&
              cudaMalloc(&s->ecol, sizeof(int) * P) == cudaSuccess &&
              cudaMalloc(&s->Ahl, sizeof(float2) * ahl.size()) == cudaSuccess &&
              cudaMemcpy(s->Bsl, bsl.data(), nb, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(s->ecol, ecol.data(), sizeof(int) * P, cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              cudaMemcpy(s->Ahl, ahl.data(), sizeof(float2) * ahl.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaFree(s->Bsl); cudaFree(s->ecol); cudaFree(s->Ahl);
      s->Bsl = nullptr; s->ecol = nullptr; s->Ahl = nullptr;
    } else {
      s->mixed_ok = true;
    }
  }
  // tensor-core normals: digits of the rows of the full A_j (K = m)
  if (s->mixed_ok && m <= kOzakiMaxK) {
    const long long Q = (long long)(n + 1) * ozaki_mpad(m);
    bool ok = cudaMalloc(&s->Bc, ozaki_contract_bytes(n, m)) == cudaSuccess &&
              cudaMalloc(&s->ecolc, sizeof(int) * Q) == cudaSuccess &&
              launch_ozaki_slice_full(s->A, n, m, P, s->Bc, s->ecolc, 0) == cudaSuccess &&
              cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaFree(s->Bc); cudaFree(s->ecolc);
      s->Bc = nullptr; s->ecolc = nullptr;
    }
  }
  *out = s;
  return SP_OK;
}

int sp_destroy_spectrahedron(sp_spec* s) {
  if (!s) return fail(SP_EINVAL, "sp_destroy_spectrahedron: null handle%s");
  cudaFree(s->A);
  cudaFree(s->pidx);
  cudaFree(s->Bsl);
  cudaFree(s->ecol);
  cudaFree(s->Bc);
  cudaFree(s->ecolc);
  cudaFree(s->Ahl);
  s->ms.release();
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

int sp_set_mixed_solver(sp_spec* s, double tol32, double tol64, double delta1, int power_iters) {
  if (!s) return fail(SP_EINVAL, "sp_set_mixed_solver: null handle%s");
  if (!(tol32 > 0.0 && tol32 < 1.0) || !(tol64 > 0.0 && tol64 < 1.0) ||
      !(delta1 > 0.0 && delta1 < 0.5) || power_iters < 1 || power_iters > 64)
    return fail(SP_EINVAL,
                "sp_set_mixed_solver: tol32, tol64 in (0,1), delta1 in (0,0.5), power_iters in "
                "[1,64]%s");
  s->tol32 = tol32;
  s->tol64 = tol64;
  s->delta1 = delta1;
  s->power_iters = power_iters;
  return SP_OK;
}

static int check_mode(int mode, const char* fn) {
  if (mode != SP_MODE_FP64 && mode != SP_MODE_MIXED && mode != SP_MODE_LEARNED)
    return fail(SP_EINVAL, "%s: unknown mode", fn);
  return SP_OK;
}

static int check_mixed(const sp_spec* s, const char* fn) {
  if (!s->mixed_ok)
    return fail(SP_EINVAL, "%s: the mixed path needs n <= 224 (tensor-core formation)", fn);
  return SP_OK;
}

// F rows (lead 1, x) and / or V rows (lead 0, v) on the tensor cores
static int form_rows_mixed(sp_spec* s, MixSpace& ms, int count, const double* x,
                           const double* v, double* F_out, double* V_out, cudaStream_t st) {
  if (x && F_out) {
    cudaError_t e = launch_ozaki_form(x, count, s->n, 1.0, s->A, s->Bsl, s->ecol, s->P, ms.digits,
                                      ms.erow, F_out, s->P, ms.err, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core formation (F)");
  }
  if (v && V_out) {
    cudaError_t e = launch_ozaki_form(v, count, s->n, 0.0, s->A, s->Bsl, s->ecol, s->P, ms.digits,
                                      ms.erow, V_out, s->P, ms.err, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core formation (V)");
  }
  return SP_OK;
}

static int run_prim_mixed(sp_spec* s, PrimParams& pp, bool learned, void* stream) {
  if (int r = check_mixed(s, "boundary oracle")) return r;
  if (learned && !s->mlp)
    return fail(SP_EINVAL, "boundary oracle: the learned mode needs a network (sp_attach_mlp)%s");
  const int ctas = std::min(pp.count, device_sms());
  int r = s->ms.ensure(s->n, s->m, std::max(ctas, 1), pp.count, s->kmax32, s->kmax64, true);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = form_rows_mixed(s, s->ms, pp.count, pp.x, pp.v, s->ms.Frows, s->ms.Vrows, st);
  if (r) return r;
  // learned warm start of REFLECTION: the network's (log t+, u) for every line
  // (INTERSECTION also needs t-, which the network does not predict: it runs
  // the plain mixed stage 1)
  if (learned && pp.op == 1) {
    MixSpace& ms = s->ms;
    if (!ms.feats &&
        (cudaMalloc(&ms.feats, sizeof(float) * (size_t)ms.rows * 2 * s->n) != cudaSuccess ||
         cudaMalloc(&ms.learned, 2 * sizeof(int)) != cudaSuccess)) {
      cudaGetLastError();
      cudaFree(ms.feats);
      ms.feats = nullptr;
      return fail(SP_ENOMEM, "learned boundary oracle: feature buffer allocation failed%s");
    }
    cudaError_t e = launch_learned_features(pp.x, pp.v, nullptr, pp.count, s->n, s->x_scale,
                                            ms.feats, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ms.learned, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "learned features");
    const float* Y = nullptr;
    int ld = 0;
    if (int rr = spg_mlp_infer(s->mlp, pp.count, ms.feats, st, &Y, &ld)) return rr;
    pp.pred = Y;
    pp.ld_pred = ld;
    pp.t_scale = s->t_scale;
    pp.margin = s->margin;
    pp.learned_ok = ms.learned;
  }
  // reflect: the normals of all lines in one tensor-core contraction
  const bool tc_normals = pp.op == 1 && s->Bc != nullptr;
  if (tc_normals) {
    if (int rr = s->ms.ensure_contract(pp.count)) return rr;
    pp.Ubuf = s->ms.Ubuf;
    pp.Wpart = s->ms.Wpart;
    pp.wtiles = s->ms.wtiles;
  }
  cudaError_t e = launch_prim_mixed(s->dev(), s->mixwork(s->ms), pp, s->ms.Frows, s->ms.Vrows, st);
  if (e != cudaSuccess) return cuda_fail(e, "mixed boundary-oracle kernel launch");
  if (tc_normals) {
    e = launch_ozaki_contract(s->ms.Ubuf, pp.count, s->n, s->m, s->Bc, s->ecolc, s->ms.udig,
                              s->ms.uerow, s->ms.Wpart, s->ms.err, st);
    if (e == cudaSuccess) e = launch_prim_reflect_finish(s->dev(), pp, 4 * device_sms(), st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core normal contraction launch");
  }
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
  if (mode != SP_MODE_FP64) return run_prim_mixed(s, pp, false, stream);
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
  if (mode != SP_MODE_FP64) return run_prim_mixed(s, pp, mode == SP_MODE_LEARNED, stream);
  return run_prim(s, pp, stream);
}

int sp_attach_mlp(sp_spec* s, sp_mlp* q, double x_scale, double t_scale, double margin,
                  int iters) {
  if (!s) return fail(SP_EINVAL, "sp_attach_mlp: null handle%s");
  if (q) {
    int din = 0, dout = 0;
    spg_mlp_io(q, &din, &dout);
    if (din != 2 * s->n || dout != 1 + s->m)
      return fail(SP_EINVAL, "sp_attach_mlp: the network must map 2n inputs to 1 + m outputs%s");
    if (!(x_scale > 0.0) || !(t_scale > 0.0) || !(margin > 0.0 && margin < 1.0) || iters < 1)
      return fail(SP_EINVAL, "sp_attach_mlp: x_scale, t_scale > 0, 0 < margin < 1, iters >= 1%s");
  }
  s->mlp = q;
  s->x_scale = x_scale;
  s->t_scale = t_scale;
  s->margin = margin;
  s->learned_iters = iters;
  return SP_OK;
}

int sp_kernel_timing(sp_chains* ch, int enable, double* out) {
  if (!ch) return fail(SP_EINVAL, "sp_kernel_timing: null handle%s");
  if (out) {
    out[0] = ch->t_fp64_ms;
    out[1] = (double)ch->n_fp64;
    out[2] = ch->t_form_ms;
    out[3] = (double)ch->n_form;
    out[4] = ch->t_wave_ms;
    out[5] = (double)ch->n_wave;
    out[6] = ch->t_mlp_ms;
    out[7] = (double)ch->n_mlp;
    out[8] = (double)ch->n_other;
    out[9] = ch->t_contract_ms;
    out[10] = (double)ch->n_contract;
    out[11] = ch->t_finish_ms;
    out[12] = (double)ch->n_finish;
  }
  if (enable >= 0) {
    ch->timing = enable != 0;
    ch->t_fp64_ms = ch->t_form_ms = ch->t_wave_ms = ch->t_mlp_ms = 0.0;
    ch->t_contract_ms = ch->t_finish_ms = 0.0;
    ch->n_fp64 = ch->n_form = ch->n_wave = ch->n_mlp = ch->n_other = 0;
    ch->n_contract = ch->n_finish = 0;
  }
  return SP_OK;
}

int sp_record_tuples(sp_chains* ch, float* x_out, float* y_out, int capacity, int* count) {
  if (!ch) return fail(SP_EINVAL, "sp_record_tuples: null handle%s");
  if (x_out && (!y_out || !count || capacity < 1))
    return fail(SP_EINVAL, "sp_record_tuples: buffers, capacity and counter go together%s");
  ch->rec_x = x_out;
  ch->rec_y = y_out;
  ch->rec_count = count;
  ch->rec_cap = x_out ? capacity : 0;
  return SP_OK;
}

int sp_learned_counts(sp_spec* s, int* accepted, int* rejected) {
  if (!s) return fail(SP_EINVAL, "sp_learned_counts: null handle%s");
  int h[2] = {0, 0};
  if (s->ms.learned) {
    if (cudaMemcpy(h, s->ms.learned, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "sp_learned_counts");
  }
  if (accepted) *accepted = h[0];
  if (rejected) *rejected = h[1];
  return SP_OK;
}

int sp_record_segments(sp_chains* ch, double* buf, int capacity, int every, int* count) {
  if (!ch) return fail(SP_EINVAL, "sp_record_segments: null handle%s");
  if (buf && (!count || capacity < 1 || every < 1))
    return fail(SP_EINVAL, "sp_record_segments: buffer, capacity >= 1, every >= 1 and counter "
                           "go together%s");
  ch->seg.buf = buf;
  ch->seg.cap = buf ? capacity : 0;
  ch->seg.every = buf ? every : 1;
  ch->seg.count = buf ? count : nullptr;
  return SP_OK;
}

int sp_set_stage_timers(sp_spec* s, long long* timers) {
  if (!s) return fail(SP_EINVAL, "sp_set_stage_timers: null handle%s");
  s->prof = timers;
  return SP_OK;
}

int sp_form_pencil(sp_spec* s, int count, const double* x, const double* v, double* F_out,
                   double* V_out, int mode, void* stream) {
  if (!s || count < 0) return fail(SP_EINVAL, "sp_form_pencil: bad argument%s");
  if ((x == nullptr) != (F_out == nullptr) || (v == nullptr) != (V_out == nullptr))
    return fail(SP_EINVAL, "sp_form_pencil: x / F_out and v / V_out go together%s");
  if (int r = check_mode(mode, "sp_form_pencil")) return r;
  if (count == 0) return SP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == SP_MODE_FP64) {
    cudaError_t e = cudaSuccess;
    if (x) e = launch_form64(s->A, s->P, s->n, x, count, 1.0, F_out, s->P, st);
    if (e == cudaSuccess && v) e = launch_form64(s->A, s->P, s->n, v, count, 0.0, V_out, s->P, st);
    if (e != cudaSuccess) return cuda_fail(e, "sp_form_pencil");
    return SP_OK;
  }
  if (int r = check_mixed(s, "sp_form_pencil")) return r;
  int r = s->ms.ensure(s->n, s->m, std::min(count, device_sms()), count, s->kmax32, s->kmax64,
                       true);
  if (r) return r;
  r = form_rows_mixed(s, s->ms, count, x, v, F_out, V_out, st);
  if (r) return r;
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(&herr, s->ms.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sp_form_pencil");
  if (herr) return fail(SP_ECUDA, "sp_form_pencil: tensor-core wait limit reached%s");
  return SP_OK;
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
  ch->release_mixed();
  delete ch;
  return SP_OK;
}

static int ensure_chain_mixed(sp_chains* ch) {
  sp_spec* s = ch->spec;
  const int C = ch->C, n = s->n;
  int r = ch->ms.ensure(n, s->m, std::min(C, device_sms()), C, s->kmax32, s->kmax64, false);
  if (r) return r;
  if (ch->F) return SP_OK;
  const size_t P = (size_t)s->P;
  bool ok = cudaMalloc(&ch->F, sizeof(double) * P * C) == cudaSuccess &&
            cudaMalloc(&ch->Xstart, sizeof(double) * (size_t)C * n) == cudaSuccess &&
            cudaMalloc(&ch->ell, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&ch->tprev, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&ch->nrefl, sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&ch->done, sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&ch->ids[0], sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&ch->ids[1], sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&ch->dirs[0], sizeof(double) * (size_t)C * n) == cudaSuccess &&
            cudaMalloc(&ch->dirs[1], sizeof(double) * (size_t)C * n) == cudaSuccess &&
            cudaMalloc(&ch->counts, 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ch->fage, sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&ch->ref_ids, sizeof(int) * C) == cudaSuccess &&
            cudaMallocHost(&ch->h_count, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ch->release_mixed();
    return fail(SP_ENOMEM, "mixed-path chain state allocation failed%s");
  }
  ch->F_valid = false;
  return SP_OK;
}

// Mixed path: waves of one segment per active chain.  Each wave forms V for
// the active chains on the tensor cores, then runs the mixed segment kernel,
// which queues the chains that still have steps to do for the next wave.
// waves with at most this many chains contract the normals in-kernel
constexpr int kDeferMinRows = 256;

static int run_walk_mixed(sp_chains* ch, int kind, int steps, double tau, int rho, double kappa,
                          bool learned, void* stream) {
  sp_spec* s = ch->spec;
  if (int r = check_mixed(s, "walk")) return r;
  if (learned && !s->mlp)
    return fail(SP_EINVAL, "walk: the learned mode needs a network (sp_attach_mlp)%s");
  if (int r = ensure_chain_mixed(ch)) return r;
  if (learned && !ch->feats &&
      cudaMalloc(&ch->feats, sizeof(float) * (size_t)ch->C * 2 * s->n) != cudaSuccess) {
    cudaGetLastError();
    return fail(SP_ENOMEM, "walk: feature buffer allocation failed%s");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const DevSpec ds = s->dev();
  {
    // F(x) of every chain formed afresh at the start of each call; within the
    // call it is carried (F <- F + t V) and re-formed after kFRefresh updates
    cudaError_t e = launch_ozaki_form(ch->X, ch->C, s->n, 1.0, s->A, s->Bsl, s->ecol, s->P,
                                      ch->ms.digits, ch->ms.erow, ch->F, s->P, ch->ms.err, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ch->fage, 0, sizeof(int) * ch->C, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ch->counts + 2, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core formation (F)");
    ch->F_valid = true;
  }
  MixWave wv{};
  wv.kind = kind;
  wv.C = ch->C;
  wv.steps = steps;
  wv.rho = rho;
  wv.step0 = ch->step;
  wv.chain0 = ch->chain0;
  wv.seed = ch->seed;
  wv.tau = tau;
  wv.kappa = kappa;
  wv.X = ch->X;
  wv.Xstart = ch->Xstart;
  wv.F = ch->F;
  wv.Vrows = ch->ms.Vrows;
  wv.ell = ch->ell;
  wv.tprev = ch->tprev;
  wv.nrefl = ch->nrefl;
  wv.done = ch->done;
  wv.status = ch->status;
  wv.stats = ch->stats;
  wv.pred = nullptr;
  wv.ld_pred = 0;
  wv.t_scale = s->t_scale;
  wv.margin = s->margin;
  wv.x_scale = s->x_scale;
  wv.rec_x = ch->rec_x;
  wv.rec_y = ch->rec_y;
  wv.rec_count = ch->rec_count;
  wv.rec_cap = ch->rec_cap;
  wv.seg = ch->seg;
  wv.fage = ch->fage;
  wv.ref_ids = ch->ref_ids;
  wv.ref_count = ch->counts + 2;
  wv.ticket = ch->counts + 3;
  // Billiard: the reflections' normals on the tensor cores, one contraction
  // per wave (deferred from the wave kernel to a finish kernel)
  const bool defer = kind == 0 && s->Bc != nullptr;
  if (defer) {
    if (int r = ch->ms.ensure_contract(ch->C)) return r;
    wv.Ubuf = ch->ms.Ubuf;
    wv.Tbuf = ch->ms.Tbuf;
    wv.pend = ch->ms.pend;
    wv.Wpart = ch->ms.Wpart;
    wv.wtiles = ch->ms.wtiles;
  }
  int cur = 0;
  wv.id_cur = ch->ids[0];
  wv.dir_cur = ch->dirs[0];
  wv.count_cur = ch->counts;
  cudaError_t e = launch_mixed_begin(ds, wv, st);
  if (e != cudaSuccess) return cuda_fail(e, "walk start kernel launch");
  const MixWork mw = s->mixwork(ch->ms);
  cudaEvent_t ev[8] = {};
  if (ch->timing)
    for (auto& x : ev) cudaEventCreate(&x);
  ch->n_other += 2;  // start kernel, count copies aside: F formation + start
  for (long long wave = 0; wave < (1ll << 40); ++wave) {
    e = cudaMemcpyAsync(ch->h_count, ch->counts + cur, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "walk wave count");
    const int count = *ch->h_count;
    if (count <= 0) break;
    wv.id_cur = ch->ids[cur];
    wv.dir_cur = ch->dirs[cur];
    wv.count_cur = ch->counts + cur;
    wv.id_next = ch->ids[cur ^ 1];
    wv.dir_next = ch->dirs[cur ^ 1];
    wv.count_next = ch->counts + (cur ^ 1);
    e = cudaMemsetAsync(wv.count_next, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(wv.ticket, 0, sizeof(int), st);
    if (ch->timing) cudaEventRecord(ev[0], st);
    // V of every listed chain on the tensor cores (CDHR reads V = A_j from
    // the stack instead)
    if (e == cudaSuccess && kind != 2) {
      e = launch_ozaki_form(wv.dir_cur, count, s->n, 0.0, s->A, s->Bsl, s->ecol, s->P, ch->ms.digits,
                            ch->ms.erow, ch->ms.Vrows, s->P, ch->ms.err, st);
      ch->n_form += 2;  // digit slicing + tensor-core formation
    }
    // fresh F(x) of the chains the last wave listed (at most this wave's
    // chains; the list's length is on the device), written into their
    // carried F; then the list starts over for this wave
    if (e == cudaSuccess)
      e = launch_ozaki_form(ch->X, count, s->n, 1.0, s->A, s->Bsl, s->ecol, s->P, ch->ms.digits,
                            ch->ms.erow, ch->F, s->P, ch->ms.err, st, ch->ref_ids, ch->counts + 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(ch->counts + 2, 0, sizeof(int), st);
    ch->n_form += 2;
    if (ch->timing) cudaEventRecord(ev[1], st);
    if (e == cudaSuccess && learned && kind == 0) {
      // warm start: the network's (log t+, u) for every listed chain
      e = launch_learned_features(ch->X, wv.dir_cur, wv.id_cur, count, s->n, s->x_scale,
                                  ch->feats, st);
      if (e != cudaSuccess) return cuda_fail(e, "learned features");
      const float* Y = nullptr;
      int ld = 0;
      if (int r = spg_mlp_infer(s->mlp, count, ch->feats, st, &Y, &ld)) return r;
      wv.pred = Y;
      wv.ld_pred = ld;
      ch->n_mlp += 5;  // features, conversion, 3 GEMMs
    }
    if (ch->timing) cudaEventRecord(ev[2], st);
    // small waves (the tail of chains with many reflections) contract
    // in-kernel: the tensor-core GEMM's cost hardly shrinks with the rows
    const bool defer_now = defer && count > kDeferMinRows;
    wv.pend = defer_now ? ch->ms.pend : nullptr;
    if (e == cudaSuccess) e = launch_mixed_wave(ds, mw, wv, st);
    if (ch->timing) cudaEventRecord(ev[3], st);
    ch->n_wave += 1;
    if (e != cudaSuccess) return cuda_fail(e, "walk wave launch");
    if (defer_now) {
      e = launch_ozaki_contract(ch->ms.Ubuf, count, s->n, s->m, s->Bc, s->ecolc, ch->ms.udig,
                                ch->ms.uerow, ch->ms.Wpart, ch->ms.err, st);
      if (ch->timing) cudaEventRecord(ev[4], st);
      if (e == cudaSuccess) e = launch_mixed_reflect(ds, wv, count, 4 * device_sms(), st);
      if (ch->timing) cudaEventRecord(ev[5], st);
      ch->n_contract += 2;  // digit slicing + tensor-core GEMM
      ch->n_finish += 1;
      if (e != cudaSuccess) return cuda_fail(e, "normal contraction / reflection launch");
    }
    cur ^= 1;
    if (ch->timing) {
      // the next wave's count copy synchronises the stream; read this wave's events
      cudaEventSynchronize(defer_now ? ev[5] : ev[3]);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
      cudaEventElapsedTime(&a0, ev[0], ev[1]);
      cudaEventElapsedTime(&a1, ev[1], ev[2]);
      cudaEventElapsedTime(&a2, ev[2], ev[3]);
      if (defer_now) {
        cudaEventElapsedTime(&a3, ev[3], ev[4]);
        cudaEventElapsedTime(&a4, ev[4], ev[5]);
      }
      ch->t_form_ms += a0;
      ch->t_mlp_ms += a1;
      ch->t_wave_ms += a2;
      ch->t_contract_ms += a3;
      ch->t_finish_ms += a4;
    }
  }
  if (ch->timing)
    for (auto& x : ev) cudaEventDestroy(x);
  int herr = 0;
  e = cudaMemcpyAsync(&herr, ch->ms.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "walk");
  if (herr) return fail(SP_ECUDA, "walk: tensor-core wait limit reached%s");
  ch->step += (uint32_t)steps;
  return SP_OK;
}

static int run_walk(sp_chains* ch, int kind, int steps, double tau, int rho, double kappa,
                    int mode, void* stream, const char* fn) {
  if (!ch) return fail(SP_EINVAL, "%s: null handle", fn);
  if (steps < 0) return fail(SP_EINVAL, "%s: steps < 0", fn);
  if (int r = check_mode(mode, fn)) return r;
  if (steps == 0) return SP_OK;
  sp_spec* s = ch->spec;
  if (mode == SP_MODE_MIXED || mode == SP_MODE_LEARNED)
    return run_walk_mixed(ch, kind, steps, tau, rho, kappa, mode == SP_MODE_LEARNED, stream);
  ch->F_valid = false;  // the FP64 path does not maintain the carried F
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
  wp.seg = ch->seg;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ch->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, (cudaStream_t)stream);
  }
  cudaError_t e = launch_walk_fp64(s->dev(), ch->ws.dev(s->tol), wp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
  ch->n_fp64 += 1;
  if (ch->timing) {
    cudaEventRecord(e1, (cudaStream_t)stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ch->t_fp64_ms += ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
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
  ch->F_valid = false;
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
