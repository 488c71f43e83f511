// C ABI of the warm-start network (include/spectra_gb.h, sp_mlp_*): handle,
// forward pass, gradients, Adam steps and training loop on the GPU.  All the
// arithmetic runs in gemm_tc.cu (tcgen05 GEMMs) and mlp.cu (elementwise).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <random>
#include <vector>

#include "../../include/spectra_gb.h"
#include "kernels.h"

using namespace spg;

extern "C" int spg_set_error(int code, const char* msg);

namespace {

int mlp_fail(int code, const char* msg) { return spg_set_error(code, msg); }

inline int round8(int x) { return (x + 7) / 8 * 8; }
inline int round16(int x) { return (x + 15) / 16 * 16; }

}  // namespace

struct sp_mlp {
  int din = 0, dinp = 0, dh = 0, dout = 0, doutp = 0, cap = 0;
  size_t offs[7] = {0};  // W1, b1, W2, b2, W3, b3, total (floats, master layout)
  float* P = nullptr;
  float* G = nullptr;
  float* M1 = nullptr;
  float* M2 = nullptr;
  void* W16[3] = {nullptr, nullptr, nullptr};  // BF16 weights (rows x cols)
  void* Wt16[3] = {nullptr, nullptr, nullptr};  // BF16 transposes
  // activations (cap rows)
  void* X16 = nullptr;
  void* H1 = nullptr;
  void* H2 = nullptr;
  float* Y = nullptr;
  void* dY = nullptr;
  void* dH2 = nullptr;
  void* dH1 = nullptr;
  void* Tr = nullptr;   // transpose scratch (largest: dh x cap)
  void* Tr2 = nullptr;  // second transpose scratch
  float* Tpad = nullptr;  // targets padded (cap x doutp)
  float* loss = nullptr;
  int* err = nullptr;
  long long t = 0;  // Adam step
  size_t rows(int l) const { return l == 0 ? dh : l == 1 ? dh : doutp; }
  size_t cols(int l) const { return l == 0 ? dinp : dh; }
};

static void mlp_free_acts(sp_mlp* q) {
  void* ps[] = {q->X16, q->H1, q->H2, q->Y, q->dY, q->dH2, q->dH1, q->Tr, q->Tr2, q->Tpad};
  for (void* p : ps) cudaFree(p);
  q->X16 = q->H1 = q->H2 = q->dY = q->dH2 = q->dH1 = q->Tr = q->Tr2 = nullptr;
  q->Y = q->Tpad = nullptr;
  q->cap = 0;
}

static int mlp_ensure(sp_mlp* q, int rows) {
  if (rows <= q->cap) return SP_OK;
  mlp_free_acts(q);
  const int cap = round8(rows);
  const size_t bf = 2;
  bool ok = cudaMalloc(&q->X16, bf * cap * q->dinp) == cudaSuccess &&
            cudaMalloc(&q->H1, bf * cap * q->dh) == cudaSuccess &&
            cudaMalloc(&q->H2, bf * cap * q->dh) == cudaSuccess &&
            cudaMalloc(&q->Y, sizeof(float) * cap * q->doutp) == cudaSuccess &&
            cudaMalloc(&q->dY, bf * cap * q->doutp) == cudaSuccess &&
            cudaMalloc(&q->dH2, bf * cap * q->dh) == cudaSuccess &&
            cudaMalloc(&q->dH1, bf * cap * q->dh) == cudaSuccess &&
            cudaMalloc(&q->Tr, bf * (size_t)cap * std::max(q->dh, std::max(q->dinp, q->doutp))) ==
                cudaSuccess &&
            cudaMalloc(&q->Tr2, bf * (size_t)cap * std::max(q->dh, q->dinp)) == cudaSuccess &&
            cudaMalloc(&q->Tpad, sizeof(float) * cap * q->doutp) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlp_free_acts(q);
    return mlp_fail(SP_ENOMEM, "sp_mlp: activation allocation failed");
  }
  q->cap = cap;
  return SP_OK;
}

// refresh the BF16 weights and their transposes from the master copy
static cudaError_t mlp_sync_weights(sp_mlp* q, cudaStream_t st) {
  for (int l = 0; l < 3; ++l) {
    const size_t n = q->rows(l) * q->cols(l);
    cudaError_t e = launch_f32_to_bf16(q->P + q->offs[2 * l], q->W16[l], (long long)n, st);
    if (e == cudaSuccess)
      e = launch_transpose_bf16(q->W16[l], (int)q->rows(l), (int)q->cols(l), (int)q->cols(l),
                                q->Wt16[l], (int)q->rows(l), st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t mlp_forward(sp_mlp* q, int B, const float* X, cudaStream_t st) {
  cudaError_t e = launch_f32_to_bf16_pad(X, B, q->din, q->dinp, q->X16, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->X16, q->dinp, q->W16[0], q->dinp, B, q->dh, q->dinp, q->P + q->offs[1],
                         1, nullptr, 0, q->H1, q->dh, q->err, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->H1, q->dh, q->W16[1], q->dh, B, q->dh, q->dh, q->P + q->offs[3], 1,
                         nullptr, 0, q->H2, q->dh, q->err, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->H2, q->dh, q->W16[2], q->dh, B, q->doutp, q->dh, q->P + q->offs[5], 0,
                         q->Y, q->doutp, nullptr, 0, q->err, st);
  return e;
}

// gradients of the batch-mean loss into q->G (after a forward pass on X)
static cudaError_t mlp_backward(sp_mlp* q, int B, const float* Tpad, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(q->loss, 0, sizeof(float), st);
  if (e == cudaSuccess) e = launch_loss_grad(q->Y, Tpad, B, q->dout, q->doutp, q->dY, q->loss, st);
  // layer 3: gW3 = dY^T H2, gb3 = colsum(dY), dH2 = dY W3
  if (e == cudaSuccess) e = launch_transpose_bf16(q->dY, B, q->doutp, q->doutp, q->Tr, B, st);
  if (e == cudaSuccess) e = launch_transpose_bf16(q->H2, B, q->dh, q->dh, q->Tr2, B, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->Tr, B, q->Tr2, B, q->doutp, q->dh, B, nullptr, 0, q->G + q->offs[4],
                         q->dh, nullptr, 0, q->err, st);
  if (e == cudaSuccess) e = launch_col_sum(q->dY, B, q->doutp, q->doutp, q->G + q->offs[5], st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->dY, q->doutp, q->Wt16[2], q->doutp, B, q->dh, q->doutp, nullptr, 0,
                         nullptr, 0, q->dH2, q->dh, q->err, st);
  if (e == cudaSuccess) e = launch_relu_back(q->dH2, q->H2, (long long)B * q->dh, st);
  // layer 2
  if (e == cudaSuccess) e = launch_transpose_bf16(q->dH2, B, q->dh, q->dh, q->Tr, B, st);
  if (e == cudaSuccess) e = launch_transpose_bf16(q->H1, B, q->dh, q->dh, q->Tr2, B, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->Tr, B, q->Tr2, B, q->dh, q->dh, B, nullptr, 0, q->G + q->offs[2],
                         q->dh, nullptr, 0, q->err, st);
  if (e == cudaSuccess) e = launch_col_sum(q->dH2, B, q->dh, q->dh, q->G + q->offs[3], st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->dH2, q->dh, q->Wt16[1], q->dh, B, q->dh, q->dh, nullptr, 0, nullptr, 0,
                         q->dH1, q->dh, q->err, st);
  if (e == cudaSuccess) e = launch_relu_back(q->dH1, q->H1, (long long)B * q->dh, st);
  // layer 1
  if (e == cudaSuccess) e = launch_transpose_bf16(q->dH1, B, q->dh, q->dh, q->Tr, B, st);
  if (e == cudaSuccess) e = launch_transpose_bf16(q->X16, B, q->dinp, q->dinp, q->Tr2, B, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(q->Tr, B, q->Tr2, B, q->dh, q->dinp, B, nullptr, 0, q->G + q->offs[0],
                         q->dinp, nullptr, 0, q->err, st);
  if (e == cudaSuccess) e = launch_col_sum(q->dH1, B, q->dh, q->dh, q->G + q->offs[1], st);
  return e;
}

static cudaError_t mlp_adam(sp_mlp* q, float lr, cudaStream_t st) {
  q->t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)q->t), c2 = 1.f - powf(b2, (float)q->t);
  for (int l = 0; l < 3; ++l) {
    const size_t wo = q->offs[2 * l], bo = q->offs[2 * l + 1];
    const size_t nw = q->rows(l) * q->cols(l), nb = q->rows(l);
    cudaError_t e = launch_adam(q->P + wo, q->G + wo, q->M1 + wo, q->M2 + wo, (long long)nw, lr, b1,
                                b2, c1, c2, eps, q->W16[l], q->Wt16[l], (int)q->rows(l),
                                (int)q->cols(l), st);
    if (e == cudaSuccess)
      e = launch_adam(q->P + bo, q->G + bo, q->M1 + bo, q->M2 + bo, (long long)nb, lr, b1, b2, c1,
                      c2, eps, nullptr, nullptr, 1, (int)nb, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// pad targets (count x dout) to (count x doutp)
static cudaError_t mlp_pad_targets(sp_mlp* q, int B, const float* T, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(q->Tpad, 0, sizeof(float) * (size_t)B * q->doutp, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(q->Tpad, sizeof(float) * q->doutp, T, sizeof(float) * q->dout,
                          sizeof(float) * q->dout, B, cudaMemcpyDeviceToDevice, st);
  return e;
}

int spg_mlp_infer(sp_mlp* q, int B, const float* X, cudaStream_t st, const float** Y, int* ld) {
  if (int r = mlp_ensure(q, B)) return r;
  if (mlp_forward(q, B, X, st) != cudaSuccess)
    return mlp_fail(SP_ECUDA, "warm-start network: launch failed");
  *Y = q->Y;
  *ld = q->doutp;
  return SP_OK;
}

int spg_mlp_io(const sp_mlp* q, int* din, int* dout) {
  *din = q->din;
  *dout = q->dout;
  return SP_OK;
}

extern "C" {

int sp_mlp_create(int din, int dh, int dout, uint64_t seed, sp_mlp** out) {
  if (!out || din < 1 || dh < 8 || dout < 2 || dh % 8)
    return mlp_fail(SP_EINVAL, "sp_mlp_create: din >= 1, dh >= 8 a multiple of 8, dout >= 2");
  sp_mlp* q = new sp_mlp();
  q->din = din;
  q->dinp = round8(din);
  q->dh = dh;
  q->dout = dout;
  q->doutp = round16(dout);
  size_t o = 0;
  const size_t sizes[6] = {(size_t)dh * q->dinp, (size_t)dh, (size_t)dh * dh, (size_t)dh,
                           (size_t)q->doutp * dh, (size_t)q->doutp};
  for (int i = 0; i < 6; ++i) {
    q->offs[i] = o;
    o += sizes[i];
  }
  q->offs[6] = o;
  // He initialisation (seeded); padded output rows stay zero
  std::vector<float> h(o, 0.f);
  std::mt19937_64 rng(seed);
  const int fan_in[3] = {din, dh, dh};
  const int ld[3] = {q->dinp, dh, dh};
  for (int l = 0; l < 3; ++l) {
    std::normal_distribution<float> nd(0.f, sqrtf(2.f / fan_in[l]));
    const size_t r = (l == 2) ? (size_t)dout : (size_t)dh;
    for (size_t i = 0; i < r; ++i)
      for (int c = 0; c < fan_in[l]; ++c) h[q->offs[2 * l] + i * ld[l] + c] = nd(rng);
  }
  bool ok = cudaMalloc(&q->P, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&q->G, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&q->M1, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&q->M2, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&q->loss, sizeof(float)) == cudaSuccess &&
            cudaMalloc(&q->err, sizeof(int)) == cudaSuccess;
  for (int l = 0; l < 3 && ok; ++l)
    ok = cudaMalloc(&q->W16[l], 2 * q->rows(l) * q->cols(l)) == cudaSuccess &&
         cudaMalloc(&q->Wt16[l], 2 * q->rows(l) * q->cols(l)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sp_mlp_destroy(q);
    return mlp_fail(SP_ENOMEM, "sp_mlp_create: allocation failed");
  }
  cudaMemcpy(q->P, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  cudaMemset(q->G, 0, sizeof(float) * o);
  cudaMemset(q->M1, 0, sizeof(float) * o);
  cudaMemset(q->M2, 0, sizeof(float) * o);
  cudaMemset(q->err, 0, sizeof(int));
  cudaError_t e = mlp_sync_weights(q, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    sp_mlp_destroy(q);
    return mlp_fail(SP_ECUDA, "sp_mlp_create: weight upload failed");
  }
  *out = q;
  return SP_OK;
}

int sp_mlp_destroy(sp_mlp* q) {
  if (!q) return mlp_fail(SP_EINVAL, "sp_mlp_destroy: null handle");
  mlp_free_acts(q);
  cudaFree(q->P); cudaFree(q->G); cudaFree(q->M1); cudaFree(q->M2);
  cudaFree(q->loss); cudaFree(q->err);
  for (int l = 0; l < 3; ++l) {
    cudaFree(q->W16[l]);
    cudaFree(q->Wt16[l]);
  }
  delete q;
  return SP_OK;
}

int sp_mlp_dims(const sp_mlp* q, int* din, int* dh, int* dout, long long* nparams) {
  if (!q) return mlp_fail(SP_EINVAL, "sp_mlp_dims: null handle");
  if (din) *din = q->din;
  if (dh) *dh = q->dh;
  if (dout) *dout = q->dout;
  if (nparams) *nparams = (long long)q->offs[6];
  return SP_OK;
}

int sp_mlp_params(sp_mlp* q, float* host_out, const float* host_in) {
  if (!q) return mlp_fail(SP_EINVAL, "sp_mlp_params: null handle");
  const size_t n = q->offs[6];
  if (host_out && cudaMemcpy(host_out, q->P, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(SP_ECUDA, "sp_mlp_params: copy failed");
  if (host_in) {
    if (cudaMemcpy(q->P, host_in, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        mlp_sync_weights(q, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return mlp_fail(SP_ECUDA, "sp_mlp_params: upload failed");
  }
  return SP_OK;
}

// file format: 8-byte magic "SPMLP\0\1\0", int32 din, dh, dout, int64 number
// of parameters, then the FP32 parameters (little-endian, the layout of
// sp_mlp_params)
static const char kMlpMagic[8] = {'S', 'P', 'M', 'L', 'P', 0, 1, 0};

int sp_mlp_save(sp_mlp* q, const char* path) {
  if (!q || !path) return mlp_fail(SP_EINVAL, "sp_mlp_save: null argument");
  const long long n = (long long)q->offs[6];
  std::vector<float> h((size_t)n);
  if (int r = sp_mlp_params(q, h.data(), nullptr)) return r;
  FILE* f = fopen(path, "wb");
  if (!f) return mlp_fail(SP_EINVAL, "sp_mlp_save: cannot open the file");
  const int32_t dims[3] = {q->din, q->dh, q->dout};
  bool ok = fwrite(kMlpMagic, 1, 8, f) == 8 && fwrite(dims, sizeof(int32_t), 3, f) == 3 &&
            fwrite(&n, sizeof(n), 1, f) == 1 &&
            fwrite(h.data(), sizeof(float), (size_t)n, f) == (size_t)n;
  ok = (fclose(f) == 0) && ok;
  return ok ? SP_OK : mlp_fail(SP_EINVAL, "sp_mlp_save: write failed");
}

int sp_mlp_load(const char* path, uint64_t seed, sp_mlp** out) {
  if (!path || !out) return mlp_fail(SP_EINVAL, "sp_mlp_load: null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return mlp_fail(SP_EINVAL, "sp_mlp_load: cannot open the file");
  char magic[8];
  int32_t dims[3];
  long long n = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMlpMagic, 8) == 0 &&
            fread(dims, sizeof(int32_t), 3, f) == 3 && fread(&n, sizeof(n), 1, f) == 1 &&
            n > 0 && n < (1ll << 34);
  std::vector<float> h;
  if (ok) {
    h.resize((size_t)n);
    ok = fread(h.data(), sizeof(float), (size_t)n, f) == (size_t)n;
  }
  fclose(f);
  if (!ok) return mlp_fail(SP_EINVAL, "sp_mlp_load: not a network file or truncated");
  sp_mlp* q = nullptr;
  if (int r = sp_mlp_create(dims[0], dims[1], dims[2], seed, &q)) return r;
  if ((long long)q->offs[6] != n) {
    sp_mlp_destroy(q);
    return mlp_fail(SP_EINVAL, "sp_mlp_load: parameter count does not match the dimensions");
  }
  if (int r = sp_mlp_params(q, nullptr, h.data())) {
    sp_mlp_destroy(q);
    return r;
  }
  *out = q;
  return SP_OK;
}

int sp_mlp_forward(sp_mlp* q, int count, const float* X, float* Y, void* stream) {
  if (!q || count < 0 || (count > 0 && (!X || !Y)))
    return mlp_fail(SP_EINVAL, "sp_mlp_forward: bad argument");
  if (count == 0) return SP_OK;
  if (int r = mlp_ensure(q, count)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = mlp_forward(q, count, X, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(Y, sizeof(float) * q->dout, q->Y, sizeof(float) * q->doutp,
                          sizeof(float) * q->dout, count, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return mlp_fail(SP_ECUDA, "sp_mlp_forward: launch failed");
  return SP_OK;
}

int sp_mlp_gradients(sp_mlp* q, int count, const float* X, const float* T, float* grads_host,
                     float* loss_host, void* stream) {
  if (!q || count < 8 || count % 8 || !X || !T)
    return mlp_fail(SP_EINVAL, "sp_mlp_gradients: count must be a positive multiple of 8");
  if (int r = mlp_ensure(q, count)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = mlp_pad_targets(q, count, T, st);
  if (e == cudaSuccess) e = mlp_forward(q, count, X, st);
  if (e == cudaSuccess) e = mlp_backward(q, count, q->Tpad, st);
  if (e == cudaSuccess && loss_host)
    e = cudaMemcpyAsync(loss_host, q->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grads_host)
    e = cudaMemcpyAsync(grads_host, q->G, sizeof(float) * q->offs[6], cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return mlp_fail(SP_ECUDA, "sp_mlp_gradients: launch failed");
  return SP_OK;
}

int sp_mlp_train(sp_mlp* q, int count, const float* X, const float* T, int epochs, int batch,
                 float lr, float* losses_host, void* stream) {
  if (!q || count < batch || batch < 8 || batch % 8 || epochs < 1 || !X || !T)
    return mlp_fail(SP_EINVAL, "sp_mlp_train: bad argument (batch: multiple of 8, <= count)");
  if (int r = mlp_ensure(q, batch)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = count / batch;
  for (int ep = 0; ep < epochs; ++ep) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
      const float* Xb = X + (size_t)b * batch * q->din;
      const float* Tb = T + (size_t)b * batch * q->dout;
      cudaError_t e = mlp_pad_targets(q, batch, Tb, st);
      if (e == cudaSuccess) e = mlp_forward(q, batch, Xb, st);
      if (e == cudaSuccess) e = mlp_backward(q, batch, q->Tpad, st);
      if (e == cudaSuccess) e = mlp_adam(q, lr, st);
      float l = 0.f;
      if (e == cudaSuccess && losses_host && b == nb - 1) {
        e = cudaMemcpyAsync(&l, q->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        acc = l;
      }
      if (e != cudaSuccess) return mlp_fail(SP_ECUDA, "sp_mlp_train: launch failed");
    }
    if (losses_host) losses_host[ep] = (float)acc;
  }
  int herr = 0;
  if (cudaMemcpy(&herr, q->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || herr)
    return mlp_fail(SP_ECUDA, "sp_mlp_train: tensor-core wait limit reached");
  return SP_OK;
}

}  // extern "C"
