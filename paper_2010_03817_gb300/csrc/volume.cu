// Volume of a spectrahedron by multiphase Monte Carlo over a sequence of
// balls (Sec. 4.1): with radii r_0 < r_1 < ... < r_q, B(r_0) inside S and S
// inside B(r_q),
//   vol(S) = vol(B(r_0)) * prod_{i=1..q} vol(S cap B(r_i)) / vol(S cap B(r_{i-1})),
// each ratio estimated as 1 / f_i, f_i the fraction of uniform samples of
// S cap B(r_i) that lie in B(r_{i-1}).  S cap B(r) is again a spectrahedron:
// the LMI of S with the ball block [[r, x^T], [x, r I_n]] (positive
// semidefinite iff |x| <= r, by the Schur complement) appended on the
// diagonal, so each phase runs the library's own walks (Alg. 5 or Alg. 4)
// on a freshly created spectrahedron.  The host drives the phases; the
// sampling and the counting run on the GPU.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "kernels.h"

extern "C" int spg_set_error(int code, const char* msg);  // defined in abi.cu

namespace spg {
namespace {

// count of the rows of X (C x n) with |x|^2 <= r2
__global__ void count_in_ball_kernel(const double* __restrict__ X, int C, int n, double r2,
                                     unsigned long long* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= C) return;
  double a = 0.0;
  for (int j = lane; j < n; j += 32) a += X[(size_t)c * n + j] * X[(size_t)c * n + j];
  a = warp_sum(a);
  if (lane == 0 && a <= r2) atomicAdd(count, 1ull);
}

// log of the volume of the n-ball of radius r: pi^(n/2) r^n / Gamma(n/2 + 1)
double log_ball_volume(int n, double r) {
  return 0.5 * n * log(M_PI) + n * log(r) - lgamma(0.5 * n + 1.0);
}

}  // namespace
}  // namespace spg

using spg::tri;

extern "C" {

int sp_volume_estimate(sp_spec* s, double r_inner, double r_outer, double ratio, int chains,
                       int burn_in, int steps, int walk, int mode, uint64_t seed, double* vol,
                       double* info, void* stream) {
  if (!s || !vol) return spg_set_error(SP_EINVAL, "sp_volume_estimate: null argument");
  if (!(r_inner > 0.0) || !(r_outer > r_inner) || !(ratio > 0.0 && ratio < 1.0) || chains < 1 ||
      burn_in < 0 || steps < 1 || (walk != 0 && walk != 1))
    return spg_set_error(SP_EINVAL, "sp_volume_estimate: bad radii, ratio or counts");
  const auto t0 = std::chrono::steady_clock::now();
  int n = 0, m = 0;
  if (int r = sp_spec_dims(s, &n, &m)) return r;
  const long long P = (long long)m * (m + 1) / 2;
  std::vector<double> packed((size_t)(n + 1) * P);
  if (int r = spg::spec_copy_stack(s, packed.data())) return r;
  // q phases: (r_{i-1} / r_i)^n = ratio for a body that fills its balls
  const int q = std::max(1, (int)ceil(n * log(r_outer / r_inner) / -log(ratio)));
  const int mb = n + 1, ma = mb + m;  // ball block, then the LMI of S
  std::vector<double> Aaug((size_t)(n + 1) * ma * ma);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* dcount = nullptr;
  if (cudaMalloc(&dcount, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return spg_set_error(SP_ENOMEM, "sp_volume_estimate: allocation failed");
  }
  double log_vol = spg::log_ball_volume(n, r_inner);
  double rel_var = 0.0;
  int ret = SP_OK;
  for (int i = 1; i <= q && ret == SP_OK; ++i) {
    const double ri = r_inner * pow(r_outer / r_inner, (double)i / q);
    const double rprev = r_inner * pow(r_outer / r_inner, (double)(i - 1) / q);
    // augmented stack: A'_0 = diag(r I_{n+1}, A_0), A'_j = diag(e_0 e_j^T + e_j e_0^T, A_j)
    std::fill(Aaug.begin(), Aaug.end(), 0.0);
    for (int j = 0; j <= n; ++j) {
      double* Aj = Aaug.data() + (size_t)j * ma * ma;
      if (j == 0) {
        for (int d = 0; d < mb; ++d) Aj[(size_t)d * ma + d] = ri;
      } else {
        Aj[j] = 1.0;
        Aj[(size_t)j * ma] = 1.0;
      }
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
          Aj[(size_t)(mb + a) * ma + mb + b] =
              packed[(size_t)j * P + (a >= b ? tri(a, b) : tri(b, a))];
    }
    sp_spec* si = nullptr;
    sp_chains* ch = nullptr;
    ret = sp_create_spectrahedron(n, ma, Aaug.data(), mode == SP_MODE_FP64 ? 1u : 0u, &si);
    if (ret == SP_OK) ret = sp_init_chains(si, chains, nullptr, seed + (uint64_t)i, 0, &ch, stream);
    auto advance = [&](int k) {
      return walk == 0 ? sp_step_billiard(ch, k, 2.0 * ri, 1000, 1e-6, mode, stream)
                       : sp_step_hnr(ch, k, mode, stream);
    };
    if (ret == SP_OK && burn_in > 0) ret = advance(burn_in);
    if (ret == SP_OK && cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), st) != cudaSuccess)
      ret = spg_set_error(SP_ECUDA, "sp_volume_estimate: memset failed");
    for (int t = 0; t < steps && ret == SP_OK; ++t) {
      ret = advance(1);
      if (ret != SP_OK) break;
      const double* X = spg::chain_points(ch);
      spg::count_in_ball_kernel<<<(chains + 7) / 8, 256, 0, st>>>(X, chains, n, rprev * rprev,
                                                                  dcount);
      if (cudaGetLastError() != cudaSuccess)
        ret = spg_set_error(SP_ECUDA, "sp_volume_estimate: count kernel launch failed");
    }
    unsigned long long hc = 0;
    if (ret == SP_OK && (cudaMemcpyAsync(&hc, dcount, sizeof(hc), cudaMemcpyDeviceToHost, st) !=
                             cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
      ret = spg_set_error(SP_ECUDA, "sp_volume_estimate: count copy failed");
    if (ch) sp_destroy_chains(ch);
    if (si) sp_destroy_spectrahedron(si);
    if (ret != SP_OK) break;
    const double N = (double)chains * steps;
    const double f = (double)hc / N;
    if (!(f > 0.0)) {
      ret = spg_set_error(SP_EINVAL,
                             "sp_volume_estimate: no sample in the smaller ball (ratio too small)");
      break;
    }
    log_vol -= log(f);
    rel_var += (1.0 - f) / (f * N);
  }
  cudaFree(dcount);
  if (ret != SP_OK) return ret;
  *vol = exp(log_vol);
  if (info) {
    info[0] = q;
    info[1] = (double)chains * steps;
    info[2] = sqrt(rel_var);
    info[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return SP_OK;
}

}  // extern "C"
