// Expected value of the indicator of a union of two half-spaces over the
// chains' current points (Sec. 4.2): f(x) = 1(c.x <= b1 or c.x >= b2), the
// Monte Carlo estimate E_N[f] = (1/N) sum f(x_i) of each group of N chains.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "kernels.h"

extern "C" int spg_set_error(int code, const char* msg);

namespace spg {
namespace {

// one warp per chain: c.x, the indicator, one atomic per chain into its group
__global__ void halfspace_count_kernel(const double* __restrict__ X, int C, int n,
                                       const double* __restrict__ c, double b1, double b2,
                                       int per_group, unsigned long long* __restrict__ hits) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < C; k += warps) {
    double a = 0.0;
    for (int j = lane; j < n; j += 32) a = fma(c[j], X[(size_t)k * n + j], a);
    a = warp_sum(a);
    if (lane == 0 && (a <= b1 || a >= b2)) atomicAdd(&hits[k / per_group], 1ull);
  }
}

}  // namespace
}  // namespace spg

extern "C" int sp_halfspace_fraction(sp_chains* ch, const double* c, double b1, double b2,
                                     int groups, double* frac_out, void* stream) {
  if (!ch || !c || !frac_out || groups < 1)
    return spg_set_error(SP_EINVAL, "sp_halfspace_fraction: bad argument");
  int n = 0, C = 0;
  const double* X = spg::chain_points(ch, &C, &n);
  if (C % groups != 0)
    return spg_set_error(SP_EINVAL, "sp_halfspace_fraction: groups must divide the chains");
  if (!(b1 < b2)) return spg_set_error(SP_EINVAL, "sp_halfspace_fraction: need b1 < b2");
  cudaStream_t st = (cudaStream_t)stream;
  double* dc = nullptr;
  unsigned long long* hits = nullptr;
  if (cudaMalloc(&dc, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&hits, sizeof(unsigned long long) * groups) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dc);
    return spg_set_error(SP_ENOMEM, "sp_halfspace_fraction: allocation failed");
  }
  cudaPointerAttributes at;
  const bool dev = cudaPointerGetAttributes(&at, c) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  cudaError_t e = cudaMemcpyAsync(dc, c, sizeof(double) * n,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(hits, 0, sizeof(unsigned long long) * groups, st);
  if (e == cudaSuccess) {
    int blocks = (C + 7) / 8;
    blocks = blocks < 4096 ? blocks : 4096;
    spg::halfspace_count_kernel<<<blocks, 256, 0, st>>>(X, C, n, dc, b1, b2, C / groups, hits);
    e = cudaGetLastError();
  }
  std::vector<unsigned long long> h(groups);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), hits, sizeof(unsigned long long) * groups,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dc);
  cudaFree(hits);
  if (e != cudaSuccess) return spg_set_error(SP_ECUDA, cudaGetErrorString(e));
  for (int g = 0; g < groups; ++g) frac_out[g] = (double)h[g] / (double)(C / groups);
  return SP_OK;
}
