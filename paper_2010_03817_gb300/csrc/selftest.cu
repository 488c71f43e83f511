// Diagnostic entry point: the reciprocal and reciprocal-square-root routines
// of the dense kernels (dense.cuh, df.cuh), evaluated on caller-given values
// so that tests can bound them against IEEE division and square root.
#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "dense.cuh"
#include "df.cuh"

namespace spg {
namespace {

__global__ void recip_kernel(int count, const double* __restrict__ x, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
    const double v = x[c];
    const dfloat d(v);
    out[4 * (size_t)c + 0] = rsqrt_t(v);
    out[4 * (size_t)c + 1] = recip_t(v);
    out[4 * (size_t)c + 2] = to_double(rsqrt_t(d));
    out[4 * (size_t)c + 3] = to_double(recip_t(d));
  }
}

}  // namespace
}  // namespace spg

extern "C" int spg_set_error(int code, const char* msg);

extern "C" int sp_selftest_recip(int count, const double* x, double* out, void* stream) {
  if (count < 0 || (count > 0 && (!x || !out)))
    return spg_set_error(SP_EINVAL, "sp_selftest_recip: bad argument");
  if (count == 0) return SP_OK;
  int grid = (count + 255) / 256;
  grid = grid < 1024 ? grid : 1024;
  spg::recip_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(count, x, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return spg_set_error(SP_ECUDA, cudaGetErrorString(e));
  return SP_OK;
}
