// Plain FP64 formation of pencil matrices for a batch of coefficient rows:
// Y[r, p] = lead * A[0, p] + sum_j vec[r, j] A[j+1, p]   (Eq. 1 / the pencil
// B_0 + t B_1 of a line).  Used by the FP64 entry points and to refresh the
// carried F(x) of the mixed path.
#include "common.cuh"
#include "kernels.h"

namespace spg {
namespace {

__global__ void form64_kernel(const double* __restrict__ A, long long P, int n,
                              const double* __restrict__ vec, int R, double lead,
                              double* __restrict__ Y, long long ldy) {
  extern __shared__ double coef[];
  const int r = blockIdx.y;
  for (int j = threadIdx.x; j < n; j += blockDim.x) coef[j] = vec[(size_t)r * n + j];
  __syncthreads();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double a0 = lead * A[p], a1 = 0.0;
  int j = 0;
#pragma unroll 4
  for (; j + 1 < n; j += 2) {
    a0 += coef[j] * A[(size_t)(j + 1) * P + p];
    a1 += coef[j + 1] * A[(size_t)(j + 2) * P + p];
  }
  if (j < n) a0 += coef[j] * A[(size_t)(j + 1) * P + p];
  Y[(size_t)r * ldy + p] = a0 + a1;
}

}  // namespace

cudaError_t launch_form64(const double* A, long long P, int n, const double* vec, int R,
                          double lead, double* Y, long long ldy, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  dim3 grid((unsigned)((P + 255) / 256), (unsigned)R);
  form64_kernel<<<grid, 256, (size_t)n * sizeof(double), st>>>(A, P, n, vec, R, lead, Y, ldy);
  return cudaGetLastError();
}

}  // namespace spg
