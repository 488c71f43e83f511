// The learned warm start: a three-layer perceptron
//   Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2),
//   Y  = H2 W3^T + b3,
// that maps a line (x, v) to (log t+, u), the step length to the boundary and
// the null vector there, used to shift the pencil and to start the
// eigen-iteration of the boundary oracle.  Weights and activations are BF16,
// accumulation FP32 on the tensor cores (gemm_tc.cu); FP32 master weights and
// Adam moments.  Training loss per sample:
//   (Y_0 - T_0)^2 + (1 - (a.b)^2/(|a|^2 |b|^2)),  a = Y_1.., b = T_1..
// (the null vector is defined up to sign: squared cosine).
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace spg {
namespace {

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                   long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// rows of din floats -> rows of dinp BF16 (zero padding)
__global__ void f32_to_bf16_pad_kernel(const float* __restrict__ in, int B, int din, int dinp,
                                       __nv_bfloat16* __restrict__ out) {
  const long long n = (long long)B * dinp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / dinp), c = (int)(i % dinp);
    out[i] = __float2bfloat16_rn(c < din ? in[(size_t)r * din + c] : 0.f);
  }
}

// out[c][r] = in[r][c] for an R x C row-major matrix (leading dims ldi, ldo)
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int R, int C, int ldi,
                                      __nv_bfloat16* __restrict__ out, int ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * ldi + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < C && r < R) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
  }
}

// per-sample loss and dL/dY (batch mean); one warp per row.  Y, T and dY16
// share the row stride ld (D <= ld meaningful columns).
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, int B,
                                 int D, int ld, __nv_bfloat16* __restrict__ dY16,
                                 float* __restrict__ loss_acc) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= B) return;
  const float* y = Y + (size_t)r * ld;
  const float* t = T + (size_t)r * ld;
  float ab = 0.f, aa = 0.f, bb = 0.f;
  for (int j = 1 + lane; j < D; j += 32) {
    ab += y[j] * t[j];
    aa += y[j] * y[j];
    bb += t[j] * t[j];
  }
  ab = warp_sum(ab);
  aa = warp_sum(aa);
  bb = warp_sum(bb);
  aa = fmaxf(aa, 1e-30f);
  bb = fmaxf(bb, 1e-30f);
  const float d0 = y[0] - t[0];
  const float cos2 = ab * ab / (aa * bb);
  const float inv_b = 1.0f / (float)B;
  if (lane == 0) {
    atomicAdd(loss_acc, (d0 * d0 + (1.f - cos2)) * inv_b);
    dY16[(size_t)r * ld] = __float2bfloat16_rn(2.f * d0 * inv_b);
  }
  const float c1 = 2.f * ab / (aa * bb), c2 = 2.f * ab * ab / (aa * aa * bb);
  for (int j = 1 + lane; j < D; j += 32)
    dY16[(size_t)r * ld + j] = __float2bfloat16_rn(-(c1 * t[j] - c2 * y[j]) * inv_b);
  for (int j = D + lane; j < ld; j += 32) dY16[(size_t)r * ld + j] = __float2bfloat16_rn(0.f);
}

// dZ = dH * (H > 0), in place on a BF16 buffer; H is the post-ReLU activation
__global__ void relu_back_kernel(__nv_bfloat16* __restrict__ dH, const __nv_bfloat16* __restrict__ H,
                                 long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(H[i]) > 0.f)) dH[i] = __float2bfloat16_rn(0.f);
}

// g[c] = sum_r dZ[r][c]
__global__ void col_sum_kernel(const __nv_bfloat16* __restrict__ dZ, int R, int C, int ld,
                               float* __restrict__ g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += __bfloat162float(dZ[(size_t)r * ld + c]);
  g[c] = s;
}

// Adam on the FP32 master copy; refreshes the BF16 copy (and its transpose
// for weight matrices: W is rows x cols, Wt is cols x rows)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, long long n, float lr,
                            float b1, float b2, float c1, float c2, float eps,
                            __nv_bfloat16* __restrict__ p16, __nv_bfloat16* __restrict__ pt16,
                            int rows, int cols) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float v = p[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    p[i] = v;
    if (p16) p16[i] = __float2bfloat16_rn(v);
    if (pt16) {
      const int r = (int)(i / cols), c = (int)(i % cols);
      pt16[(size_t)c * rows + r] = __float2bfloat16_rn(v);
    }
  }
}

inline int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

cudaError_t launch_f32_to_bf16(const float* in, void* out, long long n, cudaStream_t st) {
  f32_to_bf16_kernel<<<grid_for(n), 256, 0, st>>>(in, static_cast<__nv_bfloat16*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16_pad(const float* in, int B, int din, int dinp, void* out,
                                   cudaStream_t st) {
  f32_to_bf16_pad_kernel<<<grid_for((long long)B * dinp), 256, 0, st>>>(
      in, B, din, dinp, static_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void* in, int R, int C, int ldi, void* out, int ldo,
                                  cudaStream_t st) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  transpose_bf16_kernel<<<grid, block, 0, st>>>(static_cast<const __nv_bfloat16*>(in), R, C, ldi,
                                                static_cast<__nv_bfloat16*>(out), ldo);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const float* Y, const float* T, int B, int D, int ld, void* dY16,
                             float* loss_acc, cudaStream_t st) {
  loss_grad_kernel<<<(B + 7) / 8, 256, 0, st>>>(Y, T, B, D, ld,
                                                static_cast<__nv_bfloat16*>(dY16), loss_acc);
  return cudaGetLastError();
}

cudaError_t launch_relu_back(void* dH, const void* H, long long n, cudaStream_t st) {
  relu_back_kernel<<<grid_for(n), 256, 0, st>>>(static_cast<__nv_bfloat16*>(dH),
                                                static_cast<const __nv_bfloat16*>(H), n);
  return cudaGetLastError();
}

cudaError_t launch_col_sum(const void* dZ, int R, int C, int ld, float* g, cudaStream_t st) {
  col_sum_kernel<<<(C + 127) / 128, 128, 0, st>>>(static_cast<const __nv_bfloat16*>(dZ), R, C, ld,
                                                  g);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, long long n, float lr,
                        float b1, float b2, float c1, float c2, float eps, void* p16, void* pt16,
                        int rows, int cols, cudaStream_t st) {
  adam_kernel<<<grid_for(n), 256, 0, st>>>(p, g, m1, m2, n, lr, b1, b2, c1, c2, eps,
                                           static_cast<__nv_bfloat16*>(p16),
                                           static_cast<__nv_bfloat16*>(pt16), rows, cols);
  return cudaGetLastError();
}

}  // namespace spg
