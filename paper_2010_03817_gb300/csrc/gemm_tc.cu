// BF16 GEMM on the 5th-generation tensor cores (tcgen05.mma, accumulator in
// TMEM) for the learned warm start's MLP:
//   C[M x N] = A[M x K] * B[N x K]^T  (+ bias[N]) (ReLU), FP32 accumulation,
// A and B K-major BF16 in global memory (leading dimensions multiples of 8),
// FP32 and / or BF16 outputs.  Tiles of 128 x 128, K in stages of 64 staged
// through shared memory (double buffered; the tensor core reads stage k while
// the threads fill stage k+1), one elected thread issues the MMAs.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace spg {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kGThreads = 128;

__device__ __forceinline__ uint32_t core_off_g(int r, int g) {
  // [r/8][g][r%8][8 elems]: 8 k-groups of 16 bytes per 8-row group
  return (uint32_t)(((r >> 3) * (kBK / 8) + g) * 128 + (r & 7) * 16);
}

__global__ void __launch_bounds__(kGThreads, 1)
    gemm_bf16_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                     const __nv_bfloat16* __restrict__ B, int ldb, int M, int N, int K,
                     const float* __restrict__ bias, int relu, float* __restrict__ C32, int ldc32,
                     __nv_bfloat16* __restrict__ C16, int ldc16, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr uint32_t a_bytes = kBM * kBK * 2, b_bytes = kBN * kBK * 2;
  uint8_t* sA[2] = {smem, smem + a_bytes};
  uint8_t* sB[2] = {smem + 2 * a_bytes, smem + 2 * a_bytes + b_bytes};
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * a_bytes + 2 * b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  if (wid == 0) {
    tc::tmem_alloc(tmem_slot, kBN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc::idesc_bf16_f32(kBM, kBN);
  const uint32_t sbo = (kBK / 8) * 128;
  const int KT = (K + kBK - 1) / kBK;
  bool ok = true;
  for (int kt = 0; kt < KT; ++kt) {
    const int buf = kt & 1;
    const bool w = kt < 2 || tc::mbar_wait(&mbar[buf], ((kt - 2) >> 1) & 1);
    if (!__syncthreads_and(w)) {  // a block-uniform decision
      ok = false;
      break;
    }
    const int k0 = kt * kBK;
    for (int q = tid; q < kBM * (kBK / 8); q += kGThreads) {
      const int r = q >> 3, g = q & 7;
      uint4 v = make_uint4(0, 0, 0, 0);
      const int k = k0 + g * 8;
      if (m0 + r < M && k < K)
        v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * lda + k);
      *reinterpret_cast<uint4*>(sA[buf] + core_off_g(r, g)) = v;
    }
    for (int q = tid; q < kBN * (kBK / 8); q += kGThreads) {
      const int r = q >> 3, g = q & 7;
      uint4 v = make_uint4(0, 0, 0, 0);
      const int k = k0 + g * 8;
      if (n0 + r < N && k < K)
        v = *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * ldb + k);
      *reinterpret_cast<uint4*>(sB[buf] + core_off_g(r, g)) = v;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_base = tc::smem_u32(sA[buf]), b_base = tc::smem_u32(sB[buf]);
#pragma unroll
      for (int ks = 0; ks < kBK / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(a_base + ks * 256, 128, sbo);
        const uint64_t bd = tc::smem_desc(b_base + ks * 256, 128, sbo);
        tc::mma_bf16(tmem, ad, bd, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
      }
      tc::mma_commit(&mbar[buf]);
    }
  }
  if (ok && KT > 0) ok = tc::mbar_wait(&mbar[(KT - 1) & 1], ((KT - 1) >> 1) & 1);
  ok = __syncthreads_and(ok);  // the epilogue's TMEM loads are warp-collective
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    if (KT > 0) tc::mbar_wait(&mbar[(KT - 1) & 1], ((KT - 1) >> 1) & 1, 1ll << 20);
  }
  tc::fence_after_sync();
  if (ok) {
    const int r = m0 + wid * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(wid * 32) << 16);
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      uint32_t v[16];
      tc::tmem_ld16(lane_base + (uint32_t)c0, v);
      tc::tmem_wait_ld();
      if (r < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = n0 + c0 + i;
          if (c < N) {
            float x = (KT > 0) ? __uint_as_float(v[i]) : 0.f;
            if (bias) x += bias[c];
            if (relu) x = fmaxf(x, 0.f);
            if (C32) C32[(size_t)r * ldc32 + c] = x;
            if (C16) C16[(size_t)r * ldc16 + c] = __float2bfloat16_rn(x);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wid == 0) tc::tmem_dealloc(tmem, kBN);
}

}  // namespace

cudaError_t launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                             const float* bias, int relu, float* C32, int ldc32, void* C16,
                             int ldc16, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)(kBM + kBN) * kBK * 2 + 64;
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM));
  gemm_bf16_kernel<<<grid, kGThreads, smem, st>>>(
      static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B), ldb, M, N,
      K, bias, relu, C32, ldc32, static_cast<__nv_bfloat16*>(C16), ldc16, err);
  return cudaGetLastError();
}

}  // namespace spg
