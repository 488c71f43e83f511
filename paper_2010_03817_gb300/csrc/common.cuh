// Shared device helpers of the spectrahedron library: counter-based random
// numbers, CTA reductions, packed-triangle indexing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef SPG_THREADS
#define SPG_THREADS 512
#endif
#define SPG_WARPS (SPG_THREADS / 32)
// scratch of the blocked triangular solves: (SPG_WARPS + 1) x 32 partial sums
#define SPG_SCR ((SPG_WARPS + 2) * 32)

namespace spg {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplies with the Weyl-sequence key schedule.
// Counter = (chain, step, stream, index), key = (seed low, seed high).
// ---------------------------------------------------------------------------
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    u32x4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// 52 random bits -> (2k+1) * 2^-53: exact, strictly inside (0,1)
__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return (double)(2 * k + 1) * 0x1p-53;
}

enum Stream : uint32_t { kStreamDir = 0, kStreamEta = 1, kStreamCoord = 2 };

__device__ __forceinline__ double rng_uniform(uint64_t seed, uint32_t chain, uint32_t step,
                                              uint32_t stream) {
  u32x4 r = philox10({chain, step, stream, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
  return u01(r.x, r.y);
}

// Gaussian pair i of the direction draw (Box-Muller)
__device__ __forceinline__ void rng_gauss_pair(uint64_t seed, uint32_t chain, uint32_t step,
                                               uint32_t i, double* g0, double* g1) {
  u32x4 r = philox10({chain, step, (uint32_t)kStreamDir, i}, (uint32_t)seed,
                     (uint32_t)(seed >> 32));
  double u1 = u01(r.x, r.y), u2 = u01(r.z, r.w);
  double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincos(6.283185307179586476925286766559 * u2, &s, &c);
  *g0 = rad * c;
  *g1 = rad * s;
}

// ---------------------------------------------------------------------------
// CTA-wide reductions (blockDim.x == SPG_THREADS)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide: ask the L2 to fetch [p, p + bytes) (one prefetch per 128-byte
// line), so that later passes over the range find it there instead of
// paying the DRAM latency row by row
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)blockDim.x * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// broadcast from lane src (overloaded for the double-float type)
__device__ __forceinline__ float shfl_idx(float v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ double shfl_idx(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// sum over the CTA; red must hold SPG_WARPS elements; result broadcast to all
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
#pragma unroll
  for (int i = 0; i < SPG_WARPS; ++i) s += red[i];
  return s;
}

// CTA-wide: the slot of the calling segment in a sampled segment record, or -1
// (thread 0 takes the ticket; `ib` is a shared int used for the broadcast)
template <typename Log>
__device__ __forceinline__ int seglog_slot(const Log& lg, int* ib) {
  if (!lg.buf) return -1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k = atomicAdd(lg.count, 1);
    *ib = (k % lg.every == 0 && k / lg.every < lg.cap) ? k / lg.every : -1;
  }
  __syncthreads();
  const int slot = *ib;
  __syncthreads();
  return slot;
}

// CTA-wide: write one segment record (layout of SegLog in kernels.h)
template <typename Log>
__device__ __forceinline__ void seglog_write(const Log& lg, int slot, int n, const double* p,
                                             const double* v, const double* wh, double t_plus,
                                             double t_minus, int status, int reflected,
                                             uint32_t chain, uint32_t step, int kseg,
                                             int flags) {
  double* r = lg.buf + (size_t)slot * (3 * (size_t)n + 8);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    r[j] = p[j];
    r[n + j] = v[j];
    r[2 * n + j] = wh ? wh[j] : 0.0;
  }
  if (threadIdx.x == 0) {
    r[3 * n] = t_plus;
    r[3 * n + 1] = t_minus;
    r[3 * n + 2] = (double)status;
    r[3 * n + 3] = (double)reflected;
    r[3 * n + 4] = (double)chain;
    r[3 * n + 5] = (double)step;
    r[3 * n + 6] = (double)kseg;
    r[3 * n + 7] = (double)flags;
  }
}

// packed lower triangle, row-major: element (i, k), i >= k
__host__ __device__ __forceinline__ size_t tri(int i, int k) {
  return (size_t)i * (size_t)(i + 1) / 2 + (size_t)k;
}

}  // namespace spg
