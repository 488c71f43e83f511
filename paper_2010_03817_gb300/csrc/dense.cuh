// CTA-wide dense kernels on one chain's matrices: packed Cholesky, inverse of
// the 32x32 diagonal blocks, blocked triangular solves, full GEMV.
// All routines are called by every thread of a CTA of SPG_THREADS threads.
//
// Storage: lower triangle packed row-major, element (i, k) at i(i+1)/2 + k.
// After factor_cholesky + invert_diag_blocks the diagonal 32x32 blocks hold
// the inverses of the corresponding blocks of L; the off-diagonal blocks hold
// L.  The triangular solves use exactly that layout.
#pragma once
#include "common.cuh"

namespace spg {

constexpr int kBlk = 32;

// 1/sqrt(x) and 1/x: an FP32 seed refined by Newton steps in T (FP64 division
// and square root are long instruction sequences on this GPU's narrow FP64
// pipe; two Newton steps from 2^-23 reach full double precision)
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) {
  double r = (double)rsqrtf((float)x);
  r = r * (1.5 - 0.5 * x * r * r);
  r = r * (1.5 - 0.5 * x * r * r);
  return r;
}
__device__ __forceinline__ float recip_t(float x) { return 1.0f / x; }
__device__ __forceinline__ double recip_t(double x) {
  double r = (double)(1.0f / (float)x);
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
}

// In-place Cholesky G = L L^T of the packed lower triangle G (m x m),
// right-looking in panels of kPanel columns: the panel is factored column by
// column, then the trailing matrix receives one rank-kPanel update (kPanel
// FMAs per load and store of G).
// pan: scratch of kPanel * m elements (the panel, transposed).
// Returns true on success (CTA-uniform); on failure *flag = 1 + the first
// column whose pivot was not positive.
constexpr int kPanel = 4;
template <typename T>
__device__ bool factor_cholesky(T* G, int m, T* pan, int* flag) {
  const int tid = threadIdx.x;
  for (int jb = 0; jb < m; jb += kPanel) {
    const int nb = min(kPanel, m - jb);
    // ---- panel: columns jb .. jb+nb-1 -------------------------------------
    for (int c = 0; c < nb; ++c) {
      const int j = jb + c;
      if (tid == 0) {
        const T dj = G[tri(j, j)];
        // the FP32 seed of rsqrt_t needs dj inside the FP32 range
        if (!(dj > T(1e-37)) || !(dj < T(3e37))) {
          *flag = j + 1;
        } else {
          const T r = rsqrt_t(dj);  // 1/l
          G[tri(j, j)] = dj * r;    // l = sqrt(dj)
          pan[c * m + j] = r;
        }
      }
      __syncthreads();
      if (*flag) return false;
      const T rl = pan[c * m + j];
      for (int i = j + 1 + tid; i < m; i += SPG_THREADS) {
        const T v = G[tri(i, j)] * rl;
        G[tri(i, j)] = v;
        pan[c * m + i] = v;
      }
      __syncthreads();
      // remaining panel columns: G[i][jb+c2] -= L[i][j] L[jb+c2][j], i >= jb + c2
      const int rest = nb - 1 - c;
      if (rest > 0) {
        const int rows = m - (j + 1);
        for (int q = tid; q < rows * rest; q += SPG_THREADS) {
          const int i = j + 1 + q / rest;
          const int c2 = c + 1 + q % rest;
          const int k = jb + c2;
          if (i >= k) G[tri(i, k)] -= pan[c * m + i] * pan[c * m + k];
        }
        __syncthreads();
      }
    }
    // ---- trailing update, rows / columns >= j0: rank-nb --------------------
    const int j0 = jb + nb;
    const int s = m - j0;
    if (s <= 0) break;
    const int total = s * (s + 1) / 2;
    if (tid < total) {
      int i = j0, off = tid;  // element (i, j0 + off)
      while (off > i - j0) {
        off -= i - j0 + 1;
        ++i;
      }
      for (int q = tid; q < total; q += SPG_THREADS) {
        const int k = j0 + off;
        T acc = G[tri(i, k)];
#pragma unroll
        for (int c = 0; c < kPanel; ++c)
          if (c < nb) acc -= pan[c * m + i] * pan[c * m + k];
        G[tri(i, k)] = acc;
        off += SPG_THREADS;
        while (i < m && off > i - j0) {
          off -= i - j0 + 1;
          ++i;
        }
      }
    }
    __syncthreads();
  }
  return true;
}

// Replace each diagonal 32x32 block D of the packed factor by D^{-1} (lower
// triangular), in place.  One warp per block; row r of the inverse is built
// from the rows above it (D X = I, forward substitution by rows).
template <typename T>
__device__ void invert_diag_blocks(T* L, int m) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = (m + kBlk - 1) / kBlk;
  for (int b = wid; b < nb; b += SPG_WARPS) {
    const int r0 = b * kBlk;
    const int bs = min(kBlk, m - r0);
    for (int r = 0; r < bs; ++r) {
      // X[r][c] = -(sum_{k=c}^{r-1} D[r][k] X[k][c]) / D[r][r], X[r][r] = 1/D[r][r]
      T val = T(0);
      const T rdrr = recip_t(L[tri(r0 + r, r0 + r)]);
      if (lane < r) {
        T acc = T(0);
        for (int k = lane; k < r; ++k) acc += L[tri(r0 + r, r0 + k)] * L[tri(r0 + k, r0 + lane)];
        val = -acc * rdrr;
      } else if (lane == r) {
        val = rdrr;
      }
      __syncwarp();
      if (lane <= r) L[tri(r0 + r, r0 + lane)] = val;
      __syncwarp();
    }
  }
  __syncthreads();
}

// x <- L^{-1} x (forward), using inverted diagonal blocks.  s: scratch >= 32.
template <typename T>
__device__ void solve_lower(const T* L, T* x, int m, T* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = (m + kBlk - 1) / kBlk;
  for (int b = 0; b < nb; ++b) {
    const int r0 = b * kBlk;
    const int bs = min(kBlk, m - r0);
    // s_r = x_r - sum_{k < r0} L[r][k] x_k
    for (int rr = wid; rr < bs; rr += SPG_WARPS) {
      const int r = r0 + rr;
      const T* row = L + tri(r, 0);
      T acc = T(0);
      for (int k = lane; k < r0; k += 32) acc += row[k] * x[k];
      acc = warp_sum(acc);
      if (lane == 0) s[rr] = x[r] - acc;
    }
    __syncthreads();
    if (wid == 0 && lane < bs) {
      const T* row = L + tri(r0 + lane, r0);
      T acc = T(0);
      for (int c = 0; c <= lane; ++c) acc += row[c] * s[c];
      x[r0 + lane] = acc;
    }
    __syncthreads();
  }
}

// x <- L^{-T} x (backward), using inverted diagonal blocks.
// s: scratch >= SPG_WARPS*32 + 32.
template <typename T>
__device__ void solve_upper(const T* L, T* x, int m, T* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = (m + kBlk - 1) / kBlk;
  T* part = s + kBlk;
  for (int b = nb - 1; b >= 0; --b) {
    const int r0 = b * kBlk;
    const int bs = min(kBlk, m - r0);
    const int i = r0 + lane;
    // partial sums of sum_{r >= r0+bs} L[r][i] x_r, rows split over warps
    T acc = T(0);
    if (lane < bs)
      for (int r = r0 + bs + wid; r < m; r += SPG_WARPS) acc += L[tri(r, i)] * x[r];
    part[wid * kBlk + lane] = acc;
    __syncthreads();
    if (wid == 0 && lane < bs) {
      T t = x[i];
#pragma unroll
      for (int w = 0; w < SPG_WARPS; ++w) t -= part[w * kBlk + lane];
      s[lane] = t;
    }
    __syncthreads();
    if (wid == 0 && lane < bs) {
      // z_i = sum_{r >= i in block} Dinv[r][i] s_r
      T z = T(0);
      for (int rr = lane; rr < bs; ++rr) z += L[tri(r0 + rr, i)] * s[rr];
      x[i] = z;
    }
    __syncthreads();
  }
}

// y <- alpha * (A x), A full m x m row-major (global memory), one warp per row.
template <typename T>
__device__ void gemv_full(const T* __restrict__ A, const T* x, T* y, int m, T alpha) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = wid; r < m; r += SPG_WARPS) {
    const T* row = A + (size_t)r * m;
    T a0 = T(0), a1 = T(0);
    int k = lane;
    for (; k + 32 < m; k += 64) {
      a0 += row[k] * x[k];
      a1 += row[k + 32] * x[k + 32];
    }
    if (k < m) a0 += row[k] * x[k];
    const T acc = warp_sum(a0 + a1);
    if (lane == 0) y[r] = alpha * acc;
  }
  __syncthreads();
}

// y <- alpha * (V z) for V symmetric, stored as a packed lower triangle
// (shared or global memory).  One pass over the triangle: a warp reads row r
// (coalesced) and uses V[r][k] twice, for y_r and for y_k (k < r), keeping the
// second kind of contribution in per-lane registers (m <= 32 * kMaxColBlocks).
// part: scratch of SPG_WARPS * m elements.
constexpr int kMaxColBlocks = 16;
template <typename T>
__device__ void symv_packed(const T* __restrict__ V, const T* z, T* y, int m, T alpha, T* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T cacc[kMaxColBlocks];
#pragma unroll
  for (int i = 0; i < kMaxColBlocks; ++i) cacc[i] = T(0);
  for (int r = wid; r < m; r += SPG_WARPS) {
    const T* row = V + tri(r, 0);
    const T zr = z[r];
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < kMaxColBlocks; ++i) {
      const int k = lane + 32 * i;
      if (k <= r) {
        const T a = row[k];
        acc += a * z[k];
        if (k < r) cacc[i] += a * zr;
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) y[r] = acc;  // row part; column parts added below
  }
#pragma unroll
  for (int i = 0; i < kMaxColBlocks; ++i) {
    const int k = lane + 32 * i;
    if (k < m) part[wid * m + k] = cacc[i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += SPG_THREADS) {
    T s = y[k];
#pragma unroll
    for (int w = 0; w < SPG_WARPS; ++w) s += part[w * m + k];
    y[k] = alpha * s;
  }
  __syncthreads();
}

// y <- L^T x for the packed lower factor L (before invert_diag_blocks).
// part: scratch of SPG_WARPS * m elements.
template <typename T>
__device__ void mul_upper(const T* L, const T* x, T* y, int m, T* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T cacc[kMaxColBlocks];
#pragma unroll
  for (int i = 0; i < kMaxColBlocks; ++i) cacc[i] = T(0);
  for (int r = wid; r < m; r += SPG_WARPS) {
    const T* row = L + tri(r, 0);
    const T xr = x[r];
#pragma unroll
    for (int i = 0; i < kMaxColBlocks; ++i) {
      const int k = lane + 32 * i;
      if (k <= r) cacc[i] += row[k] * xr;  // (L^T x)_k = sum_{r >= k} L[r][k] x_r
    }
  }
#pragma unroll
  for (int i = 0; i < kMaxColBlocks; ++i) {
    const int k = lane + 32 * i;
    if (k < m) part[wid * m + k] = cacc[i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += SPG_THREADS) {
    T s = T(0);
#pragma unroll
    for (int w = 0; w < SPG_WARPS; ++w) s += part[w * m + k];
    y[k] = s;
  }
  __syncthreads();
}

}  // namespace spg
