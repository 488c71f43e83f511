// CTA-wide dense kernels on one chain's matrices: packed Cholesky, inverse of
// the 32x32 diagonal blocks, blocked triangular solves, full GEMV.
// All routines are called by every thread of a CTA of SPG_THREADS threads.
//
// Storage: lower triangle packed row-major, element (i, k) at i(i+1)/2 + k.
// After factor_cholesky + invert_diag_blocks the diagonal 32x32 blocks hold
// the inverses of the corresponding blocks of L; the off-diagonal blocks hold
// L.  The triangular solves use exactly that layout.
#pragma once
#include <string.h>

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

// acc += a b; the double-float type overloads it with a cheaper form that
// leaves the renormalisation to the end of the accumulation
template <typename T>
__device__ __forceinline__ void mac_acc(T& acc, T a, T b) {
  acc += a * b;
}

// In-place Cholesky G = L L^T of the packed lower triangle G (m x m),
// right-looking in panels of kPanel columns (8 unless the caller picks 4 or
// 16), three barriers per panel:
//   1. warp 0 factors the 8 x 8 diagonal block in registers (lane r holds
//      row r of the block; column c is broadcast by shuffles);
//   2. every row below solves against it (one thread per row, forward
//      substitution with the block read as broadcasts from shared memory) and
//      leaves its 8 entries in the transposed panel copy pan[c][i];
//   3. the trailing lower triangle receives the rank-8 update in 4 x 4
//      register tiles (8 + 8 panel loads per 128 FMAs).
// pan: scratch of cholesky_scratch(m, kPanel) elements.  Returns true on success
// (CTA-uniform); on failure *flag = 1 + the first column whose pivot was not
// positive (or outside the range where the FP32-seeded reciprocal square root
// holds).
constexpr int kPanel = 8;      // the default panel width
constexpr int kMaxPanel = 16;  // the widest panel a kernel may choose
__host__ __device__ inline int chol_ld(int m) { return (m + 6) & ~3; }
__host__ __device__ inline size_t cholesky_scratch(int m, int pw = kPanel) {
  return (size_t)pw * chol_ld(m) + 4;
}

// four consecutive elements from 16-byte aligned shared memory (vector loads)
template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&v)[4]) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    const float f[4] = {q.x, q.y, q.z, q.w};
    memcpy(v, f, sizeof(f));
  } else {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    memcpy(v, f, sizeof(f));
  }
}

// ---- the three steps of one panel (columns jb .. jb + nb) -------------------

// 1. one warp factors the nb x nb diagonal block in registers (lane r holds
//    row r; column c broadcast by shuffles): L_bb into G, its entries and the
//    reciprocal pivots into the panel copy pan.  Returns 0 or 1 + the first
//    bad column (warp-uniform).
template <typename T, int kPanel>
__device__ __forceinline__ int chol_diag_block(T* G, int jb, int nb, T* pan, int ld) {
  const int lane = threadIdx.x & 31;
  T row[kPanel];
  const bool mine = lane < nb;
#pragma unroll
  for (int c = 0; c < kPanel; ++c)
    row[c] = (mine && c <= lane) ? G[tri(jb + lane, jb + c)] : T(0);
  int bad = 0;
#pragma unroll
  for (int c = 0; c < kPanel; ++c) {
    if (c < nb && !bad) {
      const T d = shfl_idx(row[c], c);
      if (!(d > T(1e-37)) || !(d < T(3e37))) {
        bad = c + 1;
      } else {
        const T rinv = rsqrt_t(d);
        if (lane == c) row[c] = d * rinv;
        if (lane > c) row[c] *= rinv;
#pragma unroll
        for (int c2 = c + 1; c2 < kPanel; ++c2) {
          const T l2 = shfl_idx(row[c], c2);
          if (c2 <= lane) row[c2] -= row[c] * l2;
        }
        if (lane == 0) pan[c * ld + jb + c] = rinv;  // 1 / L_cc for step 2
      }
    }
  }
  if (!bad && mine) {
#pragma unroll
    for (int c = 0; c < kPanel; ++c)
      if (c <= lane) {
        G[tri(jb + lane, jb + c)] = row[c];
        if (c < lane) pan[c * ld + jb + lane] = row[c];  // L_bb[lane][c]
      }
  }
  return bad ? jb + bad : 0;
}

// 2. every row i >= j0 solves against the diagonal block (one thread per
//    row, forward substitution with the block read as broadcasts from shared
//    memory) and leaves its entries in the transposed panel copy pan[c][i];
//    rows m .. ld-1 of the copy are zeroed for the edge tiles of step 3
template <typename T, int kPanel>
__device__ __forceinline__ void chol_panel_rows(T* G, int m, int jb, int j0, T* pan, int ld) {
  const int tid = threadIdx.x;
  for (int i = j0 + tid; i < m; i += SPG_THREADS) {
    const size_t base = tri(i, jb);
    T g[kPanel];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) g[c] = G[base + c];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < c; ++k) mac_acc(acc, g[k], pan[k * ld + jb + c]);
      g[c] = (g[c] - acc) * pan[c * ld + jb + c];
    }
#pragma unroll
    for (int c = 0; c < kPanel; ++c) {
      G[base + c] = g[c];
      pan[c * ld + i] = g[c];
    }
  }
  for (int q = tid; q < kPanel * (ld - m); q += SPG_THREADS)
    pan[(q / (ld - m)) * ld + m + q % (ld - m)] = T(0);
}

// 3. the rank-kPanel update of the trailing lower triangle (rows and columns
//    >= j0) in 4 x 4 register tiles (8 + 8 panel loads per 16 kPanel MACs).
//    Thread `first` of `count` takes every count-th tile, and only rows at or
//    below `skip` (rows j0 .. skip-1 belong to a block updated elsewhere).
template <typename T, int kPanel>
__device__ __forceinline__ void chol_trailing(T* G, int m, int j0, const T* pan, int ld,
                                              int first, int count, int skip) {
  const int s = m - j0;
  const int nt = (s + 3) >> 2;
  const int ntiles = nt * (nt + 1) / 2;
  const int I0 = (skip - j0) >> 2;  // tile rows entirely above `skip`
  for (int t = I0 * (I0 + 1) / 2 + first; t < ntiles; t += count) {
    int I = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int K = t - I * (I + 1) / 2;
    const int i0 = j0 + 4 * I, k0 = j0 + 4 * K;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll
    for (int c = 0; c < kPanel; ++c) {
      T va[4], vb[4];
      load4<T>(pan + c * ld + i0, va);
      load4<T>(pan + c * ld + k0, vb);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mac_acc(acc[a][b], va[a], vb[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + a;
      if (i < m && i >= skip) {
        T* gi = G + tri(i, 0);
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (k0 + b <= i) gi[k0 + b] -= acc[a][b];
      }
    }
  }
}

// The factorisation described above: steps 1-3 per panel, three barriers.
template <typename T, int kPanel = spg::kPanel>
__device__ bool factor_cholesky(T* G, int m, T* pan_raw, int* flag) {
  const int tid = threadIdx.x, wid = tid >> 5;
  // 16-byte aligned panel base; row stride ld (a multiple of 4, >= m + 3)
  T* pan = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(pan_raw) + 15) & ~uintptr_t(15));
  const int ld = chol_ld(m);
  for (int jb = 0; jb < m; jb += kPanel) {
    const int nb = min(kPanel, m - jb);
    const int j0 = jb + nb;
    if (wid == 0) {
      const int bad = chol_diag_block<T, kPanel>(G, jb, nb, pan, ld);
      if (bad && (tid & 31) == 0) *flag = bad;
    }
    __syncthreads();
    if (*flag) return false;
    if (j0 >= m) break;
    chol_panel_rows<T, kPanel>(G, m, jb, j0, pan, ld);
    __syncthreads();
    chol_trailing<T, kPanel>(G, m, j0, pan, ld, tid, SPG_THREADS, j0);
    __syncthreads();
  }
  return true;
}

// The same factorisation with a look-ahead of one panel, two barriers per
// panel: after the panel rows of block b, warp 0 applies block b's update to
// the next diagonal block itself and factors it, while the other warps apply
// the update to the rest of the trailing triangle, so the serial chain of
// the diagonal blocks (a shuffle, a reciprocal square root and a
// multiply-add per column) overlaps the parallel update instead of stalling
// the CTA.  Two panel copies alternate (the next block's entries land in one
// while the other is read).  Every entry receives the same operations in
// the same order as in factor_cholesky, so the two give identical factors.
// pan: scratch of cholesky_scratch_la(m, kPanel) elements.
__host__ __device__ inline size_t cholesky_scratch_la(int m, int pw = kPanel) {
  return 2 * (size_t)pw * chol_ld(m) + 4;
}
template <typename T, int kPanel = spg::kPanel>
__device__ bool factor_cholesky_la(T* G, int m, T* pan_raw, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ld = chol_ld(m);
  T* pans[2];
  pans[0] = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(pan_raw) + 15) & ~uintptr_t(15));
  pans[1] = pans[0] + (size_t)kPanel * ld;  // ld is a multiple of 4: still 16-byte aligned
  if (wid == 0) {
    const int bad = chol_diag_block<T, kPanel>(G, 0, min(kPanel, m), pans[0], ld);
    if (bad && lane == 0) *flag = bad;
  }
  __syncthreads();
  if (*flag) return false;
  for (int jb = 0, p = 0; jb < m; jb += kPanel, p ^= 1) {
    const int nb = min(kPanel, m - jb);
    const int j0 = jb + nb;
    if (j0 >= m) break;
    T* cur = pans[p];
    chol_panel_rows<T, kPanel>(G, m, jb, j0, cur, ld);
    __syncthreads();
    const int nb2 = min(kPanel, m - j0);
    const int j1 = j0 + nb2;
    if (wid == 0) {
      // block b's update of the next diagonal block (lane r: row j0 + r),
      // accumulated as the 4 x 4 tiles accumulate it, then its factorisation
      if (lane < nb2) {
        const int i = j0 + lane;
        T* gi = G + tri(i, 0);
        for (int k = j0; k <= i; ++k) {
          T acc = T(0);
#pragma unroll
          for (int c = 0; c < kPanel; ++c) mac_acc(acc, cur[c * ld + i], cur[c * ld + k]);
          gi[k] -= acc;
        }
      }
      __syncwarp();
      const int bad = chol_diag_block<T, kPanel>(G, j0, nb2, pans[p ^ 1], ld);
      if (bad && lane == 0) *flag = bad;
    } else {
      chol_trailing<T, kPanel>(G, m, j0, cur, ld, tid - 32, SPG_THREADS - 32, j1);
    }
    __syncthreads();
    if (*flag) return false;
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
        for (int k = lane; k < r; ++k) mac_acc(acc, L[tri(r0 + r, r0 + k)], L[tri(r0 + k, r0 + lane)]);
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
    // s_r = x_r - sum_{k < r0} L[r][k] x_k; warp w takes the rows w + 8 q of
    // the block, their dot products interleaved
    {
      constexpr int kRows = kBlk / SPG_WARPS;
      T acc[kRows];
#pragma unroll
      for (int q = 0; q < kRows; ++q) acc[q] = T(0);
      for (int k = lane; k < r0; k += 32) {
        const T xk = x[k];
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
          const int rr = wid + SPG_WARPS * q;
          if (rr < bs) mac_acc(acc[q], L[tri(r0 + rr, k)], xk);
        }
      }
#pragma unroll
      for (int q = 0; q < kRows; ++q) acc[q] = warp_sum(acc[q]);
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
          const int rr = wid + SPG_WARPS * q;
          if (rr < bs) s[rr] = x[r0 + rr] - acc[q];
        }
      }
    }
    __syncthreads();
    if (wid == 0 && lane < bs) {
      // four independent partial sums (the chain of FMAs is the latency)
      const T* row = L + tri(r0 + lane, r0);
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int c = 0;
      for (; c + 3 <= lane; c += 4) {
        mac_acc(a0, row[c], s[c]);
        mac_acc(a1, row[c + 1], s[c + 1]);
        mac_acc(a2, row[c + 2], s[c + 2]);
        mac_acc(a3, row[c + 3], s[c + 3]);
      }
      for (; c <= lane; ++c) mac_acc(a0, row[c], s[c]);
      x[r0 + lane] = (a0 + a1) + (a2 + a3);
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
    T acc = T(0), acc2 = T(0);
    if (lane < bs) {
      int r = r0 + bs + wid;
      for (; r + SPG_WARPS < m; r += 2 * SPG_WARPS) {
        mac_acc(acc, L[tri(r, i)], x[r]);
        mac_acc(acc2, L[tri(r + SPG_WARPS, i)], x[r + SPG_WARPS]);
      }
      if (r < m) mac_acc(acc, L[tri(r, i)], x[r]);
    }
    part[wid * kBlk + lane] = acc + acc2;
    __syncthreads();
    if (wid == 0 && lane < bs) {
      T t = x[i];
#pragma unroll
      for (int w = 0; w < SPG_WARPS; ++w) t -= part[w * kBlk + lane];
      s[lane] = t;
    }
    __syncthreads();
    if (wid == 0 && lane < bs) {
      // z_i = sum_{r >= i in block} Dinv[r][i] s_r, four partial sums
      T z0 = T(0), z1 = T(0), z2 = T(0), z3 = T(0);
      int rr = lane;
      for (; rr + 3 < bs; rr += 4) {
        mac_acc(z0, L[tri(r0 + rr, i)], s[rr]);
        mac_acc(z1, L[tri(r0 + rr + 1, i)], s[rr + 1]);
        mac_acc(z2, L[tri(r0 + rr + 2, i)], s[rr + 2]);
        mac_acc(z3, L[tri(r0 + rr + 3, i)], s[rr + 3]);
      }
      for (; rr < bs; ++rr) mac_acc(z0, L[tri(r0 + rr, i)], s[rr]);
      x[i] = (z0 + z1) + (z2 + z3);
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
template <typename T, typename S = T>
__device__ void symv_packed(const S* __restrict__ V, const T* z, T* y, int m, T alpha, T* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T cacc[kMaxColBlocks];
#pragma unroll
  for (int i = 0; i < kMaxColBlocks; ++i) cacc[i] = T(0);
  for (int r = wid; r < m; r += SPG_WARPS) {
    const S* row = V + tri(r, 0);
    const T zr = z[r];
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < kMaxColBlocks; ++i) {
      const int k = lane + 32 * i;
      if (k <= r) {
        const T a = T(row[k]);
        mac_acc(acc, a, z[k]);
        if (k < r) mac_acc(cacc[i], a, zr);
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
      if (k <= r) mac_acc(cacc[i], row[k], xr);  // (L^T x)_k = sum_{r >= k} L[r][k] x_r
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

// s + e = a + b exactly (TwoSum, FP64)
__device__ __forceinline__ void two_sum64(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// CTA-wide compensated sum of the pairs (s, c) (value s + c on every
// thread): TwoSum at every level of the tree.  red: 2 SPG_WARPS doubles.
__device__ __forceinline__ double block_sum_dd(double s, double c, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double so = __shfl_xor_sync(0xffffffffu, s, o);
    const double co = __shfl_xor_sync(0xffffffffu, c, o);
    double e;
    two_sum64(s, so, s, e);
    c += co + e;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[2 * wid] = s;
    red[2 * wid + 1] = c;
  }
  __syncthreads();
  s = 0.0;
  c = 0.0;
#pragma unroll
  for (int w = 0; w < SPG_WARPS; ++w) {
    double e;
    two_sum64(s, red[2 * w], s, e);
    c += red[2 * w + 1] + e;
  }
  return s + c;
}

// Pencil Rayleigh correction of a root t0 of det(F + tV) with null-vector
// estimate u (CTA-wide, FP64), in the two forms below:
//   t = t0 - u^T (F + t0 V) u / (u^T V u),
// the Newton step of the Rayleigh quotient t(u) = -(u^T F u)/(u^T V u),
// which is stationary at the null vector: its error is quadratic in the
// error of u, and it is evaluated on the exact FP64 F and V instead of
// through a factorisation, so the factorisation's backward error (about
// m eps |F|, large when |F| >> |u^T F u|) does not enter t.  F: packed
// lower triangle (global or shared); V: packed (vfull = false) or full
// m x m row-major (vfull = true); pidx: (i << 16) | k per packed entry; u:
// shared, m.  Both return NaN if u^T V u == 0.
//
// The pencil Rayleigh correction of the FP64 path, with F(p) = A_0 + Y kept
// in two parts (Y = sum_{j>=1} p_j A_j): the large and exact A_0 part of
//   u^T (F + t0 V) u = u^T A_0 u + u^T (Y + t0 V) u
// is summed with error-free products and sums (Ogita, Rump, Oishi 2005,
// Dot2), so that neither the rounding of A_0 + Y nor that of the sum enters
// t; the small part in plain FP64.  Arguments as above (F = A0 + Y); A0 packed
// (global); red: 2 SPG_WARPS doubles.
__device__ inline double pencil_correct_split(const double* __restrict__ A0,
                                              const double* __restrict__ Y,
                                              const double* __restrict__ V, bool vfull, int m,
                                              long long P, const uint32_t* __restrict__ pidx,
                                              const double* u, double t0, double* red) {
  double s = 0.0, c = 0.0, a = 0.0, b = 0.0;
  for (long long e = threadIdx.x; e < P; e += SPG_THREADS) {
    const uint32_t ik = pidx[e];
    const int i = ik >> 16, k = ik & 0xffff;
    const double ve = vfull ? V[(size_t)i * m + k] : V[e];
    const double f = i == k ? 1.0 : 2.0;
    // U_e = f u_i u_k = uh + ul exactly
    const double uh = f * (u[i] * u[k]);
    const double ul = f * fma(u[i], u[k], -(u[i] * u[k]));
    // A_0[e] U_e: error-free product of the high part, the low part rounded
    const double ae = A0[e];
    const double ph = ae * uh;
    const double pl = fma(ae, uh, -ph) + ae * ul;
    double es;
    two_sum64(s, ph, s, es);
    c += es + pl;
    a = fma(fma(t0, ve, Y[e]), uh, a);
    b = fma(ve, uh, b);
  }
  c += a;  // the small part joins the compensation term
  const double num = block_sum_dd(s, c, red);
  b = block_sum(b, red);
  return b != 0.0 ? t0 - num / b : NAN;
}

// The pencil Rayleigh correction for an F with large entries and no A_0 + Y
// split (the mixed path's carried F): u^T (F + t0 V) u is summed with
// error-free transformations throughout (Dot2, Ogita, Rump, Oishi 2005):
// x = F + t0 V as an exact pair (TwoProduct of t0 V, TwoSum with F), the
// products x U_e exact, the running sum a TwoSum pair.  Plain FP64 summation
// of terms of size |F| |u|^2 (their magnitudes add up to about |F|, 10^3-10^4
// for the S-n-m bodies) leaves an error of about 10^-14 in a sum whose value
// is 0 at the root, which short chords at grazing incidence divide by
// t |u^T V u| ~ 10^-5.  Arguments as above (V packed); red:
// 2 SPG_WARPS doubles.
__device__ inline double pencil_correct_dot2(const double* __restrict__ F,
                                             const double* __restrict__ V, int m, long long P,
                                             const uint32_t* __restrict__ pidx, const double* u,
                                             double t0, double* red) {
  (void)m;
  double s = 0.0, c = 0.0, b = 0.0;
  for (long long e = threadIdx.x; e < P; e += SPG_THREADS) {
    const uint32_t ik = pidx[e];
    const int i = ik >> 16, k = ik & 0xffff;
    const double ve = V[e];
    const double f = i == k ? 1.0 : 2.0;
    const double uh = f * (u[i] * u[k]);
    const double ul = f * fma(u[i], u[k], -(u[i] * u[k]));
    const double tv = t0 * ve;
    const double tvl = fma(t0, ve, -tv);
    double x, xl;
    two_sum64(F[e], tv, x, xl);
    xl += tvl;
    const double ph = x * uh;
    const double pl = fma(x, uh, -ph) + (x * ul + xl * uh);
    double es;
    two_sum64(s, ph, s, es);
    c += es + pl;
    b = fma(ve, uh, b);
  }
  const double num = block_sum_dd(s, c, red);
  b = block_sum(b, red);
  return b != 0.0 ? t0 - num / b : NAN;
}

}  // namespace spg
