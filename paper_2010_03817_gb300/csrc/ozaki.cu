// FP64-quality formation of the pencil matrices on the BF16 tensor cores.
//
// For R coefficient rows c_r (length n) the kernel computes
//   Y[r, p] = lead A_0[p] + sum_{j>=1} c_r[j] A[j, p]   (A: packed LMI stack)
// i.e. V = sum v_j A_j (lead 0) and F(x) = A_0 + sum x_j A_j (lead 1) -- the
// pencil B_0 + t B_1 of a line (Lemma "PEP and S cap C").  A_0 stays out of
// the digit split (its entries are often much larger than those of A_1..A_n,
// and the split's error scales with the largest entry of its operand): it is
// added in FP64 by the epilogue.
//
// Exactness scheme (error-free splitting of both operands into integer
// digits, the Ozaki scheme; Ozaki, Ogita, Oishi, Rump 2012, and its
// tensor-core form, Mukunoki, Ozaki, Ogita, Imamura 2020):
//   c_r[j] = 2^{f_r} sum_s a_s[r, j] 2^{-7(s+1)},  A[j, p] = 2^{e_p} sum_t b_t[j, p] 2^{-7(t+1)}
// (j = 1..n)
// with integer digits |a_s|, |b_t| <= 64 (exact in BF16), S digits (7S bits:
// S = 8 for the formation, 7 for the normal contraction).  For each digit sum
// d = s + t <= S - 1 the tensor core accumulates
//   G_d[r, p] = sum_{s+t=d} sum_j a_s[r, j] b_t[j, p]
// in FP32 in TMEM; every partial sum is an integer below S * 224 * 2^12 <
// 2^24, so the accumulation is exact.  The epilogue combines the S integers
// in 64-bit integer arithmetic and scales once into FP64:
//   Y = 2^{f_r + e_p} sum_d G_d 2^{-7(d+2)}.
// The truncation (pairs with s + t > S - 1, digits beyond the S-th) is below
// n 2^{-(7S - 5)} max_j |c_r[j]| max_{j>=1} |A[j, p]| (2^-51 for S = 8), plus
// one FP64 rounding of the sum with lead A_0[p].
#include <cuda_bf16.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace spg {
namespace {

constexpr int kFormDigits = 8;      // S of the pencil formation (F and V)
constexpr int kContractDigits = 7;  // S of the normal contraction
constexpr int kMaxDigits = 8;
constexpr int kDigitBits = 7;       // beta
constexpr int kTileM = 128;         // coefficient rows per CTA
constexpr int kTileN = 32;          // packed entries per CTA
constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t core_off(int r, int g, int kgroups) {
  return (uint32_t)(((r >> 3) * kgroups + g) * 128 + (r & 7) * 16);
}

// T 2^scale rounded to the nearest double (ties to even) with integer
// operations only; |T| < 2^126, and the result stays in the normal range for
// the exponents of LMI entries and coefficients.
__device__ __forceinline__ double i128_to_double(__int128 T, int scale) {
  if (T == 0) return 0.0;
  const unsigned long long sign = T < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned __int128 a = T < 0 ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const unsigned long long ah = (unsigned long long)(a >> 64), al = (unsigned long long)a;
  int nbits = ah ? 128 - __clzll((long long)ah) : 64 - __clzll((long long)al);
  unsigned long long mant;
  const int sh = nbits - 53;
  if (sh <= 0) {
    mant = (unsigned long long)a << (-sh);
  } else {
    const unsigned __int128 q = a >> sh;
    const unsigned __int128 rem = a - (q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    mant = (unsigned long long)q;
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++nbits;
      }
    }
  }
  const long long ex = (long long)(nbits - 1 + scale) + 1023;
  return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) |
                                          (mant & 0xfffffffffffffull)));
}

// one warp per row: exponent and ND digits of c_r = vec[rows[r], 0..n-1]
// (rows null: vec[r]); rows r >= *count_dev are skipped when count_dev is given
template <int ND>
__global__ void slice_rows_kernel(const double* __restrict__ vec, int R, int n, int Kp,
                                  __nv_bfloat16* __restrict__ out, int* __restrict__ ex,
                                  const int* __restrict__ rows, const int* __restrict__ count_dev) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= R || (count_dev && r >= *count_dev)) return;
  const double* row = vec + (size_t)(rows ? rows[r] : r) * n;
  double mx = 0.0;
  for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(row[j]));
  mx = warp_max(mx);
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);  // mx < 2^e
    e += 1;         // |c| <= 2^(e-1): normalised values in [-1/2, 1/2]
  }
  if (lane == 0) ex[r] = e;
  for (int k = lane; k < Kp; k += 32) {
    double y = k < n ? ldexp(row[k], -e) : 0.0;
#pragma unroll
    for (int s = 0; s < ND; ++s) {
      y *= 128.0;
      const double d = rint(y);
      y -= d;
      out[((size_t)s * R + r) * Kp + k] = __float2bfloat16_rn((float)d);
    }
  }
}

// Epilogue of the digit-split GEMM.  kForm: Y[r][p] = value (+ lead A0[p]).
// kContract: the rows of B are the rows (j, i) of the full matrices A_j,
// padded to mpad rows per j (a tile of 32 never straddles two j), and the
// value is (A_j u_r)_i; the epilogue folds it with u_r[i] into the partial
// sum of w_j = u_r^T A_j u_r over the tile's 32 rows, written to
// Wpart[(r n1 + j) (mpad / 32) + tile] (no atomics: a fixed summation order).
constexpr int kForm = 0, kContract = 1;
struct OzEpi {
  const double* A0;
  double lead;
  double* Y;
  long long ldy;
  const int* rows;       // formation: output row of coefficient row r (null: r)
  const int* count_dev;  // formation: rows r >= *count_dev are skipped (null: R)
  const double* U;
  int m, mpad, n1;
  double* Wpart;
};

template <int kMode, int kDigits>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_kernel(const __nv_bfloat16* __restrict__ Asl, const int* __restrict__ erow, int R,
                 const __nv_bfloat16* __restrict__ Bsl, const int* __restrict__ ecol, long long P,
                 int Kp, OzEpi ep, int* err) {
  constexpr int kGroups = kDigits;  // digit sums d = 0..kDigits-1
  static_assert(kGroups * kTileN <= 256, "the digit sums must fit the 256 TMEM columns");
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // a device-side row count (formation of a list built on the GPU): rows
  // from it on are skipped and blocks past it leave before touching the
  // tensor memory.  R stays the stride of the digit planes (the slicing
  // wrote plane s of row r at s R + r); Rl bounds the live rows.
  int Rl = R;
  if (kMode == kForm && ep.count_dev) {
    const int rl = *ep.count_dev;
    Rl = rl < R ? rl : R;
  }
  if ((kMode == kForm ? (int)blockIdx.y : (int)blockIdx.x) * kTileM >= Rl) return;
  const int kgroups = Kp / 8;
  const uint32_t a_bytes = kTileM * Kp * 2;
  const uint32_t b_bytes = kTileN * Kp * 2;
  uint8_t* sB = smem;                        // kDigits x [32 x Kp]
  uint8_t* sA0 = sB + kDigits * b_bytes;     // [128 x Kp], double buffered
  uint8_t* sA1 = sA0 + a_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sA1 + a_bytes);  // 2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

  // formation: column tiles along x; contraction: row tiles along x, so that
  // consecutive blocks share (and the L2 keeps) the same B tile
  const long long p0 = (long long)(kMode == kForm ? blockIdx.x : blockIdx.y) * kTileN;
  const int r0 = (kMode == kForm ? blockIdx.y : blockIdx.x) * kTileM;

  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  if (wid == 0) {
    tc::tmem_alloc(tmem_slot, 256);
    tc::tmem_relinquish();
  }
  // All operand tiles arrive by 16-byte asynchronous copies, many in flight
  // per thread: the 7 B digit planes of this column tile (resident) and A
  // digit plane 0 first; plane s + 1 streams into the other buffer while the
  // tensor core works on plane s.
  const uint32_t sB_u = tc::smem_u32(sB), sA_u[2] = {tc::smem_u32(sA0), tc::smem_u32(sA1)};
  // (row, 16-byte group) of the copy q = tid + kThreads k, stepped without
  // divisions: consecutive threads take consecutive groups of a row
  const int r_init = tid / kgroups, g_init = tid % kgroups;
  const int dr = kThreads / kgroups, dg = kThreads % kgroups;
  for (int t = 0; t < kDigits; ++t) {
    int r = r_init, g = g_init;
    for (int q = tid; q < kTileN * kgroups; q += kThreads) {
      const bool in = p0 + r < P;
      tc::cp_async16(sB_u + t * b_bytes + core_off(r, g, kgroups),
                     in ? Bsl + ((size_t)t * P + p0 + r) * Kp + g * 8 : Bsl, in);
      r += dr;
      g += dg;
      if (g >= kgroups) {
        g -= kgroups;
        ++r;
      }
    }
  }
  tc::cp_async_commit();
  auto stage_a = [&](int s) {
    const uint32_t base = sA_u[s & 1];
    int r = r_init, g = g_init;
    for (int q = tid; q < kTileM * kgroups; q += kThreads) {
      const bool in = r0 + r < Rl;
      tc::cp_async16(base + core_off(r, g, kgroups),
                     in ? Asl + ((size_t)s * R + r0 + r) * Kp + g * 8 : Asl, in);
      r += dr;
      g += dg;
      if (g >= kgroups) {
        g -= kgroups;
        ++r;
      }
    }
    tc::cp_async_commit();
  };
  stage_a(0);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc::idesc_bf16_f32(kTileM, kTileN);
  const uint32_t sbo = (uint32_t)kgroups * 128;
  bool ok = true;

  for (int s = 0; s < kDigits; ++s) {
    if (s + 1 < kDigits) {
      // buffer (s + 1) & 1 was last read by the MMAs of plane s - 1; the
      // outcome of the bounded wait is made block-uniform
      const bool w = s < 1 || tc::mbar_wait(&mbar[(s - 1) & 1], ((s - 1) >> 1) & 1);
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
      stage_a(s + 1);
      tc::cp_async_wait<1>();  // everything but plane s + 1 has landed
    } else {
      tc::cp_async_wait<0>();
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_base = sA_u[s & 1];
      for (int t = 0; t + s < kGroups; ++t) {
        const uint32_t b_base = sB_u + t * b_bytes;
        const uint32_t d_tmem = tmem + (uint32_t)((s + t) * kTileN);
        for (int ks = 0; ks < Kp / 16; ++ks) {
          const uint64_t ad = tc::smem_desc(a_base + ks * 256, 128, sbo);
          const uint64_t bd = tc::smem_desc(b_base + ks * 256, 128, sbo);
          tc::mma_bf16(d_tmem, ad, bd, idesc, (s > 0 || ks > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&mbar[s & 1]);
    }
  }
  tc::cp_async_wait<0>();  // no copy may still be in flight when the block moves on
  // the commit of the last digit covers every MMA issued before it
  if (ok) ok = tc::mbar_wait(&mbar[(kDigits - 1) & 1], ((kDigits - 1) >> 1) & 1);
  ok = __syncthreads_and(ok);  // the epilogue's TMEM loads are warp-collective
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let in-flight MMAs drain (bounded) before the TMEM is released
    tc::mbar_wait(&mbar[(kDigits - 1) & 1], ((kDigits - 1) >> 1) & 1, 1ll << 20);
  }
  tc::fence_after_sync();
  if (ok) {
    const int r = r0 + wid * 32 + lane;
    const int er = (r < Rl) ? erow[r] : 0;
    const uint32_t lane_base = tmem + ((uint32_t)(wid * 32) << 16);
    double part = 0.0;  // kContract
    const int jc = kMode == kContract ? (int)(p0 / ep.mpad) : 0;
    const int i0 = kMode == kContract ? (int)(p0 % ep.mpad) : 0;
    for (int c0 = 0; c0 < kTileN; c0 += 16) {
      // the chunk's exponents and (contraction) u entries or (formation) A_0
      // entries first: independent loads, in flight together with the TMEM
      // reads
      int ec[16];
      double aux[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const long long p = p0 + c0 + i;
        ec[i] = p < P ? ecol[p] : 0;
        if (kMode == kForm) {
          aux[i] = (ep.lead != 0.0 && p < P) ? ep.A0[p] : 0.0;
        } else {
          const int ii = i0 + c0 + i;
          aux[i] = (r < Rl && ii < ep.m) ? ep.U[(size_t)r * ep.m + ii] : 0.0;
        }
      }
      long long hi[16], lo[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0;
      uint32_t v[kGroups][16];
#pragma unroll
      for (int d = 0; d < kGroups; ++d) tc::tmem_ld16(lane_base + (uint32_t)(d * kTileN + c0), v[d]);
      tc::tmem_wait_ld();
      // hi carries the digit sums d < kHi, lo the rest (Horner in base 2^7,
      // each below 2^(24 + 7 (kHi - 1)) < 2^63):
      //   value = 2^(e - 7 (kDigits + 1)) (hi 2^(7 (kDigits - kHi)) + lo),
      // one rounding (integer operations)
      constexpr int kHi = 4;
      constexpr int kLoShift = kDigitBits * (kDigits - kHi);
      constexpr int kScale = kDigitBits * (kDigits + 1);
#pragma unroll
      for (int d = 0; d < kGroups; ++d) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          // exact integers below 2^24 in magnitude
          const long long g = (long long)__float2int_rn(__uint_as_float(v[d][i]));
          if (d < kHi)
            hi[i] = hi[i] * (1ll << kDigitBits) + g;
          else
            lo[i] = lo[i] * (1ll << kDigitBits) + g;
        }
      }
      if (r < Rl) {
        if (kMode == kForm) {
          double* yrow = ep.Y + (size_t)(ep.rows ? ep.rows[r] : r) * ep.ldy;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const long long p = p0 + c0 + i;
            if (p < P) {
              const double y = i128_to_double(((__int128)hi[i] << kLoShift) + (__int128)lo[i],
                                              er + ec[i] - kScale);
              yrow[p] = ep.lead != 0.0 ? fma(ep.lead, aux[i], y) : y;
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i0 + c0 + i < ep.m) {
              const double y = i128_to_double(((__int128)hi[i] << kLoShift) + (__int128)lo[i],
                                              er + ec[i] - kScale);
              part = fma(y, aux[i], part);
            }
          }
        }
      }
    }
    if (kMode == kContract && r < Rl)
      ep.Wpart[((size_t)r * ep.n1 + jc) * (ep.mpad / kTileN) + i0 / kTileN] = part;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wid == 0) tc::tmem_dealloc(tmem, 256);
}

// one warp per row q = (j, i) of the contraction stack: exponent and digits
// of the row i of A_j (packed stack, FP64) over k = 0..m-1; rows i >= m of
// the padding are zero
__global__ void slice_full_kernel(const double* __restrict__ A, int n1, int m, long long P,
                                  int mpad, int Kp, __nv_bfloat16* __restrict__ out,
                                  int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const long long Q = (long long)n1 * mpad;
  const long long q = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= Q) return;
  const int j = (int)(q / mpad), i = (int)(q % mpad);
  const double* Aj = A + (size_t)j * P;
  double mx = 0.0;
  if (i < m)
    for (int k = lane; k < m; k += 32) mx = fmax(mx, fabs(Aj[i >= k ? tri(i, k) : tri(k, i)]));
  mx = warp_max(mx);
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);
    e += 1;
  }
  if (lane == 0) ex[q] = e;
  for (int k = lane; k < Kp; k += 32) {
    double y = (i < m && k < m) ? ldexp(Aj[i >= k ? tri(i, k) : tri(k, i)], -e) : 0.0;
#pragma unroll
    for (int s = 0; s < kContractDigits; ++s) {
      y *= 128.0;
      const double d = rint(y);
      y -= d;
      out[((size_t)s * Q + q) * Kp + k] = __float2bfloat16_rn((float)d);
    }
  }
}

inline size_t ozaki_smem(int Kp, int digits) {
  return (size_t)digits * kTileN * Kp * 2 + 2 * (size_t)kTileM * Kp * 2 + 64;
}

}  // namespace

int ozaki_kp(int n) { return (n + 15) / 16 * 16; }

size_t ozaki_b_bytes(long long P, int n) {
  return (size_t)kFormDigits * (size_t)P * ozaki_kp(n) * 2;
}

// host: digits of A_1..A_n, column by column (packed entry p over j = 1..n)
void ozaki_slice_stack(const double* packed, int n, long long P, uint16_t* Bsl, int* ecol) {
  const int Kp = ozaki_kp(n);
  for (long long p = 0; p < P; ++p) {
    double mx = 0.0;
    for (int j = 1; j <= n; ++j) mx = fmax(mx, fabs(packed[(size_t)j * P + p]));
    int e = 0;
    if (mx > 0.0) {
      frexp(mx, &e);
      e += 1;
    }
    ecol[p] = e;
    for (int k = 0; k < Kp; ++k) {
      double y = (k < n) ? ldexp(packed[(size_t)(k + 1) * P + p], -e) : 0.0;
      for (int s = 0; s < kFormDigits; ++s) {
        y *= 128.0;
        const double d = rint(y);
        y -= d;
        // |d| <= 64: the float is exact and its upper 16 bits are the BF16
        const float f = (float)d;
        uint32_t bits;
        memcpy(&bits, &f, 4);
        Bsl[((size_t)s * P + p) * Kp + k] = (uint16_t)(bits >> 16);
      }
    }
  }
}

size_t ozaki_row_bytes(int R, int n) { return (size_t)kMaxDigits * R * ozaki_kp(n) * 2; }

cudaError_t launch_ozaki_form(const double* vec, int R, int n, double lead, const double* A0,
                              const uint16_t* Bsl, const int* ecol, long long P, void* row_digits,
                              int* erow, double* Y, long long ldy, int* err, cudaStream_t st,
                              const int* rows, const int* count_dev) {
  if (R <= 0) return cudaSuccess;
  const int Kp = ozaki_kp(n);
  __nv_bfloat16* Asl = static_cast<__nv_bfloat16*>(row_digits);
  slice_rows_kernel<kFormDigits><<<(R + 7) / 8, 256, 0, st>>>(vec, R, n, Kp, Asl, erow, rows,
                                                               count_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = ozaki_smem(Kp, kFormDigits);
  e = cudaFuncSetAttribute(ozaki_kernel<kForm, kFormDigits>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  OzEpi ep{};
  ep.A0 = A0;
  ep.lead = lead;
  ep.Y = Y;
  ep.ldy = ldy;
  ep.rows = rows;
  ep.count_dev = count_dev;
  dim3 grid((unsigned)((P + kTileN - 1) / kTileN), (unsigned)((R + kTileM - 1) / kTileM));
  ozaki_kernel<kForm, kFormDigits><<<grid, kThreads, smem, st>>>(
      Asl, erow, R, reinterpret_cast<const __nv_bfloat16*>(Bsl), ecol, P, Kp, ep, err);
  return cudaGetLastError();
}

int ozaki_mpad(int m) { return (m + kTileN - 1) / kTileN * kTileN; }

size_t ozaki_contract_bytes(int n, int m) {
  return (size_t)kContractDigits * (size_t)(n + 1) * ozaki_mpad(m) * ozaki_kp(m) * 2;
}

cudaError_t launch_ozaki_slice_full(const double* A, int n, int m, long long P, uint16_t* Bc,
                                    int* ecolc, cudaStream_t st) {
  const long long Q = (long long)(n + 1) * ozaki_mpad(m);
  slice_full_kernel<<<(unsigned)((Q + 7) / 8), 256, 0, st>>>(
      A, n + 1, m, P, ozaki_mpad(m), ozaki_kp(m), reinterpret_cast<__nv_bfloat16*>(Bc), ecolc);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_contract(const double* U, int R, int n, int m, const uint16_t* Bc,
                                  const int* ecolc, void* row_digits, int* erow, double* Wpart,
                                  int* err, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int Kp = ozaki_kp(m), mpad = ozaki_mpad(m);
  __nv_bfloat16* Asl = static_cast<__nv_bfloat16*>(row_digits);
  slice_rows_kernel<kContractDigits><<<(R + 7) / 8, 256, 0, st>>>(U, R, m, Kp, Asl, erow,
                                                                   nullptr, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = ozaki_smem(Kp, kContractDigits);
  e = cudaFuncSetAttribute(ozaki_kernel<kContract, kContractDigits>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  OzEpi ep{};
  ep.U = U;
  ep.m = m;
  ep.mpad = mpad;
  ep.n1 = n + 1;
  ep.Wpart = Wpart;
  const long long Q = (long long)(n + 1) * mpad;
  dim3 grid((unsigned)((R + kTileM - 1) / kTileM), (unsigned)(Q / kTileN));
  ozaki_kernel<kContract, kContractDigits><<<grid, kThreads, smem, st>>>(
      Asl, erow, R, reinterpret_cast<const __nv_bfloat16*>(Bc), ecolc, Q, Kp, ep, err);
  return cudaGetLastError();
}

}  // namespace spg
