// Double-float (FP32 pair) arithmetic for the mixed-precision path.
//
// A value is held as hi + lo with |lo| <= ulp(hi)/2 (about 48 significant
// bits).  Products are split exactly with an FMA and sums with TwoSum (Knuth;
// Dekker 1971; Ogita, Rump, Oishi 2005 for the compensated dot products), so
// that FP64-level residuals run on the FP32 pipe: on this GPU the FP64 pipe
// runs at about 1/58 of the FP32 rate.
#pragma once
#include "common.cuh"

namespace spg {

// FP64 -> (hi, lo) by integer operations (no FP64 instruction): hi keeps the
// sign, exponent and leading 24 significand bits of x, lo the remaining 29
// bits rounded to 24, so |x - hi - lo| <= 2^-47 |x|.  Magnitudes below 2^-63
// lose lo (absolute error below 2^-86), below 2^-126 both parts are 0;
// magnitudes of 2^128 and above overflow to infinity.
__device__ __forceinline__ float2 split_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7ffu);
  float hi = 0.f, lo = 0.f;
  if (e > 896) {
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    hi = e < 1151 ? __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23)
                  : __uint_as_float(sign | 0x7f800000u);
    const unsigned rem = l32 & 0x1fffffffu;
    if (e > 960 && e < 1151 && rem) {
      // rem * 2^(e - 1075): an exact power-of-two scale
      const float r = __uint2float_rn(rem) * __uint_as_float((unsigned)(e - 948) << 23);
      lo = __uint_as_float(__float_as_uint(r) | sign);
    }
  }
  return make_float2(hi, lo);
}

// the leading 24 significand bits of x as a float (truncation), integer ops only
__device__ __forceinline__ float trunc_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int e = (int)((h32 >> 20) & 0x7ffu);
  if (e <= 896) return 0.f;
  const unsigned sign = h32 & 0x80000000u;
  if (e >= 1151) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((h32 & 0xfffffu) << 3) |
                         (l32 >> 29));
}

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (acc_h, acc_l) += (ah + al) (bh + bl); the rounding errors of the product
// and of the running sum go to acc_l
__device__ __forceinline__ void df_mac(float& acc_h, float& acc_l, float ah, float al, float bh,
                                       float bl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, fmaf(al, bh, pe));
  float s, e;
  two_sum(acc_h, p, s, e);
  acc_h = s;
  acc_l += e + pe;
}

// (h, l) += (bh, bl)
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  h = s;
  l += e + bl;
}

// renormalise so that |l| <= ulp(h)/2
__device__ __forceinline__ void df_norm(float& h, float& l) {
  const float s = h + l;
  l = l - (s - h);
  h = s;
}

__device__ __forceinline__ double df_to_double(float h, float l) { return (double)h + (double)l; }

// warp-wide double-float sum (result on every lane)
__device__ __forceinline__ void warp_sum_df(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
  df_norm(h, l);
}

}  // namespace spg

namespace spg {

// A double-float number as a value type, for the CTA-wide dense routines
// (templated on the element type): hi + lo, FP32 operations only.  Sums use
// TwoSum on the high parts and products an exact FMA split, each followed by
// a renormalisation (Dekker's add2 / mul2), relative error about 2^-47 of the
// operands' magnitudes.
struct dfloat {
  float h, l;
  dfloat() = default;
  __device__ __forceinline__ dfloat(float a) : h(a), l(0.f) {}
  __device__ __forceinline__ dfloat(int a) : h((float)a), l(0.f) {}
  __device__ __forceinline__ explicit dfloat(double a) {
    const float2 s = split_df(a);
    h = s.x;
    l = s.y;
  }
  __device__ __forceinline__ dfloat(float hi, float lo) : h(hi), l(lo) {}
};

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  const float hs = s + e;
  return dfloat(hs, e - (hs - s));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.h, -a.l); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float hs = p + e;
  return dfloat(hs, e - (hs - p));
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) {
  return a.h < b.h || (a.h == b.h && a.l < b.l);
}
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }

__device__ __forceinline__ double to_double(dfloat a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double to_double(double a) { return a; }

// 1/x: IEEE FP32 reciprocal refined by one Newton step in double-float
__device__ __forceinline__ dfloat recip_t(dfloat x) {
  const dfloat r0(1.0f / x.h);
  const dfloat e = dfloat(1.0f) - x * r0;
  return r0 + r0 * e;
}
// 1/sqrt(x): FP32 seed and two Newton steps in double-float
__device__ __forceinline__ dfloat rsqrt_t(dfloat x) {
  dfloat r(rsqrtf(x.h));
#pragma unroll
  for (int it = 0; it < 2; ++it) r = r * (dfloat(1.5f) - dfloat(0.5f) * (x * (r * r)));
  return r;
}

// acc += a b without renormalising acc (Dot2-style: the product's error and
// the sum's error collect in acc.l; the next full operation renormalises)
__device__ __forceinline__ void mac_acc(dfloat& acc, dfloat a, dfloat b) {
  df_mac(acc.h, acc.l, a.h, a.l, b.h, b.l);
}

__device__ __forceinline__ dfloat shfl_idx(dfloat v, int src) {
  return dfloat(__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src));
}

__device__ __forceinline__ dfloat warp_sum(dfloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = v + dfloat(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
  return v;
}

}  // namespace spg
