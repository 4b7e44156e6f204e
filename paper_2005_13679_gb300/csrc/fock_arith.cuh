// fock_arith.cuh -- arithmetic policies of the H C kernels.
//
// GB300 executes FP64 FMAs at about 1/74 of the FP32 rate (measured 1.0 versus
// 74 TFLOP/s), so the FP64-accurate apply runs on the FP32 pipes with values
// held as unevaluated sums of two floats, hi + lo (Dekker's product with FMA,
// Knuth's TwoSum; 48-bit significands), and only the final conversion uses
// FP64 instructions.  Error-free transformations use the _rn intrinsics so the
// compiler cannot contract a rounded product into a following addition.
//
//   PolF64   : complex128 storage, native FP64 FMA arithmetic (reference arm)
//   PolDF    : complex128 storage (pre-split into float hi/lo), FP32-pair arithmetic
//   PolMixed : complex64 storage, FP32 products and partial sums, FP32-pair
//              accumulation per configuration
#pragma once

#include <cuda_runtime.h>

#include "fock_pack.cuh"

// ---- FP32-pair primitives --------------------------------------------------
// (h, l) += a * b with a = (ah, al), b = (bh, bl).  The product's high part
// p = fl(ah*bh) and its rounding error come from one FMA; the cross terms
// ah*bl + al*bh are added in FP32 (their error is below 2^-46 relative); the
// sum h + p is split exactly by TwoSum and the error joins the low word.
__device__ __forceinline__ void df_prod_acc(float &h, float &l, float ah, float al, float bh, float bl) {
  float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float s = __fadd_rn(h, p);
  float bb = __fsub_rn(s, h);
  float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, e));
}

// (h, l) += (bh, bl)
__device__ __forceinline__ void df_add_acc(float &h, float &l, float bh, float bl) {
  float s = __fadd_rn(h, bh);
  float bb = __fsub_rn(s, h);
  float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, bl));
}

// Normalised product of two pairs.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float s = __fadd_rn(p, e);
  return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

// ---- conversions between FP64 and FP32 pairs with integer operations -------
// This part runs FP64 instructions at about 1/74 of the FP32 rate, so the
// conversions at the ends of the FP32-pair path work on the bit patterns.

// x 2^sh as an FP32 pair: hi = x 2^sh rounded to nearest-even, lo = the exact
// remainder rounded to nearest.  Requires |x 2^sh| < 2^127; values below
// 2^-125 (after scaling) become (0, 0), as do zeros and FP64 subnormals.
__device__ __forceinline__ float2 df_split_bits(double x, int sh) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  const int e0 = ex - 1075 + sh;                       // |x| 2^sh = m 2^e0, m the 53-bit significand
  if (ex == 0 || e0 + 52 < -125) return make_float2(0.f, 0.f);
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint64_t mh = m >> 29;
  const uint64_t r = m & 0x1FFFFFFFull;
  if (r > 0x10000000ull || (r == 0x10000000ull && (mh & 1))) ++mh;   // round to 24 bits, ties to even
  const int lo_i = (int)((int64_t)m - (int64_t)(mh << 29));          // |lo_i| <= 2^28
  // 2^(e0 + 29) and 2^e0 as two float factors each (e0 + 29 <= 98 here)
  const int a1 = max(e0 + 29, -126), a2 = e0 + 29 - a1;
  const int c1 = max(e0, -126), c2 = e0 - c1;
  float hi = __fmul_rn(__fmul_rn((float)(int)mh, __int_as_float((a1 + 127) << 23)), __int_as_float((max(a2, -126) + 127) << 23));
  float lo = __fmul_rn(__fmul_rn(__int2float_rn(lo_i), __int_as_float((c1 + 127) << 23)), __int_as_float((max(c2, -126) + 127) << 23));
  if (b >> 63) {
    hi = -hi;
    lo = -lo;
  }
  return make_float2(hi, lo);
}

// (hi + lo) 2^e as a double.  The pair is first renormalised by TwoSum (an
// accumulated low word may exceed the high word's ulp after cancellation),
// then the sum is formed exactly on the 2^-52 grid of the high significand
// (bits of the low word below it are dropped, a relative error below 2^-52)
// and rounded to 53 bits.
__device__ __forceinline__ double df_to_double_bits(float h0, float l0, int e) {
  const float hi = __fadd_rn(h0, l0);
  const float bb = __fsub_rn(hi, h0);
  const float lo = __fadd_rn(__fsub_rn(h0, __fsub_rn(hi, bb)), __fsub_rn(l0, bb));
  const uint32_t bh = __float_as_uint(hi), bl = __float_as_uint(lo);
  if ((bh & 0x7fffffffu) == 0u) return 0.0;
  const int fh = (int)((bh >> 23) & 0xff), fl = (int)((bl >> 23) & 0xff);
  int64_t mh = (int64_t)((bh & 0x7fffffu) | (fh ? 0x800000u : 0u));
  int64_t ml = (int64_t)((bl & 0x7fffffu) | (fl ? 0x800000u : 0u));
  const int eh = (fh ? fh : 1) - 150, el = (fl ? fl : 1) - 150;   // value = m 2^e
  if (bh >> 31) mh = -mh;
  if (bl >> 31) ml = -ml;
  int64_t S = mh * (1ll << 29);                         // units of 2^(eh - 29)
  const int d = el - (eh - 29);
  if (ml != 0 && d > -40) S += d >= 0 ? ml * (1ll << d) : (ml >> -d);
  if (S == 0) return 0.0;
  const uint64_t sgn = S < 0 ? 0x8000000000000000ull : 0ull;
  uint64_t u = (uint64_t)(S < 0 ? -S : S);
  int shift = 63 - __clzll((long long)u) - 52;          // bring the leading 1 to bit 52
  uint64_t mant;
  if (shift > 0) {
    const uint64_t rem = u & ((1ull << shift) - 1), half = 1ull << (shift - 1);
    mant = u >> shift;
    if (rem > half || (rem == half && (mant & 1))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++shift;
      }
    }
  } else {
    mant = u << -shift;
  }
  const int ex = eh - 29 + e + shift + 52 + 1023;
  return __longlong_as_double((long long)(sgn | ((uint64_t)ex << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// ---- native FP64 -----------------------------------------------------------
struct PolF64 {
  using vec_t = double2;   // one complex element of C / sigma
  using amp_t = double;    // real amplitude (square-root products)
  using coef_t = double2;  // complex coefficient
  using acc_t = double2;
  using inner_t = double2;
  static constexpr bool kInner = false;

  static __device__ __forceinline__ amp_t amul(amp_t a, amp_t b) { return a * b; }
  static __device__ __forceinline__ void zero(acc_t &a) { a = make_double2(0.0, 0.0); }
  static __device__ __forceinline__ coef_t scale(coef_t c, amp_t x) { return make_double2(c.x * x, c.y * x); }
  static __device__ __forceinline__ void mac(acc_t &a, coef_t k, vec_t v, bool real) {
    a.x = fma(k.x, v.x, a.x);
    a.y = fma(k.x, v.y, a.y);
    if (!real) {
      a.x = fma(-k.y, v.y, a.x);
      a.y = fma(k.y, v.x, a.y);
    }
  }
  static __device__ __forceinline__ void flush(acc_t &a, const inner_t &i) { a.x += i.x; a.y += i.y; }
  static __device__ __forceinline__ vec_t finish(const acc_t &a, double scale, bool = false) {
    return make_double2(a.x * scale, a.y * scale);
  }
};

// ---- FP32 pairs ------------------------------------------------------------
struct PolDF {
  using vec_t = float4;    // (re_hi, im_hi, re_lo, im_lo), pre-split copy of C
  using amp_t = float2;    // (hi, lo)
  using coef_t = float4;   // (re_hi, im_hi, re_lo, im_lo)
  using acc_t = float4;    // (re_hi, re_lo, im_hi, im_lo), low words not renormalised
  using inner_t = float4;
  static constexpr bool kInner = false;

  static __device__ __forceinline__ amp_t amul(amp_t a, amp_t b) { return df_mul(a, b); }
  static __device__ __forceinline__ void zero(acc_t &a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ coef_t scale(coef_t c, amp_t x) {
    float2 re = df_mul(make_float2(c.x, c.z), x);
    float2 im = df_mul(make_float2(c.y, c.w), x);
    return make_float4(re.x, im.x, re.y, im.y);
  }
  static __device__ __forceinline__ void mac(acc_t &a, coef_t k, vec_t v, bool real) {
    df_prod_acc(a.x, a.y, k.x, k.z, v.x, v.z);        // + Re k Re v
    df_prod_acc(a.z, a.w, k.x, k.z, v.y, v.w);        // + Re k Im v
    if (!real) {
      df_prod_acc(a.x, a.y, -k.y, -k.w, v.y, v.w);    // - Im k Im v
      df_prod_acc(a.z, a.w, k.y, k.w, v.x, v.z);      // + Im k Re v
    }
  }
  static __device__ __forceinline__ void flush(acc_t &a, const inner_t &i) {
    df_add_acc(a.x, a.y, i.x, i.y);
    df_add_acc(a.z, a.w, i.z, i.w);
  }
  // value = (hi + lo) * scale, in FP64 (two conversions and one add per part)
  static __device__ __forceinline__ double2 finish(const acc_t &a, double scale, bool = false) {
    return make_double2(((double)a.x + (double)a.y) * scale, ((double)a.z + (double)a.w) * scale);
  }
};

// ---- FP32 storage, FP32-pair accumulation ----------------------------------
struct PolMixed {
  using vec_t = float2;
  using amp_t = float;
  using coef_t = float2;
  using acc_t = float4;    // (re_hi, re_lo, im_hi, im_lo)
  using inner_t = float2;  // FP32 partial sum over the additions of one removal
  static constexpr bool kInner = true;

  static __device__ __forceinline__ amp_t amul(amp_t a, amp_t b) { return a * b; }
  static __device__ __forceinline__ void zero(acc_t &a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void izero(inner_t &a) { a = make_float2(0.f, 0.f); }
  static __device__ __forceinline__ coef_t scale(coef_t c, amp_t x) { return make_float2(c.x * x, c.y * x); }
  static __device__ __forceinline__ void imac(inner_t &a, coef_t k, vec_t v, bool real) {
    a.x = fmaf(k.x, v.x, a.x);
    a.y = fmaf(k.x, v.y, a.y);
    if (!real) {
      a.x = fmaf(-k.y, v.y, a.x);
      a.y = fmaf(k.y, v.x, a.y);
    }
  }
  static __device__ __forceinline__ void flush(acc_t &a, const inner_t &i) {
    df_add_acc(a.x, a.y, i.x, 0.f);
    df_add_acc(a.z, a.w, i.y, 0.f);
  }
  // FP32 result: no FP64 instruction on this path.
  static __device__ __forceinline__ float2 finish(const acc_t &a, double scale, bool = false) {
    const float f = (float)scale;
    return make_float2(__fadd_rn(a.x, a.y) * f, __fadd_rn(a.z, a.w) * f);
  }
};

// ---- packed variants (sparse kernel) ---------------------------------------
// FP32 pairs on packed lanes.  With a real coefficient K the two lanes hold
// (Re, Im) of K C directly; with a complex one they hold P1 = (Re K Re C,
// Im K Im C) and P2 = (Im K Re C, Re K Im C), combined once at the end.
struct PolDFP {
  using vec_t = float4;    // (re_hi, im_hi, re_lo, im_lo)
  using amp_t = float2;
  using coef_t = float4;   // (re_hi, im_hi, re_lo, im_lo)
  struct acc_t { fp2_t h1, l1, h2, l2; };
  using inner_t = acc_t;
  static constexpr bool kInner = false;

  static __device__ __forceinline__ amp_t amul(amp_t a, amp_t b) { return df_mul(a, b); }
  static __device__ __forceinline__ void zero(acc_t &a) { a.h1 = a.l1 = a.h2 = a.l2 = 0ull; }
  static __device__ __forceinline__ coef_t scale(coef_t c, amp_t x) {
    fp2_t p, e;
    fp2_dprod(fp2_make(c.x, c.y), fp2_make(c.z, c.w), fp2_make(x.x, x.x), fp2_make(x.y, x.y), p, e);
    return make_float4(fp2_x(p), fp2_y(p), fp2_x(e), fp2_y(e));
  }
  static __device__ __forceinline__ void mac(acc_t &a, coef_t k, vec_t v, bool real) {
    const fp2_t Ch = fp2_make(v.x, v.y), Cl = fp2_make(v.z, v.w);
    fp2_t p, e;
    if (real) {
      fp2_dprod(fp2_make(k.x, k.x), fp2_make(k.z, k.z), Ch, Cl, p, e);
      fp2_dacc(a.h1, a.l1, p, e);
    } else {
      const fp2_t Kh = fp2_make(k.x, k.y), Kl = fp2_make(k.z, k.w);
      fp2_dprod(Kh, Kl, Ch, Cl, p, e);
      fp2_dacc(a.h1, a.l1, p, e);
      fp2_dprod(fp2_swap(Kh), fp2_swap(Kl), Ch, Cl, p, e);
      fp2_dacc(a.h2, a.l2, p, e);
    }
  }
  static __device__ __forceinline__ double2 finish(const acc_t &a, double scale, bool real) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (real) {
      df_add_acc(rh, rl, fp2_x(a.h1), fp2_x(a.l1));
      df_add_acc(ih, il, fp2_y(a.h1), fp2_y(a.l1));
    } else {
      df_add_acc(rh, rl, fp2_x(a.h1), fp2_x(a.l1));
      df_add_acc(rh, rl, -fp2_y(a.h1), -fp2_y(a.l1));
      df_add_acc(ih, il, fp2_x(a.h2), fp2_x(a.l2));
      df_add_acc(ih, il, fp2_y(a.h2), fp2_y(a.l2));
    }
    return make_double2(((double)rh + (double)rl) * scale, ((double)ih + (double)il) * scale);
  }
};

struct PolMixedP {
  using vec_t = float2;
  using amp_t = float;
  using coef_t = float2;
  struct acc_t { fp2_t h, l; };        // (Re, Im) as FP32 pairs
  struct inner_t { fp2_t i1, i2; };    // FP32 partial sums of one removal
  static constexpr bool kInner = true;

  static __device__ __forceinline__ amp_t amul(amp_t a, amp_t b) { return a * b; }
  static __device__ __forceinline__ void zero(acc_t &a) { a.h = a.l = 0ull; }
  static __device__ __forceinline__ void izero(inner_t &a) { a.i1 = a.i2 = 0ull; }
  static __device__ __forceinline__ coef_t scale(coef_t c, amp_t x) { return make_float2(c.x * x, c.y * x); }
  static __device__ __forceinline__ void imac(inner_t &a, coef_t k, vec_t v, bool real) {
    const fp2_t Cv = fp2_make(v.x, v.y);
    if (real) {
      a.i1 = fp2_fma(fp2_make(k.x, k.x), Cv, a.i1);
    } else {
      const fp2_t Kp = fp2_make(k.x, k.y);
      a.i1 = fp2_fma(Kp, Cv, a.i1);
      a.i2 = fp2_fma(fp2_swap(Kp), Cv, a.i2);
    }
  }
  static __device__ __forceinline__ void flush(acc_t &a, const inner_t &i, bool real) {
    const fp2_t part = real ? i.i1
                            : fp2_make(fp2_x(i.i1) - fp2_y(i.i1), fp2_x(i.i2) + fp2_y(i.i2));
    fp2_dacc(a.h, a.l, part, 0ull);
  }
  static __device__ __forceinline__ float2 finish(const acc_t &a, double scale, bool) {
    const float f = (float)scale;
    const fp2_t v = fp2_add(a.h, a.l);
    return make_float2(fp2_x(v) * f, fp2_y(v) * f);
  }
};
