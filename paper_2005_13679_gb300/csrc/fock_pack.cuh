// fock_pack.cuh -- packed FP32x2 arithmetic (sm_100+ `add/sub/mul/fma.rn.f32x2`)
// and FP32-pair (hi + lo) building blocks on packed lanes.
//
// A packed value holds two independent floats in one 64-bit register pair; one
// instruction updates both lanes.  The FP32-pair kernels keep the real and the
// imaginary parts of a complex quantity in the two lanes, so the error-free
// transformations (Dekker's product with FMA, Knuth's TwoSum) run on both parts
// with one instruction each.  Inline PTX keeps the compiler from contracting or
// reassociating the error-free sequences.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

typedef unsigned long long fp2_t;  // two packed floats: low word = .x, high word = .y

__device__ __forceinline__ fp2_t fp2_make(float x, float y) {
  fp2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float fp2_x(fp2_t a) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a));
  return x;
}
__device__ __forceinline__ float fp2_y(fp2_t a) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a));
  return y;
}
__device__ __forceinline__ fp2_t fp2_swap(fp2_t a) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a));
  return fp2_make(y, x);
}
__device__ __forceinline__ fp2_t fp2_add(fp2_t a, fp2_t b) {
  fp2_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ fp2_t fp2_sub(fp2_t a, fp2_t b) {
  fp2_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ fp2_t fp2_mul(fp2_t a, fp2_t b) {
  fp2_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ fp2_t fp2_fma(fp2_t a, fp2_t b, fp2_t c) {
  fp2_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// -a on both lanes (sign-bit flip; exact)
__device__ __forceinline__ fp2_t fp2_neg(fp2_t a) { return a ^ 0x8000000080000000ull; }
// d = a * b - c  (one rounding)
__device__ __forceinline__ fp2_t fp2_fms(fp2_t a, fp2_t b, fp2_t c) { return fp2_fma(a, b, fp2_neg(c)); }

// Product of pairs a = ah + al and b = bh + bl on both lanes: returns the
// rounded high product in *p and its error plus the cross terms in *e
// (al*bl is below 2^-46 relative and dropped).
__device__ __forceinline__ void fp2_dprod(fp2_t ah, fp2_t al, fp2_t bh, fp2_t bl, fp2_t &p, fp2_t &e) {
  p = fp2_mul(ah, bh);
  e = fp2_fms(ah, bh, p);
  e = fp2_fma(ah, bl, e);
  e = fp2_fma(al, bh, e);
}

// (h, l) += (p, e): TwoSum on the high words, errors into the low words.
__device__ __forceinline__ void fp2_dacc(fp2_t &h, fp2_t &l, fp2_t p, fp2_t e) {
  const fp2_t s = fp2_add(h, p);
  const fp2_t bb = fp2_sub(s, h);
  const fp2_t err = fp2_add(fp2_sub(h, fp2_sub(s, bb)), fp2_sub(p, bb));
  h = s;
  l = fp2_add(l, fp2_add(err, e));
}
