// fock_device.cuh -- device helpers of libfock: decode (unrank) and rank with
// the binomial tables of a space.  See fock_common.cuh for the closed form of
// the hash these implement.
#pragma once

#include "fock_common.cuh"

// Greedy decoding of the combinatorial-number-system code (Algorithm 2 in
// closed form).  Fills the prefix sums S[0..M-1] (S[M-1] = N) of the
// configuration with index gamma.  `sat` is the saturated table of the index
// width; the inner search walks x downward and never passes C(m, m+1) = 0, so
// the total number of steps is at most N + M.
template <class Idx, int MAXM>
__device__ __forceinline__ void fock_decode_prefix(Idx gamma, int N, int M, Idx nc,
                                                   const Idx *__restrict__ sat, int xdim,
                                                   int (&S)[MAXM]) {
  Idx rem = nc - (Idx)1 - gamma;
  int x = N + M - 1;
#pragma unroll
  for (int m = MAXM - 2; m >= 0; --m) {
    if (m <= M - 2) {
      const Idx *row = sat + (size_t)m * xdim;
      int xx = x - 1;
      Idx v = row[xx];
      while (v > rem) {
        --xx;
        v = row[xx];
      }
      rem -= v;
      S[m] = xx - m;
      x = xx;
    }
  }
#pragma unroll
  for (int m = 0; m < MAXM; ++m)
    if (m >= M - 1) S[m] = N;
}

// Greedy decoding as fock_decode_prefix for a compile-time number of
// orbitals and 32-bit indices, with each search started at the closed-form
// estimate x ~ (k! r)^(1/k) + (k - 1)/2 of the largest x with C(x, k) <= r
// (k = m + 1, r the remaining rank) and corrected by single steps.  The table
// is non-decreasing in x, so the corrections end at the same x as the linear
// walk; they take one or two table reads instead of up to N + M.
template <int M>
__device__ __forceinline__ void fock_decode_fast(uint32_t gamma, int N, uint32_t nc, const uint32_t *__restrict__ sat,
                                                 int xdim, int (&S)[M]) {
  uint32_t rem = nc - 1u - gamma;
  int x = N + M - 1;
#pragma unroll
  for (int m = M - 2; m >= 0; --m) {
    const uint32_t *row = sat + m * xdim;
    int xx;
    if (m == 0) {
      xx = (int)min(rem, (uint32_t)(x - 1));            // C(x, 1) = x
    } else {
      float kf = 1.f;                                    // (m + 1)!
#pragma unroll
      for (int i = 2; i <= m + 1; ++i) kf *= (float)i;
      const float est = exp2f(__log2f((float)rem * kf) * (1.f / (m + 1))) + 0.5f * m;
      xx = min(max((int)est, m), x - 1);
      while (xx < x - 1 && row[xx + 1] <= rem) ++xx;
      while (row[xx] > rem) --xx;
    }
    rem -= row[xx];
    S[m] = xx - m;
    x = xx;
  }
  S[M - 1] = N;
}

// Index of the configuration with prefix sums S (S[M-1] = N).
template <class Idx, int MAXM>
__device__ __forceinline__ Idx fock_rank_prefix(const int (&S)[MAXM], int M, Idx nc,
                                                const Idx *__restrict__ mod, int xdim) {
  Idx acc = nc - (Idx)1;
#pragma unroll
  for (int m = 0; m < MAXM - 1; ++m)
    if (m <= M - 2) acc -= mod[(size_t)m * xdim + S[m] + m];
  return acc;
}

// 2^e for -1022 <= e <= 1023, built from the exponent field (exact, no call).
__device__ __forceinline__ double fock_pow2(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}
