// fock_apply_tc.cuh -- phase 1 of the two-phase apply (fock_apply_twophase.cuh)
// on the fifth-generation tensor cores, with FP64-class accuracy.
//
// Phase 1 is the dense product Y = R X with R the P x P reduced coefficients
// and X[a][n'] = B_a(n') C[n' + a] over the (N-2)-particle configurations.  In
// real form (rows and columns interleaved as (Re, Im)) it is a 2P x 2P matrix
// times a 2P x (configurations x rhs) matrix.  Both factors are split into
// signed base-2^9 digits with a power-of-two scale per row of R and per column
// of X (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59 (2012)):
//
//     R~[rho][k] = 2^(e_rho - 8) sum_{i=1..6} rho_i 2^(-9(i-1)) + dR,   |rho_i| <= 256,
//     X[k][c]    = 2^(e_c - 8)   sum_{j=1..5} xi_j  2^(-9(j-1)) + dX,
//                  |xi_1|, |xi_2|, |xi_5| <= 256, |xi_3| <= 268, |xi_4| <= 513,
//
// with |R~[rho][k]| < 2^e_rho over the row and |X[k][c]| < 2^e_c over the
// column.  Digits are integers, exact in fp16.  The level sums
// S_l = sum_{i+j=l} sum_k rho_i xi_j, l = 2..7, hold at most five digit pairs,
// so |S_l| <= 2P * 256 * (256 + 256 + 268 + 513 + 256) = 16,654,848 < 2^24 at
// M = 6 (2P = 42): every partial sum is an integer below 2^24 and the tensor
// core's FP32 accumulation of S_l is exact in any order.  The epilogue forms
//
//     Y = 2^(e_rho + e_c - 16) sum_{l=2..7} 2^(-9(l-2)) S_l
//
// as an FP32 pair.  What the product leaves out, per entry (rho, c), with the
// unit u = 2^(e_rho + e_c - 16) of the level sums:
//   * levels 8..11 (i + j >= 8): at most 2P * 256 * 1293 * 2^-54 u, below
//     2^-46.2 2^(e_rho + e_c) at M = 6;
//   * the remainder of R~ after six digits, |dR| <= 2^-54 2^e_rho: below
//     2P 2^-54 2^(e_rho + e_c);
//   * the remainder of X after five digits, |dX| <= (2^-45 + 2^-59) 2^e_c:
//     below 2^-45 2^e_c ||R~_rho||_1;
//   * the combination into a pair: S2, S3 2^-9 and S4 2^-18 are added by TwoSum
//     (errors kept); S5 2^-27 + S6 2^-36 + S7 2^-45 (below 2^-3 u) is formed in
//     FP32, an error below 2^-27 u = 2^-43 2^(e_rho + e_c); the low word's own
//     rounding is below 2^-47 sum_k |R~[rho][k] X[k][c]|.
// With 2^e_c < 2 max_k |X[k][c]| and 2^e_rho < 2 max_k |R~[rho][k]| <= 2 ||R~_rho||_1,
//
//     |Y^[rho][c] - Y[rho][c]| <= 2^-40.5 ||R~_rho||_1 max_k |X[k][c]|,
//
// i.e. 6.3e-13 of the largest value the row can produce on that column (the
// X remainder alone gives 2^-44; the others count only when one coefficient
// dominates its row).
//
// The MMA computes the transposed product: its M = 128 rows are the tile's
// (configuration, rhs) columns, so tensor-memory lane c holds everything of
// column c, and its N columns are (real row, level) combinations in two
// blocks: columns 3 rho + (7 - l) hold levels l = 7, 6, 5 of real row rho
// (0 <= rho < 2P), column 3 * 2P receives the column exponent, and from N2 on
// columns N2 + 3 rho + (4 - l) hold levels 4, 3, 2.  K is ordered
// [digits 1..3 of every real index, interleaved, and the column exponent |
//  digits 4, 5 interleaved].  Digits 4 and 5 of X only meet levels 5..7, so
// the product runs as two MMA chains into the same accumulators: part 1, K1
// positions (digits 1..3) against all N1 columns, and part 2, K2 positions
// (digits 4, 5) against the first N2 columns only.  An epilogue thread reads
// its own lane, so no data crosses lanes.
#pragma once

#include <cuda_fp16.h>

#include "fock_apply_twophase.cuh"
#include "fock_tc.cuh"

constexpr int kTcCols = 128;        // (configuration, rhs) columns per tile = MMA M
constexpr int kTcProducers = 128;   // producer group: 4 warps, one thread per column
constexpr int kTcThreads = 512;     // two producer groups (warps 0-3 even tiles, 4-7 odd tiles),
                                    // warps 8-15 epilogue (warp 8 + q + 4h: tile columns 32q .. 32q+31,
                                    // alternate passes of rows by h); lane 0 of warp 8 also issues the MMAs
constexpr int kTcEpiWarps = 8;
constexpr int kTcMmaWarp = 8;
constexpr int kTcTmemCols = 512;    // two tiles x NT (<= 256) columns, at 0 and 256
constexpr uint32_t kTcPolls = 1u << 20;
constexpr int kTcExpCol = 15;       // tensor-memory column of the column exponent

// Shape of the real-form product for M orbitals (2 <= M <= 6).
struct TcShape {
  int P, R2, K1, K2, KT, N2, N1;
  __host__ __device__ constexpr explicit TcShape(int m)
      : P(m * (m + 1) / 2), R2(m * (m + 1)), K1((3 * m * (m + 1) + 1 + 15) / 16 * 16),
        K2((2 * m * (m + 1) + 15) / 16 * 16),
        KT((3 * m * (m + 1) + 1 + 15) / 16 * 16 + (2 * m * (m + 1) + 15) / 16 * 16),
        N2((3 * m * (m + 1) + 1 + 15) / 16 * 16),
        N1(((3 * m * (m + 1) + 1 + 15) / 16 * 16 + 3 * m * (m + 1) + 15) / 16 * 16) {}
  // bytes of the coefficient image: part 1 (N1 rows x K1), then part 2 (N2 rows x K2), fp16
  __host__ __device__ constexpr int r1_bytes() const { return N1 * K1 * 2; }
  __host__ __device__ constexpr int r_bytes() const { return N1 * K1 * 2 + N2 * K2 * 2; }
  // bytes of one digit tile (128 columns x KT)
  __host__ __device__ constexpr int b_bytes() const { return kTcCols * KT * 2; }
  // K position of the column exponent (the last of part 1, never a digit)
  __host__ __device__ constexpr int exp_pos() const { return K1 - 1; }
  // tensor-memory column of the column exponent
  __host__ __device__ constexpr int exp_col() const { return 3 * R2; }
  // additions swept by the producer, padding included, so that every 16-byte
  // chunk of both K parts is written
  __host__ __device__ constexpr int a_end() const {
    const int c1 = (K1 + 5) / 6, c2 = K2 / 4;
    const int m = P > c1 ? (P > c2 ? P : c2) : (c1 > c2 ? c1 : c2);
    return (m + 3) / 4 * 4;
  }
  // tensor-memory column of level l (2..7) of real row rho
  __host__ __device__ constexpr int col(int rho, int l) const {
    return l >= 5 ? 6 * (rho >> 1) + 2 * (7 - l) + (rho & 1) : N2 + 6 * (rho >> 1) + 2 * (4 - l) + (rho & 1);
  }
};

// Shared-memory layout of the kernel for a policy with an image of r_bytes,
// kt-deep digit tiles, r2 row exponents and a square-root table of sq_bytes
// per entry.
struct TcSmem {
  size_t off_r, off_b0, off_b1, off_er, off_mod, off_sat, off_sq, off_bar, total;
  __host__ __device__ TcSmem(int r_bytes, int kt, int r2, int M, int xdim, int nsq, int sq_bytes) {
    const int rows = M > 1 ? M - 1 : 1;
    size_t o = 0;
    off_r = o;    o += (size_t)r_bytes;
    off_b0 = o;   o += (size_t)kTcCols * kt * 2;
    off_b1 = o;   o += (size_t)kTcCols * kt * 2;
    off_er = o;   o = fock_align16(o + 4 * (size_t)r2 + 8 * (size_t)r2 + 16);
    off_mod = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sat = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sq = o;   o = fock_align16(o + (size_t)sq_bytes * nsq);
    off_bar = o;  o = fock_align16(o + 6 * 8 + 8);
    total = o;
  }
};

// Shape of the FP32-mixed product: one accumulator per real row, K holds
// [X_h | 2^11 X_l | X_h] of the 2P real indices and the column exponent.
struct TcMixedShape {
  int P, R2, NT, KT;
  __host__ __device__ constexpr explicit TcMixedShape(int m)
      : P(m * (m + 1) / 2), R2(m * (m + 1)), NT((m * (m + 1) + 1 + 15) / 16 * 16),
        KT((3 * m * (m + 1) + 1 + 15) / 16 * 16) {}
  __host__ __device__ constexpr int r_bytes() const { return NT * KT * 2; }
  __host__ __device__ constexpr int exp_pos() const { return 3 * R2; }
};

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float tc_pow2(int e) { return __int_as_float((e + 127) << 23); }

// Multiply a pair by 2^e exactly for any e (two factors when e leaves the
// single-float range; that happens only for columns or rows ~2^-118 below the
// largest amplitude).
__device__ __forceinline__ void tc_scale(float &h, float &l, int e) {
  if (e >= -126 && e <= 127) {
    const float f = tc_pow2(e);
    h = __fmul_rn(h, f);
    l = __fmul_rn(l, f);
  } else {
    const int e1 = max(-126, min(127, e)), e2 = max(-126, min(127, e - e1));
    const float f1 = tc_pow2(e1), f2 = tc_pow2(e2);
    h = __fmul_rn(__fmul_rn(h, f1), f2);
    l = __fmul_rn(__fmul_rn(l, f1), f2);
  }
}

// The row (hi, lo) packed pair scaled by 2^e0 (Re) and 2^e1 (Im), any
// exponents: the rare path of the epilogue, kept out of line.
__device__ __noinline__ float4 tc_scale_row(fp2_t hi, fp2_t lo, int e0, int e1) {
  float h0 = fp2_x(hi), h1 = fp2_y(hi), l0 = fp2_x(lo), l1 = fp2_y(lo);
  tc_scale(h0, l0, e0);
  tc_scale(h1, l1, e1);
  return make_float4(h0, h1, l0, l1);
}

constexpr float kTcMagic = 12582912.f;   // 1.5 * 2^23

// One digit on both packed lanes without negations: from x (true sign) with
// m and nm = -m, d = RN(x m) and y = d - x m (the remainder, negated); from a
// negated remainder y with the constants -512 and 512, d = RN(512 r) and the
// next negated remainder d - 512 r.  |x m| < 2^22, m a power of two, so
// every step is exact (the 1.5 * 2^23 rounding of the FP32 significand).
__device__ __forceinline__ fp2_t tc_digit2(fp2_t x, fp2_t m, fp2_t nm, fp2_t &y) {
  const fp2_t mg = fp2_make(kTcMagic, kTcMagic);
  const fp2_t d = fp2_sub(fp2_fma(x, m, mg), mg);
  y = fp2_fma(x, nm, d);
  return d;
}

// Digits of v = (xh + xl) 2^E on both lanes (the real and imaginary parts of
// one complex value of X at its column scale; f = 2^E, f18 = 2^(E+18),
// |xh f| < 256, |xl f| <= 3 2^-16):
//     v = c1 + c2 2^-9 + c3 2^-18 + c4 2^-27 + c5 2^-36 + r,   |r| <= 2^-37 (+ 2^-51).
// The high word gives c1..c4 with exact remainders, the low word adds to c3
// and c4, the two remainders share c5 (their FP32 sum is rounded far below
// the digit's unit), and one carry folds c5 back into [-256, 256]:
// |c1|, |c2|, |c5| <= 256, |c3| <= 268, |c4| <= 513.  27 packed operations.
__device__ __forceinline__ void tc_digits2(fp2_t xh, fp2_t xl, fp2_t f, fp2_t nf, fp2_t f18, fp2_t nf18,
                                           fp2_t (&c)[5]) {
  const fp2_t k512 = fp2_make(512.f, 512.f), n512 = fp2_make(-512.f, -512.f);
  const fp2_t i512 = fp2_make(1.f / 512.f, 1.f / 512.f), mg = fp2_make(kTcMagic, kTcMagic);
  fp2_t y, u;
  c[0] = tc_digit2(xh, f, nf, y);            // y = -(remainder)
  c[1] = tc_digit2(y, n512, k512, y);
  const fp2_t d3 = tc_digit2(y, n512, k512, y);
  const fp2_t d4 = tc_digit2(y, n512, k512, y);
  const fp2_t e3 = tc_digit2(xl, f18, nf18, u);
  const fp2_t e4 = tc_digit2(u, n512, k512, u);
  const fp2_t c5 = fp2_sub(fp2_fma(fp2_add(y, u), n512, mg), mg);    // RN(512 (r_hi + r_lo))
  const fp2_t q = fp2_sub(fp2_fma(c5, i512, mg), mg);
  c[4] = fp2_fma(q, n512, c5);
  c[3] = fp2_add(fp2_add(d4, e4), q);
  c[2] = fp2_add(d3, e3);
}

__device__ __forceinline__ uint32_t tc_pack(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Addition pairs (s, l), s <= l, in lexicographic order, as compile-time tables.
template <int M>
struct TcPairs {
  int s[M * (M + 1) / 2], l[M * (M + 1) / 2];
  __host__ __device__ constexpr TcPairs() : s(), l() {
    int a = 0;
    for (int i = 0; i < M; ++i)
      for (int j = i; j < M; ++j) {
        s[a] = i;
        l[a] = j;
        ++a;
      }
  }
};

// Addition pair (s, l), s <= l, of index a in lexicographic order.
__host__ __device__ constexpr int tc_pair_s(int M, int a) {
  int s = 0;
  while (a >= M - s) { a -= M - s; ++s; }
  return s;
}
__host__ __device__ constexpr int tc_pair_l(int M, int a) {
  int s = 0;
  while (a >= M - s) { a -= M - s; ++s; }
  return s + a;
}

// ---------------------------------------------------------------------------
// mbarrier helpers of the pipeline
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tc_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem_addr(bar)) : "memory");
}

// Bounded wait (at most `polls` polls) that also gives up as soon as another
// role raised the abort flag.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *flag, uint32_t polls) {
  for (uint32_t i = 0; i < polls; ++i) {
    if (tc_mbar_try_wait(bar, parity)) return true;
    if (*flag) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_abort(volatile int *flag, int *status) {
  *flag = 1;
  if (status) atomicExch(status, 1);
}

// ---------------------------------------------------------------------------
// Producer: digits of one column of X (all P additions) into the B operand
// (K-major, 128 columns x KT), the column exponent at K position exp_pos().
// The P gathers of C are issued together before any arithmetic.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void tc_produce(const TwoPhaseArgs &t, uint32_t tile, uint32_t total, int cl,
                                           unsigned char *bbuf, const uint32_t *s_mod, const uint32_t *s_sat,
                                           const float2 *s_sq) {
  constexpr TcShape sh(M);
  constexpr int P = sh.P;
  constexpr int AE = sh.a_end();
  constexpr int CH1 = sh.K1 / 8, CH2 = sh.K2 / 8, CHT = sh.KT / 8;
  const ApplyArgs<uint32_t> &a = t.a;
  const uint32_t col = tile * (uint32_t)kTcCols + cl;
  const uint32_t cc = col < total ? col : total - 1u;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const uint32_t np = nrhs == 1u ? cc : cc / nrhs;
  const int jr = (int)(cc - np * nrhs);

  int S[M];
  fock_decode_fast<M>(np, a.N - 2, t.nc2, s_sat, a.xdim, S);
  uint32_t U[M], V[M];
  const uint32_t base = twophase_targets<M>(S, s_mod, a.xdim, a.nc, U, V);
  float2 sq1[M], sq2[M];                                // sqrt(n'_m + 1), sqrt(n'_m + 2) as pairs
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int occ = S[m] - (m > 0 ? S[m - 1] : 0);
    sq1[m] = s_sq[occ + 1];
    sq2[m] = s_sq[occ + 2];
  }

  // all P gathers first, then X = B_a(n') C[n' + a] as FP32 pairs in place
  constexpr TcPairs<M> pr;
  const float4 *__restrict__ C = (const float4 *)a.C;
  float4 v[P];
#pragma unroll
  for (int ai = 0; ai < P; ++ai) {
    const int s = pr.s[ai], l = pr.l[ai];
    v[ai] = __ldg(C + (size_t)(base - U[s] - V[l]) * nrhs + jr);
  }
  float vmax = 0.f;
#pragma unroll
  for (int ai = 0; ai < P; ++ai) {
    const int s = pr.s[ai], l = pr.l[ai];
    const float2 amp = df_mul(sq1[s], s == l ? sq2[s] : sq1[l]);
    fp2_t Xh, Xl;
    fp2_dprod(fp2_make(v[ai].x, v[ai].y), fp2_make(v[ai].z, v[ai].w), fp2_make(amp.x, amp.x),
              fp2_make(amp.y, amp.y), Xh, Xl);
    v[ai] = make_float4(fp2_x(Xh), fp2_y(Xh), fp2_x(Xl), fp2_y(Xl));   // (Re hi, Im hi, Re lo, Im lo)
    vmax = fmaxf(vmax, fmaxf(fabsf(v[ai].x), fabsf(v[ai].y)));
  }
  const int field = (int)((__float_as_uint(vmax) >> 23) & 0xffu);
  const int e_c = field > 0 ? field - 126 : 0;         // |X| < 2^e_c; all-zero column: digits 0
  int E = 8 - e_c;                                      // v = X 2^E, |v| < 256
  if (E > 109) {                                        // columns ~2^-100 below the largest amplitude:
#pragma unroll                                          // pre-scale so that 2^(E+18) stays a float
    for (int ai = 0; ai < P; ++ai) {
      v[ai].x = __fmul_rn(v[ai].x, 0x1p64f); v[ai].y = __fmul_rn(v[ai].y, 0x1p64f);
      v[ai].z = __fmul_rn(v[ai].z, 0x1p64f); v[ai].w = __fmul_rn(v[ai].w, 0x1p64f);
    }
    E -= 64;
  }
  const float f = tc_pow2(E), f18 = tc_pow2(E + 18);
  const fp2_t F = fp2_make(f, f), NF = fp2_make(-f, -f), F18 = fp2_make(f18, f18), NF18 = fp2_make(-f18, -f18);

  unsigned char *colbase = bbuf + (size_t)(cl >> 3) * (CHT * 128) + (cl & 7) * 16;
#pragma unroll
  for (int bi = 0; bi < AE / 4; ++bi) {
    fp2_t dig[4][5];                                    // four additions, (Re, Im) lanes
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int ai = 4 * bi + r;
      if (ai < P) {
        const float4 x = v[ai];
        tc_digits2(fp2_make(x.x, x.y), fp2_make(x.z, x.w), F, NF, F18, NF18, dig[r]);
      } else {
#pragma unroll
        for (int j = 0; j < 5; ++j) dig[r][j] = 0ull;
      }
    }
    // digit j (1-based) of real index 8 bi + rr, rr = 2 (addition) + (0 Re, 1 Im)
    auto D = [&](int rr, int j) -> float { return (rr & 1) ? fp2_y(dig[rr >> 1][j - 1]) : fp2_x(dig[rr >> 1][j - 1]); };
    // part 1: positions 3k + (j - 1), j = 1..3; the exponent at exp_pos()
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const int chunk = 3 * bi + ch;
      if (chunk < CH1) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p0 = 8 * ch + 2 * e, p1 = p0 + 1;
          const float lo = D(p0 / 3, p0 % 3 + 1);
          const float hi = 8 * chunk + 2 * e + 1 == sh.exp_pos() ? (float)e_c : D(p1 / 3, p1 % 3 + 1);
          w[e] = tc_pack(lo, hi);
        }
        *(uint4 *)(colbase + chunk * 128) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    // part 2: positions 2k + (j - 4), j = 4, 5
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
      const int chunk = 2 * bi + ch;
      if (chunk < CH2) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = tc_pack(D((8 * ch + 2 * e) / 2, 4), D((8 * ch + 2 * e) / 2, 5));
        *(uint4 *)(colbase + (CH1 + chunk) * 128) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// Combination of the six level sums of two real rows (packed lanes) into
// FP32 pairs: V = s2 + s3 2^-9 + s4 2^-18 + s5 2^-27 + s6 2^-36 + s7 2^-45
// with the s_l exact integers below 2^24.  The scalings are exact; s2, s3 2^-9
// and s4 2^-18 are added by TwoSum (errors collected in e); the lower levels,
// below 2^-3 of the unit, are formed in FP32 (error below 2^-27 of the unit)
// and join e.
__device__ __forceinline__ void tc_combine2(fp2_t s2, fp2_t s3, fp2_t s4, fp2_t s5, fp2_t s6, fp2_t s7, fp2_t &hi,
                                            fp2_t &lo) {
  const fp2_t a3 = fp2_mul(s3, fp2_make(0x1p-9f, 0x1p-9f));
  const fp2_t a4 = fp2_mul(s4, fp2_make(0x1p-18f, 0x1p-18f));
  const fp2_t a57 = fp2_fma(s7, fp2_make(0x1p-45f, 0x1p-45f),
                            fp2_fma(s6, fp2_make(0x1p-36f, 0x1p-36f), fp2_mul(s5, fp2_make(0x1p-27f, 0x1p-27f))));
  fp2_t s = fp2_add(s2, a3);
  fp2_t bb = fp2_sub(s, s2);
  fp2_t e = fp2_add(fp2_sub(s2, fp2_sub(s, bb)), fp2_sub(a3, bb));
  const fp2_t t = fp2_add(s, a4);
  bb = fp2_sub(t, s);
  e = fp2_add(e, fp2_add(fp2_sub(s, fp2_sub(t, bb)), fp2_sub(a4, bb)));
  e = fp2_add(e, a57);
  hi = fp2_add(t, e);
  lo = fp2_sub(e, fp2_sub(hi, t));
}

// ---------------------------------------------------------------------------
// FP32-mixed producer: X = B_a(n') C[n' + a] in FP32 from complex64 C, the
// column scaled by 2^E so that |X 2^E| < 2^15, and each real value split into
// fp16 x_h = RN(X 2^E) and x_l = RN(2^11 (X 2^E - x_h)).
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void tc_produce_mixed(const TwoPhaseArgs &t, uint32_t tile, uint32_t total, int cl,
                                                 unsigned char *bbuf, const uint32_t *s_mod, const uint32_t *s_sat,
                                                 const float *s_sq) {
  constexpr TcMixedShape sh(M);
  constexpr int P = sh.P, R2 = sh.R2, CHT = sh.KT / 8;
  const ApplyArgs<uint32_t> &a = t.a;
  const uint32_t col = tile * (uint32_t)kTcCols + cl;
  const uint32_t cc = col < total ? col : total - 1u;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const uint32_t np = nrhs == 1u ? cc : cc / nrhs;
  const int jr = (int)(cc - np * nrhs);
  int S[M];
  fock_decode_fast<M>(np, a.N - 2, t.nc2, s_sat, a.xdim, S);
  uint32_t U[M], V[M];
  const uint32_t base = twophase_targets<M>(S, s_mod, a.xdim, a.nc, U, V);
  float sq1[M], sq2[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int occ = S[m] - (m > 0 ? S[m - 1] : 0);
    sq1[m] = s_sq[occ + 1];
    sq2[m] = s_sq[occ + 2];
  }
  constexpr TcPairs<M> pr;
  const float2 *__restrict__ C = (const float2 *)a.C;
  float x[R2];
#pragma unroll
  for (int ai = 0; ai < P; ++ai) {
    const float2 v = __ldg(C + (size_t)(base - U[pr.s[ai]] - V[pr.l[ai]]) * nrhs + jr);
    x[2 * ai] = v.x;
    x[2 * ai + 1] = v.y;
  }
  uint32_t ebits = 0;
#pragma unroll
  for (int ai = 0; ai < P; ++ai) {
    const int s = pr.s[ai], l = pr.l[ai];
    const float amp = sq1[s] * (s == l ? sq2[s] : sq1[l]);
    x[2 * ai] *= amp;
    x[2 * ai + 1] *= amp;
    ebits = max(ebits, max(__float_as_uint(x[2 * ai]) & 0x7f800000u, __float_as_uint(x[2 * ai + 1]) & 0x7f800000u));
  }
  const int field = (int)(ebits >> 23);
  const int e_c = field > 0 ? field - 126 : 0;          // |X| < 2^e_c
  int E = 15 - e_c;
  if (E > 127) {                                         // columns ~2^-112 below the largest amplitude
#pragma unroll
    for (int k = 0; k < R2; ++k) x[k] = __fmul_rn(x[k], 0x1p64f);
    E -= 64;
  }
  const float f = tc_pow2(E);
  __half xh[R2], xl[R2];
#pragma unroll
  for (int k = 0; k < R2; ++k) {
    const float v = __fmul_rn(x[k], f);
    xh[k] = __float2half_rn(v);
    xl[k] = __float2half_rn(__fmul_rn(__fsub_rn(v, __half2float(xh[k])), 2048.f));
  }
  const __half hexp = __float2half_rn((float)e_c);
  const __half hz = __float2half_rn(0.f);
  unsigned char *colbase = bbuf + (size_t)(cl >> 3) * (CHT * 128) + (cl & 7) * 16;
#pragma unroll
  for (int ch = 0; ch < CHT; ++ch) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __half hv[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int p = 8 * ch + 2 * e + u;
        hv[u] = p < R2 ? xh[p] : p < 2 * R2 ? xl[p - R2] : p < 3 * R2 ? xh[p - 2 * R2] : p == 3 * R2 ? hexp : hz;
      }
      w[e] = (uint32_t)__half_as_ushort(hv[0]) | ((uint32_t)__half_as_ushort(hv[1]) << 16);
    }
    *(uint4 *)(colbase + ch * 128) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------------------
// Policies: shapes, producer, square-root table and epilogue of the two forms.
// ---------------------------------------------------------------------------
template <int M>
struct TcPolDF {                                         // FP64-class: exact digits, level sums
  static constexpr TcShape sh{M};
  static constexpr int NT = sh.N1, KT = sh.KT, R2 = sh.R2, R_BYTES = sh.r_bytes();
  using sq_t = float2;
  __device__ static void produce(const TwoPhaseArgs &t, uint32_t tile, uint32_t total, int cl, unsigned char *bbuf,
                                 const uint32_t *s_mod, const uint32_t *s_sat, const void *s_sq) {
    tc_produce<M>(t, tile, total, cl, bbuf, s_mod, s_sat, (const float2 *)s_sq);
  }
  // The two MMA chains of one tile into the accumulators at d: part 1 (digits
  // 1..3 and the exponent, K1) against all N1 columns, then part 2 (digits 4,
  // 5, K2) against the first N2 columns (levels 5..7).
  __device__ static void issue(uint32_t d, uint32_t x_addr, uint32_t r_addr) {
    constexpr int CHT = KT / 8, CH1 = sh.K1 / 8, CH2 = sh.K2 / 8;
    constexpr uint32_t idesc1 = tc_idesc_f16(kTcCols, sh.N1), idesc2 = tc_idesc_f16(kTcCols, sh.N2);
    const uint32_t r2_addr = r_addr + (uint32_t)sh.r1_bytes();
#pragma unroll
    for (int kk = 0; kk < sh.K1 / 16; ++kk)
      tc_mma_f16(d, tc_desc_kmajor(x_addr + kk * 256, 128, CHT * 128), tc_desc_kmajor(r_addr + kk * 256, 128, CH1 * 128),
                 idesc1, kk > 0);
#pragma unroll
    for (int kk = 0; kk < sh.K2 / 16; ++kk)
      tc_mma_f16(d, tc_desc_kmajor(x_addr + CH1 * 128 + kk * 256, 128, CHT * 128),
                 tc_desc_kmajor(r2_addr + kk * 256, 128, CH2 * 128), idesc2, 1u);
  }
  // Lane-local epilogue in passes of four complex rows: levels 7, 6, 5 of a
  // complex row r sit in columns 6r .. 6r+5 (Re row, then Im row) and levels
  // 4, 3, 2 in N2 + 6r .. N2 + 6r + 5, read as 16- and 8-column loads (a
  // full pass; 8-column loads for the last, partial one).  The two warps
  // of a lane quarter take alternate passes (half = pass & 1), last pass
  // first; the column exponent is read with a warp's first loads.
  __device__ static void drain(const TwoPhaseArgs &t, uint32_t tq, uint32_t colg, bool live, const int *s_er, int half) {
    constexpr int P = sh.P, NPASS = (P + 3) / 4;
    float4 *__restrict__ Y = (float4 *)t.Y;
    const float ecf = tc_ld_x1(tq + (uint32_t)sh.exp_col());
    int ec = 0;
    bool fast = false, first = true;
    fp2_t FC = 0ull;
    const float *s_fr = (const float *)(s_er + 2 * P + ((2 * P) & 1));
    // this warp's passes: p0, p0 - 2, ... (p0 the last pass of its parity)
    const int p0 = (NPASS - 1) - (((NPASS - 1) & 1) ^ half);
#pragma unroll 1
    for (int pass = p0; pass >= 0; pass -= 2) {
      const int nrow = P - 4 * pass < 4 ? P - 4 * pass : 4;
      float A[24], B[24];
      if (nrow == 4) {
        tc_ld_x16(tq + (uint32_t)(24 * pass), *reinterpret_cast<float(*)[16]>(&A[0]));
        tc_ld_x8(tq + (uint32_t)(24 * pass + 16), *reinterpret_cast<float(*)[8]>(&A[16]));
        tc_ld_x16(tq + (uint32_t)(sh.N2 + 24 * pass), *reinterpret_cast<float(*)[16]>(&B[0]));
        tc_ld_x8(tq + (uint32_t)(sh.N2 + 24 * pass + 16), *reinterpret_cast<float(*)[8]>(&B[16]));
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (6 * nrow > 8 * c) {
            tc_ld_x8(tq + (uint32_t)(24 * pass + 8 * c), *reinterpret_cast<float(*)[8]>(&A[8 * c]));
            tc_ld_x8(tq + (uint32_t)(sh.N2 + 24 * pass + 8 * c), *reinterpret_cast<float(*)[8]>(&B[8 * c]));
          }
      }
      tc_wait_ld();
      if (first) {
        first = false;
        ec = (int)ecf - 16;
        const int *rng = (const int *)(s_fr + 2 * P);
        // both factors and their product stay normal floats: one product per row
        fast = rng[0] >= -126 && rng[1] <= 127 && ec >= -126 && ec <= 127 && rng[0] + ec >= -126 && rng[1] + ec <= 127;
        FC = fp2_make(tc_pow2(max(-126, min(127, ec))), tc_pow2(max(-126, min(127, ec))));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j < nrow) {
          const int r = 4 * pass + j;                    // complex row
          fp2_t hi, lo;
          tc_combine2(fp2_make(B[6 * j + 4], B[6 * j + 5]), fp2_make(B[6 * j + 2], B[6 * j + 3]),
                      fp2_make(B[6 * j], B[6 * j + 1]), fp2_make(A[6 * j + 4], A[6 * j + 5]),
                      fp2_make(A[6 * j + 2], A[6 * j + 3]), fp2_make(A[6 * j], A[6 * j + 1]), hi, lo);
          float4 y;
          if (fast) {
            const float2 fr = *(const float2 *)(s_fr + 2 * r);
            const fp2_t sc = fp2_mul(fp2_make(fr.x, fr.y), FC);
            hi = fp2_mul(hi, sc);
            lo = fp2_mul(lo, sc);
            y = make_float4(fp2_x(hi), fp2_y(hi), fp2_x(lo), fp2_y(lo));
          } else {
            y = tc_scale_row(hi, lo, s_er[2 * r] + ec, s_er[2 * r + 1] + ec);
          }
          if (live) __stcs(&Y[twophase_yidx(r, colg, P)], y);
        }
      }
    }
  }
};

template <int M>
struct TcPolMixed {                                      // FP32-mixed: fp16 hi/lo split, one accumulator per row
  static constexpr TcMixedShape sh{M};
  static constexpr int NT = sh.NT, KT = sh.KT, R2 = sh.R2, R_BYTES = sh.r_bytes();
  using sq_t = float;
  __device__ static void produce(const TwoPhaseArgs &t, uint32_t tile, uint32_t total, int cl, unsigned char *bbuf,
                                 const uint32_t *s_mod, const uint32_t *s_sat, const void *s_sq) {
    tc_produce_mixed<M>(t, tile, total, cl, bbuf, s_mod, s_sat, (const float *)s_sq);
  }
  // One MMA chain of the tile: K = KT against all NT columns.
  __device__ static void issue(uint32_t d, uint32_t x_addr, uint32_t r_addr) {
    constexpr int CHT = KT / 8;
    constexpr uint32_t idesc = tc_idesc_f16(kTcCols, NT);
#pragma unroll
    for (int kk = 0; kk < KT / 16; ++kk)
      tc_mma_f16(d, tc_desc_kmajor(x_addr + kk * 256, 128, CHT * 128), tc_desc_kmajor(r_addr + kk * 256, 128, CHT * 128),
                 idesc, kk > 0);
  }
  // Y = D 2^(e_rho + e_c - 30): the row scale 2^(15 - e_rho) of the image and
  // the column scale 2^(15 - e_c) of the digits taken out.  The epilogue is
  // light (one scaling per value), so only the second warp of a lane quarter
  // drains (the first warp of the first quarter issues the MMAs); the others
  // only keep the barrier count.
  __device__ static void drain(const TwoPhaseArgs &t, uint32_t tq, uint32_t colg, bool live, const int *s_er, int half) {
    constexpr int P = M * (M + 1) / 2;
    float2 *__restrict__ Y = (float2 *)t.Y;
    if (!half) return;
    float d[NT];
#pragma unroll
    for (int i = 0; i < NT / 16; ++i) tc_ld_x16(tq + (uint32_t)(16 * i), *reinterpret_cast<float(*)[16]>(&d[16 * i]));
    tc_wait_ld();
    const int ec = (int)d[R2] - 30;
#pragma unroll
    for (int r = 0; r < P; ++r) {
      float v[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int e = s_er[2 * r + c] + ec;
        v[c] = e >= -126 ? __fmul_rn(d[2 * r + c], tc_pow2(e))
                         : __fmul_rn(__fmul_rn(d[2 * r + c], tc_pow2(-126)), tc_pow2(max(e + 126, -126)));
      }
      if (live) __stcs(&Y[twophase_yidx(r, colg, P)], make_float2(v[0], v[1]));
    }
  }
};

template <class Pol, int M>
__host__ __device__ inline TcSmem tc_smem_of(int xdim, int nsq) {
  return TcSmem(Pol::R_BYTES, Pol::KT, Pol::R2, M, xdim, nsq, (int)sizeof(typename Pol::sq_t));
}

// ---------------------------------------------------------------------------
// The kernel: persistent, one CTA per SM, tiles of 128 columns, three roles
// joined by mbarriers (slot s = tile & 1 for the digit tile and the tensor
// memory of a tile):
//   producers (warps 0-3 for even k, warps 4-7 for odd k)
//                           wait done[s] of tile k-2, write B[s], arrive full[s]
//   MMA (warp 8, lane 0)    after draining tile k: wait full[s] of tile k+2 and empty[s] of
//                           tile k, issue, commit done[s] (tiles 0 and 1 before the loop)
//   epilogue (warps 8-15)   wait done[s], drain tensor memory (warp w reads TMEM lanes
//                           32 (w % 4) .. +31; warps w and w + 4 take alternate passes
//                           of four complex rows), write Y, arrive empty[s] (8 arrivals)
// ---------------------------------------------------------------------------
template <int M, class Pol>
__global__ void __launch_bounds__(kTcThreads, 1) fock_twophase_x_tc(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const TcSmem L = tc_smem_of<Pol, M>(a.xdim, a.nsq);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows = M > 1 ? M - 1 : 1;

  // stage the coefficient image, row exponents and tables
  {
    const uint4 *src = (const uint4 *)t.tc_a;
    uint4 *dst = (uint4 *)(smem + L.off_r);
    for (int i = tid; i < Pol::R_BYTES / 16; i += kTcThreads) dst[i] = __ldg(src + i);
    int *s_er = (int *)(smem + L.off_er);
    for (int i = tid; i < Pol::R2; i += kTcThreads) s_er[i] = __ldg(t.tc_er + i);
    float *s_fr = (float *)(s_er + Pol::R2 + (Pol::R2 & 1));       // 2^e_rho as floats (clamped)
    for (int i = tid; i < Pol::R2; i += kTcThreads) {
      const int e = __ldg(t.tc_er + i);
      s_fr[i] = tc_pow2(max(-126, min(127, e)));
    }
    if (tid == 0) {
      int lo = 1 << 30, hi = -(1 << 30);
      for (int i = 0; i < Pol::R2; ++i) { lo = min(lo, __ldg(t.tc_er + i)); hi = max(hi, __ldg(t.tc_er + i)); }
      ((int *)(s_fr + Pol::R2))[0] = lo;
      ((int *)(s_fr + Pol::R2))[1] = hi;
    }
    uint32_t *s_mod = (uint32_t *)(smem + L.off_mod), *s_sat = (uint32_t *)(smem + L.off_sat);
    for (int i = tid; i < rows * a.xdim; i += kTcThreads) {
      s_mod[i] = a.mod[i];
      s_sat[i] = a.sat[i];
    }
    using sq_t = typename Pol::sq_t;
    sq_t *s_sq = (sq_t *)(smem + L.off_sq);
    for (int i = tid; i < a.nsq; i += kTcThreads) s_sq[i] = ((const sq_t *)a.sq)[i];
  }
  tc_fence_proxy_async();                                // the image is read by the tensor core
  uint64_t *full = (uint64_t *)(smem + L.off_bar), *done = full + 2, *empty = full + 4;
  uint32_t *tslot = (uint32_t *)(full + 6);
  volatile int *flag = (volatile int *)(tslot + 1);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc_mbar_init(&full[i], kTcProducers);
      tc_mbar_init(&done[i], 1);
      tc_mbar_init(&empty[i], kTcEpiWarps);
    }
    *flag = 0;
    tc_fence_mbar_init();
  }
  if (warp == kTcMmaWarp) tc_tmem_alloc(tslot, kTcTmemCols);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = *tslot;

  // tiles [tb, te) of this launch: columns [c_begin, c_end), c_begin a multiple of the tile
  const uint32_t total = (uint32_t)t.c_end;
  const uint32_t tb = (uint32_t)(t.c_begin / kTcCols), te = (total + kTcCols - 1) / kTcCols;
  const uint32_t ntiles = te - tb;
  const uint32_t mytiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  uint32_t issued = 0;                                   // MMA role: tiles committed

  if (warp < 8) {
    // ---------------- producers: group g = warp / 4 takes tiles k = g, g + 2, ... ----------------
    const int g = warp >> 2, cl = tid & (kTcProducers - 1);
    const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
    const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
    const void *s_sq = smem + L.off_sq;
    unsigned char *bbuf = smem + (g ? L.off_b1 : L.off_b0);
    for (uint32_t k = g; k < mytiles; k += 2) {
      if (k >= 2 && !tc_wait(&done[g], ((k - 2) >> 1) & 1u, flag, t.polls)) {
        tc_abort(flag, t.status);
        break;
      }
      Pol::produce(t, tb + blockIdx.x + k * gridDim.x, total, cl, bbuf, s_mod, s_sat, s_sq);
      tc_fence_proxy_async();
      tc_arrive(&full[g]);
    }
  } else {
    // ---------------- epilogue (tile columns 32q .. 32q+31, one per lane; rows of half h) ----------------
    // ---------------- and, on lane 0 of warp 8, the MMA issue ----------------
    const int q = (warp - 8) & 3, half = (warp - 8) >> 2;
    const bool issuer = warp == kTcMmaWarp;
    const int *s_er = (const int *)(smem + L.off_er);
    const uint32_t r_addr = tc_smem_addr(smem + L.off_r);
    bool ok = true;
    // tile k into tensor-memory slot k & 1: its digits written (full) and
    // tile k - 2 drained from the slot by all epilogue warps (empty)
    auto issue = [&](uint32_t k) -> bool {
      const int s = k & 1;
      if (!tc_wait(&full[s], (k >> 1) & 1u, flag, t.polls) ||
          (k >= 2 && !tc_wait(&empty[s], ((k - 2) >> 1) & 1u, flag, t.polls))) {
        tc_abort(flag, t.status);
        return false;
      }
      tc_fence_after_sync();
      Pol::issue(tbase + (uint32_t)s * 256u, tc_smem_addr(smem + (s ? L.off_b1 : L.off_b0)), r_addr);
      tc_commit(&done[s]);
      issued = k + 1;
      return true;
    };
    if (issuer && lane == 0)
      for (uint32_t k = 0; k < 2 && k < mytiles && ok; ++k) ok = issue(k);
    __syncwarp();
    for (uint32_t k = 0; k < mytiles; ++k) {
      const int s = k & 1;
      if (!tc_wait(&done[s], (k >> 1) & 1u, flag, t.polls)) {
        tc_abort(flag, t.status);
        break;
      }
      tc_fence_after_sync();
      const uint32_t colg = (tb + blockIdx.x + k * gridDim.x) * (uint32_t)kTcCols + (uint32_t)(32 * q + lane);
      Pol::drain(t, tbase + (uint32_t)s * 256u + ((uint32_t)(32 * q) << 16), colg, colg < total, s_er, half);
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) tc_arrive(&empty[s]);
      if (issuer) {
        if (lane == 0 && ok && k + 2 < mytiles) ok = issue(k + 2);
        __syncwarp();
      }
    }
  }

  __syncthreads();
  if (warp == kTcMmaWarp) {
    // after an abort, let the MMAs already committed finish before the
    // columns are released
    if (*flag && lane == 0 && issued > 0) {
      const uint32_t last = issued - 1;
      tc_mbar_wait(&done[last & 1], (last >> 1) & 1u, kTcPolls);
    }
    __syncwarp();
    tc_fence_after_sync();
    tc_tmem_dealloc(tbase, kTcTmemCols);
  }
}
