// fock_apply_tc.cuh -- phase 1 of the two-phase apply (fock_apply_twophase.cuh)
// on the fifth-generation tensor cores, with FP64-class accuracy.
//
// Phase 1 is the dense product Y = R X with R the P x P reduced coefficients
// and X[a][n'] = B_a(n') C[n' + a] over the (N-2)-particle configurations.  In
// real form (rows and columns interleaved as (Re, Im)) it is a 2P x 2P matrix
// times a 2P x (configurations x rhs) matrix.  Both factors are split into five
// signed base-2^9 digits with a power-of-two scale per row of R and per column
// of X (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59 (2012)):
//
//     R~[rho][k] = 2^(e_rho - 8) sum_{i=1..5} rho_i 2^(-9(i-1)),   |rho_i| <= 256,
//     X~[k][c]   = 2^(e_c - 8)   sum_{j=1..5} xi_j  2^(-9(j-1)),   |xi_j|  <= 265.
//
// Digits are integers held exactly in fp16.  For a level l = i + j the sum
// S_l = sum_{i+j=l} sum_k rho_i xi_j has at most 5 pairs x 42 terms of
// magnitude <= 256 * 265, below 2^24, so the tensor core's FP32 accumulation
// of S_l is exact whatever its internal order.  Levels 2..6 are kept:
//
//     Y = 2^(e_rho + e_c - 16) sum_{l=2..6} 2^(-9(l-2)) S_l,
//
// whose dropped terms and digit remainders are below 2^-44 of
// max|R~ row| * max|X~ column| * 2P; the five level sums are combined into an
// FP32 pair (TwoSum) for phase 2.
//
// The MMA computes the transposed product: its M = 128 rows are the tile's
// (configuration, rhs) columns, so tensor-memory lane c holds everything of
// column c, and its N columns are (real row, level) combinations.  Real rows
// come in groups of three, 16 tensor-memory columns per group: column
// 16 g + 5 i + (6 - l) holds level l of real row 3 g + i, and column 15 (the
// spare of group 0) receives the column exponent, which the producer stores at
// K position K1 - 1 and a unit row of the coefficient image copies.  An
// epilogue thread reads its own lane: two groups (32 columns) hold three
// complex rows (Re and Im), so no data crosses lanes.  K is ordered
// [digits 1..3 of every real index, interleaved | digits 4, 5 interleaved].
#pragma once

#include <cuda_fp16.h>

#include "fock_apply_twophase.cuh"
#include "fock_tc.cuh"

constexpr int kTcCols = 128;        // (configuration, rhs) columns per tile = MMA M
constexpr int kTcProducers = 128;   // producer group: 4 warps, one thread per column
constexpr int kTcThreads = 416;     // two producer groups (warps 0-3 even tiles, 4-7 odd tiles),
                                    // warps 8-11 epilogue (warp 8 + q: tile columns 32q .. 32q+31), warp 12 MMA
constexpr int kTcTmemCols = 512;    // two tiles x NT (<= 224) columns, at 0 and 256
constexpr uint32_t kTcPolls = 1u << 20;
constexpr int kTcExpCol = 15;       // tensor-memory column of the column exponent

// Shape of the real-form product for M orbitals (2 <= M <= 6).
struct TcShape {
  int P, R2, NG, NT, K1, K2, KT;
  __host__ __device__ constexpr explicit TcShape(int m)
      : P(m * (m + 1) / 2), R2(m * (m + 1)), NG((m * (m + 1) + 2) / 3), NT(16 * ((m * (m + 1) + 2) / 3)),
        K1((3 * m * (m + 1) + 15) / 16 * 16), K2((2 * m * (m + 1) + 15) / 16 * 16),
        KT((3 * m * (m + 1) + 15) / 16 * 16 + (2 * m * (m + 1) + 15) / 16 * 16) {}
  // bytes of the coefficient image (NT rows x KT, fp16) and of one digit tile
  __host__ __device__ constexpr int r_bytes() const { return NT * KT * 2; }
  __host__ __device__ constexpr int b_bytes() const { return kTcCols * KT * 2; }
  // K position of the column exponent (the last of part 1, never a digit)
  __host__ __device__ constexpr int exp_pos() const { return K1 - 1; }
  // additions swept by the producer, padding included, so that every 16-byte
  // chunk of both K parts is written
  __host__ __device__ constexpr int a_end() const {
    const int c1 = (K1 + 5) / 6, c2 = K2 / 4;
    const int m = P > c1 ? (P > c2 ? P : c2) : (c1 > c2 ? c1 : c2);
    return (m + 3) / 4 * 4;
  }
  // tensor-memory column of level l of real row rho
  __host__ __device__ constexpr int col(int rho, int l) const { return 16 * (rho / 3) + 5 * (rho % 3) + (6 - l); }
};

// Shared-memory layout of the kernel for a policy with an nt x kt coefficient
// image, kt-deep digit tiles, r2 row exponents and a square-root table of
// sq_bytes per entry.
struct TcSmem {
  size_t off_r, off_b0, off_b1, off_er, off_mod, off_sat, off_sq, off_bar, total;
  __host__ __device__ TcSmem(int nt, int kt, int r2, int M, int xdim, int nsq, int sq_bytes) {
    const int rows = M > 1 ? M - 1 : 1;
    size_t o = 0;
    off_r = o;    o += (size_t)nt * kt * 2;
    off_b0 = o;   o += (size_t)kTcCols * kt * 2;
    off_b1 = o;   o += (size_t)kTcCols * kt * 2;
    off_er = o;   o = fock_align16(o + 4 * (size_t)r2);
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

constexpr float kTcMagic = 12582912.f;   // 1.5 * 2^23

// d = x m rounded to the nearest integer (ties to even) and the exact
// remainder r = x m - d, for m a power of two and |x m| < 2^22.
__device__ __forceinline__ float tc_digit(float x, float m, float &r) {
  const float d = __fsub_rn(__fmaf_rn(x, m, kTcMagic), kTcMagic);
  r = __fmaf_rn(x, m, -d);
  return d;
}

__device__ __forceinline__ float tc_round(float x, float m) {
  return __fsub_rn(__fmaf_rn(x, m, kTcMagic), kTcMagic);
}

// Digits of v = (xh + xl) 2^E, the pair of one real value of X at its column
// scale (f = 2^E, f18 = 2^(E+18), |xh f| < 256, |xl f| <= 3 2^-16):
//     v = c1 + c2 2^-9 + c3 2^-18 + c4 2^-27 + c5 2^-36 + r,   |r| <= 2^-37 (+ 2^-51).
// The high word gives c1..c4 with exact remainders, the low word adds to c3
// and c4, the two remainders share c5 (their FP32 sum is rounded far below
// the digit's unit), and one carry folds c5 back into [-256, 256]:
// |c1|, |c2|, |c5| <= 256, |c3| <= 268, |c4| <= 513.
__device__ __forceinline__ void tc_digits(float xh, float xl, float f, float f18, float (&c)[5]) {
  float r, u;
  c[0] = tc_digit(xh, f, r);
  c[1] = tc_digit(r, 512.f, r);
  const float d3 = tc_digit(r, 512.f, r);
  const float d4 = tc_digit(r, 512.f, r);
  const float e3 = tc_digit(xl, f18, u);
  const float e4 = tc_digit(u, 512.f, u);
  const float c5 = tc_round(__fadd_rn(r, u), 512.f);
  const float q = tc_round(c5, 1.f / 512.f);
  c[4] = __fmaf_rn(q, -512.f, c5);
  c[3] = __fadd_rn(__fadd_rn(d4, e4), q);
  c[2] = __fadd_rn(d3, e3);
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

// Bounded wait that also gives up as soon as another role raised the abort flag.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *flag) {
  for (uint32_t i = 0; i < kTcPolls; ++i) {
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
  uint32_t ebits = 0;
#pragma unroll
  for (int ai = 0; ai < P; ++ai) {
    const int s = pr.s[ai], l = pr.l[ai];
    const float2 amp = df_mul(sq1[s], s == l ? sq2[s] : sq1[l]);
    fp2_t Xh, Xl;
    fp2_dprod(fp2_make(v[ai].x, v[ai].y), fp2_make(v[ai].z, v[ai].w), fp2_make(amp.x, amp.x),
              fp2_make(amp.y, amp.y), Xh, Xl);
    v[ai] = make_float4(fp2_x(Xh), fp2_y(Xh), fp2_x(Xl), fp2_y(Xl));   // (Re hi, Im hi, Re lo, Im lo)
    ebits = max(ebits, max(__float_as_uint(v[ai].x) & 0x7f800000u, __float_as_uint(v[ai].y) & 0x7f800000u));
  }
  const int field = (int)(ebits >> 23);
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

  unsigned char *colbase = bbuf + (size_t)(cl >> 3) * (CHT * 128) + (cl & 7) * 16;
#pragma unroll
  for (int bi = 0; bi < AE / 4; ++bi) {
    float dig[8][5];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int k = 8 * bi + r;                         // real index 2a + (0 Re, 1 Im)
      if (k < 2 * P) {
        const float4 x = v[k >> 1];
        tc_digits((k & 1) ? x.y : x.x, (k & 1) ? x.w : x.z, f, f18, dig[r]);
      } else {
#pragma unroll
        for (int j = 0; j < 5; ++j) dig[r][j] = 0.f;
      }
    }
    // part 1: positions 3k + (j - 1), j = 1..3; the exponent at exp_pos()
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const int chunk = 3 * bi + ch;
      if (chunk < CH1) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p0 = 8 * ch + 2 * e, p1 = p0 + 1;
          const float lo = dig[p0 / 3][p0 % 3];
          const float hi = 8 * chunk + 2 * e + 1 == sh.exp_pos() ? (float)e_c : dig[p1 / 3][p1 % 3];
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
        for (int e = 0; e < 4; ++e) w[e] = tc_pack(dig[(8 * ch + 2 * e) / 2][3], dig[(8 * ch + 2 * e) / 2][4]);
        *(uint4 *)(colbase + (CH1 + chunk) * 128) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// Combination of the five level sums of one real row into an FP32 pair.
__device__ __forceinline__ void tc_combine(float s2, float s3, float s4, float s5, float s6, float &hi, float &lo) {
  const float a3 = __fmul_rn(s3, 1.f / 512.f);
  const float a4 = __fmul_rn(s4, 1.f / 262144.f);
  const float a56 = __fmaf_rn(s6, 1.f / 68719476736.f, __fmul_rn(s5, 1.f / 134217728.f));
  float s = __fadd_rn(s2, a3);
  float bb = __fsub_rn(s, s2);
  float e = __fadd_rn(__fsub_rn(s2, __fsub_rn(s, bb)), __fsub_rn(a3, bb));
  const float s1 = __fadd_rn(s, a4);
  bb = __fsub_rn(s1, s);
  e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(a4, bb)));
  e = __fadd_rn(e, a56);
  hi = __fadd_rn(s1, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s1));
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
  static constexpr int NT = sh.NT, KT = sh.KT, R2 = sh.R2, R_BYTES = sh.r_bytes();
  using sq_t = float2;
  __device__ static void produce(const TwoPhaseArgs &t, uint32_t tile, uint32_t total, int cl, unsigned char *bbuf,
                                 const uint32_t *s_mod, const uint32_t *s_sat, const void *s_sq) {
    tc_produce<M>(t, tile, total, cl, bbuf, s_mod, s_sat, (const float2 *)s_sq);
  }
  // Lane-local epilogue: 32 tensor-memory columns (three complex rows) per
  // pass; the next pass's load overlaps the combination of the current one.
  __device__ static void drain(const TwoPhaseArgs &t, uint32_t tq, uint32_t colg, bool live, const int *s_er) {
    constexpr int NPASS = (NT + 31) / 32;
    constexpr TcShape shp(M);
    float4 *__restrict__ Y = (float4 *)t.Y;
    float v[32];
    tc_ld_x16(tq, *reinterpret_cast<float(*)[16]>(&v[0]));
    tc_ld_x16(tq + 16u, *reinterpret_cast<float(*)[16]>(&v[16]));
    int ec = 0;
#pragma unroll
    for (int pass = 0; pass < NPASS; ++pass) {
      tc_wait_ld();
      float w[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) w[i] = v[i];
      if (pass + 1 < NPASS) {
        tc_ld_x16(tq + (uint32_t)(32 * (pass + 1)), *reinterpret_cast<float(*)[16]>(&v[0]));
        if (32 * (pass + 1) + 16 < NT)
          tc_ld_x16(tq + (uint32_t)(32 * (pass + 1) + 16), *reinterpret_cast<float(*)[16]>(&v[16]));
      }
      if (pass == 0) ec = (int)w[kTcExpCol] - 16;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int r = 3 * pass + j;                      // complex row
        if (2 * r < R2) {
          float hv[2], lv[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int rho = 2 * r + c;
            const int b = shp.col(rho, 6) - 32 * pass;   // levels 6..2 at b .. b+4
            tc_combine(w[b + 4], w[b + 3], w[b + 2], w[b + 1], w[b], hv[c], lv[c]);
            const int e = s_er[rho] + ec;
            if (e >= -126) {
              const float sc = tc_pow2(e);
              hv[c] = __fmul_rn(hv[c], sc);
              lv[c] = __fmul_rn(lv[c], sc);
            } else {
              tc_scale(hv[c], lv[c], e);
            }
          }
          if (live) Y[twophase_yidx(r, colg, shp.P)] = make_float4(hv[0], hv[1], lv[0], lv[1]);
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
  // Y = D 2^(e_rho + e_c - 30): the row scale 2^(15 - e_rho) of the image and
  // the column scale 2^(15 - e_c) of the digits taken out.
  __device__ static void drain(const TwoPhaseArgs &t, uint32_t tq, uint32_t colg, bool live, const int *s_er) {
    constexpr int P = M * (M + 1) / 2;
    float2 *__restrict__ Y = (float2 *)t.Y;
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
      if (live) Y[twophase_yidx(r, colg, P)] = make_float2(v[0], v[1]);
    }
  }
};

template <class Pol, int M>
__host__ __device__ inline TcSmem tc_smem_of(int xdim, int nsq) {
  return TcSmem(Pol::NT, Pol::KT, Pol::R2, M, xdim, nsq, (int)sizeof(typename Pol::sq_t));
}

// ---------------------------------------------------------------------------
// The kernel: persistent, one CTA per SM, tiles of 128 columns, three roles
// joined by mbarriers (slot s = tile & 1 for the digit tile and the tensor
// memory of a tile):
//   producers (warps 0-3 for even k, warps 4-7 for odd k)
//                           wait done[s] of tile k-2, write B[s], arrive full[s]
//   MMA (warp 12, one lane) wait full[s] and empty[s] of tile k-2, issue, commit done[s]
//   epilogue (warps 8-11)   wait done[s], drain tensor memory, write Y, arrive empty[s]
// ---------------------------------------------------------------------------
template <int M, class Pol>
__global__ void __launch_bounds__(kTcThreads, 1) fock_twophase_x_tc(const TwoPhaseArgs t) {
  constexpr int NT = Pol::NT, CHT = Pol::KT / 8;
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
      tc_mbar_init(&empty[i], 4);
    }
    *flag = 0;
    tc_fence_mbar_init();
  }
  if (warp == 12) tc_tmem_alloc(tslot, kTcTmemCols);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = *tslot;

  const uint32_t total = t.nc2 * (uint32_t)a.nrhs;
  const uint32_t ntiles = (total + kTcCols - 1) / kTcCols;
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
      if (k >= 2 && !tc_wait(&done[g], ((k - 2) >> 1) & 1u, flag)) {
        tc_abort(flag, t.status);
        break;
      }
      Pol::produce(t, blockIdx.x + k * gridDim.x, total, cl, bbuf, s_mod, s_sat, s_sq);
      tc_fence_proxy_async();
      tc_arrive(&full[g]);
    }
  } else if (warp == 12) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_f16(kTcCols, NT);
      const uint32_t r_addr = tc_smem_addr(smem + L.off_r);
      for (uint32_t k = 0; k < mytiles; ++k) {
        const int s = k & 1;
        if (!tc_wait(&full[s], (k >> 1) & 1u, flag) ||
            (k >= 2 && !tc_wait(&empty[s], ((k - 2) >> 1) & 1u, flag))) {
          tc_abort(flag, t.status);
          break;
        }
        tc_fence_after_sync();
        const uint32_t d = tbase + (uint32_t)s * 256u;
        const uint32_t x_addr = tc_smem_addr(smem + (s ? L.off_b1 : L.off_b0));
#pragma unroll
        for (int kk = 0; kk < Pol::KT / 16; ++kk)
          tc_mma_f16(d, tc_desc_kmajor(x_addr + kk * 256, 128, CHT * 128),
                     tc_desc_kmajor(r_addr + kk * 256, 128, CHT * 128), idesc, kk > 0);
        tc_commit(&done[s]);
        issued = k + 1;
      }
    }
  } else {
    // ---------------- epilogue: tile columns 32q .. 32q+31, one per lane ----------------
    const int q = warp - 8;
    const int *s_er = (const int *)(smem + L.off_er);
    for (uint32_t k = 0; k < mytiles; ++k) {
      const int s = k & 1;
      if (!tc_wait(&done[s], (k >> 1) & 1u, flag)) {
        tc_abort(flag, t.status);
        break;
      }
      tc_fence_after_sync();
      const uint32_t colg = (blockIdx.x + k * gridDim.x) * (uint32_t)kTcCols + (uint32_t)(32 * q + lane);
      Pol::drain(t, tbase + (uint32_t)s * 256u + ((uint32_t)(32 * q) << 16), colg, colg < total, s_er);
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) tc_arrive(&empty[s]);
    }
  }

  __syncthreads();
  if (warp == 12) {
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
