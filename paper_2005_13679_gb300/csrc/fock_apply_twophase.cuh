// fock_apply_twophase.cuh -- sigma = H C for dense reduced coefficients,
// evaluated through the (N-2)-particle space.
//
// With n' = gamma - e_k - e_q the configuration left after a removal r, the
// pull form reads sigma_gamma = sum_r A_r(gamma) Y[r][n'], where
//
//     X[a][n'] = B_a(n') C[n' + a],         B_a(n') = sqrt((n'_s + 1)(n'_l + 1 + delta_sl)),
//     Y[r][n'] = sum_a R[r][a] X[a][n'],    A_r(gamma) = sqrt(n_k (n_q - delta_kq)).
//
// Phase 1 runs one thread per n' in H(N-2, M): P gathers of C build X in the
// thread's slice of shared memory, a dense P x P product with the staged R
// gives Y, written r-major (consecutive n' consecutive in memory).  Phase 2 runs
// one thread per gamma and gathers P entries of Y.  The multiply-accumulate
// count is the same as the direct pull form, but each C value is gathered once
// per n' instead of once per (gamma, r), and the inner product needs no index
// or amplitude arithmetic.
#pragma once

#include "fock_apply_dense.cuh"

// Y is stored in blocks of kYBlock consecutive (configuration, rhs) columns:
// block b holds rows r = 0..P-1 of columns [b kYBlock, (b + 1) kYBlock), each
// row contiguous.  A tile of phase 1 writes one contiguous block, and the P
// entries that phase 2 reads for one configuration lie within one block.
// Every phase 1 writes Y with evict-first stores (st.global.cs): nothing reads
// it before phase 2 starts, and the gathers of C keep more of L2 (measured:
// the tensor-core phase 1 at N = 100, M = 6 from 14.48 to 14.12 ms; the same
// hint on phase 2's loads of Y made phase 2 slower).
constexpr int kYBlock = 128;
__host__ __device__ __forceinline__ size_t twophase_yidx(int r, size_t col, int P) {
  return (col / kYBlock) * ((size_t)P * kYBlock) + (size_t)r * kYBlock + (col % kYBlock);
}

struct TwoPhaseArgs {
  ApplyArgs<uint32_t> a;          // N-space tables, coefficients (dense, r*P + a), C, sigma, nrhs, scales
  uint32_t nc2;                   // N_c(N - 2, M)
  void *Y;                        // blocks of kYBlock columns x P rows (twophase_yidx)
  const float4 *g1, *g2;          // FP32-pair form: Gauss coefficients (see fock_apply.cu)
  const void *tc_a;               // tensor-core phase 1: digit image of R (fock_apply_tc.cuh), or NULL
  const int *tc_er;               // its row exponents
  const void *blk;                // pair-weight blocks: coefficient tables by block (fock_twophase_block.cu), or NULL
  int *status;                    // nonzero after a bounded wait of phase 1 expired, or NULL
  uint32_t polls;                 // poll budget of each bounded wait of the tensor-core phase 1
  cudaEvent_t phase1_done;        // recorded between the two phases when non-null (profiling hook)
  int phases;                     // 1: phase 1 only, 2: phase 2 only, 3: both
  uint32_t g_begin, g_end;        // configurations phase 2 computes
  uint64_t c_begin, c_end;        // (configuration, rhs) columns of H(N-2, M) phase 1 computes
};

template <int M>
struct TwoPhaseSmem {
  static constexpr int P = M * (M + 1) / 2;
  size_t off_coef, off_pair, off_mod, off_sat, off_sq, off_x, total;
  // priv_bytes: bytes of each thread's private area
  __host__ __device__ TwoPhaseSmem(int xdim, int nsq, size_t coef_bytes, size_t priv_bytes, int threads) {
    const int rows = M > 1 ? M - 1 : 1;
    size_t o = 0;
    off_coef = o; o = fock_align16(o + coef_bytes * P * P);
    off_pair = o; o = fock_align16(o + 2 * P);
    off_mod = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sat = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sq = o;   o = fock_align16(o + 8 * (size_t)nsq);
    off_x = o;    o = fock_align16(o + priv_bytes * (size_t)threads);
    total = o;
  }
};

// Target base and prefix differences of n' for adding two particles back
// (the (N-2)-space configuration itself, no removal).
template <int M>
__device__ __forceinline__ uint32_t twophase_targets(const int (&S)[M], const uint32_t *s_mod, int xdim, uint32_t nc,
                                                     uint32_t (&U)[M], uint32_t (&V)[M]) {
  uint32_t F0 = 0, F1 = 0, F2 = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    U[m] = F0 - F1;
    V[m] = F1 - F2;
    if (m < M - 1) {
      const uint32_t *row = s_mod + m * xdim + (S[m] + m);
      F0 += row[0];
      F1 += row[1];
      F2 += row[2];
    }
  }
  return nc - 1u - F2;
}

// Index in H(N-2, M) of gamma minus particles at k and q.
template <int M>
__device__ __forceinline__ uint32_t twophase_rank2(const int (&S)[M], int kk, int qq, const uint32_t *s_mod, int xdim,
                                                   uint32_t nc2) {
  uint32_t acc = nc2 - 1u;
#pragma unroll
  for (int m = 0; m < M - 1; ++m) acc -= s_mod[m * xdim + (S[m] - (kk <= m) - (qq <= m) + m)];
  return acc;
}

// Per-thread slice of phase 1: prefix differences and square roots of n'.
struct TwoPhaseSlot {
  uint32_t U, V;
  float bh, bl;       // sqrt(n'_m + 1) as a pair
  float ch, cl;       // sqrt(n'_m + 2) as a pair
};

// Stage coefficients, addition pairs, binomial tables and square roots.
template <int M, class CoefT, class SqT>
__device__ __forceinline__ void twophase_stage(const ApplyArgs<uint32_t> &a, const TwoPhaseSmem<M> &L,
                                               unsigned char *smem, bool stage_coef = true) {
  constexpr int P = TwoPhaseSmem<M>::P;
  CoefT *s_coef = (CoefT *)(smem + L.off_coef);
  int8_t *s_pair = (int8_t *)(smem + L.off_pair);
  uint32_t *s_mod = (uint32_t *)(smem + L.off_mod);
  uint32_t *s_sat = (uint32_t *)(smem + L.off_sat);
  SqT *s_sq = (SqT *)(smem + L.off_sq);
  const int rows = M > 1 ? M - 1 : 1;
  if (stage_coef)
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) s_coef[i] = ((const CoefT *)a.coef)[i];
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    // addition pair i = (s, l), s <= l, lexicographic
    int s = 0, r = i;
    while (r >= M - s) {
      r -= M - s;
      ++s;
    }
    s_pair[2 * i] = (int8_t)s;
    s_pair[2 * i + 1] = (int8_t)(s + r);
  }
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const SqT *)a.sq)[i];
  __syncthreads();
}

// Decode n' and fill the thread's slots; returns the target base in H(N, M).
template <int M, class SqT>
__device__ __forceinline__ uint32_t twophase_slots(uint32_t gc, const ApplyArgs<uint32_t> &a, uint32_t nc2,
                                                   const uint32_t *s_mod, const uint32_t *s_sat, const SqT *s_sq,
                                                   TwoPhaseSlot *slot, int nt) {
  int S[M];
  fock_decode_fast<M>(gc, a.N - 2, nc2, s_sat, a.xdim, S);
  uint32_t U[M], V[M];
  const uint32_t base = twophase_targets<M>(S, s_mod, a.xdim, a.nc, U, V);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int np = S[m] - (m > 0 ? S[m - 1] : 0);
    TwoPhaseSlot z;
    z.U = U[m];
    z.V = V[m];
    if constexpr (sizeof(SqT) == 8) {
      const float2 b = ((const float2 *)s_sq)[np + 1], c = ((const float2 *)s_sq)[np + 2];
      z.bh = b.x; z.bl = b.y; z.ch = c.x; z.cl = c.y;
    } else {
      z.bh = ((const float *)s_sq)[np + 1]; z.bl = 0.f;
      z.ch = ((const float *)s_sq)[np + 2]; z.cl = 0.f;
    }
    slot[m * nt] = z;
  }
  return base;
}


// Phase 2 per configuration: with Q = N_c(N-2,M) - 1 - sum_m C(S_m + m, m+1)
// and prefix sums P1[j], P2[j] of C(S_m + m - d, m+1) - C(S_m + m, m+1)
// (d = 1, 2) over m < j, removing particles at k <= q gives the index
//     rank2 = Q - (P1[q] - P1[k]) - (P2[M-1] - P2[q])
// (S_m drops by one on [k, q) and by two from q on).
template <int M>
__device__ __forceinline__ uint32_t twophase_prefix2(const int (&S)[M], const uint32_t *s_mod, int xdim,
                                                     uint32_t nc2, uint32_t (&P1)[M], uint32_t (&P2)[M]) {
  uint32_t q0 = nc2 - 1u, a1 = 0u, a2 = 0u;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    P1[m] = a1;
    P2[m] = a2;
    if (m < M - 1) {
      const int x = S[m] + m;
      const uint32_t t0 = s_mod[m * xdim + x];
      q0 -= t0;
      a1 += (x >= 1 ? s_mod[m * xdim + x - 1] : 0u) - t0;
      a2 += (x >= 2 ? s_mod[m * xdim + x - 2] : 0u) - t0;
    }
  }
  return q0;
}

// ---------------------------------------------------------------------------
// FP32 pairs
// ---------------------------------------------------------------------------
// Phase 1 in FP32 pairs with Gauss's three products per complex term:
//   k1 = Re R (Re X + Im X),  k2 = (Re R + Im R) Im X,  k3 = (Im R - Re R) Re X,
//   Re(R X) = k1 - k2,  Im(R X) = k1 + k3.
// (k1, k2) share one packed product and accumulation; k3 of two neighbouring
// removals share the other, so a complex term costs 1.5 packed products and
// accumulations instead of 2.
template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4)
fock_twophase_x_df(const TwoPhaseArgs t) {
  constexpr int P = TwoPhaseSmem<M>::P;
  constexpr int PP = (P + 1) / 2;
  constexpr int RB = 8;   // removals accumulated in registers per sweep over the additions (even)
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const TwoPhaseSmem<M> L(a.xdim, a.nsq, 2 * sizeof(float4), sizeof(TwoPhaseSlot) * M, blockDim.x);
  {
    // stage: Gauss coefficients (g1 rows, then g2 row pairs), tables, pairs
    float4 *s_g = (float4 *)(smem + L.off_coef);
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) s_g[i] = t.g1[i];
    for (int i = threadIdx.x; i < PP * P; i += blockDim.x) s_g[P * P + i] = t.g2[i];
  }
  twophase_stage<M, float4, float2>(a, L, smem, false);
  const float4 *s_g1 = (const float4 *)(smem + L.off_coef);
  const float4 *s_g2 = s_g1 + P * P;
  const int8_t *s_pair = (const int8_t *)(smem + L.off_pair);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float2 *s_sq = (const float2 *)(smem + L.off_sq);
  const int tid = threadIdx.x, nt = blockDim.x;
  TwoPhaseSlot *slot = (TwoPhaseSlot *)(smem + L.off_x) + tid;   // slot[m * nt]
  const uint32_t nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float4 *__restrict__ C = (const float4 *)a.C;
  float4 *__restrict__ Y = (float4 *)t.Y;

  // one thread per (configuration, right-hand side): the nrhs values of one
  // gathered configuration are adjacent, so a warp's gathers stay coalesced
  const size_t total = t.c_end;                         // columns [c_begin, c_end) of this launch
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < t.c_end; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + tid;
    const bool live = col < total;
    const size_t cc = live ? col : total - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    const uint32_t base = twophase_slots<M, float2>(g, a, nc2, s_mod, s_sat, s_sq, slot, nt);
    {
      for (int r0 = 0; r0 < P; r0 += RB) {
        fp2_t K12h[RB], K12l[RB], K3h[RB / 2], K3l[RB / 2];
#pragma unroll
        for (int q = 0; q < RB; ++q) K12h[q] = K12l[q] = 0ull;
#pragma unroll
        for (int q = 0; q < RB / 2; ++q) K3h[q] = K3l[q] = 0ull;
#pragma unroll 2
        for (int ai = 0; ai < P; ++ai) {
          // X = B_a(n') C[n' + a] as FP32 pairs (lanes: Re, Im)
          const int s = s_pair[2 * ai], l = s_pair[2 * ai + 1];
          const TwoPhaseSlot zs = slot[s * nt], zl = slot[l * nt];
          const float2 amp = df_mul(make_float2(zs.bh, zs.bl), s == l ? make_float2(zs.ch, zs.cl)
                                                                       : make_float2(zl.bh, zl.bl));
          const float4 v = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + j);
          fp2_t Xh, Xl;
          fp2_dprod(fp2_make(v.x, v.y), fp2_make(v.z, v.w), fp2_make(amp.x, amp.x), fp2_make(amp.y, amp.y), Xh, Xl);
          const float xrh = fp2_x(Xh), xih = fp2_y(Xh), xrl = fp2_x(Xl), xil = fp2_y(Xl);
          float th = 0.f, tl = 0.f;                         // Re X + Im X as a pair
          df_add_acc(th, tl, xrh, xrl);
          df_add_acc(th, tl, xih, xil);
          const fp2_t Bh = fp2_make(th, xih), Bl = fp2_make(tl, xil);     // (Re X + Im X, Im X)
          const fp2_t Rh = fp2_make(xrh, xrh), Rl = fp2_make(xrl, xrl);   // (Re X, Re X)
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (r0 + q < P) {
              const float4 w = s_g1[(r0 + q) * P + ai];       // (Re R, Re R + Im R)
              fp2_t p, e;
              fp2_dprod(fp2_make(w.x, w.y), fp2_make(w.z, w.w), Bh, Bl, p, e);
              fp2_dacc(K12h[q], K12l[q], p, e);               // (k1, k2)
            }
          }
#pragma unroll
          for (int q = 0; q < RB / 2; ++q) {
            if (r0 + 2 * q < P) {
              const float4 w = s_g2[((r0 >> 1) + q) * P + ai]; // (Im R - Re R) of two removals
              fp2_t p, e;
              fp2_dprod(fp2_make(w.x, w.y), fp2_make(w.z, w.w), Rh, Rl, p, e);
              fp2_dacc(K3h[q], K3l[q], p, e);                 // (k3, k3')
            }
          }
        }
        if (live) {
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (r0 + q < P) {
              const float k1h = fp2_x(K12h[q]), k1l = fp2_x(K12l[q]);
              const float k3h = (q & 1) ? fp2_y(K3h[q / 2]) : fp2_x(K3h[q / 2]);
              const float k3l = (q & 1) ? fp2_y(K3l[q / 2]) : fp2_x(K3l[q / 2]);
              float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
              df_add_acc(rh, rl, k1h, k1l);
              df_add_acc(rh, rl, -fp2_y(K12h[q]), -fp2_y(K12l[q]));
              df_add_acc(ih, il, k1h, k1l);
              df_add_acc(ih, il, k3h, k3l);
              __stcs(&Y[twophase_yidx(r0 + q, (size_t)g * nrhs + j, P)], make_float4(rh, ih, rl, il));
            }
          }
        }
      }
    }
  }
}

// Phase 2 is a gather: each target reads up to P rows of Y at hashed
// addresses.  For the FP32-pair form the minimum-block hint of 3 blocks of
// 128 threads per SM for M <= 6 leaves the registers to keep all P gathers of
// a configuration in flight (measured 3.5 % faster over the whole apply at
// N = 100, M = 6 than 8 blocks of 64 registers); for M = 7, 8 (P = 28, 36
// gathers) 2 blocks per SM (N = 20, M = 8, 16 right-hand sides: 24.5 ms
// against 27.7 ms at 5 blocks).
template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, (M <= 6 ? 3 : (M <= 8 ? 2 : 4)))
fock_twophase_sigma_df(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_mod = (uint32_t *)(smem + 256);
  const int rows = M > 1 ? M - 1 : 1;
  uint32_t *s_sat = s_mod + rows * a.xdim;
  float2 *s_sq = (float2 *)(s_sat + rows * a.xdim + 4);
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const float2 *)a.sq)[i];
  __syncthreads();
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nc = a.nc, nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float4 *__restrict__ Y = (const float4 *)t.Y;
  // output scale 2^e_out: the coefficient scale (a power of two) and the input scale
  int e_out = (int)(((unsigned long long)__double_as_longlong(a.out_scale) >> 52) & 0x7ff) - 1023;
  if (a.in_exp) e_out += __ldg(a.in_exp);
  // Y is incomplete if phase 1 gave up a wait: report NaN rather than a wrong sigma
  const bool failed = t.status && *(volatile const int *)t.status;

  const uint32_t g_end = t.g_end;
  // one thread per (configuration, right-hand side) of [g_begin, g_end)
  const size_t cbeg = (size_t)t.g_begin * nrhs, cend = (size_t)g_end * nrhs;
  for (size_t tile = cbeg + blockIdx.x * (size_t)nt; tile < cend; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + tid;
    const bool live = col < cend;
    const size_t cc = live ? col : cend - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    int S[M], n[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
#pragma unroll
    for (int m = 0; m < M; ++m) n[m] = S[m] - (m > 0 ? S[m - 1] : 0);
    float2 sq0[M], sq1[M];                                  // sqrt(n_m), sqrt(n_m - 1) as pairs
#pragma unroll
    for (int m = 0; m < M; ++m) {
      sq0[m] = s_sq[n[m]];
      sq1[m] = s_sq[max(n[m] - 1, 0)];
    }
    uint32_t P1[M], P2[M];
    const uint32_t q0 = twophase_prefix2<M>(S, s_mod, a.xdim, nc2, P1, P2);
    {
      fp2_t Ah = 0ull, Al = 0ull;
      // every removal is evaluated: an impossible one has amplitude 0
      // (sqrt(0) or sqrt(n - 1) = 0 for n = 1) and reads the block start
#pragma unroll
      for (int k = 0; k < M; ++k) {
#pragma unroll
        for (int q = k; q < M; ++q) {
          const int r = k * M - (k * (k - 1)) / 2 + (q - k);
          const bool valid = k == q ? n[k] >= 2 : (n[k] >= 1 && n[q] >= 1);
          const uint32_t r2 = valid ? q0 - (P1[q] - P1[k]) - (P2[M - 1] - P2[q]) : 0u;
          const float2 A = df_mul(sq0[k], k == q ? sq1[k] : sq0[q]);
          const float4 y = __ldg(Y + twophase_yidx(r, (size_t)r2 * nrhs + j, M * (M + 1) / 2));
          fp2_t p, e;
          fp2_dprod(fp2_make(y.x, y.y), fp2_make(y.z, y.w), fp2_make(A.x, A.x), fp2_make(A.y, A.y), p, e);
          fp2_dacc(Ah, Al, p, e);
        }
      }
      if (live) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        df_add_acc(rh, rl, fp2_x(Ah), fp2_x(Al));
        df_add_acc(ih, il, fp2_y(Ah), fp2_y(Al));
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        ((double2 *)a.sigma)[(size_t)g * nrhs + j] =
            failed ? make_double2(nan, nan)
                   : make_double2(df_to_double_bits(rh, rl, e_out), df_to_double_bits(ih, il, e_out));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP32-mixed
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4)
fock_twophase_x_mixed(const TwoPhaseArgs t) {
  constexpr int P = TwoPhaseSmem<M>::P;
  constexpr int RB = 12;
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const TwoPhaseSmem<M> L(a.xdim, a.nsq, sizeof(float2), sizeof(TwoPhaseSlot) * M, blockDim.x);
  twophase_stage<M, float2, float>(a, L, smem);
  const float2 *s_coef = (const float2 *)(smem + L.off_coef);
  const int8_t *s_pair = (const int8_t *)(smem + L.off_pair);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float *s_sq = (const float *)(smem + L.off_sq);
  const int tid = threadIdx.x, nt = blockDim.x;
  TwoPhaseSlot *slot = (TwoPhaseSlot *)(smem + L.off_x) + tid;
  const uint32_t nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float2 *__restrict__ C = (const float2 *)a.C;
  float2 *__restrict__ Y = (float2 *)t.Y;

  const size_t total = t.c_end;                         // columns [c_begin, c_end) of this launch        // one thread per (configuration, right-hand side)
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < t.c_end; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + tid;
    const bool live = col < total;
    const size_t cc = live ? col : total - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    const uint32_t base = twophase_slots<M, float>(g, a, nc2, s_mod, s_sat, s_sq, slot, nt);
    {
      for (int r0 = 0; r0 < P; r0 += RB) {
        fp2_t A1[RB], A2[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) A1[q] = A2[q] = 0ull;
#pragma unroll 2
        for (int ai = 0; ai < P; ++ai) {
          const int s = s_pair[2 * ai], l = s_pair[2 * ai + 1];
          const TwoPhaseSlot zs = slot[s * nt], zl = slot[l * nt];
          const float amp = zs.bh * (s == l ? zs.ch : zl.bh);
          const float2 v = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + j);
          const fp2_t Xp = fp2_make(v.x * amp, v.y * amp), Xs = fp2_make(v.y * amp, v.x * amp);
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (r0 + q < P) {
              const float2 w = s_coef[(r0 + q) * P + ai];
              const fp2_t Rp = fp2_make(w.x, w.y);
              A1[q] = fp2_fma(Rp, Xp, A1[q]);   // (Re R Re X, Im R Im X)
              A2[q] = fp2_fma(Rp, Xs, A2[q]);   // (Re R Im X, Im R Re X)
            }
          }
        }
        if (live) {
#pragma unroll
          for (int q = 0; q < RB; ++q)
            if (r0 + q < P)
              __stcs(&Y[twophase_yidx(r0 + q, (size_t)g * nrhs + j, P)],
                     make_float2(fp2_x(A1[q]) - fp2_y(A1[q]), fp2_x(A2[q]) + fp2_y(A2[q])));
        }
      }
    }
  }
}

// The FP32-mixed form, branch-free like the FP32-pair one: 4 blocks per SM
// for M <= 6 keep the P gathers of a configuration in flight (whole mixed
// apply at N = 100, M = 6: 10.4 ms, against 13.5 ms with a warp vote that
// skipped impossible removals at 8 blocks); 2 blocks for M = 7, 8 (N = 20,
// M = 8, 16 right-hand sides: 9.0 ms against 12.4 ms at 5 blocks).
template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, (M <= 6 ? 4 : (M <= 8 ? 2 : 4)))
fock_twophase_sigma_mixed(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_mod = (uint32_t *)(smem + 256);
  const int rows = M > 1 ? M - 1 : 1;
  uint32_t *s_sat = s_mod + rows * a.xdim;
  float *s_sq = (float *)(s_sat + rows * a.xdim + 4);
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const float *)a.sq)[i];
  __syncthreads();
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nc = a.nc, nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float2 *__restrict__ Y = (const float2 *)t.Y;
  // Y is incomplete if the tensor-core phase 1 gave up a wait: report NaN
  const float out_scale = (t.status && *(volatile const int *)t.status) ? __int_as_float(0x7fc00000)
                                                                        : (float)a.out_scale;

  const uint32_t g_end = t.g_end;
  // one thread per (configuration, right-hand side) of [g_begin, g_end)
  const size_t cbeg = (size_t)t.g_begin * nrhs, cend = (size_t)g_end * nrhs;
  for (size_t tile = cbeg + blockIdx.x * (size_t)nt; tile < cend; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + tid;
    const bool live = col < cend;
    const size_t cc = live ? col : cend - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    int S[M], n[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
#pragma unroll
    for (int m = 0; m < M; ++m) n[m] = S[m] - (m > 0 ? S[m - 1] : 0);
    float sq0[M], sq1[M];                                   // sqrt(n_m), sqrt(n_m - 1)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      sq0[m] = s_sq[n[m]];
      sq1[m] = s_sq[max(n[m] - 1, 0)];
    }
    uint32_t P1[M], P2[M];
    const uint32_t q0 = twophase_prefix2<M>(S, s_mod, a.xdim, nc2, P1, P2);
    {
      fp2_t Sh = 0ull, Sl = 0ull;
      // every removal is evaluated: an impossible one has amplitude 0
      // (sqrt(0) or sqrt(n - 1) = 0 for n = 1) and reads the block start
#pragma unroll
      for (int k = 0; k < M; ++k) {
#pragma unroll
        for (int q = k; q < M; ++q) {
          const int r = k * M - (k * (k - 1)) / 2 + (q - k);
          const bool valid = k == q ? n[k] >= 2 : (n[k] >= 1 && n[q] >= 1);
          const uint32_t r2 = valid ? q0 - (P1[q] - P1[k]) - (P2[M - 1] - P2[q]) : 0u;
          const float A = sq0[k] * (k == q ? sq1[k] : sq0[q]);
          const float2 y = __ldg(Y + twophase_yidx(r, (size_t)r2 * nrhs + j, M * (M + 1) / 2));
          fp2_dacc(Sh, Sl, fp2_mul(fp2_make(y.x, y.y), fp2_make(A, A)), 0ull);
        }
      }
      if (live) {
        const fp2_t v = fp2_add(Sh, Sl);
        ((float2 *)a.sigma)[(size_t)g * nrhs + j] = make_float2(fp2_x(v) * out_scale, fp2_y(v) * out_scale);
      }
    }
  }
}

// Phase 2 shared memory: pair table, binomial tables, square roots.
__host__ __device__ inline size_t twophase_sigma_smem(int rows, int xdim, int nsq) {
  return 256 + 8 * (size_t)rows * xdim + 16 + 8 * (size_t)nsq;
}

template <class K>
int fock_launch_grid(K kern, const TwoPhaseArgs &t, uint64_t n, size_t smem, int device, cudaStream_t stream) {
  const int threads = FOCK_APPLY_THREADS;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fock_cuda_status(e);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return fock_cuda_status(e);
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t tiles = ((int64_t)n + threads - 1) / threads;
  int64_t grid = (int64_t)per_sm * fock_get_sm_count(device);
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, threads, smem, stream>>>(t);
  e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}
