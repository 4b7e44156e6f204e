// fock_twophase_pairs.cu -- the two-phase apply for pair-weight-conserving
// operators whose pair blocks are rank one off the diagonal:
//
//     R[r][a] = c_K o_r o_a + D_r d_ra      (r, a pairs of sum K),
//
// with o = 2 for a pair of two orbitals and 1 for a doubly occupied one.  The
// Lieb-Liniger ring in plane waves (Sec. 6, Eq. LLHamiltonian) is of this
// form: W_kqsl = g/L whenever k + q = s + l gives c_K = g/2L, and the folded
// one-body energies h_kk/(N - 1) give D.  The two-body part is then
// sum_K c_K A_K^dag A_K with the pair operator A_K = sum_{s+l=K} a_s a_l
// (ordered pairs), and the apply factors through the 2M - 1 pair-momentum
// amplitudes of every (N-2)-particle configuration n':
//
//   phase 1:  Z_K(n') = c_K sum_{a in K} o_a B_a(n') C[n' + a]      (c_K A_K C),
//   phase 2:  sigma_gamma = sum_r o_r A_r(gamma) Z_{K(r)}(gamma - r)
//                          + (sum_r D_r n_k (n_q - d_kq)) C_gamma,
//
// the last term being the diagonal part (A_r(gamma) B_r(gamma - r) =
// n_k (n_q - d_kq) for r = {k, q}).  Against the general block form
// (fock_twophase_block.cu) the intermediate holds 2M - 1 instead of
// M(M + 1)/2 rows (19 against 55 at M = 10), phase 1 takes one coefficient
// product per pair momentum and phase 2 none per removal.  FP32 pairs
// (FOCK_PREC_F64) or FP32 (FOCK_PREC_F32_MIXED).
#include <math.h>

#include <complex>
#include <vector>

#include "fock_apply_twophase.cuh"

namespace {

// Per-thread slot of phase 1: target offsets and square roots of n'.
template <class SqT>
struct PairSlot {
  uint32_t U, V;
  SqT b, c;                 // sqrt(n'_m + 1), sqrt(n'_m + 2)
};

template <int M, class SqT>
struct PairSmem {
  size_t off_mod, off_sat, off_sq, off_slot, total;
  __host__ __device__ PairSmem(int xdim, int nsq, int threads) {
    const int rows = M - 1;
    size_t o = 0;
    off_mod = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sat = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sq = o;   o = fock_align16(o + 8 * (size_t)nsq);
    off_slot = o; o = fock_align16(o + sizeof(PairSlot<SqT>) * M * (size_t)threads);
    total = o;
  }
};

template <int M, class SqT>
__device__ __forceinline__ void pair_stage(const ApplyArgs<uint32_t> &a, const PairSmem<M, SqT> &L,
                                           unsigned char *smem) {
  uint32_t *s_mod = (uint32_t *)(smem + L.off_mod), *s_sat = (uint32_t *)(smem + L.off_sat);
  for (int i = threadIdx.x; i < (M - 1) * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  SqT *s_sq = (SqT *)(smem + L.off_sq);
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const SqT *)a.sq)[i];
  __syncthreads();
}

template <int M, class SqT>
__device__ __forceinline__ uint32_t pair_slots(uint32_t np, const ApplyArgs<uint32_t> &a, uint32_t nc2,
                                               const uint32_t *s_mod, const uint32_t *s_sat, const SqT *s_sq,
                                               PairSlot<SqT> *slot, int nt) {
  int S[M];
  fock_decode_fast<M>(np, a.N - 2, nc2, s_sat, a.xdim, S);
  uint32_t U[M], V[M];
  const uint32_t base = twophase_targets<M>(S, s_mod, a.xdim, a.nc, U, V);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int occ = S[m] - (m > 0 ? S[m - 1] : 0);
    PairSlot<SqT> z;
    z.U = U[m];
    z.V = V[m];
    z.b = s_sq[occ + 1];
    z.c = s_sq[occ + 2];
    slot[m * nt] = z;
  }
  return base;
}

// ---------------------------------------------------------------------------
// Phase 1, FP32 pairs: Z_K = c_K sum_a o_a B_a C[n' + a] (the factor o = 2
// is exact on both words of a pair), one pair-momentum block of NB pairs.
// ---------------------------------------------------------------------------
template <int M, int NB>
__device__ __forceinline__ void pairs_df(int K, int lo, uint32_t base, const PairSlot<float2> *slot, int nt,
                                         const float4 *__restrict__ C, float4 *__restrict__ Z, uint32_t nrhs,
                                         uint32_t jr, size_t col, bool live, float2 cK) {
  float4 v[NB];
  float2 amp[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int s = lo + i, l = K - s;
    const PairSlot<float2> zs = slot[s * nt], zl = slot[l * nt];
    v[i] = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + jr);
    amp[i] = df_mul(zs.b, s == l ? zs.c : zl.b);
    if (s != l) amp[i] = make_float2(2.f * amp[i].x, 2.f * amp[i].y);
  }
  fp2_t h = 0ull, lw = 0ull;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    fp2_t p, e;
    fp2_dprod(fp2_make(v[i].x, v[i].y), fp2_make(v[i].z, v[i].w), fp2_make(amp[i].x, amp[i].x),
              fp2_make(amp[i].y, amp[i].y), p, e);
    fp2_dacc(h, lw, p, e);
  }
  // times c_K, renormalised (fast TwoSum: |e| is below 2^-22 |p|)
  fp2_t p, e;
  fp2_dprod(h, lw, fp2_make(cK.x, cK.x), fp2_make(cK.y, cK.y), p, e);
  h = fp2_add(p, e);
  lw = fp2_sub(e, fp2_sub(h, p));
  if (live) __stcs(&Z[twophase_yidx(K, col, 2 * M - 1)], make_float4(fp2_x(h), fp2_y(h), fp2_x(lw), fp2_y(lw)));
}

template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_pairs_z_df(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const PairSmem<M, float2> L(a.xdim, a.nsq, blockDim.x);
  pair_stage<M, float2>(a, L, smem);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float2 *s_sq = (const float2 *)(smem + L.off_sq);
  const int nt = blockDim.x;
  PairSlot<float2> *slot = (PairSlot<float2> *)(smem + L.off_slot) + threadIdx.x;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const float4 *__restrict__ C = (const float4 *)a.C;
  float4 *__restrict__ Z = (float4 *)t.Y;
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < t.c_end; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < t.c_end;
    const size_t cc = live ? col : t.c_end - 1u;
    const uint32_t np = (uint32_t)(cc / nrhs);
    const uint32_t jr = (uint32_t)(cc - (size_t)np * nrhs);
    const uint32_t base = pair_slots<M, float2>(np, a, t.nc2, s_mod, s_sat, s_sq, slot, nt);
#pragma unroll 1
    for (int K = 0; K < 2 * M - 1; ++K) {
      const int lo = K - (M - 1) > 0 ? K - (M - 1) : 0, nb = K / 2 - lo + 1;
      const float2 cK = __ldg((const float2 *)t.blk + K);
      switch (nb) {
        case 1: pairs_df<M, 1>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 2: pairs_df<M, 2>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 3: pairs_df<M, 3>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 4: pairs_df<M, 4>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 5: pairs_df<M, 5>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        default: pairs_df<M, 6>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Phase 1, FP32-mixed: the same sums in FP32 from complex64 C.
// ---------------------------------------------------------------------------
template <int M, int NB>
__device__ __forceinline__ void pairs_mixed(int K, int lo, uint32_t base, const PairSlot<float> *slot, int nt,
                                            const float2 *__restrict__ C, float2 *__restrict__ Z, uint32_t nrhs,
                                            uint32_t jr, size_t col, bool live, float cK) {
  fp2_t acc = 0ull;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int s = lo + i, l = K - s;
    const PairSlot<float> zs = slot[s * nt], zl = slot[l * nt];
    const float2 v = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + jr);
    const float amp = (s == l ? 1.f : 2.f) * zs.b * (s == l ? zs.c : zl.b);
    acc = fp2_fma(fp2_make(amp, amp), fp2_make(v.x, v.y), acc);
  }
  acc = fp2_mul(acc, fp2_make(cK, cK));
  if (live) __stcs(&Z[twophase_yidx(K, col, 2 * M - 1)], make_float2(fp2_x(acc), fp2_y(acc)));
}

template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_pairs_z_mixed(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const PairSmem<M, float> L(a.xdim, a.nsq, blockDim.x);
  pair_stage<M, float>(a, L, smem);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float *s_sq = (const float *)(smem + L.off_sq);
  const int nt = blockDim.x;
  PairSlot<float> *slot = (PairSlot<float> *)(smem + L.off_slot) + threadIdx.x;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const float2 *__restrict__ C = (const float2 *)a.C;
  float2 *__restrict__ Z = (float2 *)t.Y;
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < t.c_end; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < t.c_end;
    const size_t cc = live ? col : t.c_end - 1u;
    const uint32_t np = (uint32_t)(cc / nrhs);
    const uint32_t jr = (uint32_t)(cc - (size_t)np * nrhs);
    const uint32_t base = pair_slots<M, float>(np, a, t.nc2, s_mod, s_sat, s_sq, slot, nt);
#pragma unroll 1
    for (int K = 0; K < 2 * M - 1; ++K) {
      const int lo = K - (M - 1) > 0 ? K - (M - 1) : 0, nb = K / 2 - lo + 1;
      const float cK = __ldg((const float *)t.blk + K);
      switch (nb) {
        case 1: pairs_mixed<M, 1>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 2: pairs_mixed<M, 2>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 3: pairs_mixed<M, 3>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 4: pairs_mixed<M, 4>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        case 5: pairs_mixed<M, 5>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
        default: pairs_mixed<M, 6>(K, lo, base, slot, nt, C, Z, nrhs, jr, col, live, cK); break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Phase 2: sigma_gamma = sum_r o_r A_r Z_K(gamma - r) + diag(gamma) C_gamma.
// The table t.blk holds c_K (K = 0 .. 2M - 2), 2 c_K, then D_r (r = 0 ..
// P - 1), divided by the coefficient scale for FP32 pairs; phase 1 has taken
// c_K into Z.  The diagonal sum_r D_r n_k (n_q - d_kq) takes two removals
// per packed operation (the integer product exact as a pair).
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_pairs_sigma_df(const TwoPhaseArgs t) {
  constexpr int P = M * (M + 1) / 2, NK = 2 * M - 1;
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_mod = (uint32_t *)(smem + 256);
  const int rows = M - 1;
  uint32_t *s_sat = s_mod + rows * a.xdim;
  float2 *s_sq = (float2 *)(s_sat + rows * a.xdim + 4);
  float2 *s_tab = s_sq + a.nsq;                          // c_K o (NK entries, o = 1: [K], o = 2 after), D_r (P)
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const float2 *)a.sq)[i];
  for (int i = threadIdx.x; i < 2 * NK + P; i += blockDim.x) s_tab[i] = ((const float2 *)t.blk)[i];
  __syncthreads();
  const int nt = blockDim.x;
  const uint32_t nc = a.nc, nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float4 *__restrict__ Z = (const float4 *)t.Y;
  const float4 *__restrict__ C = (const float4 *)a.C;
  int e_out = (int)(((unsigned long long)__double_as_longlong(a.out_scale) >> 52) & 0x7ff) - 1023;
  if (a.in_exp) e_out += __ldg(a.in_exp);
  const size_t cbeg = (size_t)t.g_begin * nrhs, cend = (size_t)t.g_end * nrhs;
  for (size_t tile = cbeg + blockIdx.x * (size_t)nt; tile < cend; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < cend;
    const size_t cc = live ? col : cend - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    int S[M], n[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
#pragma unroll
    for (int m = 0; m < M; ++m) n[m] = S[m] - (m > 0 ? S[m - 1] : 0);
    float2 sq0[M], sq1[M];                               // sqrt(n_m), sqrt(n_m - 1) as pairs
#pragma unroll
    for (int m = 0; m < M; ++m) {
      sq0[m] = s_sq[n[m]];
      sq1[m] = s_sq[max(n[m] - 1, 0)];
    }
    uint32_t P1[M], P2[M];
    const uint32_t q0 = twophase_prefix2<M>(S, s_mod, a.xdim, nc2, P1, P2);
    fp2_t Ah = 0ull, Al = 0ull;
    fp2_t dH = 0ull, dL = 0ull;                          // diag(gamma): two partial pairs
    float pa = 0.f, pb = 0.f;                            // pending removal of the diagonal
    float2 pD = make_float2(0.f, 0.f);
    bool pend = false;                                   // resolved at compile time (full unroll)
#pragma unroll
    for (int k = 0; k < M; ++k) {
#pragma unroll
      for (int q = k; q < M; ++q) {
        const int r = k * M - (k * (k - 1)) / 2 + (q - k);
        const bool valid = k == q ? n[k] >= 2 : (n[k] >= 1 && n[q] >= 1);
        const uint32_t r2 = valid ? q0 - (P1[q] - P1[k]) - (P2[M - 1] - P2[q]) : 0u;
        float2 A = df_mul(sq0[k], k == q ? sq1[k] : sq0[q]);         // 0 for an impossible removal
        if (k != q) A = make_float2(2.f * A.x, 2.f * A.y);            // o_r, exact
        const float4 z = __ldg(Z + twophase_yidx(k + q, (size_t)r2 * nrhs + j, NK));
        fp2_t p, e;
        fp2_dprod(fp2_make(z.x, z.y), fp2_make(z.z, z.w), fp2_make(A.x, A.x), fp2_make(A.y, A.y), p, e);
        fp2_dacc(Ah, Al, p, e);
        // diagonal part D_r n_k (n_q - d_kq), two removals per packed step
        const float fa = (float)n[k], fb = (float)(n[q] - (k == q ? 1 : 0));
        const float2 D = s_tab[2 * NK + r];
        if (!pend) {
          pa = fa; pb = fb; pD = D; pend = true;
        } else {
          const fp2_t a2 = fp2_make(pa, fa), b2 = fp2_make(pb, fb);
          const fp2_t mh = fp2_mul(a2, b2), ml = fp2_fms(a2, b2, mh);   // exact product
          const fp2_t Dh = fp2_make(pD.x, D.x), Dl = fp2_make(pD.y, D.y);
          fp2_t dp = fp2_mul(Dh, mh), de = fp2_fms(Dh, mh, dp);
          de = fp2_fma(Dh, ml, de);
          de = fp2_fma(Dl, mh, de);
          fp2_dacc(dH, dL, dp, de);
          pend = false;
        }
      }
    }
    if (pend) {                                          // odd number of removals
      const fp2_t a2 = fp2_make(pa, 0.f), b2 = fp2_make(pb, 0.f);
      const fp2_t mh = fp2_mul(a2, b2), ml = fp2_fms(a2, b2, mh);
      const fp2_t Dh = fp2_make(pD.x, 0.f), Dl = fp2_make(pD.y, 0.f);
      fp2_t dp = fp2_mul(Dh, mh), de = fp2_fms(Dh, mh, dp);
      de = fp2_fma(Dh, ml, de);
      de = fp2_fma(Dl, mh, de);
      fp2_dacc(dH, dL, dp, de);
    }
    float dh = fp2_x(dH), dl = fp2_x(dL);
    df_add_acc(dh, dl, fp2_y(dH), fp2_y(dL));
    const float4 c = __ldg(C + (size_t)g * nrhs + j);
    fp2_t p, e;
    fp2_dprod(fp2_make(c.x, c.y), fp2_make(c.z, c.w), fp2_make(dh, dh), fp2_make(dl, dl), p, e);
    fp2_dacc(Ah, Al, p, e);
    if (live) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      df_add_acc(rh, rl, fp2_x(Ah), fp2_x(Al));
      df_add_acc(ih, il, fp2_y(Ah), fp2_y(Al));
      ((double2 *)a.sigma)[(size_t)g * nrhs + j] =
          make_double2(df_to_double_bits(rh, rl, e_out), df_to_double_bits(ih, il, e_out));
    }
  }
}

template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_pairs_sigma_mixed(const TwoPhaseArgs t) {
  constexpr int P = M * (M + 1) / 2, NK = 2 * M - 1;
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_mod = (uint32_t *)(smem + 256);
  const int rows = M - 1;
  uint32_t *s_sat = s_mod + rows * a.xdim;
  float *s_sq = (float *)(s_sat + rows * a.xdim + 4);
  float *s_tab = s_sq + a.nsq;
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const float *)a.sq)[i];
  for (int i = threadIdx.x; i < 2 * NK + P; i += blockDim.x) s_tab[i] = ((const float *)t.blk)[i];
  __syncthreads();
  const int nt = blockDim.x;
  const uint32_t nc = a.nc, nc2 = t.nc2;
  const int nrhs = a.nrhs;
  const float2 *__restrict__ Z = (const float2 *)t.Y;
  const float2 *__restrict__ C = (const float2 *)a.C;
  const float out_scale = (float)a.out_scale;
  const size_t cbeg = (size_t)t.g_begin * nrhs, cend = (size_t)t.g_end * nrhs;
  for (size_t tile = cbeg + blockIdx.x * (size_t)nt; tile < cend; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < cend;
    const size_t cc = live ? col : cend - 1u;
    const uint32_t g = (uint32_t)(cc / (size_t)nrhs);
    const int j = (int)(cc - (size_t)g * nrhs);
    int S[M], n[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
#pragma unroll
    for (int m = 0; m < M; ++m) n[m] = S[m] - (m > 0 ? S[m - 1] : 0);
    float sq0[M], sq1[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      sq0[m] = s_sq[n[m]];
      sq1[m] = s_sq[max(n[m] - 1, 0)];
    }
    uint32_t P1[M], P2[M];
    const uint32_t q0 = twophase_prefix2<M>(S, s_mod, a.xdim, nc2, P1, P2);
    fp2_t Sh = 0ull, Sl = 0ull;
    float diag = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
#pragma unroll
      for (int q = k; q < M; ++q) {
        const int r = k * M - (k * (k - 1)) / 2 + (q - k);
        const bool valid = k == q ? n[k] >= 2 : (n[k] >= 1 && n[q] >= 1);
        const uint32_t r2 = valid ? q0 - (P1[q] - P1[k]) - (P2[M - 1] - P2[q]) : 0u;
        const float A = (k == q ? 1.f : 2.f) * sq0[k] * (k == q ? sq1[k] : sq0[q]);
        const float2 z = __ldg(Z + twophase_yidx(k + q, (size_t)r2 * nrhs + j, NK));
        fp2_dacc(Sh, Sl, fp2_mul(fp2_make(z.x, z.y), fp2_make(A, A)), 0ull);
        diag = fmaf((float)(n[k] * (n[q] - (k == q ? 1 : 0))), s_tab[2 * NK + r], diag);
      }
    }
    const float2 c = __ldg(C + (size_t)g * nrhs + j);
    fp2_dacc(Sh, Sl, fp2_mul(fp2_make(c.x, c.y), fp2_make(diag, diag)), 0ull);
    if (live) {
      const fp2_t v = fp2_add(Sh, Sl);
      ((float2 *)a.sigma)[(size_t)g * nrhs + j] = make_float2(fp2_x(v) * out_scale, fp2_y(v) * out_scale);
    }
  }
}

template <int M>
size_t pairs_sigma_smem(int xdim, int nsq, bool mixed) {
  constexpr int P = M * (M + 1) / 2, NK = 2 * M - 1;
  return twophase_sigma_smem(M - 1, xdim, nsq) + (mixed ? 4 : 8) * (size_t)(2 * NK + P);
}

template <int M>
int launch_pairs(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  const ApplyArgs<uint32_t> &a = t.a;
  if (t.phases & 1) {
    const uint64_t n = t.c_end - t.c_begin;
    const int st = mixed ? fock_launch_grid(fock_pairs_z_mixed<M>, t, n, PairSmem<M, float>(a.xdim, a.nsq, FOCK_APPLY_THREADS).total,
                                            dev, s)
                         : fock_launch_grid(fock_pairs_z_df<M>, t, n, PairSmem<M, float2>(a.xdim, a.nsq, FOCK_APPLY_THREADS).total,
                                            dev, s);
    if (st) return st;
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  const uint64_t n = (uint64_t)(t.g_end - t.g_begin) * a.nrhs;
  const size_t sm = pairs_sigma_smem<M>(a.xdim, a.nsq, mixed);
  return mixed ? fock_launch_grid(fock_pairs_sigma_mixed<M>, t, n, sm, dev, s)
               : fock_launch_grid(fock_pairs_sigma_df<M>, t, n, sm, dev, s);
}

}  // namespace

int fock_launch_twophase_pairs(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_PAIRS_CASE(MM) \
    case MM: return launch_pairs<MM>(t, mixed, dev, s);
    FOCK_PAIRS_CASE(2)
    FOCK_PAIRS_CASE(3)
    FOCK_PAIRS_CASE(4)
    FOCK_PAIRS_CASE(5)
    FOCK_PAIRS_CASE(6)
    FOCK_PAIRS_CASE(7)
    FOCK_PAIRS_CASE(8)
    FOCK_PAIRS_CASE(9)
    FOCK_PAIRS_CASE(10)
    FOCK_PAIRS_CASE(11)
    FOCK_PAIRS_CASE(12)
#undef FOCK_PAIRS_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}

// Host: the rank-one form of a pair-weight-conserving reduced matrix R (P x P,
// lexicographic pairs), if it has one: per block K a real c_K with
// R[r][a] = c_K o_r o_a for r != a, and real diagonal remainders D_r.  Tables
// (for the FP32-pair form divided by `scale`): [c_K]_{K} [2 c_K]_{K} [D_r]_{r}
// as (hi, lo) pairs and as floats.  False when R is not of that form (to within
// tol times the largest coefficient).
bool fock_pairs_tables(int M, const std::complex<double> *R, double scale, double tol, std::vector<float2> &df,
                       std::vector<float> &mx) {
  const int P = M * (M + 1) / 2, NK = 2 * M - 1;
  double rmax = 0.0;
  for (int i = 0; i < P * P; ++i) rmax = fmax(rmax, std::abs(R[i]));
  const double eps = tol * rmax;
  auto pidx = [M](int s, int l) { return s * M - (s * (s - 1)) / 2 + (l - s); };
  std::vector<double> c(NK, 0.0), D(P, 0.0);
  for (int K = 0; K < NK; ++K) {
    const int lo = K - (M - 1) > 0 ? K - (M - 1) : 0, nb = K / 2 - lo + 1;
    auto o = [&](int i) { return (lo + i) != (K - lo - i) ? 2.0 : 1.0; };
    auto at = [&](int i, int j) { return R[(size_t)pidx(lo + i, K - lo - i) * P + pidx(lo + j, K - lo - j)]; };
    if (nb == 1) {
      c[K] = at(0, 0).real() / (o(0) * o(0));
      if (fabs(at(0, 0).imag()) > eps) return false;
    } else {
      c[K] = at(0, 1).real() / (o(0) * o(1));
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
          const std::complex<double> v = at(i, j);
          if (fabs(v.imag()) > eps) return false;
          if (i != j && fabs(v.real() - c[K] * o(i) * o(j)) > eps) return false;
        }
    }
    for (int i = 0; i < nb; ++i) D[pidx(lo + i, K - lo - i)] = at(i, i).real() - c[K] * o(i) * o(i);
  }
  // every entry outside the blocks must vanish (the pair weight is conserved)
  for (int r = 0; r < P; ++r)
    for (int a2 = 0; a2 < P; ++a2) {
      int sr = 0, sa = 0, x = r, y = a2;
      for (int s = 0; s < M; ++s)
        if (x < M - s) { sr = s + (s + x); break; } else x -= M - s;
      for (int s = 0; s < M; ++s)
        if (y < M - s) { sa = s + (s + y); break; } else y -= M - s;
      if (sr != sa && std::abs(R[(size_t)r * P + a2]) > eps) return false;
    }
  auto put = [&](double v, int i) {
    const double x = v / scale;
    const float h = (float)x;
    df[i] = make_float2(h, (float)(x - (double)h));
    mx[i] = (float)v;
  };
  df.assign(2 * NK + P, make_float2(0.f, 0.f));
  mx.assign(2 * NK + P, 0.f);
  for (int K = 0; K < NK; ++K) {
    put(c[K], K);
    put(2.0 * c[K], NK + K);
  }
  for (int r = 0; r < P; ++r) put(D[r], 2 * NK + r);
  return true;
}
