// fock_twophase_block.cu -- the two-phase apply (fock_apply_twophase.cuh) for
// operators that conserve the pair weight: the reduced coefficient R[r][a] of
// removal pair r = {k, q} and addition pair a = {s, l} vanishes unless
// k + q = s + l.  R is then block diagonal by the pair sum K = 0 .. 2M - 2
// (a block holds the pairs {s, K - s}, at most floor(M/2) + 1 of them).  For
// the Lieb-Liniger ring in plane waves (Sec. 6, Eq. LLHamiltonian) K is the
// total momentum of the pair: W_kqsl = g/L when k + q = s + l.
//
// Phase 1, one thread per (N-2)-configuration n' (and right-hand side):
//     Y[r][n'] = sum_{a in block(r)} R[r][a] B_a(n') C[n' + a],
// block by block: the block's gathers of C, the amplitudes B_a, then the
// block's rows of Y (sum_K |block K|^2 products instead of P^2; 195 instead
// of 3025 at M = 10).  Y has the blocked layout of the dense two-phase apply,
// so phase 2 (sigma_gamma = sum_r A_r(gamma) Y[r][gamma - r]) is the dense
// form's kernel.  FP32 pairs (FOCK_PREC_F64) or FP32 (FOCK_PREC_F32_MIXED),
// as the dense two-phase kernels.
#include <complex>
#include <vector>

#include "fock_apply_twophase.cuh"

// Pairs (s, l), s <= l, grouped by their sum K, with each block's offset in the
// pair list and in the block coefficient table (rows r, columns a of one
// block, row-major), as compile-time tables.
template <int M>
struct PairBlocks {
  static constexpr int P = M * (M + 1) / 2, NB = 2 * M - 1, MAXB = M / 2 + 1;
  int cnt[NB], off[NB], coff[NB], pidx[P], s[P], l[P];
  __host__ __device__ constexpr PairBlocks() : cnt(), off(), coff(), pidx(), s(), l() {
    int o = 0, c = 0;
    for (int K = 0; K < NB; ++K) {
      off[K] = o;
      coff[K] = c;
      int n = 0;
      for (int a = K - (M - 1) > 0 ? K - (M - 1) : 0; 2 * a <= K; ++a) {
        const int b = K - a;
        s[o + n] = a;
        l[o + n] = b;
        pidx[o + n] = a * M - (a * (a - 1)) / 2 + (b - a);
        ++n;
      }
      cnt[K] = n;
      o += n;
      c += n * n;
    }
  }
  __host__ __device__ constexpr int coef_entries() const { return coff[NB - 1] + cnt[NB - 1] * cnt[NB - 1]; }
};

// Host: the block coefficient tables from the full reduced matrix R (P x P,
// row r = removal pair, column a = addition pair, lexicographic indices).
// Returns false when some coefficient links pairs of different sums.
template <int M>
static bool block_tables(const std::complex<double> *R, double scale, std::vector<float4> &df,
                         std::vector<float2> &mx) {
  constexpr PairBlocks<M> pb;
  constexpr int P = PairBlocks<M>::P;
  std::vector<int> sum_of(P);
  for (int i = 0; i < P; ++i) sum_of[pb.pidx[i]] = pb.s[i] + pb.l[i];
  for (int r = 0; r < P; ++r)
    for (int a = 0; a < P; ++a)
      if (R[(size_t)r * P + a] != 0.0 && sum_of[r] != sum_of[a]) return false;
  df.assign(pb.coef_entries(), make_float4(0.f, 0.f, 0.f, 0.f));
  mx.assign(pb.coef_entries(), make_float2(0.f, 0.f));
  for (int K = 0; K < PairBlocks<M>::NB; ++K)
    for (int i = 0; i < pb.cnt[K]; ++i)
      for (int j = 0; j < pb.cnt[K]; ++j) {
        const std::complex<double> v = R[(size_t)pb.pidx[pb.off[K] + i] * P + pb.pidx[pb.off[K] + j]];
        const double re = v.real() / scale, im = v.imag() / scale;
        const float rh = (float)re, ih = (float)im;
        df[pb.coff[K] + i * pb.cnt[K] + j] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
        mx[pb.coff[K] + i * pb.cnt[K] + j] = make_float2((float)v.real(), (float)v.imag());
      }
  return true;
}

// Phase 1 runs a loop over the blocks at run time, each block by code
// specialised for its size (1 .. floor(M/2) + 1 pairs), instead of one fully
// unrolled body of all 2M - 1 blocks (about 4,800 instructions per column at
// M = 10, 40 % of the issue slots stalled on instruction fetch).  The
// column's per-orbital values (target offsets U, V and square roots) live in
// a shared-memory slot per thread so that the run-time orbital indices of a
// block need no local memory.
template <class SqT>
struct BlockSlot {
  uint32_t U, V;
  SqT b, c;                 // sqrt(n'_m + 1), sqrt(n'_m + 2)
};

template <int M, class SqT>
__device__ __forceinline__ uint32_t block_slots(uint32_t np, const ApplyArgs<uint32_t> &a, uint32_t nc2,
                                                const uint32_t *s_mod, const uint32_t *s_sat, const SqT *s_sq,
                                                BlockSlot<SqT> *slot, int nt) {
  int S[M];
  fock_decode_fast<M>(np, a.N - 2, nc2, s_sat, a.xdim, S);
  uint32_t U[M], V[M];
  const uint32_t base = twophase_targets<M>(S, s_mod, a.xdim, a.nc, U, V);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int occ = S[m] - (m > 0 ? S[m - 1] : 0);
    BlockSlot<SqT> z;
    z.U = U[m];
    z.V = V[m];
    z.b = s_sq[occ + 1];
    z.c = s_sq[occ + 2];
    slot[m * nt] = z;
  }
  return base;
}

// Shared memory of phase 1: block coefficients, binomial tables, square roots,
// the threads' slots.
template <int M>
struct BlockSmemRT {
  size_t off_coef, off_mod, off_sat, off_sq, off_slot, total;
  __host__ __device__ BlockSmemRT(int xdim, int nsq, size_t coef_bytes, size_t slot_bytes, int threads) {
    constexpr PairBlocks<M> pb;
    const int rows = M - 1;
    size_t o = 0;
    off_coef = o; o = fock_align16(o + coef_bytes * pb.coef_entries());
    off_mod = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sat = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sq = o;   o = fock_align16(o + 8 * (size_t)nsq);
    off_slot = o; o = fock_align16(o + slot_bytes * M * (size_t)threads);
    total = o;
  }
};

template <int M, class CoefT, class SqT>
__device__ __forceinline__ void block_stage_rt(const TwoPhaseArgs &t, const BlockSmemRT<M> &L, unsigned char *smem) {
  constexpr PairBlocks<M> pb;
  const ApplyArgs<uint32_t> &a = t.a;
  CoefT *s_coef = (CoefT *)(smem + L.off_coef);
  for (int i = threadIdx.x; i < pb.coef_entries(); i += blockDim.x) s_coef[i] = ((const CoefT *)t.blk)[i];
  uint32_t *s_mod = (uint32_t *)(smem + L.off_mod), *s_sat = (uint32_t *)(smem + L.off_sat);
  for (int i = threadIdx.x; i < (M - 1) * a.xdim; i += blockDim.x) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  SqT *s_sq = (SqT *)(smem + L.off_sq);
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const SqT *)a.sq)[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Phase 1, FP32 pairs: X_a = B_a C[n' + a] by Dekker products (lanes Re, Im),
// Y_r = sum_a R[r][a] X_a with the coefficient's real part times (Re X, Im X)
// and, for complex coefficients, (-Im R, Im R) times (Im X, Re X).  One block
// of NB pairs (s, K - s), s = lo .. lo + NB - 1, coefficients from s_coef[co].
// ---------------------------------------------------------------------------
template <int M, int NB>
__device__ __forceinline__ void block_df(int K, int lo, int co, uint32_t base, const BlockSlot<float2> *slot, int nt,
                                         const float4 *__restrict__ C, float4 *__restrict__ Y, const float4 *s_coef,
                                         uint32_t nrhs, uint32_t jr, size_t col, bool live, bool real) {
  constexpr int P = M * (M + 1) / 2;
  float4 v[NB];
  float2 amp[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int s = lo + i, l = K - s;
    const BlockSlot<float2> zs = slot[s * nt], zl = slot[l * nt];
    v[i] = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + jr);
    amp[i] = df_mul(zs.b, s == l ? zs.c : zl.b);
  }
  fp2_t Xh[NB], Xl[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i)
    fp2_dprod(fp2_make(v[i].x, v[i].y), fp2_make(v[i].z, v[i].w), fp2_make(amp[i].x, amp[i].x),
              fp2_make(amp[i].y, amp[i].y), Xh[i], Xl[i]);
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    fp2_t h = 0ull, lw = 0ull;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const float4 w = s_coef[co + r * NB + i];            // (Re R hi, Im R hi, Re R lo, Im R lo)
      fp2_t p, e;
      fp2_dprod(Xh[i], Xl[i], fp2_make(w.x, w.x), fp2_make(w.z, w.z), p, e);
      fp2_dacc(h, lw, p, e);
      if (!real) {
        fp2_dprod(fp2_swap(Xh[i]), fp2_swap(Xl[i]), fp2_make(-w.y, w.y), fp2_make(-w.w, w.w), p, e);
        fp2_dacc(h, lw, p, e);
      }
    }
    const int s = lo + r, l = K - s;
    if (live)
      __stcs(&Y[twophase_yidx(s * M - (s * (s - 1)) / 2 + (l - s), col, P)],
             make_float4(fp2_x(h), fp2_y(h), fp2_x(lw), fp2_y(lw)));
  }
}

template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_twophase_x_block_df(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const BlockSmemRT<M> L(a.xdim, a.nsq, sizeof(float4), sizeof(BlockSlot<float2>), blockDim.x);
  block_stage_rt<M, float4, float2>(t, L, smem);
  const float4 *s_coef = (const float4 *)(smem + L.off_coef);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float2 *s_sq = (const float2 *)(smem + L.off_sq);
  const int nt = blockDim.x;
  BlockSlot<float2> *slot = (BlockSlot<float2> *)(smem + L.off_slot) + threadIdx.x;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const size_t total = t.c_end;                           // columns [c_begin, c_end) of this launch
  const bool real = a.real;
  const float4 *__restrict__ C = (const float4 *)a.C;
  float4 *__restrict__ Y = (float4 *)t.Y;
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < total; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < total;
    const size_t cc = live ? col : total - 1u;
    const uint32_t np = (uint32_t)(cc / nrhs);
    const uint32_t jr = (uint32_t)(cc - (size_t)np * nrhs);
    const uint32_t base = block_slots<M, float2>(np, a, t.nc2, s_mod, s_sat, s_sq, slot, nt);
    int co = 0;
#pragma unroll 1
    for (int K = 0; K < 2 * M - 1; ++K) {
      const int lo = K - (M - 1) > 0 ? K - (M - 1) : 0, nb = K / 2 - lo + 1;
      switch (nb) {
        case 1: block_df<M, 1>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
        case 2: block_df<M, 2>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
        case 3: block_df<M, 3>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
        case 4: block_df<M, 4>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
        case 5: block_df<M, 5>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
        default: block_df<M, 6>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live, real); break;
      }
      co += nb * nb;
    }
  }
}

// ---------------------------------------------------------------------------
// Phase 1, FP32-mixed: X_a = B_a C[n' + a] in FP32 from complex64 C, FP32
// products and sums per block row, Y as complex64.
// ---------------------------------------------------------------------------
template <int M, int NB>
__device__ __forceinline__ void block_mixed(int K, int lo, int co, uint32_t base, const BlockSlot<float> *slot, int nt,
                                            const float2 *__restrict__ C, float2 *__restrict__ Y, const float2 *s_coef,
                                            uint32_t nrhs, uint32_t jr, size_t col, bool live) {
  constexpr int P = M * (M + 1) / 2;
  fp2_t Xp[NB], Xs[NB];                                   // (Re X, Im X) and (Im X, Re X)
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int s = lo + i, l = K - s;
    const BlockSlot<float> zs = slot[s * nt], zl = slot[l * nt];
    const float2 v = __ldg(C + (size_t)(base - zs.U - zl.V) * nrhs + jr);
    const float amp = zs.b * (s == l ? zs.c : zl.b);
    Xp[i] = fp2_make(v.x * amp, v.y * amp);
    Xs[i] = fp2_make(v.y * amp, v.x * amp);
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    fp2_t A1 = 0ull, A2 = 0ull;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const float2 w = s_coef[co + r * NB + i];
      const fp2_t Rp = fp2_make(w.x, w.y);
      A1 = fp2_fma(Rp, Xp[i], A1);                         // (Re R Re X, Im R Im X)
      A2 = fp2_fma(Rp, Xs[i], A2);                         // (Re R Im X, Im R Re X)
    }
    const int s = lo + r, l = K - s;
    if (live)
      __stcs(&Y[twophase_yidx(s * M - (s * (s - 1)) / 2 + (l - s), col, P)],
             make_float2(fp2_x(A1) - fp2_y(A1), fp2_x(A2) + fp2_y(A2)));
  }
}

template <int M>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_twophase_x_block_mixed(const TwoPhaseArgs t) {
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const BlockSmemRT<M> L(a.xdim, a.nsq, sizeof(float2), sizeof(BlockSlot<float>), blockDim.x);
  block_stage_rt<M, float2, float>(t, L, smem);
  const float2 *s_coef = (const float2 *)(smem + L.off_coef);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float *s_sq = (const float *)(smem + L.off_sq);
  const int nt = blockDim.x;
  BlockSlot<float> *slot = (BlockSlot<float> *)(smem + L.off_slot) + threadIdx.x;
  const uint32_t nrhs = (uint32_t)a.nrhs;
  const size_t total = t.c_end;                           // columns [c_begin, c_end) of this launch
  const float2 *__restrict__ C = (const float2 *)a.C;
  float2 *__restrict__ Y = (float2 *)t.Y;
  for (size_t tile = t.c_begin + blockIdx.x * (size_t)nt; tile < total; tile += gridDim.x * (size_t)nt) {
    const size_t col = tile + threadIdx.x;
    const bool live = col < total;
    const size_t cc = live ? col : total - 1u;
    const uint32_t np = (uint32_t)(cc / nrhs);
    const uint32_t jr = (uint32_t)(cc - (size_t)np * nrhs);
    const uint32_t base = block_slots<M, float>(np, a, t.nc2, s_mod, s_sat, s_sq, slot, nt);
    int co = 0;
#pragma unroll 1
    for (int K = 0; K < 2 * M - 1; ++K) {
      const int lo = K - (M - 1) > 0 ? K - (M - 1) : 0, nb = K / 2 - lo + 1;
      switch (nb) {
        case 1: block_mixed<M, 1>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
        case 2: block_mixed<M, 2>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
        case 3: block_mixed<M, 3>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
        case 4: block_mixed<M, 4>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
        case 5: block_mixed<M, 5>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
        default: block_mixed<M, 6>(K, lo, co, base, slot, nt, C, Y, s_coef, nrhs, jr, col, live); break;
      }
      co += nb * nb;
    }
  }
}

template <int M>
static int launch_block(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  const ApplyArgs<uint32_t> &a = t.a;
  if (t.phases & 1) {
    const uint64_t n = t.c_end - t.c_begin;
    const int st =
        mixed ? fock_launch_grid(fock_twophase_x_block_mixed<M>, t, n,
                                 BlockSmemRT<M>(a.xdim, a.nsq, sizeof(float2), sizeof(BlockSlot<float>), FOCK_APPLY_THREADS).total,
                                 dev, s)
              : fock_launch_grid(fock_twophase_x_block_df<M>, t, n,
                                 BlockSmemRT<M>(a.xdim, a.nsq, sizeof(float4), sizeof(BlockSlot<float2>), FOCK_APPLY_THREADS).total,
                                 dev, s);
    if (st) return st;
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  const uint64_t n = (uint64_t)(t.g_end - t.g_begin) * a.nrhs;
  const size_t sm = twophase_sigma_smem(a.rows, a.xdim, a.nsq);
  return mixed ? fock_launch_grid(fock_twophase_sigma_mixed<M>, t, n, sm, dev, s)
               : fock_launch_grid(fock_twophase_sigma_df<M>, t, n, sm, dev, s);
}

int fock_launch_twophase_block(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_BLK_CASE(MM) \
    case MM: return launch_block<MM>(t, mixed, dev, s);
    FOCK_BLK_CASE(2)
    FOCK_BLK_CASE(3)
    FOCK_BLK_CASE(4)
    FOCK_BLK_CASE(5)
    FOCK_BLK_CASE(6)
    FOCK_BLK_CASE(7)
    FOCK_BLK_CASE(8)
    FOCK_BLK_CASE(9)
    FOCK_BLK_CASE(10)
    FOCK_BLK_CASE(11)
    FOCK_BLK_CASE(12)
#undef FOCK_BLK_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}

// Block coefficient tables of a pair-weight-conserving operator; false when
// R links pairs of different sums (the path does not apply).
bool fock_block_tables(int M, const std::complex<double> *R, double scale, std::vector<float4> &df,
                       std::vector<float2> &mx) {
  switch (M) {
#define FOCK_BLK_TAB(MM) \
    case MM: return block_tables<MM>(R, scale, df, mx);
    FOCK_BLK_TAB(2)
    FOCK_BLK_TAB(3)
    FOCK_BLK_TAB(4)
    FOCK_BLK_TAB(5)
    FOCK_BLK_TAB(6)
    FOCK_BLK_TAB(7)
    FOCK_BLK_TAB(8)
    FOCK_BLK_TAB(9)
    FOCK_BLK_TAB(10)
    FOCK_BLK_TAB(11)
    FOCK_BLK_TAB(12)
#undef FOCK_BLK_TAB
  }
  return false;
}

size_t fock_block_smem(int M, int xdim, int nsq, bool mixed) {
  switch (M) {
#define FOCK_BLK_SM(MM) \
    case MM: return mixed ? BlockSmemRT<MM>(xdim, nsq, sizeof(float2), sizeof(BlockSlot<float>), FOCK_APPLY_THREADS).total \
                          : BlockSmemRT<MM>(xdim, nsq, sizeof(float4), sizeof(BlockSlot<float2>), FOCK_APPLY_THREADS).total;
    FOCK_BLK_SM(2)
    FOCK_BLK_SM(3)
    FOCK_BLK_SM(4)
    FOCK_BLK_SM(5)
    FOCK_BLK_SM(6)
    FOCK_BLK_SM(7)
    FOCK_BLK_SM(8)
    FOCK_BLK_SM(9)
    FOCK_BLK_SM(10)
    FOCK_BLK_SM(11)
    FOCK_BLK_SM(12)
#undef FOCK_BLK_SM
  }
  return (size_t)-1;
}
