// fock_apply_sparse.cuh -- sigma = H C for any coefficient sparsity (e.g. the
// momentum-conserving Lieb-Liniger W, or one-body operators), pull form.
//
// Moving particles changes the prefix sums S_m of a configuration by a step
// function d(m) = [s <= m] + [l <= m] - [k <= m] - [q <= m] (removal {k, q},
// addition {s, l}); with the hash of Eq. TotalCost in closed form,
//
//     target = gamma - sum_{m} D_m(d(m)),   D_m(d) = C(S_m + m + d, m + 1) - C(S_m + m, m + 1).
//
// Each thread tabulates, once per configuration, the prefix sums
// PD_d[j] = sum_{m<j} D_m(d) for d in {-2, -1, 1, 2} in its slice of shared
// memory.  The breakpoints of d(m) and its values on the (at most three)
// intervals between them depend only on the term, not on the configuration, so
// the host precomputes them: a term's target is six table reads.  Amplitudes
// come from the occupations (shared memory) and a table of square roots:
//     sqrt(n_k (n_q - delta_kq)) * sqrt((n_s - ds + 1) (n_l - dl + 1)),
// with ds, dl the host-precomputed corrections for orbitals shared between the
// removal and the addition.  No per-removal setup pass is needed.
#pragma once

#include "fock_apply_kernel.cuh"
#include "fock_pack.cuh"

// One (removal, addition) term of the coefficient list, 16 bytes.  off[] are
// the byte offsets, inside a thread's prefix table (rows d + 2 = 0..4 of MAXM
// entries, FOCK_APPLY_THREADS words apart), of the six reads
//     + PD_{d0}[x1] - PD_{d0}[x0] + PD_{d1}[x2] - PD_{d1}[x1] + PD_{d2}[x3] - PD_{d2}[x2]
// where x0 <= x1 <= x2 <= x3 are the breakpoints of d(m) and d0, d1, d2 its
// values between them.
struct FockTerm {
  uint16_t off[6];
  int8_t s;         // first added orbital (-1 for a one-particle addition)
  int8_t l;         // second added orbital
  int8_t ds, dl;    // n'_s + 1 = n_s - ds + 1,  n''_l + 1 = n_l - dl + 1
};

__host__ __device__ inline int fock_sparse_maxm(int M) { return M <= 4 ? 4 : (M <= 8 ? 8 : 12); }

struct SparseArgs {
  ApplyArgs<uint32_t> base;      // sizes, tables, vectors, removal list, coefficients
  const FockTerm *terms;         // [nadd]
  const int32_t *slots;          // [nadd] map slot of each term (maps arm)
  int nadd;
};

struct SparseSmemLayout {
  size_t off_terms, off_coef, off_mod, off_sat, off_sq, off_pd, off_n, total;
};

template <int MAXM>
__host__ __device__ inline SparseSmemLayout sparse_layout(int nadd, size_t coef_bytes, int rows, int xdim, int nsq,
                                                          size_t sq_bytes, int threads) {
  SparseSmemLayout L;
  size_t o = 0;
  L.off_terms = o; o = fock_align16(o + sizeof(FockTerm) * (size_t)nadd);
  L.off_coef = o;  o = fock_align16(o + coef_bytes * (size_t)nadd);
  L.off_mod = o;   o = fock_align16(o + 4 * (size_t)rows * (xdim + 2));
  L.off_sat = o;   o = fock_align16(o + 4 * (size_t)rows * xdim);
  L.off_sq = o;    o = fock_align16(o + sq_bytes * (size_t)nsq);
  L.off_pd = o;    o = fock_align16(o + 4 * (size_t)5 * MAXM * threads);
  L.off_n = o;     o = fock_align16(o + 4 * (size_t)MAXM * threads);
  L.total = o;
  return L;
}

// Everything one configuration needs, with the problem's tables staged in
// shared memory (shared by the single-problem and the batched kernels).
struct SparseView {
  int N, M, nrem, xs, xdim, nrhs;
  uint32_t nc;
  const uint32_t *mod;           // shared, rows of xs = xdim + 2 (two leading zeros)
  const uint32_t *sat;           // shared, rows of xdim
  const void *sq;                // shared square-root table (policy amp_t)
  const FockTerm *terms;         // shared
  const void *coef;              // shared (policy coef_t)
  const FockRemoval *rem;        // removal list
  const void *C;                 // vectors of this problem, [nc][nrhs]
  void *sigma;
  const int32_t *map, *slots;    // maps arm
  double out_scale;
};

// sigma for configuration g of the problem (g >= nc: a dead lane that only
// takes part in the warp-wide votes).  pd/nn are this thread's slices.
template <int MAXM, class P, bool REAL, int CH, bool MAPS>
__device__ __forceinline__ void sparse_config(const SparseView &v, uint32_t g, uint32_t *pd, int *nn, int nt) {
  using amp_t = typename P::amp_t;
  using vec_t = typename P::vec_t;
  using coef_t = typename P::coef_t;
  const amp_t *s_sq = (const amp_t *)v.sq;
  const coef_t *coef = (const coef_t *)v.coef;
  const vec_t *__restrict__ C = (const vec_t *)v.C;
  const int M = v.M, nrhs = v.nrhs;
  const uint32_t nc = v.nc;
  const bool live = g < nc;
  const uint32_t gc = live ? g : nc - 1u;
  int S[MAXM];
  fock_decode_prefix<uint32_t, MAXM>(gc, v.N, M, nc, v.sat, v.xdim, S);
  // occupations and the prefix sums of the table deltas
  uint32_t Pm2 = 0, Pm1 = 0, Pp1 = 0, Pp2 = 0;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (m < M) {
      nn[m * nt] = S[m] - (m > 0 ? S[m - 1] : 0);
      pd[(0 * MAXM + m) * nt] = Pm2;
      pd[(1 * MAXM + m) * nt] = Pm1;
      pd[(3 * MAXM + m) * nt] = Pp1;
      pd[(4 * MAXM + m) * nt] = Pp2;
      if (m < M - 1) {
        const uint32_t *row = v.mod + m * v.xs + (S[m] + m + 2);
        const uint32_t t0 = row[0];
        Pm2 += row[-2] - t0;
        Pm1 += row[-1] - t0;
        Pp1 += row[1] - t0;
        Pp2 += row[2] - t0;
      }
    }
  }
  for (int c0 = 0; c0 < nrhs; c0 += CH) {
    typename P::acc_t acc[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) P::zero(acc[j]);
    for (int ri = 0; ri < v.nrem; ++ri) {
      const FockRemoval R = v.rem[ri];
      const int k = R.k, q = R.q;
      const bool two = R.size == 2;
      const int nk = nn[k * nt];
      const int nq = two ? nn[q * nt] : 0;
      const bool valid = live && (two ? (k == q ? nk >= 2 : (nk >= 1 && nq >= 1)) : nk >= 1);
      if (!__any_sync(0xffffffffu, valid)) continue;
      amp_t A = s_sq[valid ? nk : 0];
      if (two) A = P::amul(A, s_sq[valid ? nq - (k == q) : 0]);
      typename P::inner_t inner[P::kInner ? CH : 1];
      if constexpr (P::kInner) {
#pragma unroll
        for (int j = 0; j < CH; ++j) P::izero(inner[j]);
      }
#pragma unroll 4
      for (int e = R.a_beg; e < R.a_end; ++e) {
        const uint4 w = ((const uint4 *)v.terms)[e];
        uint32_t t;
        if (MAPS) {
          t = (uint32_t)__ldg(v.map + (size_t)__ldg(v.slots + e) * nc + gc);
        } else {
          const unsigned char *pb = (const unsigned char *)pd;
          const uint32_t sum = *(const uint32_t *)(pb + (w.x & 0xffffu)) - *(const uint32_t *)(pb + (w.x >> 16)) +
                               *(const uint32_t *)(pb + (w.y & 0xffffu)) - *(const uint32_t *)(pb + (w.y >> 16)) +
                               *(const uint32_t *)(pb + (w.z & 0xffffu)) - *(const uint32_t *)(pb + (w.z >> 16));
          t = g - sum;
        }
        t = valid ? t : gc;
        const int ts = (int)(int8_t)(w.w & 0xffu), tl = (int)(int8_t)((w.w >> 8) & 0xffu);
        const int tds = (int)(int8_t)((w.w >> 16) & 0xffu), tdl = (int)(int8_t)(w.w >> 24);
        const int il = max(nn[tl * nt] - tdl + 1, 0);
        amp_t amp = P::amul(A, s_sq[il]);
        if (ts >= 0) amp = P::amul(amp, s_sq[max(nn[ts * nt] - tds + 1, 0)]);
        const coef_t K = P::scale(coef[e], amp);
        const vec_t *src = C + (size_t)t * nrhs + c0;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          if (CH == 1 || c0 + j < nrhs) {
            if constexpr (P::kInner) P::imac(inner[j], K, __ldg(src + j), REAL);
            else P::mac(acc[j], K, __ldg(src + j), REAL);
          }
        }
      }
      if constexpr (P::kInner) {
#pragma unroll
        for (int j = 0; j < CH; ++j) P::flush(acc[j], inner[j], REAL);
      }
    }
    if (live) {
      auto *out = (decltype(P::finish(acc[0], 1.0, REAL)) *)v.sigma + (size_t)g * nrhs + c0;
#pragma unroll
      for (int j = 0; j < CH; ++j)
        if (CH == 1 || c0 + j < nrhs) out[j] = P::finish(acc[j], v.out_scale, REAL);
    }
  }
}

// Stage one problem's tables in shared memory (all threads of the block).
template <class P>
__device__ __forceinline__ void sparse_stage(unsigned char *smem, const SparseSmemLayout &L, int rows, int xdim,
                                             const uint32_t *mod, const uint32_t *sat, int nsq, const void *sq,
                                             int nadd, const FockTerm *terms, const void *coef) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  uint32_t *s_mod = (uint32_t *)(smem + L.off_mod);
  uint32_t *s_sat = (uint32_t *)(smem + L.off_sat);
  amp_t *s_sq = (amp_t *)(smem + L.off_sq);
  FockTerm *s_terms = (FockTerm *)(smem + L.off_terms);
  coef_t *s_coef = (coef_t *)(smem + L.off_coef);
  const int tid = threadIdx.x, nt = blockDim.x, xs = xdim + 2;
  for (int i = tid; i < rows * xs; i += nt) {
    const int m = i / xs, x = i - m * xs;
    s_mod[i] = x < 2 ? 0u : mod[m * xdim + x - 2];
  }
  for (int i = tid; i < rows * xdim; i += nt) s_sat[i] = sat[i];
  for (int i = tid; i < nadd; i += nt) {
    s_terms[i] = terms[i];
    s_coef[i] = ((const coef_t *)coef)[i];
  }
  for (int i = tid; i < nsq; i += nt) s_sq[i] = ((const amp_t *)sq)[i];
}

// 6 blocks per SM (85 registers): measured 3-6 % faster than 4 or 8 on the
// Lieb-Liniger rings (N = 22 and 30, M = 10).
template <int MAXM, class P, bool REAL, int CH, bool MAPS>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 6)
fock_apply_sparse(const SparseArgs sa) {
  const ApplyArgs<uint32_t> &a = sa.base;
  extern __shared__ __align__(16) unsigned char smem[];
  const SparseSmemLayout L = sparse_layout<MAXM>(sa.nadd, sizeof(typename P::coef_t), a.rows, a.xdim, a.nsq,
                                                 sizeof(typename P::amp_t), blockDim.x);
  sparse_stage<P>(smem, L, a.rows, a.xdim, a.mod, a.sat, a.nsq, a.sq, sa.nadd, sa.terms, a.coef);
  const int tid = threadIdx.x, nt = blockDim.x;
  uint32_t *pd = (uint32_t *)(smem + L.off_pd) + tid;   // pd[(d+2)*MAXM*nt + j*nt]
  int *nn = (int *)(smem + L.off_n) + tid;               // nn[m*nt]
#pragma unroll
  for (int j = 0; j < MAXM; ++j) pd[(2 * MAXM + j) * nt] = 0u;  // d = 0 row
  __syncthreads();
  SparseView v;
  v.N = a.N; v.M = a.M; v.nrem = a.nrem; v.xs = a.xdim + 2; v.xdim = a.xdim; v.nrhs = a.nrhs; v.nc = a.nc;
  v.mod = (const uint32_t *)(smem + L.off_mod);
  v.sat = (const uint32_t *)(smem + L.off_sat);
  v.sq = smem + L.off_sq;
  v.terms = (const FockTerm *)(smem + L.off_terms);
  v.coef = smem + L.off_coef;
  v.rem = a.rem;
  v.C = a.C;
  v.sigma = a.sigma;
  v.map = a.map;
  v.slots = sa.slots;
  v.out_scale = a.out_scale;
  if (a.in_exp) v.out_scale *= fock_pow2(__ldg(a.in_exp));
  for (uint32_t tile = blockIdx.x * (uint32_t)nt; tile < a.nc; tile += gridDim.x * (uint32_t)nt)
    sparse_config<MAXM, P, REAL, CH, MAPS>(v, tile + tid, pd, nn, nt);
}

template <int MAXM, class P, bool REAL, int CH, bool MAPS>
int fock_launch_sparse_one(const SparseArgs &sa, int device, cudaStream_t stream) {
  auto kern = fock_apply_sparse<MAXM, P, REAL, CH, MAPS>;
  const int threads = FOCK_APPLY_THREADS;
  const SparseSmemLayout L = sparse_layout<MAXM>(sa.nadd, sizeof(typename P::coef_t), sa.base.rows, sa.base.xdim,
                                                 sa.base.nsq, sizeof(typename P::amp_t), threads);
  if (L.total > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return fock_cuda_status(e);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, L.total);
  if (e != cudaSuccess) return fock_cuda_status(e);
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t tiles = ((int64_t)sa.base.nc + threads - 1) / threads;
  int64_t grid = (int64_t)per_sm * fock_get_sm_count(device);
  if (grid > tiles) grid = tiles;
  kern<<<(unsigned)grid, threads, L.total, stream>>>(sa);
  e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

// Dispatch on (MAXM, real coefficients, block of right-hand sides, maps arm).
template <class P, int CHB>
int fock_launch_sparse_policy(const SparseArgs &sa, bool block, bool maps, int device, cudaStream_t s) {
  const int M = sa.base.M;
  const bool real = sa.base.real;
  if (maps && block) return FOCK_ERR_UNSUPPORTED;
#define FOCK_SPARSE_CASE(MM)                                                                        \
  if (M <= MM) {                                                                                   \
    if (maps) return real ? fock_launch_sparse_one<MM, P, true, 1, true>(sa, device, s)            \
                          : fock_launch_sparse_one<MM, P, false, 1, true>(sa, device, s);          \
    if (block) return real ? fock_launch_sparse_one<MM, P, true, CHB, false>(sa, device, s)        \
                           : fock_launch_sparse_one<MM, P, false, CHB, false>(sa, device, s);      \
    return real ? fock_launch_sparse_one<MM, P, true, 1, false>(sa, device, s)                     \
                : fock_launch_sparse_one<MM, P, false, 1, false>(sa, device, s);                   \
  }
  FOCK_SPARSE_CASE(4)
  FOCK_SPARSE_CASE(8)
  FOCK_SPARSE_CASE(12)
#undef FOCK_SPARSE_CASE
  return FOCK_ERR_UNSUPPORTED;
}
