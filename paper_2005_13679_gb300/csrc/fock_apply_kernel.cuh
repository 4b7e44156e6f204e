// fock_apply_kernel.cuh -- the sigma = H C kernel (Eq. Haction), pull form.
//
// One thread owns one output configuration gamma (consecutive threads hold
// consecutive gamma, so the gathers of a warp for one operator string land on
// nearly consecutive addresses).  With the occupation n of gamma decoded in
// registers, the thread walks the Hamiltonian's removal list: for a removal r
// (a_k a_q, or a_k alone) that gamma allows, the remaining configuration
// n' = n - e_k - e_q is summarised per orbital j by
//
//     U_j = F0_j - F1_j,  V_j = F1_j - F2_j,   F_d_j = sum_{m<j} C(S'_m + m + d, m + 1),
//
// so that adding the two particles back at s <= l lands on index
// N_c - 1 - F2_{M-1} - U_s - V_l (two subtractions per term; one-particle
// additions use N_c - 1 - F1_{M-1} - U_l), and by the square-root amplitudes
// c_j = A sqrt(n'_j + 1), d_j = c_j sqrt(n'_j + 2), b_j = sqrt(n'_j + 1) with
// A = sqrt(n_k (n_q - delta_kq)).  The term of the addition (s, l) is then
//
//     coef(r, a) * (s == l ? d_s : c_s b_l) * C[target].
//
// These per-orbital values live in a per-thread slice of shared memory, so the
// additions of any sparsity pattern index them directly.  With the jump maps
// the target index is read from the map instead (MAPS = true).
#pragma once

#include "fock_arith.cuh"
#include "fock_common.cuh"
#include "fock_device.cuh"

#define FOCK_APPLY_THREADS 128

template <class Idx>
struct ApplyArgs {
  int N, M;
  Idx nc;
  int xdim, rows;
  const Idx *mod, *sat;          // binomial tables (global)
  const FockRemoval *rem;
  int nrem;
  const FockAddition *add;
  const void *coef;              // policy coefficient array [nadd]
  const void *sq;                // policy square-root table [N + 4]
  int nsq;
  const void *C;                 // policy vector type, [nc][nrhs]
  void *sigma;                   // output, [nc][nrhs]
  int nrhs;
  const int32_t *map;            // jump map (MAPS) or NULL
  const int *in_exp;             // device word: input scale exponent (PolDF) or NULL
  double out_scale;              // host part of the output scale
  bool real;                     // coefficients are real
};

template <class T>
__device__ __forceinline__ T sel_small(const T (&a)[FOCK_MAXM], int i) {
  T r = a[0];
#pragma unroll
  for (int j = 1; j < FOCK_MAXM; ++j) r = (j == i) ? a[j] : r;
  return r;
}

template <int MAXM>
__device__ __forceinline__ int sel_occ(const int (&n)[MAXM], int i) {
  int r = n[0];
#pragma unroll
  for (int j = 1; j < MAXM; ++j) r = (j == i) ? n[j] : r;
  return r;
}

__host__ __device__ inline size_t fock_align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class Idx, int MAXM, class P>
struct ApplySmem {
  // byte offsets inside dynamic shared memory
  size_t off_mod, off_sat, off_sq, off_U, off_V, off_c, off_b, off_d, total;
  __host__ __device__ ApplySmem(int rows, int xdim, int nsq, int threads) {
    size_t o = 0;
    off_mod = o; o = fock_align16(o + sizeof(Idx) * (size_t)rows * xdim);
    off_sat = o; o = fock_align16(o + sizeof(Idx) * (size_t)rows * xdim);
    off_sq = o;  o = fock_align16(o + sizeof(typename P::amp_t) * (size_t)nsq);
    off_U = o;   o = fock_align16(o + sizeof(Idx) * (size_t)MAXM * threads);
    off_V = o;   o = fock_align16(o + sizeof(Idx) * (size_t)MAXM * threads);
    off_c = o;   o = fock_align16(o + sizeof(typename P::amp_t) * (size_t)MAXM * threads);
    off_b = o;   o = fock_align16(o + sizeof(typename P::amp_t) * (size_t)MAXM * threads);
    off_d = o;   o = fock_align16(o + sizeof(typename P::amp_t) * (size_t)MAXM * threads);
    total = o;
  }
};

template <class Idx, int MAXM, class P, int NRHS, bool MAPS>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS)
fock_apply_list_kernel(const ApplyArgs<Idx> a) {
  using amp_t = typename P::amp_t;
  using vec_t = typename P::vec_t;
  using coef_t = typename P::coef_t;
  extern __shared__ __align__(16) unsigned char smem[];
  const ApplySmem<Idx, MAXM, P> L(a.rows, a.xdim, a.nsq, blockDim.x);
  Idx *s_mod = (Idx *)(smem + L.off_mod);
  Idx *s_sat = (Idx *)(smem + L.off_sat);
  amp_t *s_sq = (amp_t *)(smem + L.off_sq);
  Idx *s_U = (Idx *)(smem + L.off_U);
  Idx *s_V = (Idx *)(smem + L.off_V);
  amp_t *s_c = (amp_t *)(smem + L.off_c);
  amp_t *s_b = (amp_t *)(smem + L.off_b);
  amp_t *s_d = (amp_t *)(smem + L.off_d);

  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < a.rows * a.xdim; i += nt) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = tid; i < a.nsq; i += nt) s_sq[i] = ((const amp_t *)a.sq)[i];
  __syncthreads();

  const int N = a.N, M = a.M;
  const Idx nc = a.nc;
  const vec_t *__restrict__ C = (const vec_t *)a.C;
  const coef_t *__restrict__ coef = (const coef_t *)a.coef;
  double out_scale = a.out_scale;
  if (a.in_exp) out_scale *= fock_pow2(__ldg(a.in_exp));
  const int nrhs = NRHS == 1 ? 1 : a.nrhs;

  for (Idx tile = (Idx)blockIdx.x * nt; tile < nc; tile += (Idx)gridDim.x * nt) {
    const Idx g = tile + tid;
    const bool live = g < nc;
    const Idx gd = live ? g : nc - 1;
    int S[MAXM], n[MAXM];
    fock_decode_prefix<Idx, MAXM>(gd, N, M, nc, s_sat, a.xdim, S);
#pragma unroll
    for (int m = 0; m < MAXM; ++m) n[m] = S[m] - (m > 0 ? S[m - 1] : 0);

    typename P::acc_t acc[NRHS];
#pragma unroll
    for (int j = 0; j < NRHS; ++j) P::zero(acc[j]);

    for (int ri = 0; ri < a.nrem; ++ri) {
      const FockRemoval R = a.rem[ri];
      const int k = R.k, q = R.q;
      const bool two = R.size == 2;
      const int nk = sel_occ<MAXM>(n, k);
      const int nq = two ? sel_occ<MAXM>(n, q) : 0;
      const bool valid = live && (two ? (k == q ? nk >= 2 : (nk >= 1 && nq >= 1)) : nk >= 1);
      if (!__any_sync(0xffffffffu, valid)) continue;

      // removal amplitude A = sqrt(n_k (n_q - delta_kq))  (sqrt(n_k) for one particle)
      amp_t A = s_sq[valid ? nk : 0];
      if (two) A = P::amul(A, s_sq[valid ? nq - (k == q) : 0]);
      Idx F0 = 0, F1 = 0, F2 = 0;
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          const int dm = valid ? ((k <= m) + (two && q <= m)) : 0;
          const int np = n[m] - (valid ? ((m == k) + (two && m == q)) : 0);
          if (!MAPS) {
            s_U[m * nt + tid] = F0 - F1;
            s_V[m * nt + tid] = F1 - F2;
            if (m < M - 1) {
              const Idx *row = s_mod + m * a.xdim + (S[m] - dm + m);
              F0 += row[0];
              F1 += row[1];
              F2 += row[2];
            }
          }
          const amp_t b = s_sq[np + 1];
          const amp_t c = P::amul(A, b);
          s_b[m * nt + tid] = b;
          s_c[m * nt + tid] = c;
          s_d[m * nt + tid] = P::amul(c, s_sq[np + 2]);
        }
      }
      const Idx base = nc - (Idx)1 - (two ? F2 : F1);

      typename P::inner_t inner[P::kInner ? NRHS : 1];
      if constexpr (P::kInner) {
#pragma unroll
        for (int j = 0; j < NRHS; ++j) P::izero(inner[j]);
      }
      for (int e = R.a_beg; e < R.a_end; ++e) {
        const FockAddition ad = a.add[e];
        const int s = ad.s, l = ad.l;
        Idx t;
        amp_t amp;
        if (two) {
          if (!MAPS) t = base - s_U[s * nt + tid] - s_V[l * nt + tid];
          amp = (s == l) ? s_d[s * nt + tid] : P::amul(s_c[s * nt + tid], s_b[l * nt + tid]);
        } else {
          if (!MAPS) t = base - s_U[l * nt + tid];
          amp = s_c[l * nt + tid];
        }
        if (valid) {
          if (MAPS) t = (Idx)__ldg(a.map + (size_t)(R.slot_base + ad.a_index) * (size_t)nc + g);
          const coef_t K = P::scale(__ldg(coef + e), amp);
          const vec_t *src = C + (size_t)t * nrhs;
#pragma unroll
          for (int j = 0; j < NRHS; ++j) {
            if (j < nrhs) {
              const vec_t v = __ldg(src + j);
              if constexpr (P::kInner) P::imac(inner[j], K, v, a.real);
              else P::mac(acc[j], K, v, a.real);
            }
          }
        }
      }
      if constexpr (P::kInner) {
#pragma unroll
        for (int j = 0; j < NRHS; ++j) P::flush(acc[j], inner[j]);
      }
    }
    if (live) {
      auto *out = (decltype(P::finish(acc[0], 1.0, false)) *)a.sigma + (size_t)g * nrhs;
#pragma unroll
      for (int j = 0; j < NRHS; ++j)
        if (j < nrhs) out[j] = P::finish(acc[j], out_scale, a.real);
    }
  }
}

// Launch with the occupancy-derived persistent grid.  Defined per policy in
// fock_apply_<policy>.cu through FOCK_INSTANTIATE_APPLY.
template <class Idx, int MAXM, class P, int NRHS, bool MAPS>
int fock_launch_list(const ApplyArgs<Idx> &a, int device, cudaStream_t stream) {
  auto kern = fock_apply_list_kernel<Idx, MAXM, P, NRHS, MAPS>;
  const int threads = FOCK_APPLY_THREADS;
  ApplySmem<Idx, MAXM, P> L(a.rows, a.xdim, a.nsq, threads);
  if (L.total > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return fock_cuda_status(e);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, L.total);
  if (e != cudaSuccess) return fock_cuda_status(e);
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t tiles = ((int64_t)a.nc + threads - 1) / threads;
  int64_t grid = (int64_t)per_sm * fock_get_sm_count(device);
  if (grid > tiles) grid = tiles;
  kern<<<(unsigned)grid, threads, L.total, stream>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}
