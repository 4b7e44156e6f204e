// fock_sector.cu -- configurations of one total orbital weight
//     Q = sum_i i n_i,
// with plane-wave orbitals (orbital i of momentum (i - floor(M/2)) 2 pi / L,
// Sec. 6) the sector of total momentum (Q - N floor(M/2)) 2 pi / L.  An
// operator with diagonal h and W_kqsl = 0 unless k + q = s + l (the
// Lieb-Liniger selection rule) maps a sector into itself, so its eigenproblem
// splits into sectors of about N_c / (N (M - 1) + 1) configurations or fewer.
//
// Order and hash.  The sector keeps the order of the full space (ascending
// lexicographic order of (n_{M-1}, ..., n_0), Algorithm 1), restricted to its
// members.  With D_m(s, q) the number of configurations of s particles in
// orbitals 0..m-1 of weight q (D_1(s, q) = [q = 0],
// D_{m+1}(s, q) = D_m(s, q) + D_{m+1}(s - 1, q - m)), the configurations that
// agree with n on orbitals m+1..M-1 and have fewer particles in orbital m
// number sum_{v < n_m} D_m(S_m - v, Q_m - m v) = D_{m+1}(S_m, Q_m) -
// D_{m+1}(S_{m-1}, Q_{m-1}), with the prefix sums S_m = sum_{i<=m} n_i and
// Q_m = sum_{i<=m} i n_i.  Summing over m and telescoping,
//     rank(n) = N_sec - 1 - sum_{m=1}^{M-2} T_m(S_m, Q_m),
//     T_m(s, q) = D_{m+2}(s, q) - D_{m+1}(s, q) = D_{m+2}(s - 1, q - m - 1),
// the weighted counterpart of the hash of Eq. TotalCost (with all weights zero
// T_m(s) = C(s + m, m + 1)).  Decoding walks m = M-1..1 and picks n_m as the
// largest c with D_{m+1}(S_m, Q_m) - D_{m+1}(S_m - c, Q_m - m c) <= the
// remaining index (a binary search; the count is monotone in c).
//
// Apply.  Pull form as in the full space: for each removal (k, q) valid in
// gamma and each addition (s, l) of its coefficient list the target is
// gamma - e_k - e_q + e_s + e_l, whose prefix sums differ from gamma's only
// for m in [min(k, s), max(q, l)); the target's rank is gamma minus the
// change of sum_m T_m over that range (one table read per orbital in it).
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "fock_apply_kernel.cuh"

struct fock_sector {
  const fock_space *sp;
  int N, M, Q;
  int64_t ns;                 // configurations in the sector
  int device;
  std::vector<uint64_t> D;    // host: D_m(s, q), m = 1..M, [m - 1][s][q]
  uint32_t *d_G;              // [M - 1][N + 1][Q + 1]: D_{m+1}(s, q) mod 2^32, m = 1..M-1
  uint32_t *d_T;              // [M - 2][N + 1][Q + 1]: T_m(s, q) mod 2^32, m = 1..M-2
  uint32_t *d_flag;
  void *ws;                   // workspace owned by the sector (callers passing none)
  size_t ws_bytes;
};

namespace {

constexpr int kSecThreads = 128;

static int check_dev(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  return cur == dev ? FOCK_OK : FOCK_ERR_DEVICE;
}

struct SecTables {
  const uint32_t *G, *T;
  int N, Q;
  __device__ __forceinline__ uint32_t g(int m, int s, int q) const {
    return __ldg(G + ((size_t)(m - 1) * (N + 1) + s) * (Q + 1) + q);
  }
  __device__ __forceinline__ uint32_t t(int m, int s, int q) const {
    return __ldg(T + ((size_t)(m - 1) * (N + 1) + s) * (Q + 1) + q);
  }
};

// Occupations of sector index r (r < N_sec).
template <int M>
__device__ __forceinline__ void sec_decode(uint32_t r, const SecTables &tb, int (&n)[M]) {
  int s = tb.N, q = tb.Q;
  uint32_t rem = r;
#pragma unroll
  for (int m = M - 1; m >= 1; --m) {
    const uint32_t top = tb.g(m, s, q);
    int lo = 0, hi = min(s, q / m);
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (top - tb.g(m, s - mid, q - m * mid) <= rem) lo = mid;
      else hi = mid - 1;
    }
    rem -= top - tb.g(m, s - lo, q - m * lo);
    n[m] = lo;
    s -= lo;
    q -= m * lo;
  }
  n[0] = s;
}

__global__ void sec_rank_kernel(SecTables tb, int M, uint32_t ns, const int32_t *__restrict__ occ,
                                int64_t count, int64_t *__restrict__ idx, uint32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *o = occ + i * M;
    bool ok = true;
    int S = 0, W = 0;
    for (int m = 0; m < M; ++m) {
      const int v = o[m];
      ok = ok && v >= 0 && v <= tb.N;
      if (ok) {
        S += v;
        W += m * v;
      }
      ok = ok && S <= tb.N && W <= tb.Q;
    }
    ok = ok && S == tb.N && W == tb.Q;
    if (!ok) {
      idx[i] = -1;
      atomicOr(flag, FOCK_DEVFLAG_INVALID);
      continue;
    }
    uint32_t acc = ns - 1u;
    S = o[0];
    W = 0;
    for (int m = 1; m <= M - 2; ++m) {
      S += o[m];
      W += m * o[m];
      acc -= tb.t(m, S, W);
    }
    idx[i] = (int64_t)acc;
  }
}

template <int M>
__global__ void sec_unrank_kernel(SecTables tb, uint32_t ns, const int64_t *__restrict__ idx, int64_t count,
                                  int32_t *__restrict__ occ, uint32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = idx[i];
    int32_t *o = occ + i * M;
    if (g < 0 || g >= (int64_t)ns) {
      for (int m = 0; m < M; ++m) o[m] = -1;
      atomicOr(flag, FOCK_DEVFLAG_RANGE);
      continue;
    }
    int n[M];
    sec_decode<M>((uint32_t)g, tb, n);
#pragma unroll
    for (int m = 0; m < M; ++m) o[m] = n[m];
  }
}

struct SecArgs {
  SecTables tb;
  uint32_t ns;
  int nsq, nrem, nadd, nrhs;
  bool real;
  const FockRemoval *rem;
  const FockAddition *add;
  const void *coef, *sq;
  const void *C;
  void *sigma;
  const int *in_exp;
  double out_scale;
};

// A term's prefix-sum change.  Removing (k, q) and adding (s, l) changes
// (S_m, Q_m) by a constant (dS, dQ) between consecutive positions of the
// sorted list {k, q, s, l}: at most three segments of orbitals, each with a
// constant offset dS (Q + 1) + dQ into a plane of the T table.  Computed once
// per block for every term, clamped to the orbitals 1..M-2 of the hash.
struct SecSeg {
  int8_t st[3], en[3];
  int16_t pad;
  int32_t off[3];
};

__device__ __forceinline__ SecSeg sec_segments(int k, int q, int s, int l, int M, int qd) {
  int p[4] = {k, q, s, l}, d[4] = {-1, -1, 1, 1};
  const int np = q < 0 ? 2 : 4;
  if (q < 0) {                                         // one-body: remove k, add l
    p[1] = l;
    d[1] = 1;
  }
  for (int i = 1; i < np; ++i)                         // insertion sort of the positions
    for (int j = i; j > 0 && p[j - 1] > p[j]; --j) {
      const int tp = p[j], td = d[j];
      p[j] = p[j - 1];
      d[j] = d[j - 1];
      p[j - 1] = tp;
      d[j - 1] = td;
    }
  SecSeg g;
  g.pad = 0;
  int dS = 0, dQ = 0;
  for (int i = 0; i < 3; ++i) {
    int a = 0, b = 0;
    if (i < np - 1) {
      dS += d[i];
      dQ += p[i] * d[i];
      a = max(p[i], 1);
      b = min(p[i + 1], M - 1);
    }
    g.st[i] = (int8_t)a;
    g.en[i] = (int8_t)(b > a ? b : a);
    g.off[i] = dS * qd + dQ;
  }
  return g;
}

// Shared-memory layout of the sector kernel, every section 16-byte aligned.
struct SecSmem {
  size_t coef, it, seg, sq, rem, add, n, total;
  __host__ __device__ SecSmem(int M, int nadd, int nsq, int nrem, size_t coef_bytes, size_t amp_bytes) {
    size_t o = 0;
    coef = o; o = fock_align16(o + coef_bytes * nadd);
    it = o;   o = fock_align16(o + 8 * (size_t)M * kSecThreads);
    seg = o;  o = fock_align16(o + sizeof(SecSeg) * nadd);
    sq = o;   o = fock_align16(o + amp_bytes * nsq);
    rem = o;  o = fock_align16(o + sizeof(FockRemoval) * nrem);
    add = o;  o = fock_align16(o + sizeof(FockAddition) * nadd);
    n = o;    o = fock_align16(o + 4 * (size_t)M * kSecThreads);
    total = o;
  }
};

// One thread per sector configuration.  Per orbital m the thread keeps, in a
// shared-memory column, the flat index of T_m(S_m, Q_m) and its value; a
// target's rank is gamma minus sum over the term's segments of
// T[index_m + offset] - T_m(S_m, Q_m).  Occupations sit in another column
// (runtime orbital indices, no local-memory arrays).  The term lists and
// segments, coefficients and square roots are staged once per block.
template <int M, class P>
__global__ void __launch_bounds__(kSecThreads) fock_sector_apply_kernel(const SecArgs a) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  using vec_t = typename P::vec_t;
  extern __shared__ __align__(16) unsigned char smem[];
  const SecSmem L(M, a.nadd, a.nsq, a.nrem, sizeof(coef_t), sizeof(amp_t));
  coef_t *s_coef = (coef_t *)(smem + L.coef);                        // [nadd]
  int2 *s_it = (int2 *)(smem + L.it);                                // [M][threads]: (T index, T value)
  SecSeg *s_seg = (SecSeg *)(smem + L.seg);                          // [nadd]
  amp_t *s_sq = (amp_t *)(smem + L.sq);                              // [nsq]
  FockRemoval *s_rem = (FockRemoval *)(smem + L.rem);                // [nrem]
  FockAddition *s_add = (FockAddition *)(smem + L.add);              // [nadd]
  int *s_n = (int *)(smem + L.n);                                    // [M][threads]
  const int qd = a.tb.Q + 1;
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const amp_t *)a.sq)[i];
  for (int i = threadIdx.x; i < a.nrem; i += blockDim.x) s_rem[i] = a.rem[i];
  __syncthreads();
  for (int r = 0; r < a.nrem; ++r) {
    const FockRemoval R = s_rem[r];
    for (int i = R.a_beg + threadIdx.x; i < R.a_end; i += blockDim.x) {
      const FockAddition ad = a.add[i];
      s_coef[i] = ((const coef_t *)a.coef)[i];
      s_add[i] = ad;
      s_seg[i] = R.size == 2 ? sec_segments(R.k, R.q, ad.s, ad.l, M, qd) : sec_segments(R.k, -1, -1, ad.l, M, qd);
    }
  }
  __syncthreads();
  const int tid = threadIdx.x;
  double out_scale = a.out_scale;
  if (a.in_exp) out_scale *= fock_pow2(__ldg(a.in_exp));
  const vec_t *__restrict__ C = (const vec_t *)a.C;
  const uint32_t *__restrict__ T = a.tb.T;
  const int nrhs = a.nrhs;

  for (uint32_t g = blockIdx.x * blockDim.x + tid; g < a.ns; g += gridDim.x * blockDim.x) {
    {
      int n[M];
      sec_decode<M>(g, a.tb, n);
      int S = 0, W = 0;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        S += n[m];
        W += m * n[m];
        s_n[m * kSecThreads + tid] = n[m];
        if (m >= 1 && m <= M - 2) {
          const int idx = ((m - 1) * (a.tb.N + 1) + S) * qd + W;
          s_it[m * kSecThreads + tid] = make_int2(idx, (int)__ldg(T + idx));
        }
      }
    }
    for (int j = 0; j < nrhs; ++j) {
      typename P::acc_t acc;
      P::zero(acc);
      for (int ri = 0; ri < a.nrem; ++ri) {
        const FockRemoval R = s_rem[ri];
        const int k = R.k, q = R.q;
        const bool two = R.size == 2;
        const int nk = s_n[k * kSecThreads + tid];
        const int nq = two ? s_n[q * kSecThreads + tid] : 0;
        const bool valid = two ? (k == q ? nk >= 2 : (nk >= 1 && nq >= 1)) : nk >= 1;
        if (!valid) continue;
        // removal amplitude sqrt(n_k (n_q - delta_kq)) (sqrt(n_k) for one particle)
        amp_t A = s_sq[nk];
        if (two) A = P::amul(A, s_sq[nq - (k == q)]);
        typename P::inner_t inner;
        if constexpr (P::kInner) P::izero(inner);
        for (int e = R.a_beg; e < R.a_end; ++e) {
          const FockAddition ad = s_add[e];
          const int l = ad.l;
          // occupations after the removal, then the addition amplitude
          const int nl = s_n[l * kSecThreads + tid] - (l == k) - (two && l == q);
          amp_t amp;
          if (two) {
            const int s = ad.s;
            const int ns_ = s_n[s * kSecThreads + tid] - (s == k) - (s == q);
            amp = P::amul(P::amul(A, s_sq[ns_ + 1]), s_sq[nl + 1 + (s == l)]);
          } else {
            amp = P::amul(A, s_sq[nl + 1]);
          }
          // target rank: gamma minus the change of sum_m T_m over the segments
          const SecSeg sg = s_seg[e];
          uint32_t diff = 0;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const int off = sg.off[i];
            for (int m = sg.st[i]; m < sg.en[i]; ++m) {
              const int2 it = s_it[m * kSecThreads + tid];
              diff += __ldg(T + (it.x + off)) - (uint32_t)it.y;
            }
          }
          const uint32_t t = g - diff;
          const coef_t K = P::scale(s_coef[e], amp);
          const vec_t v = __ldg(C + (size_t)t * nrhs + j);
          if constexpr (P::kInner) P::imac(inner, K, v, a.real);
          else P::mac(acc, K, v, a.real);
        }
        if constexpr (P::kInner) P::flush(acc, inner, a.real);
      }
      auto *out = (decltype(P::finish(acc, 1.0, false)) *)a.sigma;
      out[(size_t)g * nrhs + j] = P::finish(acc, out_scale, a.real);
    }
  }
}

template <int M, class P>
int launch_sector_m(const SecArgs &a, int device, cudaStream_t s) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  const size_t smem = SecSmem(M, a.nadd, a.nsq, a.nrem, sizeof(coef_t), sizeof(amp_t)).total;
  auto kern = fock_sector_apply_kernel<M, P>;
  if (smem > 48 * 1024) FOCK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FOCK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSecThreads, smem));
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t blocks = ((int64_t)a.ns + kSecThreads - 1) / kSecThreads;
  const int64_t cap = (int64_t)per_sm * fock_get_sm_count(device);
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)(blocks < 1 ? 1 : blocks), kSecThreads, smem, s>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

template <class P>
int launch_sector(const SecArgs &a, int M, int device, cudaStream_t s) {
  switch (M) {
#define FOCK_SEC_CASE(MM) \
    case MM: return launch_sector_m<MM, P>(a, device, s);
    FOCK_SEC_CASE(1)
    FOCK_SEC_CASE(2)
    FOCK_SEC_CASE(3)
    FOCK_SEC_CASE(4)
    FOCK_SEC_CASE(5)
    FOCK_SEC_CASE(6)
    FOCK_SEC_CASE(7)
    FOCK_SEC_CASE(8)
    FOCK_SEC_CASE(9)
    FOCK_SEC_CASE(10)
    FOCK_SEC_CASE(11)
    FOCK_SEC_CASE(12)
#undef FOCK_SEC_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}

template <int M>
void launch_unrank_m(const SecTables &tb, uint32_t ns, const int64_t *idx, int64_t count, int32_t *occ,
                     uint32_t *flag, unsigned grid, cudaStream_t s) {
  sec_unrank_kernel<M><<<grid, 256, 0, s>>>(tb, ns, idx, count, occ, flag);
}

static unsigned grid_for(int64_t count, int device) {
  int64_t blocks = (count + 255) / 256;
  const int64_t cap = (int64_t)fock_get_sm_count(device) * 16;
  if (blocks > cap) blocks = cap;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

static int finish_checked(const fock_sector *sec, cudaStream_t st, uint32_t mask, int err) {
  uint32_t flag = 0;
  FOCK_CUDA_TRY(cudaGetLastError());
  FOCK_CUDA_TRY(cudaMemcpyAsync(&flag, sec->d_flag, 4, cudaMemcpyDeviceToHost, st));
  FOCK_CUDA_TRY(cudaStreamSynchronize(st));
  return (flag & mask) ? err : FOCK_OK;
}

static void free_sector(fock_sector *sec) {
  if (!sec) return;
  cudaFree(sec->d_G);
  cudaFree(sec->d_T);
  cudaFree(sec->d_flag);
  cudaFree(sec->ws);
  delete sec;
}

// Every term of the operator keeps the total weight: removal weight k + q (k
// for one particle) equals addition weight s + l (l).
static bool conserves(const fock_ham *ham) {
  for (int r = 0; r < ham->nrem; ++r) {
    const FockRemoval &e = ham->h_rem[r];
    const int wr = e.size == 2 ? e.k + e.q : e.k;
    for (int i = e.a_beg; i < e.a_end; ++i) {
      const FockAddition &d = ham->h_add[i];
      const int wa = e.size == 2 ? d.s + d.l : d.l;
      if (wa != wr) return false;
    }
  }
  return true;
}

static uint64_t host_D(const fock_sector *sec, int m, int s, int q) {
  if (m < 1 || s < 0 || q < 0 || s > sec->N || q > sec->Q) return 0;
  return sec->D[((size_t)(m - 1) * (sec->N + 1) + s) * (sec->Q + 1) + q];
}

static size_t sector_ws_bytes(const fock_sector *sec, int nrhs, int precision) {
  if (precision != FOCK_PREC_F64) return 0;
  return FOCK_WS_HEADER + (size_t)sec->ns * (size_t)nrhs * sizeof(float4);
}

}  // namespace

static int fock_sector_apply_internal(const fock_sector *sec, const fock_ham *ham, const void *C, void *sigma, int nrhs,
                               int precision, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (sec->ns == 0) return FOCK_OK;
  const size_t elem = precision == FOCK_PREC_F32_MIXED ? 8 : 16;
  const size_t bytes = (size_t)sec->ns * (size_t)nrhs * elem;
  const char *c0 = (const char *)C, *s0 = (const char *)sigma;
  if (c0 < s0 + bytes && s0 < c0 + bytes) return FOCK_ERR_ALIAS;
  if (ham->nrem == 0) {
    FOCK_CUDA_TRY(cudaMemsetAsync(sigma, 0, bytes, stream));
    return FOCK_OK;
  }
  SecArgs a;
  a.tb.G = sec->d_G;
  a.tb.T = sec->d_T;
  a.tb.N = sec->N;
  a.tb.Q = sec->Q;
  a.ns = (uint32_t)sec->ns;
  a.nsq = sec->N + 4;
  a.nrem = ham->nrem;
  a.nadd = ham->nadd;
  a.nrhs = nrhs;
  a.real = ham->real;
  a.rem = ham->d_rem;
  a.add = ham->d_add;
  a.C = C;
  a.sigma = sigma;
  a.in_exp = nullptr;
  const int M = sec->M;
  if (precision == FOCK_PREC_F64) {
    if (!ws || ws_bytes < sector_ws_bytes(sec, nrhs, precision)) return FOCK_ERR_ARG;
    const int st = fock_prepare_df(C, sec->ns * (int64_t)nrhs, ws, sec->device, stream);
    if (st) return st;
    a.C = (const char *)ws + FOCK_WS_HEADER;
    a.in_exp = (const int *)ws + 1;
  }
  // the caller's events (fock_apply_set_events) bracket the main kernel
  if (ham->ev_start) FOCK_CUDA_TRY(cudaEventRecord(ham->ev_start, stream));
  int st;
  switch (precision) {
    case FOCK_PREC_F64:
      a.coef = ham->d_coefdf;
      a.sq = ham->d_sqrtdf;
      a.out_scale = ham->coef_scale;
      st = launch_sector<PolDFP>(a, M, sec->device, stream);
      break;
    case FOCK_PREC_F64_NATIVE:
      a.coef = ham->d_coef64;
      a.sq = ham->d_sqrt64;
      a.out_scale = 1.0;
      st = launch_sector<PolF64>(a, M, sec->device, stream);
      break;
    default:
      a.coef = ham->d_coef32;
      a.sq = ham->d_sqrt32;
      a.out_scale = 1.0;
      st = launch_sector<PolMixedP>(a, M, sec->device, stream);
      break;
  }
  if (st == FOCK_OK && ham->ev_stop) FOCK_CUDA_TRY(cudaEventRecord(ham->ev_stop, stream));
  return st;
}

static int sector_create(const fock_space *sp, int64_t Q, fock_sector **out);

// The counting tables grow as M (N + 1) (Q + 1); beyond 2^28 entries (2 GB on
// the host) the call returns FOCK_ERR_UNSUPPORTED, and a host allocation that
// fails below that returns FOCK_ERR_NOMEM (no C++ exception crosses the ABI).
extern "C" int fock_sector_create(const fock_space *sp, int64_t Q, fock_sector **out) {
  if (!sp || !out) return FOCK_ERR_ARG;
  int st = check_dev(sp->device);
  if (st) return st;
  const int N = sp->N, M = sp->M;
  if (Q < 0 || Q > (int64_t)N * (M - 1)) return FOCK_ERR_ARG;
  if ((double)M * (N + 1) * ((double)Q + 1) > (double)(1u << 28)) return FOCK_ERR_UNSUPPORTED;
  try {
    return sector_create(sp, Q, out);
  } catch (const std::bad_alloc &) {
    return FOCK_ERR_NOMEM;
  }
}

static int sector_create(const fock_space *sp, int64_t Q, fock_sector **out) {
  int st = FOCK_OK;
  const int N = sp->N, M = sp->M;
  fock_sector *sec = new fock_sector();
  sec->sp = sp;
  sec->N = N;
  sec->M = M;
  sec->Q = (int)Q;
  sec->device = sp->device;
  const size_t plane = (size_t)(N + 1) * (Q + 1);
  sec->D.assign((size_t)M * plane, 0);
  // D_1(s, q) = [q = 0]; D_{m+1}(s, q) = D_m(s, q) + D_{m+1}(s - 1, q - m)
  for (int s = 0; s <= N; ++s) sec->D[(size_t)s * (Q + 1)] = 1;
  for (int m = 1; m < M; ++m)
    for (int s = 0; s <= N; ++s)
      for (int q = 0; q <= Q; ++q) {
        uint64_t v = sec->D[((size_t)(m - 1) * (N + 1) + s) * (Q + 1) + q];
        if (s >= 1 && q >= m) v += sec->D[((size_t)m * (N + 1) + s - 1) * (Q + 1) + q - m];
        sec->D[((size_t)m * (N + 1) + s) * (Q + 1) + q] = v;   // counts <= N_c(N, M) < 2^63
      }
  sec->ns = (int64_t)host_D(sec, M, N, (int)Q);
  if (sec->ns >= ((int64_t)1 << 31)) {
    free_sector(sec);
    return FOCK_ERR_OVERFLOW;
  }
  std::vector<uint32_t> G((size_t)(M > 1 ? M - 1 : 1) * plane, 0u), T((size_t)(M > 2 ? M - 2 : 1) * plane, 0u);
  for (int m = 1; m <= M - 1; ++m)
    for (int s = 0; s <= N; ++s)
      for (int q = 0; q <= Q; ++q) G[((size_t)(m - 1) * (N + 1) + s) * (Q + 1) + q] = (uint32_t)host_D(sec, m + 1, s, q);
  for (int m = 1; m <= M - 2; ++m)
    for (int s = 0; s <= N; ++s)
      for (int q = 0; q <= Q; ++q)
        T[((size_t)(m - 1) * (N + 1) + s) * (Q + 1) + q] = (uint32_t)host_D(sec, m + 2, s - 1, q - m - 1);
  auto upload = [](uint32_t **dst, const std::vector<uint32_t> &v) -> int {
    if (cudaMalloc(dst, v.size() * 4) != cudaSuccess) return FOCK_ERR_NOMEM;
    return cudaMemcpy(*dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
  };
  st = upload(&sec->d_G, G);
  if (!st) st = upload(&sec->d_T, T);
  if (!st) st = cudaMalloc(&sec->d_flag, 4) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM;
  if (st) {
    free_sector(sec);
    return st;
  }
  *out = sec;
  return FOCK_OK;
}

extern "C" int fock_sector_destroy(fock_sector *sec) {
  free_sector(sec);
  return FOCK_OK;
}

extern "C" int fock_sector_size(const fock_sector *sec, int64_t *ns) {
  if (!sec || !ns) return FOCK_ERR_ARG;
  *ns = sec->ns;
  return FOCK_OK;
}

extern "C" int fock_sector_rank(const fock_sector *sec, const int32_t *occ_dev, int64_t count, int64_t *idx_dev,
                                void *stream) {
  if (!sec || count < 0 || (count > 0 && (!occ_dev || !idx_dev))) return FOCK_ERR_ARG;
  int st = check_dev(sec->device);
  if (st) return st;
  if (count == 0) return FOCK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  FOCK_CUDA_TRY(cudaMemsetAsync(sec->d_flag, 0, 4, s));
  SecTables tb{sec->d_G, sec->d_T, sec->N, sec->Q};
  sec_rank_kernel<<<grid_for(count, sec->device), 256, 0, s>>>(tb, sec->M, (uint32_t)sec->ns, occ_dev, count,
                                                                 idx_dev, sec->d_flag);
  return finish_checked(sec, s, FOCK_DEVFLAG_INVALID, FOCK_ERR_INVALID_CONFIG);
}

extern "C" int fock_sector_unrank(const fock_sector *sec, const int64_t *idx_dev, int64_t count, int32_t *occ_dev,
                                  void *stream) {
  if (!sec || count < 0 || (count > 0 && (!occ_dev || !idx_dev))) return FOCK_ERR_ARG;
  int st = check_dev(sec->device);
  if (st) return st;
  if (count == 0) return FOCK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  FOCK_CUDA_TRY(cudaMemsetAsync(sec->d_flag, 0, 4, s));
  SecTables tb{sec->d_G, sec->d_T, sec->N, sec->Q};
  const unsigned grid = grid_for(count, sec->device);
  const uint32_t ns = (uint32_t)sec->ns;
  switch (sec->M) {
#define FOCK_SEC_UNRANK(MM) \
    case MM: launch_unrank_m<MM>(tb, ns, idx_dev, count, occ_dev, sec->d_flag, grid, s); break;
    FOCK_SEC_UNRANK(1)
    FOCK_SEC_UNRANK(2)
    FOCK_SEC_UNRANK(3)
    FOCK_SEC_UNRANK(4)
    FOCK_SEC_UNRANK(5)
    FOCK_SEC_UNRANK(6)
    FOCK_SEC_UNRANK(7)
    FOCK_SEC_UNRANK(8)
    FOCK_SEC_UNRANK(9)
    FOCK_SEC_UNRANK(10)
    FOCK_SEC_UNRANK(11)
    FOCK_SEC_UNRANK(12)
#undef FOCK_SEC_UNRANK
    default: return FOCK_ERR_UNSUPPORTED;
  }
  return finish_checked(sec, s, FOCK_DEVFLAG_RANGE, FOCK_ERR_RANGE);
}

extern "C" int fock_sector_terms(const fock_sector *sec, const fock_ham *ham, int64_t *terms) {
  if (!sec || !ham || !terms || ham->sp != sec->sp) return FOCK_ERR_ARG;
  if (!conserves(ham)) return FOCK_ERR_NOT_CONSERVING;
  // a removal (k, q) is valid in exactly the sector configurations of the
  // (N - 2)-particle sector of weight Q - k - q with (k, q) added back
  int64_t t = 0;
  for (int r = 0; r < ham->nrem; ++r) {
    const FockRemoval &e = ham->h_rem[r];
    const int wr = e.size == 2 ? e.k + e.q : e.k;
    t += (int64_t)(e.a_end - e.a_beg) * (int64_t)host_D(sec, sec->M, sec->N - e.size, sec->Q - wr);
  }
  *terms = t;
  return FOCK_OK;
}

extern "C" int fock_sector_workspace_size(const fock_sector *sec, int32_t nrhs, int precision, size_t *bytes) {
  if (!sec || !bytes || nrhs < 1 || nrhs > FOCK_MAX_NRHS) return FOCK_ERR_ARG;
  if (precision < FOCK_PREC_F64 || precision > FOCK_PREC_F32_MIXED) return FOCK_ERR_ARG;
  *bytes = sector_ws_bytes(sec, nrhs, precision);
  return FOCK_OK;
}

extern "C" int fock_sector_apply_H(const fock_sector *sec, const fock_ham *ham, const void *C_dev, void *sigma_dev,
                                   int32_t nrhs, int precision, void *workspace_dev, size_t workspace_bytes,
                                   void *stream) {
  if (!sec || !ham || ham->sp != sec->sp || nrhs < 1 || nrhs > FOCK_MAX_NRHS) return FOCK_ERR_ARG;
  if (precision < FOCK_PREC_F64 || precision > FOCK_PREC_F32_MIXED) return FOCK_ERR_ARG;
  if (sec->ns > 0 && (!C_dev || !sigma_dev)) return FOCK_ERR_ARG;
  int st = check_dev(sec->device);
  if (st) return st;
  if (!conserves(ham)) return FOCK_ERR_NOT_CONSERVING;
  void *ws = workspace_dev;
  size_t wsb = workspace_bytes;
  const size_t need = sector_ws_bytes(sec, nrhs, precision);
  if (need && (!ws || wsb < need)) {
    fock_sector *mut = (fock_sector *)sec;
    if (mut->ws_bytes < need) {
      cudaFree(mut->ws);
      mut->ws = nullptr;
      mut->ws_bytes = 0;
      FOCK_CUDA_TRY(cudaMalloc(&mut->ws, need));
      mut->ws_bytes = need;
    }
    ws = mut->ws;
    wsb = mut->ws_bytes;
  }
  return fock_sector_apply_internal(sec, ham, C_dev, sigma_dev, nrhs, precision, ws, wsb, (cudaStream_t)stream);
}

extern "C" int fock_sector_lanczos_ground(const fock_sector *sec, const fock_ham *ham, int32_t max_iter,
                                          int32_t restart_len, double tol, uint64_t seed, int precision,
                                          const void *start_dev, double *E0, double *residual, void *vec_dev,
                                          int32_t *iters, void *stream) {
  if (!sec || !ham || ham->sp != sec->sp) return FOCK_ERR_ARG;
  int st = check_dev(sec->device);
  if (st) return st;
  if (!conserves(ham)) return FOCK_ERR_NOT_CONSERVING;
  if (sec->ns == 0) return FOCK_ERR_ARG;
  const size_t wsb = sector_ws_bytes(sec, 1, FOCK_PREC_F64);
  FockApplyFn apply = [sec, ham](int prec, const void *x, void *y, void *ws, size_t ws_bytes, cudaStream_t s) {
    return fock_sector_apply_internal(sec, ham, x, y, 1, prec, ws, ws_bytes, s);
  };
  return fock_lanczos_run(sec->ns, ham->real, sec->device, apply, wsb, wsb, max_iter, restart_len, tol, seed,
                          precision, start_dev, E0, residual, vec_dev, iters, (cudaStream_t)stream);
}
