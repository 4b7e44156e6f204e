// fock_apply_nn.cu -- sigma = H C for nearest-neighbour operators: h_kl = 0
// unless l = k or l, k are neighbouring sites (a chain, or a ring when the
// corner h_{0,M-1} is present), and W only on-site (W_kkkk), the Bose-Hubbard
// class.  Each configuration has the diagonal
//     sum_k h_kk n_k + (1/2) sum_k W_kkkk n_k (n_k - 1)
// and two hops per bond (k, l): h_kl sqrt(n_k (n_l + 1)) C[gamma - e_k + e_l]
// and h_lk sqrt(n_l (n_k + 1)) C[gamma - e_l + e_k] (pull form of Eq. Haction).
// Moving a particle across a chain bond (m, m + 1) changes only the prefix
// sum S_m, by -1 (m -> m + 1) or +1 (m + 1 -> m), so the target is gamma minus
// one difference of the table C(S_m + m, m + 1); across the ring bond
// (M - 1, 0) every S_m with m < M - 1 changes, and the target offset is the
// sum of those differences.  O(M) terms and table reads per configuration.
// The site energies E_k(n) and, for the native FP64 policy with N < 32, the
// hop amplitudes sqrt(a (b + 1)) are host-built tables staged in shared
// memory with the hash tables.
#include <type_traits>

#include "fock_apply_kernel.cuh"

namespace {

constexpr int kNNThreads = 128;
constexpr int kNNMinBlocks = 8;   // 32 warps per SM (64 registers) to hide the gather latency

// Real amplitudes of the three policies: double, float, or an FP32 pair.
__device__ __forceinline__ double nn_add(double a, double b) { return a + b; }
__device__ __forceinline__ float nn_add(float a, float b) { return a + b; }
__device__ __forceinline__ float2 nn_add(float2 a, float2 b) {
  float h = a.x, l = a.y;
  df_add_acc(h, l, b.x, b.y);
  return make_float2(h, l);
}
// a real amplitude as the policy's complex coefficient
__device__ __forceinline__ double2 nn_real_coef(double d) { return make_double2(d, 0.0); }
__device__ __forceinline__ float2 nn_real_coef(float d) { return make_float2(d, 0.f); }
__device__ __forceinline__ float4 nn_real_coef(float2 d) { return make_float4(d.x, 0.f, d.y, 0.f); }

// Two terms added to the accumulator; the policies with an FP32 inner sum
// (FP32-mixed) add both there and fold the sum into the FP32 pair once.
template <class P>
__device__ __forceinline__ void nn_mac2(typename P::acc_t &acc, typename P::coef_t k1, typename P::vec_t v1,
                                        typename P::coef_t k2, typename P::vec_t v2, bool real) {
  if constexpr (P::kInner) {
    typename P::inner_t in;
    P::izero(in);
    P::imac(in, k1, v1, real);
    P::imac(in, k2, v2, real);
    P::flush(acc, in, real);
  } else {
    P::mac(acc, k1, v1, real);
    P::mac(acc, k2, v2, real);
  }
}

template <class P>
__device__ __forceinline__ void nn_mac1(typename P::acc_t &acc, typename P::coef_t k, typename P::vec_t v,
                                        bool real) {
  if constexpr (P::kInner) {
    typename P::inner_t in;
    P::izero(in);
    P::imac(in, k, v, real);
    P::flush(acc, in, real);
  } else {
    P::mac(acc, k, v, real);
  }
}

// Output of one configuration.  The FP32-pair policy converts with integer
// operations (FP64 instructions run at about 1/74 of the FP32 rate); the
// others use their own conversion.
template <class P>
__device__ __forceinline__ auto nn_finish(const typename P::acc_t &acc, double out_scale, int e_out, bool real) {
  if constexpr (std::is_same<P, PolDFP>::value) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    df_add_acc(rh, rl, fp2_x(acc.h1), fp2_x(acc.l1));
    if (real) {
      df_add_acc(ih, il, fp2_y(acc.h1), fp2_y(acc.l1));
    } else {
      df_add_acc(rh, rl, -fp2_y(acc.h1), -fp2_y(acc.l1));
      df_add_acc(ih, il, fp2_x(acc.h2), fp2_x(acc.l2));
      df_add_acc(ih, il, fp2_y(acc.h2), fp2_y(acc.l2));
    }
    return make_double2(df_to_double_bits(rh, rl, e_out), df_to_double_bits(ih, il, e_out));
  } else {
    return P::finish(acc, out_scale, real);
  }
}

struct NNArgs {
  ApplyArgs<uint32_t> a;      // sizes, tables, C, sigma, nrhs, scales
  const void *bond;           // [2 * nb] policy coef_t: h_kl, h_lk of bond b = (k, k + 1 mod M)
  const void *etab;           // [M][N + 1] policy amp_t: E_k(n) = h_kk n + W_kkkk n (n - 1) / 2
  const void *ttab;           // [N + 1][N + 1] policy amp_t: sqrt(a (b + 1)), or null
  int nb;                     // bonds: M - 1, or M for a ring (M > 2)
  uint32_t g_begin, g_end;    // configurations computed
};

// TT: hop amplitudes sqrt(n_k (n_l + 1)) from the (N + 1)^2 table (one
// rounding, one read) rather than the product of two square roots.
template <int M, class P, bool TT>
__global__ void __launch_bounds__(kNNThreads, kNNMinBlocks) fock_apply_nn(const NNArgs t) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  using vec_t = typename P::vec_t;
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const int rows = M > 1 ? M - 1 : 1, xs = a.xdim + 2, np1 = a.N + 1;
  const int namp = TT ? np1 * np1 : a.nsq;
  coef_t *s_bond = (coef_t *)smem;                                   // [2 nb]
  amp_t *s_E = (amp_t *)(s_bond + 2 * M);                            // [M][N + 1]
  amp_t *s_A = s_E + M * np1;                                        // T table, or sqrt(i)
  uint32_t *s_mod = (uint32_t *)(s_A + namp + 1);                    // rows of xs (two leading zeros)
  uint32_t *s_sat = s_mod + rows * xs;
  for (int i = threadIdx.x; i < 2 * t.nb; i += blockDim.x) s_bond[i] = ((const coef_t *)t.bond)[i];
  for (int i = threadIdx.x; i < M * np1; i += blockDim.x) s_E[i] = ((const amp_t *)t.etab)[i];
  for (int i = threadIdx.x; i < namp; i += blockDim.x) s_A[i] = ((const amp_t *)(TT ? t.ttab : a.sq))[i];
  for (int i = threadIdx.x; i < rows * xs; i += blockDim.x) {
    const int m = i / xs, x = i - m * xs;
    s_mod[i] = x < 2 ? 0u : a.mod[m * a.xdim + x - 2];
  }
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) s_sat[i] = a.sat[i];
  __syncthreads();
  double out_scale = a.out_scale;
  int e_out = (int)(((unsigned long long)__double_as_longlong(a.out_scale) >> 52) & 0x7ff) - 1023;
  if (a.in_exp) {
    const int ein = __ldg(a.in_exp);
    out_scale *= fock_pow2(ein);
    e_out += ein;
  }
  const vec_t *__restrict__ C = (const vec_t *)a.C;
  const uint32_t nc = a.nc;
  const int nrhs = a.nrhs;
  const bool real = a.real != 0;
  const bool ring = t.nb == M && M > 2;
  // sqrt(n_k (n_l + 1)) for a hop k -> l
  auto amp = [&](int nk, int nl) -> amp_t {
    if constexpr (TT) return s_A[nk * np1 + nl];
    else return P::amul(s_A[nk], s_A[nl + 1]);
  };

  for (uint32_t g = t.g_begin + blockIdx.x * blockDim.x + threadIdx.x; g < t.g_end; g += gridDim.x * blockDim.x) {
    int S[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
    // diagonal: sum_k E_k(n_k), a real amplitude
    amp_t dg = s_E[S[0]];
#pragma unroll
    for (int m = 1; m < M; ++m) dg = nn_add(dg, s_E[m * np1 + S[m] - S[m - 1]]);
    for (int j = 0; j < nrhs; ++j) {
      typename P::acc_t acc;
      P::zero(acc);
      // the accumulator layout of the FP32-pair policy follows the operator's
      // real flag, so the (real) diagonal goes in with the same flag
      nn_mac1<P>(acc, nn_real_coef(dg), __ldg(C + (size_t)g * nrhs + j), real);
      // chain bonds (m, m + 1): moving a particle across the bond changes only
      // S_m, so each target is one table difference away from gamma
      uint32_t fm = 0, fp = 0;
#pragma unroll
      for (int m = 0; m < M - 1; ++m) {
        const int nk = S[m] - (m > 0 ? S[m - 1] : 0), nl = S[m + 1] - S[m];
        const uint32_t *row = s_mod + m * xs + (S[m] + m + 2);
        const uint32_t c0 = row[0], dm = row[-1] - c0, dp = row[1] - c0;
        fm += dm;
        fp += dp;
        const uint32_t tkl = nk > 0 ? g - dm : g;        // particle m -> m + 1, h_{m,m+1}
        const uint32_t tlk = nl > 0 ? g - dp : g;        // particle m + 1 -> m, h_{m+1,m}
        const coef_t Kkl = P::scale(s_bond[2 * m], amp(nk, nl));
        const coef_t Klk = P::scale(s_bond[2 * m + 1], amp(nl, nk));
        nn_mac2<P>(acc, Kkl, __ldg(C + (size_t)tkl * nrhs + j), Klk, __ldg(C + (size_t)tlk * nrhs + j), real);
      }
      if (ring) {
        // bond (M - 1, 0): S_0 .. S_{M-2} all change, by +1 (particle M-1 -> 0)
        // or by -1 (particle 0 -> M-1): the summed differences
        const int nk = S[M - 1] - S[M - 2], nl = S[0];
        const uint32_t tkl = nk > 0 ? g - fp : g;
        const uint32_t tlk = nl > 0 ? g - fm : g;
        const coef_t Kkl = P::scale(s_bond[2 * (M - 1)], amp(nk, nl));
        const coef_t Klk = P::scale(s_bond[2 * (M - 1) + 1], amp(nl, nk));
        nn_mac2<P>(acc, Kkl, __ldg(C + (size_t)tkl * nrhs + j), Klk, __ldg(C + (size_t)tlk * nrhs + j), real);
      }
      auto *out = (decltype(nn_finish<P>(acc, 1.0, 0, real)) *)a.sigma;
      out[(size_t)g * nrhs + j] = nn_finish<P>(acc, out_scale, e_out, real);
    }
  }
}

template <int M, class P, bool TT>
int launch_nn_m(const NNArgs &t, int device, cudaStream_t s) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  const ApplyArgs<uint32_t> &a = t.a;
  const int rows = M > 1 ? M - 1 : 1;
  const size_t np1 = (size_t)a.N + 1, namp = TT ? np1 * np1 : (size_t)a.nsq;
  const size_t smem = sizeof(coef_t) * 2 * M + sizeof(amp_t) * (M * np1 + namp + 1) +
                      4 * (size_t)rows * (a.xdim + 2) + 4 * (size_t)rows * a.xdim + 16;
  auto kern = fock_apply_nn<M, P, TT>;
  if (smem > 48 * 1024) FOCK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FOCK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNNThreads, smem));
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t blocks = ((int64_t)(t.g_end - t.g_begin) + kNNThreads - 1) / kNNThreads;
  const int64_t cap = (int64_t)per_sm * fock_get_sm_count(device);
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)(blocks < 1 ? 1 : blocks), kNNThreads, smem, s>>>(t);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

template <class P, bool TT>
int launch_nn(const NNArgs &t, int device, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_NN_CASE(MM) \
    case MM: return launch_nn_m<MM, P, TT>(t, device, s);
    FOCK_NN_CASE(2)
    FOCK_NN_CASE(3)
    FOCK_NN_CASE(4)
    FOCK_NN_CASE(5)
    FOCK_NN_CASE(6)
    FOCK_NN_CASE(7)
    FOCK_NN_CASE(8)
    FOCK_NN_CASE(9)
    FOCK_NN_CASE(10)
    FOCK_NN_CASE(11)
    FOCK_NN_CASE(12)
#undef FOCK_NN_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}

// The amplitude table pays for the native FP64 policy (one FP64 multiply
// fewer per hop); for the FP32 policies it measured slower (more registers).
template <class P>
int launch_nn_p(const NNArgs &t, int device, cudaStream_t s) {
  if constexpr (std::is_same<P, PolF64>::value) {
    if (t.ttab) return launch_nn<P, true>(t, device, s);
  }
  return launch_nn<P, false>(t, device, s);
}

}  // namespace

// Launch for one of the precisions over configurations [g_begin, g_end); bond,
// etab and ttab hold that precision's arrays (ttab null: hop amplitudes from
// the square-root table of `a`).
int fock_launch_nn(const ApplyArgs<uint32_t> &a, const void *bond, const void *etab, const void *ttab, int nb,
                   int precision, uint32_t g_begin, uint32_t g_end, int device, cudaStream_t s) {
  NNArgs t;
  t.a = a;
  t.bond = bond;
  t.etab = etab;
  t.ttab = ttab;
  t.nb = nb;
  t.g_begin = g_begin;
  t.g_end = g_end;
  if (g_begin >= g_end) return FOCK_OK;
  if (precision == FOCK_PREC_F64) return launch_nn_p<PolDFP>(t, device, s);
  if (precision == FOCK_PREC_F32_MIXED) return launch_nn_p<PolMixedP>(t, device, s);
  return launch_nn_p<PolF64>(t, device, s);
}
