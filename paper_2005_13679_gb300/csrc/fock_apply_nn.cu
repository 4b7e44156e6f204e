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
// a x with x a small integer or half-integer (exact in FP32)
__device__ __forceinline__ double nn_scale(double a, float x) { return a * (double)x; }
__device__ __forceinline__ float nn_scale(float a, float x) { return a * x; }
__device__ __forceinline__ float2 nn_scale(float2 a, float x) { return df_mul(a, make_float2(x, 0.f)); }
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

struct NNArgs {
  ApplyArgs<uint32_t> a;      // sizes, tables, C, sigma, nrhs, scales
  const void *bond;           // [2 * nb] policy coef_t: h_kl, h_lk of bond b = (k, k + 1 mod M)
  const void *diag;           // [2 * M] policy amp_t: h_kk, then W_kkkk
  int nb;                     // bonds: M - 1, or M for a ring (M > 2)
};

template <int M, class P>
__global__ void __launch_bounds__(kNNThreads, kNNMinBlocks) fock_apply_nn(const NNArgs t) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  using vec_t = typename P::vec_t;
  const ApplyArgs<uint32_t> &a = t.a;
  extern __shared__ __align__(16) unsigned char smem[];
  const int rows = M > 1 ? M - 1 : 1, xs = a.xdim + 2;
  coef_t *s_bond = (coef_t *)smem;                                   // [2 nb]
  amp_t *s_diag = (amp_t *)(s_bond + 2 * M);                         // [2 M]
  amp_t *s_sq = s_diag + 2 * M;                                      // [nsq]
  uint32_t *s_mod = (uint32_t *)(s_sq + a.nsq + 1);                  // rows of xs (two leading zeros)
  uint32_t *s_sat = s_mod + rows * xs;
  for (int i = threadIdx.x; i < 2 * t.nb; i += blockDim.x) s_bond[i] = ((const coef_t *)t.bond)[i];
  for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) s_diag[i] = ((const amp_t *)t.diag)[i];
  for (int i = threadIdx.x; i < a.nsq; i += blockDim.x) s_sq[i] = ((const amp_t *)a.sq)[i];
  for (int i = threadIdx.x; i < rows * xs; i += blockDim.x) {
    const int m = i / xs, x = i - m * xs;
    s_mod[i] = x < 2 ? 0u : a.mod[m * a.xdim + x - 2];
  }
  for (int i = threadIdx.x; i < rows * a.xdim; i += blockDim.x) s_sat[i] = a.sat[i];
  __syncthreads();
  double out_scale = a.out_scale;
  if (a.in_exp) out_scale *= fock_pow2(__ldg(a.in_exp));
  const vec_t *__restrict__ C = (const vec_t *)a.C;
  const uint32_t nc = a.nc;
  const int nrhs = a.nrhs;
  const bool real = a.real != 0;
  const bool ring = t.nb == M && M > 2;

  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nc; g += gridDim.x * blockDim.x) {
    int S[M];
    fock_decode_fast<M>(g, a.N, nc, s_sat, a.xdim, S);
    // diagonal: sum_k h_kk n_k + 1/2 W_kkkk n_k (n_k - 1), as a real amplitude
    amp_t dg{};
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const float nm = (float)(S[m] - (m > 0 ? S[m - 1] : 0));
      dg = nn_add(dg, nn_scale(s_diag[m], nm));
      dg = nn_add(dg, nn_scale(s_diag[M + m], 0.5f * nm * (nm - 1.f)));
    }
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
        const coef_t Kkl = P::scale(s_bond[2 * m], P::amul(s_sq[nk], s_sq[nl + 1]));
        const coef_t Klk = P::scale(s_bond[2 * m + 1], P::amul(s_sq[nl], s_sq[nk + 1]));
        nn_mac2<P>(acc, Kkl, __ldg(C + (size_t)tkl * nrhs + j), Klk, __ldg(C + (size_t)tlk * nrhs + j), real);
      }
      if (ring) {
        // bond (M - 1, 0): S_0 .. S_{M-2} all change, by +1 (particle M-1 -> 0)
        // or by -1 (particle 0 -> M-1): the summed differences
        const int nk = S[M - 1] - S[M - 2], nl = S[0];
        const uint32_t tkl = nk > 0 ? g - fp : g;
        const uint32_t tlk = nl > 0 ? g - fm : g;
        const coef_t Kkl = P::scale(s_bond[2 * (M - 1)], P::amul(s_sq[nk], s_sq[nl + 1]));
        const coef_t Klk = P::scale(s_bond[2 * (M - 1) + 1], P::amul(s_sq[nl], s_sq[nk + 1]));
        nn_mac2<P>(acc, Kkl, __ldg(C + (size_t)tkl * nrhs + j), Klk, __ldg(C + (size_t)tlk * nrhs + j), real);
      }
      ((decltype(P::finish(acc, 1.0, real)) *)a.sigma)[(size_t)g * nrhs + j] = P::finish(acc, out_scale, real);
    }
  }
}

}  // namespace

namespace {

template <int M, class P>
int launch_nn_m(const NNArgs &t, int device, cudaStream_t s) {
  using amp_t = typename P::amp_t;
  using coef_t = typename P::coef_t;
  const ApplyArgs<uint32_t> &a = t.a;
  const int rows = M > 1 ? M - 1 : 1;
  const size_t smem = sizeof(coef_t) * 2 * M + sizeof(amp_t) * (2 * M + a.nsq + 1) + 4 * (size_t)rows * (a.xdim + 2) +
                      4 * (size_t)rows * a.xdim + 16;
  auto kern = fock_apply_nn<M, P>;
  if (smem > 48 * 1024) FOCK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FOCK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNNThreads, smem));
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t blocks = ((int64_t)a.nc + kNNThreads - 1) / kNNThreads;
  const int64_t cap = (int64_t)per_sm * fock_get_sm_count(device);
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)(blocks < 1 ? 1 : blocks), kNNThreads, smem, s>>>(t);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

template <class P>
int launch_nn(const NNArgs &t, int device, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_NN_CASE(MM) \
    case MM: return launch_nn_m<MM, P>(t, device, s);
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

}  // namespace

// Launch for one of the precisions; bond/diag hold that precision's arrays.
int fock_launch_nn(const ApplyArgs<uint32_t> &a, const void *bond, const void *diag, int nb, int precision,
                   int device, cudaStream_t s) {
  NNArgs t;
  t.a = a;
  t.bond = bond;
  t.diag = diag;
  t.nb = nb;
  if (precision == FOCK_PREC_F64) return launch_nn<PolDFP>(t, device, s);
  if (precision == FOCK_PREC_F32_MIXED) return launch_nn<PolMixedP>(t, device, s);
  return launch_nn<PolF64>(t, device, s);
}
