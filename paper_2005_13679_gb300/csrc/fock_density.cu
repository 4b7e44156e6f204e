// fock_density.cu -- one- and two-body density matrices (Eqs. rho1, rho2):
//
//     rho1[k][l]       = <Psi| a^dag_k a_l |Psi>           = sum_{m'} conj(Z_k[m']) Z_l[m'],
//     rho2[k][l][q][s] = <Psi| a^dag_k a^dag_l a_q a_s |Psi> = sum_{n'} conj(X_{kl}[n']) X_{qs}[n'],
//
// with Z_l[m'] = <m'| a_l |Psi> = sqrt(m'_l + 1) C[m' + e_l] over the
// (N-1)-particle configurations and X_{qs}[n'] = <n'| a_q a_s |Psi> =
// sqrt(n'_q + 1) sqrt(n'_s + 1 + delta_qs) C[n' + e_q + e_s] over the
// (N-2)-particle configurations (a_q a_s = a_s a_q, so one vector per unordered
// pair).  Both are Hermitian Gram matrices of small vectors over a large
// space: one thread builds the vector of one configuration in a shared tile
// of 128 columns; the upper triangle is cut into 3 x 3 blocks of entries, and
// a thread takes one block over one of G interleaved column groups of the
// tile (9 complex products per 6 shared-memory reads), accumulating in FP32
// pairs.  Each thread adds its tile sums in FP64 to its own shared slots;
// the groups, then the per-block partials, are summed in a fixed order
// (deterministic).  This replaces the paper's element-by-element sums over
// beta with a reduction that reads each C gather once per configuration of
// the smaller space.
#include <math.h>

#include <vector>

#include "fock_apply_twophase.cuh"

namespace {

constexpr int kGramWarp = 32;   // columns of a warp's tile (one per lane)

// Shapes of one Gram reduction: K vectors per column, E upper-triangle
// entries, in BS x BS blocks of entries (W blocks in the upper triangle).
template <int M, bool TWO>
struct GramShape {
  static constexpr int K = TWO ? M * (M + 1) / 2 : M;     // vectors per configuration
  static constexpr int E = K * (K + 1) / 2;               // upper-triangle entries
  static constexpr int W3 = ((K + 2) / 3) * ((K + 2) / 3 + 1) / 2, W2 = ((K + 1) / 2) * ((K + 1) / 2 + 1) / 2;
  static constexpr int BS = W3 >= 28 ? 3 : (W2 >= 28 ? 2 : 1);  // entry block edge: most reuse with >= 28 lanes busy
  static constexpr int NB = (K + BS - 1) / BS;
  static constexpr int KP = BS * NB;                      // tile row length (zero padded)
  static constexpr int W = NB * (NB + 1) / 2;             // upper-triangle blocks
  static constexpr int TILE = kGramWarp * KP * 16;        // bytes of a warp's column tile
  static constexpr int SLOTS = W * BS * BS;              // entry slots (blocks x BS^2)
  static constexpr int ACC = SLOTS * 16;                  // bytes of a warp's FP32-pair sums
  static constexpr int WARP_BYTES = TILE + ACC;
};

struct GramArgs {
  int N, M, xdim, nsq;
  uint32_t nc, ncol;                // N-space size; columns (configurations of the smaller space)
  const uint32_t *mod, *sat;        // binomial tables of the N-space (wrapping and saturated)
  const float4 *C;                  // FP32-pair split of C (re_hi, im_hi, re_lo, im_lo), scaled
  double2 *slots;                   // [warps][SLOTS] FP64 sums
  double2 *partial;                 // [warps][E]
};

constexpr int kGramFlush = 16;      // tiles between the FP32-pair and FP64 sums

// sqrt(i) as an FP32 pair: the correctly rounded root and the residual
// (i - hi^2, exact by FMA) divided by 2 hi.
__device__ __forceinline__ float2 gram_sqrt_pair(int i) {
  const float x = (float)i;
  const float hi = __fsqrt_rn(x);
  const float lo = hi > 0.f ? __fdiv_rn(__fmaf_rn(-hi, hi, x), 2.f * hi) : 0.f;
  return make_float2(hi, lo);
}

// (re, im) of conj(a) b accumulated into the packed pair (h, l), a and b as
// float4 (re_hi, im_hi, re_lo, im_lo):
//   Re = ar br + ai bi,  Im = ar bi - ai br.
__device__ __forceinline__ void gram_mac(fp2_t &h, fp2_t &l, float4 a, float4 b) {
  fp2_t p, e;
  fp2_dprod(fp2_make(a.x, a.x), fp2_make(a.z, a.z), fp2_make(b.x, b.y), fp2_make(b.z, b.w), p, e);
  fp2_dacc(h, l, p, e);
  fp2_dprod(fp2_make(a.y, a.y), fp2_make(a.w, a.w), fp2_make(b.y, -b.x), fp2_make(b.w, -b.z), p, e);
  fp2_dacc(h, l, p, e);
}

// Block (bi, bj), bi <= bj, of the row-major upper triangle of an NB x NB grid.
__device__ __forceinline__ void gram_block(int it, int nb, int &bi, int &bj) {
  int r = it, i = 0;
  while (r >= nb - i) {
    r -= nb - i;
    ++i;
  }
  bi = i;
  bj = i + r;
}

// Every warp works alone (no block barrier in the loop): it builds the
// vectors of 32 consecutive columns in its own shared tile, one lane per
// column, then each lane takes blocks of BS x BS entries over the 32 columns
// (FP32 pairs, BS^2 independent sums) and adds them by TwoSum to the warp's
// shared FP32-pair sums, which go into the warp's FP64 sums in global memory
// every kGramFlush tiles (the FP64 pipe runs at 1/64 of the FP32 rate).  The
// warps' sums go to `partial` in entry order.
template <int M, bool TWO>
__global__ void __launch_bounds__(256) fock_gram_kernel(const GramArgs g) {
  using Sh = GramShape<M, TWO>;
  constexpr int K = Sh::K, E = Sh::E, KP = Sh::KP, W = Sh::W, BS = Sh::BS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int rows = M > 1 ? M - 1 : 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwb = blockDim.x >> 5;
  uint32_t *s_mod = (uint32_t *)smem;
  uint32_t *s_sat = s_mod + rows * g.xdim;
  float2 *s_sq = (float2 *)(s_sat + rows * g.xdim + 2);
  const size_t tab = ((size_t)(8 * rows * g.xdim + 8 + 8 * g.nsq) + 15) & ~(size_t)15;
  unsigned char *mine = smem + tab + (size_t)warp * Sh::WARP_BYTES;
  float4 *Xt = (float4 *)mine;                                        // [32][KP]
  float4 *acc = (float4 *)(mine + Sh::TILE);                          // [SLOTS] (re_h, im_h, re_l, im_l)
  for (int i = tid; i < rows * g.xdim; i += blockDim.x) {
    s_mod[i] = g.mod[i];
    s_sat[i] = g.sat[i];
  }
  for (int i = tid; i < g.nsq; i += blockDim.x) s_sq[i] = gram_sqrt_pair(i);
  const uint32_t gw = blockIdx.x * (uint32_t)nwb + warp, nw = gridDim.x * (uint32_t)nwb;
  double2 *gacc = g.slots + (size_t)gw * Sh::SLOTS;
  for (int i = lane; i < Sh::SLOTS; i += 32) {
    acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    gacc[i] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  // FP32-pair sums into the FP64 sums
  auto flush = [&]() {
    for (int i = lane; i < Sh::SLOTS; i += 32) {
      const float4 v = acc[i];
      double2 d = gacc[i];
      d.x += (double)v.x + (double)v.z;
      d.y += (double)v.y + (double)v.w;
      gacc[i] = d;
      acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };

  int ntile = 0;
  for (uint32_t tile = gw; tile * kGramWarp < g.ncol; tile += nw) {
    // ---- this lane's column vector into the warp's tile ----
    const uint32_t col = tile * kGramWarp + lane;
    float4 *xrow = Xt + lane * KP;
    for (int a = K; a < KP; ++a) xrow[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col < g.ncol) {
      int S[M];
      if (TWO) {
        fock_decode_fast<M>(col, g.N - 2, g.ncol, s_sat, g.xdim, S);
        uint32_t U[M], V[M];
        const uint32_t base = twophase_targets<M>(S, s_mod, g.xdim, g.nc, U, V);
        float2 sq1[M], sq2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int occ = S[m] - (m > 0 ? S[m - 1] : 0);
          sq1[m] = s_sq[occ + 1];
          sq2[m] = s_sq[occ + 2];
        }
        float4 v[TWO ? K : 1];
        int a = 0;
#pragma unroll
        for (int s = 0; s < M; ++s)
#pragma unroll
          for (int l = s; l < M; ++l, ++a) v[a] = __ldg(g.C + (base - U[s] - V[l]));
        a = 0;
#pragma unroll
        for (int s = 0; s < M; ++s)
#pragma unroll
          for (int l = s; l < M; ++l, ++a) {
            const float2 amp = df_mul(sq1[s], s == l ? sq2[s] : sq1[l]);
            fp2_t Xh, Xl;
            fp2_dprod(fp2_make(v[a].x, v[a].y), fp2_make(v[a].z, v[a].w), fp2_make(amp.x, amp.x),
                      fp2_make(amp.y, amp.y), Xh, Xl);
            xrow[a] = make_float4(fp2_x(Xh), fp2_y(Xh), fp2_x(Xl), fp2_y(Xl));
          }
      } else {
        fock_decode_fast<M>(col, g.N - 1, g.ncol, s_sat, g.xdim, S);
        // rank(m' + e_l) = (nc - 1 - F1[M-1]) - (F0[l] - F1[l]) with F_d[j] the
        // prefix sums of C(S_m + m + d, m + 1) over m < j
        uint32_t F0 = 0, F1 = 0, D[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          D[m] = F0 - F1;
          if (m < M - 1) {
            const uint32_t *row = s_mod + m * g.xdim + (S[m] + m);
            F0 += row[0];
            F1 += row[1];
          }
        }
        const uint32_t base = g.nc - 1u - F1;
#pragma unroll
        for (int l = 0; l < M; ++l) {
          const float4 v = __ldg(g.C + (base - D[l]));
          const int occ = S[l] - (l > 0 ? S[l - 1] : 0);
          const float2 amp = s_sq[occ + 1];
          fp2_t Xh, Xl;
          fp2_dprod(fp2_make(v.x, v.y), fp2_make(v.z, v.w), fp2_make(amp.x, amp.x), fp2_make(amp.y, amp.y), Xh,
                    Xl);
          xrow[l] = make_float4(fp2_x(Xh), fp2_y(Xh), fp2_x(Xl), fp2_y(Xl));
        }
      }
    } else {
      for (int a = 0; a < K; ++a) xrow[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    // ---- BS x BS entry blocks over the tile's 32 columns ----
    for (int it = lane; it < W; it += 32) {
      int bi, bj;
      gram_block(it, Sh::NB, bi, bj);
      const int a0 = BS * bi, b0 = BS * bj;
      fp2_t h[BS * BS], l[BS * BS];
#pragma unroll
      for (int i = 0; i < BS * BS; ++i) h[i] = l[i] = 0ull;
#pragma unroll 2
      for (int c = 0; c < kGramWarp; ++c) {
        const float4 *x = Xt + c * KP;
        float4 A[BS], B[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
          A[i] = x[a0 + i];
          B[i] = x[b0 + i];
        }
#pragma unroll
        for (int i = 0; i < BS; ++i)
#pragma unroll
          for (int j = 0; j < BS; ++j) gram_mac(h[BS * i + j], l[BS * i + j], A[i], B[j]);
      }
      float4 *dst = acc + BS * BS * it;
#pragma unroll
      for (int i = 0; i < BS * BS; ++i) {
        const float4 v = dst[i];
        fp2_t H = fp2_make(v.x, v.y), L = fp2_make(v.z, v.w);
        fp2_dacc(H, L, h[i], l[i]);
        dst[i] = make_float4(fp2_x(H), fp2_y(H), fp2_x(L), fp2_y(L));
      }
    }
    __syncwarp();
    if (++ntile == kGramFlush) {
      flush();
      ntile = 0;
      __syncwarp();
    }
  }
  flush();
  __syncwarp();
  // this warp's upper-triangle entries
  for (int e = lane; e < E; e += 32) {
    int a = 0, r = e;
    while (r >= K - a) {
      r -= K - a;
      ++a;
    }
    const int b = a + r, bi = a / BS, bj = b / BS;
    const int it = bi * Sh::NB - (bi * (bi - 1)) / 2 + (bj - bi);
    g.partial[(size_t)gw * E + e] = gacc[BS * BS * it + BS * (a - BS * bi) + (b - BS * bj)];
  }
}

// out[e] = sum over warps of partial[w][e], in warp order.
__global__ void fock_gram_reduce(const double2 *__restrict__ partial, int blocks, int E, double2 *__restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < blocks; ++b) {
    const double2 v = partial[(size_t)b * E + e];
    s.x += v.x;
    s.y += v.y;
  }
  out[e] = s;
}

// Shared memory of a block of `warps` warps: the tables, then one tile and
// FP64 sums per warp.
template <int M, bool TWO>
size_t gram_smem(int xdim, int nsq, int warps) {
  using Sh = GramShape<M, TWO>;
  const int rows = M > 1 ? M - 1 : 1;
  const size_t tab = ((size_t)(8 * rows * xdim + 8 + 8 * nsq) + 15) & ~(size_t)15;
  return tab + (size_t)warps * Sh::WARP_BYTES;
}

// Runs one Gram reduction; G receives the upper triangle (E entries).
// Device buffer of at least `bytes`, kept in *buf between calls (grown when needed).
static int grow(void **buf, size_t *cap, size_t bytes) {
  if (*cap >= bytes) return FOCK_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  FOCK_CUDA_TRY(cudaMalloc(buf, bytes));
  *cap = bytes;
  return FOCK_OK;
}

template <int M, bool TWO>
int gram_run(const GramArgs &g0, int device, cudaStream_t s, std::vector<double> &G, fock_space *sp) {
  constexpr int E = GramShape<M, TWO>::E;
  GramArgs g = g0;
  auto kern = fock_gram_kernel<M, TWO>;
  int optin = 0;
  FOCK_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  // warps per block: the most resident warps per SM (shared memory and
  // registers), fewest blocks on a tie
  int warps = 0, per_sm = 0;
  for (int w = 8; w >= 1; w /= 2) {
    const size_t sm_w = gram_smem<M, TWO>(g.xdim, g.nsq, w);
    if (sm_w > (size_t)optin) continue;
    FOCK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_w));
    int b = 0;
    FOCK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * w, sm_w));
    if (b * w > per_sm * warps) {
      warps = w;
      per_sm = b;
    }
  }
  if (warps < 1 || per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  const size_t smem = gram_smem<M, TWO>(g.xdim, g.nsq, warps);
  FOCK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t tiles = ((int64_t)g.ncol + kGramWarp - 1) / kGramWarp;
  int64_t grid = (int64_t)per_sm * fock_get_sm_count(device);
  if (grid * warps > tiles) grid = (tiles + warps - 1) / warps;
  if (grid < 1) grid = 1;
  const int64_t nwarps = grid * warps;
  const size_t nslots = (size_t)GramShape<M, TWO>::SLOTS * nwarps;
  const int gst = grow(&sp->dm_part, &sp->dm_part_bytes, sizeof(double2) * ((size_t)E * (nwarps + 1) + nslots));
  if (gst) return gst;
  double2 *buf = (double2 *)sp->dm_part;
  g.partial = buf;
  g.slots = buf + (size_t)E * (nwarps + 1);
  kern<<<(unsigned)grid, 32 * warps, smem, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    fock_gram_reduce<<<(E + 127) / 128, 128, 0, s>>>(buf, (int)nwarps, E, buf + (size_t)E * nwarps);
    e = cudaGetLastError();
  }
  G.assign(2 * (size_t)E, 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(G.data(), buf + (size_t)E * nwarps, sizeof(double2) * E, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

template <bool TWO>
int gram_dispatch(int M, const GramArgs &g, int device, cudaStream_t s, std::vector<double> &G, fock_space *sp) {
  switch (M) {
#define FOCK_GRAM_CASE(MM) \
    case MM: return gram_run<MM, TWO>(g, device, s, G, sp);
    FOCK_GRAM_CASE(1)
    FOCK_GRAM_CASE(2)
    FOCK_GRAM_CASE(3)
    FOCK_GRAM_CASE(4)
    FOCK_GRAM_CASE(5)
    FOCK_GRAM_CASE(6)
    FOCK_GRAM_CASE(7)
    FOCK_GRAM_CASE(8)
    FOCK_GRAM_CASE(9)
    FOCK_GRAM_CASE(10)
    FOCK_GRAM_CASE(11)
    FOCK_GRAM_CASE(12)
#undef FOCK_GRAM_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}

int64_t nc_of(int n, int m) {
  if (n < 0 || m < 1) return 0;
  // C(n + m - 1, m - 1) by the multiplicative formula (fits: the caller's
  // space is 32-bit)
  uint64_t r = 1;
  for (int i = 1; i <= m - 1; ++i) r = r * (uint64_t)(n + i) / (uint64_t)i;
  return (int64_t)r;
}

}  // namespace

int fock_prepare_df(const void *C, int64_t n, void *ws, int device, cudaStream_t stream);

extern "C" int fock_density_matrices(const fock_space *sp, const void *C_dev, double *rho1_host, double *rho2_host,
                                     void *stream) {
  if (!sp || !C_dev || (!rho1_host && !rho2_host)) return FOCK_ERR_ARG;
  if (!sp->idx32 || sp->M > 12) return FOCK_ERR_UNSUPPORTED;
  int dev = -1;
  FOCK_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != sp->device) return FOCK_ERR_DEVICE;
  const int N = sp->N, M = sp->M;
  cudaStream_t s = (cudaStream_t)stream;
  // FP32-pair split of C, scaled by a power of two (the apply's preparation)
  fock_space *spw = (fock_space *)sp;                    // the space keeps the workspace between calls
  int st = grow(&spw->dm_ws, &spw->dm_ws_bytes, 256 + 16 * (size_t)sp->nc);
  if (st) return st;
  void *ws = spw->dm_ws;
  st = fock_prepare_df(C_dev, sp->nc, ws, sp->device, s);
  int words[2] = {0, 0};
  if (!st) {
    cudaError_t e = cudaMemcpyAsync(words, ws, sizeof(words), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fock_cuda_status(e);
  }
  GramArgs g;
  g.N = N;
  g.M = M;
  g.xdim = sp->tab.xdim;
  g.nsq = N + 4;
  g.nc = (uint32_t)sp->nc;
  g.mod = sp->tab.mod32;
  g.sat = sp->tab.sat32;
  g.C = (const float4 *)((const char *)ws + 256);
  g.partial = nullptr;
  g.slots = nullptr;
  const double scale2 = ldexp(1.0, 2 * words[1]);       // |C|^2 units of the split
  auto pair_index = [M](int k, int l) {                  // unordered pair {k, l} in the kernel's order
    const int s = k < l ? k : l, t = k < l ? l : k;
    return s * M - s * (s - 1) / 2 + (t - s);
  };
  if (!st && rho2_host) {
    const size_t m4 = (size_t)M * M * M * M;
    if (N < 2) {
      for (size_t i = 0; i < 2 * m4; ++i) rho2_host[i] = 0.0;
    } else {
      g.ncol = (uint32_t)nc_of(N - 2, M);
      std::vector<double> G;
      st = gram_dispatch<true>(M, g, sp->device, s, G, (fock_space *)sp);
      if (!st) {
        const int P = M * (M + 1) / 2;
        std::vector<double> full(2 * (size_t)P * P);
        int e = 0;
        for (int a = 0; a < P; ++a)
          for (int b = a; b < P; ++b, ++e) {
            full[2 * ((size_t)a * P + b)] = G[2 * e] * scale2;
            full[2 * ((size_t)a * P + b) + 1] = G[2 * e + 1] * scale2;
            full[2 * ((size_t)b * P + a)] = G[2 * e] * scale2;
            full[2 * ((size_t)b * P + a) + 1] = -G[2 * e + 1] * scale2;
          }
        for (int k = 0; k < M; ++k)
          for (int l = 0; l < M; ++l)
            for (int q = 0; q < M; ++q)
              for (int r = 0; r < M; ++r) {
                const size_t o = ((((size_t)k * M + l) * M + q) * M + r);
                const size_t src = (size_t)pair_index(k, l) * P + pair_index(q, r);
                rho2_host[2 * o] = full[2 * src];
                rho2_host[2 * o + 1] = full[2 * src + 1];
              }
      }
    }
  }
  if (!st && rho1_host && rho2_host && N >= 2) {
    // rho1 as the partial trace of rho2: sum_x a^dag_k a^dag_x a_x a_l =
    // a^dag_k N^ a_l, and N^ a_l = (N - 1) a_l on N particles, so
    // rho1[k][l] = sum_x rho2[k][x][x][l] / (N - 1)
    for (int k = 0; k < M; ++k)
      for (int l = 0; l < M; ++l) {
        double re = 0.0, im = 0.0;
        for (int x = 0; x < M; ++x) {
          const size_t o = ((((size_t)k * M + x) * M + x) * M + l);
          re += rho2_host[2 * o];
          im += rho2_host[2 * o + 1];
        }
        rho1_host[2 * (k * M + l)] = re / (N - 1);
        rho1_host[2 * (k * M + l) + 1] = im / (N - 1);
      }
  } else if (!st && rho1_host) {
    g.ncol = (uint32_t)nc_of(N - 1, M);
    std::vector<double> G;
    st = gram_dispatch<false>(M, g, sp->device, s, G, (fock_space *)sp);
    if (!st) {
      int e = 0;
      for (int a = 0; a < M; ++a)
        for (int b = a; b < M; ++b, ++e) {
          const double re = G[2 * e] * scale2, im = G[2 * e + 1] * scale2;
          rho1_host[2 * (a * M + b)] = re;
          rho1_host[2 * (a * M + b) + 1] = im;
          rho1_host[2 * (b * M + a)] = re;
          rho1_host[2 * (b * M + a) + 1] = -im;
        }
    }
  }
  return st;
}
