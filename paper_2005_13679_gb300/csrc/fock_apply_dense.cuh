// fock_apply_dense.cuh -- sigma = H C when every reduced two-body coefficient
// R[r][a] is present (generic h and W), for a compile-time number of orbitals M.
//
// Same pull form as fock_apply_kernel.cuh, but the additions of a removal are
// all M(M+1)/2 pairs in a fixed order, so the addition loop is unrolled at
// compile time: the per-orbital prefix values U_j, V_j and the amplitudes
// b_j = sqrt(n'_j + 1), c_j = A b_j, d_j = c_j sqrt(n'_j + 2) stay in
// registers, each term costs two integer subtractions for its target, and the
// compiler can issue the gathers of many terms before their products.
//
// FP32-pair arithmetic runs on packed f32x2 lanes: for a term with complex
// coefficient K = R[r][a] * amp and gathered value C, the products
//     P1 = (Re K Re C, Im K Im C),  P2 = (Im K Re C, Re K Im C)
// are accumulated separately (two packed TwoSum chains), and sigma is formed
// once per configuration as Re = P1.x - P1.y, Im = P2.x + P2.y.
#pragma once

#include "fock_apply_kernel.cuh"
#include "fock_pack.cuh"

template <int M>
struct DenseSmem {
  static constexpr int P = M * (M + 1) / 2;
  size_t off_coef, off_pair, off_mod, off_sat, off_sq, total;
  __host__ __device__ DenseSmem(int xdim, int nsq, size_t coef_bytes) {
    const int rows = M > 1 ? M - 1 : 1;
    size_t o = 0;
    off_coef = o; o = fock_align16(o + coef_bytes * P * P);
    off_pair = o; o = fock_align16(o + 2 * P);
    off_mod = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sat = o;  o = fock_align16(o + 4 * (size_t)rows * xdim);
    off_sq = o;   o = fock_align16(o + 8 * (size_t)nsq);
    total = o;
  }
};

// Stage coefficients, pair list, binomial tables and square roots in shared memory.
template <int M, class CoefT, class SqT>
__device__ __forceinline__ void dense_stage(const ApplyArgs<uint32_t> &a, const DenseSmem<M> &L,
                                            unsigned char *smem) {
  constexpr int P = DenseSmem<M>::P;
  CoefT *s_coef = (CoefT *)(smem + L.off_coef);
  int8_t *s_pair = (int8_t *)(smem + L.off_pair);
  uint32_t *s_mod = (uint32_t *)(smem + L.off_mod);
  uint32_t *s_sat = (uint32_t *)(smem + L.off_sat);
  SqT *s_sq = (SqT *)(smem + L.off_sq);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < P * P; i += nt) s_coef[i] = ((const CoefT *)a.coef)[i];
  for (int i = tid; i < P; i += nt) {
    s_pair[2 * i] = a.rem[i].k;
    s_pair[2 * i + 1] = a.rem[i].q;
  }
  const int rows = M > 1 ? M - 1 : 1;
  for (int i = tid; i < rows * a.xdim; i += nt) {
    s_mod[i] = a.mod[i];
    s_sat[i] = a.sat[i];
  }
  for (int i = tid; i < a.nsq; i += nt) s_sq[i] = ((const SqT *)a.sq)[i];
  __syncthreads();
}

// Decoded configuration of one thread.
template <int M>
struct DenseCfg {
  int S[M], n[M];
};

// Per-removal values (prefix differences for the targets); invalid lanes use
// n' = n so that every table index stays inside its row.
template <int M>
__device__ __forceinline__ uint32_t dense_targets(const DenseCfg<M> &cf, int kk, int qq,
                                                  const uint32_t *s_mod, int xdim, uint32_t nc,
                                                  uint32_t (&U)[M], uint32_t (&V)[M]) {
  uint32_t F0 = 0, F1 = 0, F2 = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    U[m] = F0 - F1;
    V[m] = F1 - F2;
    if (m < M - 1) {
      const int dm = (kk <= m) + (qq <= m);
      const uint32_t *row = s_mod + m * xdim + (cf.S[m] - dm + m);
      F0 += row[0];
      F1 += row[1];
      F2 += row[2];
    }
  }
  return nc - 1u - F2;
}

// ---------------------------------------------------------------------------
// FP32-pair (FOCK_PREC_F64) dense kernel.  CH = right-hand sides per pass.
// ---------------------------------------------------------------------------
template <int M, int CH, bool MAPS>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS)
fock_apply_dense_df(const ApplyArgs<uint32_t> a) {
  constexpr int P = DenseSmem<M>::P;
  extern __shared__ __align__(16) unsigned char smem[];
  const DenseSmem<M> L(a.xdim, a.nsq, sizeof(float4));
  dense_stage<M, float4, float2>(a, L, smem);
  const float4 *s_coef = (const float4 *)(smem + L.off_coef);
  const int8_t *s_pair = (const int8_t *)(smem + L.off_pair);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float2 *s_sq = (const float2 *)(smem + L.off_sq);

  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nc = a.nc;
  const float4 *__restrict__ C = (const float4 *)a.C;
  const int nrhs = a.nrhs;
  double out_scale = a.out_scale;
  if (a.in_exp) out_scale *= fock_pow2(__ldg(a.in_exp));

  for (uint32_t tile = blockIdx.x * (uint32_t)nt; tile < nc; tile += gridDim.x * (uint32_t)nt) {
    const uint32_t g = tile + tid;
    const bool live = g < nc;
    const uint32_t gc = live ? g : nc - 1u;
    DenseCfg<M> cf;
    fock_decode_prefix<uint32_t, M>(live ? g : nc - 1u, a.N, M, nc, s_sat, a.xdim, cf.S);
#pragma unroll
    for (int m = 0; m < M; ++m) cf.n[m] = cf.S[m] - (m > 0 ? cf.S[m - 1] : 0);

    for (int c0 = 0; c0 < nrhs; c0 += CH) {
      fp2_t A1h[CH], A1l[CH], A2h[CH], A2l[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) A1h[j] = A1l[j] = A2h[j] = A2l[j] = 0ull;

      for (int r = 0; r < P; ++r) {
        const int k = s_pair[2 * r], q = s_pair[2 * r + 1];
        const int nk = sel_occ<M>(cf.n, k), nq = sel_occ<M>(cf.n, q);
        const bool valid = live && (k == q ? nk >= 2 : (nk >= 1 && nq >= 1));
        if (!__any_sync(0xffffffffu, valid)) continue;
        const int kk = valid ? k : M, qq = valid ? q : M;
        const float2 Ar = df_mul(s_sq[valid ? nk : 0], s_sq[valid ? nq - (k == q) : 0]);
        uint32_t U[M], V[M];
        uint32_t base = 0;
        if (!MAPS) base = dense_targets<M>(cf, kk, qq, s_mod, a.xdim, nc, U, V);
        float bh[M], bl[M], ch[M], cl[M], dh[M], dl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int np = cf.n[m] - (m == kk) - (m == qq);
          const float2 b = s_sq[np + 1];
          const float2 c = df_mul(Ar, b);
          const float2 d = df_mul(c, s_sq[np + 2]);
          bh[m] = b.x; bl[m] = b.y; ch[m] = c.x; cl[m] = c.y; dh[m] = d.x; dl[m] = d.y;
        }
        const float4 *cr = s_coef + r * P;
        const int32_t *mp = MAPS ? a.map + (size_t)r * P * nc + gc : nullptr;
#pragma unroll
        for (int s = 0; s < M; ++s) {
#pragma unroll
          for (int l = s; l < M; ++l) {
            const int ai = s * M - (s * (s - 1)) / 2 + (l - s);
            float ah, al;
            if (s == l) {
              ah = dh[s];
              al = dl[s];
            } else {
              ah = __fmul_rn(ch[s], bh[l]);
              al = __fmaf_rn(ch[s], bh[l], -ah);
              al = __fmaf_rn(ch[s], bl[l], al);
              al = __fmaf_rn(cl[s], bh[l], al);
            }
            const float4 w = cr[ai];
            fp2_t Kph, Kpl;
            fp2_dprod(fp2_make(w.x, w.y), fp2_make(w.z, w.w), fp2_make(ah, ah), fp2_make(al, al), Kph, Kpl);
            const fp2_t Ksh = fp2_swap(Kph), Ksl = fp2_swap(Kpl);
            // Branch-free: a lane whose removal is not allowed has A = 0, so K = 0
            // and its term adds exactly zero; it reads its own entry instead.
            uint32_t t = MAPS ? (uint32_t)__ldg(mp + (size_t)ai * nc) : base - U[s] - V[l];
            t = valid ? t : gc;
            const float4 *src = C + (size_t)t * nrhs + c0;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
              if (CH == 1 || c0 + j < nrhs) {
                const float4 v = __ldg(src + j);
                const fp2_t Ch = fp2_make(v.x, v.y), Cl = fp2_make(v.z, v.w);
                fp2_t p, e;
                fp2_dprod(Kph, Kpl, Ch, Cl, p, e);
                fp2_dacc(A1h[j], A1l[j], p, e);
                fp2_dprod(Ksh, Ksl, Ch, Cl, p, e);
                fp2_dacc(A2h[j], A2l[j], p, e);
              }
            }
          }
        }
      }
      if (live) {
        double2 *out = (double2 *)a.sigma + (size_t)g * nrhs + c0;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          if (CH == 1 || c0 + j < nrhs) {
            // Re = P1.x - P1.y and Im = P2.x + P2.y as FP32 pairs, then FP64
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            df_add_acc(rh, rl, fp2_x(A1h[j]), fp2_x(A1l[j]));
            df_add_acc(rh, rl, -fp2_y(A1h[j]), -fp2_y(A1l[j]));
            df_add_acc(ih, il, fp2_x(A2h[j]), fp2_x(A2l[j]));
            df_add_acc(ih, il, fp2_y(A2h[j]), fp2_y(A2l[j]));
            out[j] = make_double2(((double)rh + (double)rl) * out_scale, ((double)ih + (double)il) * out_scale);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP32-mixed (FOCK_PREC_F32_MIXED) dense kernel: FP32 products and per-removal
// partial sums on packed lanes, FP32-pair accumulation per configuration.
// ---------------------------------------------------------------------------
template <int M, int CH, bool MAPS>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS)
fock_apply_dense_mixed(const ApplyArgs<uint32_t> a) {
  constexpr int P = DenseSmem<M>::P;
  extern __shared__ __align__(16) unsigned char smem[];
  const DenseSmem<M> L(a.xdim, a.nsq, sizeof(float2));
  dense_stage<M, float2, float>(a, L, smem);
  const float2 *s_coef = (const float2 *)(smem + L.off_coef);
  const int8_t *s_pair = (const int8_t *)(smem + L.off_pair);
  const uint32_t *s_mod = (const uint32_t *)(smem + L.off_mod);
  const uint32_t *s_sat = (const uint32_t *)(smem + L.off_sat);
  const float *s_sq = (const float *)(smem + L.off_sq);

  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nc = a.nc;
  const float2 *__restrict__ C = (const float2 *)a.C;
  const int nrhs = a.nrhs;
  const float out_scale = (float)a.out_scale;

  for (uint32_t tile = blockIdx.x * (uint32_t)nt; tile < nc; tile += gridDim.x * (uint32_t)nt) {
    const uint32_t g = tile + tid;
    const bool live = g < nc;
    const uint32_t gc = live ? g : nc - 1u;
    DenseCfg<M> cf;
    fock_decode_prefix<uint32_t, M>(live ? g : nc - 1u, a.N, M, nc, s_sat, a.xdim, cf.S);
#pragma unroll
    for (int m = 0; m < M; ++m) cf.n[m] = cf.S[m] - (m > 0 ? cf.S[m - 1] : 0);

    for (int c0 = 0; c0 < nrhs; c0 += CH) {
      fp2_t Sh[CH], Sl[CH];  // (Re, Im) sigma as FP32 pairs
#pragma unroll
      for (int j = 0; j < CH; ++j) Sh[j] = Sl[j] = 0ull;

      for (int r = 0; r < P; ++r) {
        const int k = s_pair[2 * r], q = s_pair[2 * r + 1];
        const int nk = sel_occ<M>(cf.n, k), nq = sel_occ<M>(cf.n, q);
        const bool valid = live && (k == q ? nk >= 2 : (nk >= 1 && nq >= 1));
        if (!__any_sync(0xffffffffu, valid)) continue;
        const int kk = valid ? k : M, qq = valid ? q : M;
        const float Ar = s_sq[valid ? nk : 0] * s_sq[valid ? nq - (k == q) : 0];
        uint32_t U[M], V[M];
        uint32_t base = 0;
        if (!MAPS) base = dense_targets<M>(cf, kk, qq, s_mod, a.xdim, nc, U, V);
        float b[M], c[M], d[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int np = cf.n[m] - (m == kk) - (m == qq);
          b[m] = s_sq[np + 1];
          c[m] = Ar * b[m];
          d[m] = c[m] * s_sq[np + 2];
        }
        fp2_t I1[CH], I2[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) I1[j] = I2[j] = 0ull;
        const float2 *cr = s_coef + r * P;
        const int32_t *mp = MAPS ? a.map + (size_t)r * P * nc + gc : nullptr;
#pragma unroll
        for (int s = 0; s < M; ++s) {
#pragma unroll
          for (int l = s; l < M; ++l) {
            const int ai = s * M - (s * (s - 1)) / 2 + (l - s);
            const float amp = (s == l) ? d[s] : c[s] * b[l];
            const float2 w = cr[ai];
            const fp2_t Kp = fp2_mul(fp2_make(w.x, w.y), fp2_make(amp, amp));
            const fp2_t Ks = fp2_swap(Kp);
            uint32_t t = MAPS ? (uint32_t)__ldg(mp + (size_t)ai * nc) : base - U[s] - V[l];
            t = valid ? t : gc;
            const float2 *src = C + (size_t)t * nrhs + c0;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
              if (CH == 1 || c0 + j < nrhs) {
                const float2 v = __ldg(src + j);
                const fp2_t Cv = fp2_make(v.x, v.y);
                I1[j] = fp2_fma(Kp, Cv, I1[j]);   // (Re K Re C, Im K Im C)
                I2[j] = fp2_fma(Ks, Cv, I2[j]);   // (Im K Re C, Re K Im C)
              }
            }
          }
        }
        if (valid) {
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            const fp2_t part = fp2_make(fp2_x(I1[j]) - fp2_y(I1[j]), fp2_x(I2[j]) + fp2_y(I2[j]));
            fp2_dacc(Sh[j], Sl[j], part, 0ull);
          }
        }
      }
      if (live) {
        float2 *out = (float2 *)a.sigma + (size_t)g * nrhs + c0;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          if (CH == 1 || c0 + j < nrhs) {
            const fp2_t v = fp2_add(Sh[j], Sl[j]);
            out[j] = make_float2(fp2_x(v) * out_scale, fp2_y(v) * out_scale);
          }
        }
      }
    }
  }
}

template <class K>
int fock_launch_dense(K kern, const ApplyArgs<uint32_t> &a, size_t smem_bytes, int device, cudaStream_t stream) {
  const int threads = FOCK_APPLY_THREADS;
  if (smem_bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return fock_cuda_status(e);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem_bytes);
  if (e != cudaSuccess) return fock_cuda_status(e);
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  int64_t tiles = ((int64_t)a.nc + threads - 1) / threads;
  int64_t grid = (int64_t)per_sm * fock_get_sm_count(device);
  if (grid > tiles) grid = tiles;
  kern<<<(unsigned)grid, threads, smem_bytes, stream>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}
