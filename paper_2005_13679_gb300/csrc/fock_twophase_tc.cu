// fock_twophase_tc.cu -- the two-phase apply with its phase 1 on the tensor
// cores (fock_apply_tc.cuh), M = 2..6: host construction of the digit image
// of R, launch of phase 1 and of the FP32-pair phase 2.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <complex>
#include <type_traits>
#include <vector>

#include "fock_apply_tc.cuh"

// Digit image of the real form of R (P x P complex, row r = removal pair,
// column a = addition pair, already divided by the coefficient scale):
// rows 2r, 2r+1 are (Re, Im) of Y_r, columns 2a, 2a+1 multiply (Re, Im) of X_a.
// Each real row rho gets e_rho with |R~[rho][k]| < 2^e_rho for all k and five
// base-2^9 digits of R~ 2^(8 - e_rho), computed exactly in FP64.  The image is
// the MMA's B operand (N = (real row, level) combinations, K-major) in
// tensor-core shared-memory layout.
int fock_tc_image(int M, const std::complex<double> *R, std::vector<unsigned char> &img, std::vector<int> &er) {
  if (M < 2 || M > 6) return FOCK_ERR_UNSUPPORTED;
  const TcShape sh(M);
  const int P = sh.P, R2 = sh.R2;
  std::vector<double> Rt((size_t)R2 * R2);
  for (int r = 0; r < P; ++r)
    for (int a = 0; a < P; ++a) {
      const std::complex<double> v = R[(size_t)r * P + a];
      Rt[(size_t)(2 * r) * R2 + 2 * a] = v.real();
      Rt[(size_t)(2 * r) * R2 + 2 * a + 1] = -v.imag();
      Rt[(size_t)(2 * r + 1) * R2 + 2 * a] = v.imag();
      Rt[(size_t)(2 * r + 1) * R2 + 2 * a + 1] = v.real();
    }
  er.assign(R2, 0);
  std::vector<float> dig((size_t)R2 * R2 * 5, 0.f);
  for (int rho = 0; rho < R2; ++rho) {
    int e = INT_MIN;
    for (int k = 0; k < R2; ++k) {
      const double x = Rt[(size_t)rho * R2 + k];
      if (x != 0.0) {
        int ex;
        frexp(x, &ex);   // |x| < 2^ex
        if (ex > e) e = ex;
      }
    }
    if (e == INT_MIN) e = 0;
    er[rho] = e;
    for (int k = 0; k < R2; ++k) {
      double v = ldexp(Rt[(size_t)rho * R2 + k], 8 - e);
      for (int i = 0; i < 5; ++i) {
        const double d = nearbyint(v);
        dig[((size_t)rho * R2 + k) * 5 + i] = (float)d;
        v = (v - d) * 512.0;
      }
    }
  }
  // rows of the image: level l of real row rho at sh.col(rho, l); row 15
  // copies the column exponent stored at K position exp_pos()
  const int CHT = sh.KT / 8;
  img.assign(sh.r_bytes(), 0);
  for (int rho = 0; rho < R2; ++rho)
    for (int level = 2; level <= 6; ++level) {
      const int row = sh.col(rho, level);
      for (int p = 0; p < sh.KT; ++p) {
        int k, j;
        if (p < sh.K1) {
          k = p / 3;
          j = p % 3 + 1;
        } else {
          k = (p - sh.K1) / 2;
          j = 4 + (p - sh.K1) % 2;
        }
        const int i = level - j;
        if (k >= R2 || i < 1 || i > 5) continue;
        const __half h = __float2half(dig[((size_t)rho * R2 + k) * 5 + (i - 1)]);
        memcpy(img.data() + tc_kmajor_offset(row, p, CHT), &h, 2);
      }
    }
  const __half one = __float2half(1.f);
  memcpy(img.data() + tc_kmajor_offset(kTcExpCol, sh.exp_pos(), CHT), &one, 2);
  return FOCK_OK;
}

// Image of the FP32-mixed form: real row rho of R (unscaled) gets a scale
// 2^(15 - e_rho) with |R~[rho][k]| < 2^e_rho and the fp16 split
// R_h = RN(R~ 2^s), R_l = RN(R~ 2^s - R_h); its image row holds
// [R_h | 2^-11 R_h | R_l] against the digit tile's [x_h | 2^11 x_l | x_h], and
// row R2 copies the column exponent at K position 3 R2.
int fock_tc_image_mixed(int M, const std::complex<double> *R, std::vector<unsigned char> &img, std::vector<int> &er) {
  if (M < 2 || M > 6) return FOCK_ERR_UNSUPPORTED;
  const TcMixedShape sh(M);
  const int P = sh.P, R2 = sh.R2, CHT = sh.KT / 8;
  std::vector<double> Rt((size_t)R2 * R2);
  for (int r = 0; r < P; ++r)
    for (int a = 0; a < P; ++a) {
      const std::complex<double> v = R[(size_t)r * P + a];
      Rt[(size_t)(2 * r) * R2 + 2 * a] = v.real();
      Rt[(size_t)(2 * r) * R2 + 2 * a + 1] = -v.imag();
      Rt[(size_t)(2 * r + 1) * R2 + 2 * a] = v.imag();
      Rt[(size_t)(2 * r + 1) * R2 + 2 * a + 1] = v.real();
    }
  er.assign(R2, 0);
  img.assign(sh.r_bytes(), 0);
  auto put = [&](int row, int p, float v) {
    const __half h = __float2half_rn(v);
    memcpy(img.data() + tc_kmajor_offset(row, p, CHT), &h, 2);
  };
  for (int rho = 0; rho < R2; ++rho) {
    int e = INT_MIN;
    for (int k = 0; k < R2; ++k) {
      const double x = Rt[(size_t)rho * R2 + k];
      if (x != 0.0) {
        int ex;
        frexp(x, &ex);
        if (ex > e) e = ex;
      }
    }
    if (e == INT_MIN) e = 0;
    er[rho] = e;
    for (int k = 0; k < R2; ++k) {
      const double v = ldexp(Rt[(size_t)rho * R2 + k], 15 - e);
      const float vh = __half2float(__float2half_rn((float)v));
      put(rho, k, vh);
      put(rho, R2 + k, ldexpf(vh, -11));
      put(rho, 2 * R2 + k, (float)(v - (double)vh));
    }
  }
  put(R2, sh.exp_pos(), 1.f);
  return FOCK_OK;
}

size_t fock_tc_smem(int M, int xdim, int nsq, bool mixed) {
  switch (M) {
#define FOCK_TC_SMEM(MM) \
    case MM: return mixed ? tc_smem_of<TcPolMixed<MM>, MM>(xdim, nsq).total : tc_smem_of<TcPolDF<MM>, MM>(xdim, nsq).total;
    FOCK_TC_SMEM(2)
    FOCK_TC_SMEM(3)
    FOCK_TC_SMEM(4)
    FOCK_TC_SMEM(5)
    FOCK_TC_SMEM(6)
#undef FOCK_TC_SMEM
  }
  return (size_t)-1;
}

template <int M, class Pol>
static int launch_tc(const TwoPhaseArgs &t, int dev, cudaStream_t s) {
  const ApplyArgs<uint32_t> &a = t.a;
  if (t.phases & 1) {
    const size_t smem = tc_smem_of<Pol, M>(a.xdim, a.nsq).total;
    cudaError_t e = cudaFuncSetAttribute(fock_twophase_x_tc<M, Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fock_cuda_status(e);
    const uint64_t total = (uint64_t)t.nc2 * (uint64_t)a.nrhs;
    const uint64_t tiles = (total + kTcCols - 1) / kTcCols;
    uint64_t grid = (uint64_t)fock_get_sm_count(dev);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    fock_twophase_x_tc<M, Pol><<<(unsigned)grid, kTcThreads, smem, s>>>(t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fock_cuda_status(e);
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  const uint32_t n = t.g_end - t.g_begin;
  if (std::is_same<Pol, TcPolMixed<M>>::value)
    return fock_launch_grid(fock_twophase_sigma_mixed<M>, t, n, twophase_sigma_smem(a.rows, a.xdim, a.nsq), dev, s);
  return fock_launch_grid(fock_twophase_sigma_df<M>, t, n, twophase_sigma_smem(a.rows, a.xdim, a.nsq), dev, s);
}

int fock_launch_twophase_tc(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_TC_CASE(MM) \
    case MM: return mixed ? launch_tc<MM, TcPolMixed<MM>>(t, dev, s) : launch_tc<MM, TcPolDF<MM>>(t, dev, s);
    FOCK_TC_CASE(2)
    FOCK_TC_CASE(3)
    FOCK_TC_CASE(4)
    FOCK_TC_CASE(5)
    FOCK_TC_CASE(6)
#undef FOCK_TC_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}
