// fock_twophase_tc.cu -- the two-phase apply with its phase 1 on the tensor
// cores (fock_apply_tc.cuh), M = 2..6: host construction of the digit image
// of R, launch of phase 1 and of the FP32-pair phase 2.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <complex>
#include <type_traits>
#include <vector>

#include "fock_apply_tc.cuh"

// Digit image of the real form of R (P x P complex, row r = removal pair,
// column a = addition pair, already divided by the coefficient scale):
// rows 2r, 2r+1 are (Re, Im) of Y_r, columns 2a, 2a+1 multiply (Re, Im) of X_a.
// Each real row rho gets e_rho with |R~[rho][k]| < 2^e_rho for all k and six
// base-2^9 digits of R~ 2^(8 - e_rho), computed exactly in FP64.  The image is
// the MMA's B operand in tensor-core shared-memory layout (K-major), in two
// parts: part 1 has N1 rows (tensor-memory columns, TcShape::col) by K1
// positions 3k + (j - 1) for X digits j = 1..3, plus the exponent row, which
// copies the column exponent stored at K position exp_pos(); part 2 has N2
// rows (levels 5..7) by K2 positions 2k + (j - 4) for X digits j = 4, 5.  The
// entry of row (rho, level l) at (k, j) is digit i = l - j of R~[rho][k]
// (zero when i is outside 1..6).
int fock_tc_image(int M, const std::complex<double> *R, std::vector<unsigned char> &img, std::vector<int> &er) {
  if (M < 2 || M > 6) return FOCK_ERR_UNSUPPORTED;
  const TcShape sh(M);
  const int P = sh.P, R2 = sh.R2;
  constexpr int kDig = 6;
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
  std::vector<float> dig((size_t)R2 * R2 * kDig, 0.f);
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
      for (int i = 0; i < kDig; ++i) {
        const double d = nearbyint(v);
        dig[((size_t)rho * R2 + k) * kDig + i] = (float)d;
        v = (v - d) * 512.0;
      }
    }
  }
  img.assign(sh.r_bytes(), 0);
  unsigned char *part2 = img.data() + sh.r1_bytes();
  const int ch1 = sh.K1 / 8, ch2 = sh.K2 / 8;
  auto put = [&](unsigned char *base, int row, int p, int chunks, float v) {
    const __half h = __float2half(v);
    memcpy(base + tc_kmajor_offset(row, p, chunks), &h, 2);
  };
  for (int rho = 0; rho < R2; ++rho)
    for (int level = 2; level <= 7; ++level) {
      const int row = sh.col(rho, level);
      for (int k = 0; k < R2; ++k) {
        for (int j = 1; j <= 5; ++j) {
          const int i = level - j;
          if (i < 1 || i > kDig) continue;
          const float d = dig[((size_t)rho * R2 + k) * kDig + (i - 1)];
          if (j <= 3)
            put(img.data(), row, 3 * k + (j - 1), ch1, d);
          else if (level >= 5)
            put(part2, row, 2 * k + (j - 4), ch2, d);
        }
      }
    }
  put(img.data(), sh.exp_col(), sh.exp_pos(), ch1, 1.f);
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

// Poll budget of the bounded waits inside phase 1 (producers, MMA issue,
// epilogue).  The default is kTcPolls (about a second); fock_debug_set_wait_polls
// lowers it so that tests can make the waits give up.  The wait that lets
// committed MMAs finish before tensor memory is freed always keeps kTcPolls.
static std::atomic<uint32_t> g_tc_polls{kTcPolls};

extern "C" int fock_debug_set_wait_polls(int64_t polls) {
  if (polls > (int64_t)kTcPolls) return FOCK_ERR_ARG;
  g_tc_polls.store(polls < 0 ? kTcPolls : (uint32_t)polls);
  return FOCK_OK;
}

template <int M, class Pol>
static int launch_tc(const TwoPhaseArgs &targ, int dev, cudaStream_t s) {
  TwoPhaseArgs t = targ;
  t.polls = g_tc_polls.load();
  const ApplyArgs<uint32_t> &a = t.a;
  if (t.phases & 1) {
    const size_t smem = tc_smem_of<Pol, M>(a.xdim, a.nsq).total;
    cudaError_t e = cudaFuncSetAttribute(fock_twophase_x_tc<M, Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fock_cuda_status(e);
    const uint64_t tiles = (t.c_end + kTcCols - 1) / kTcCols - t.c_begin / kTcCols;
    uint64_t grid = (uint64_t)fock_get_sm_count(dev);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    fock_twophase_x_tc<M, Pol><<<(unsigned)grid, kTcThreads, smem, s>>>(t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fock_cuda_status(e);
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  const uint64_t n = (uint64_t)(t.g_end - t.g_begin) * a.nrhs;
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
