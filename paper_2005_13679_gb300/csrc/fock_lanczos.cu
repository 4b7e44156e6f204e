// fock_lanczos.cu -- Lanczos ground state of H (Sec. 5).
//
// Krylov vectors are complex128 in device memory.  Inside a cycle of at most
// restart_len vectors every new vector is orthogonalised against all previous
// ones of the cycle (classical Gram-Schmidt applied twice); a cycle ends with
// the Ritz vector of the lowest Ritz value, which starts the next cycle.  The
// tridiagonal eigen-problem is solved on the host: Sturm-sequence bisection for
// the lowest eigenvalue, inverse iteration for its vector.
//
// With FOCK_PREC_F32_MIXED products the solver first converges to the mixed
// floor (the apply's own error), then continues with FOCK_PREC_F64 products
// from the current Ritz vector (final FP64 refinement).  The returned energy is
// the Rayleigh quotient <v, H v> of the final unit vector with an FP64-class
// product, and the residual is || H v - E v ||.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "fock_common.cuh"

namespace {

const int kDotBlocks = 512;
const int kChunk = 8;  // vectors per fused pass

struct Coeffs {
  double2 c[kChunk];
};

// partial[b][i] = sum over this block's elements of conj(V_i[x]) w[x]
__global__ void dots_kernel(const double2 *__restrict__ V, int64_t ld, int k, int64_t n,
                            const double2 *__restrict__ w, double2 *__restrict__ partial) {
  double2 acc[kChunk];
#pragma unroll
  for (int i = 0; i < kChunk; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    const double2 wx = w[x];
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
      if (i < k) {
        const double2 v = V[i * ld + x];
        acc[i].x = fma(v.x, wx.x, fma(v.y, wx.y, acc[i].x));
        acc[i].y = fma(v.x, wx.y, fma(-v.y, wx.x, acc[i].y));
      }
  }
  __shared__ double2 red[kChunk][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < kChunk; ++i) {
    double2 a = acc[i];
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) red[i][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x < kChunk) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < nw; ++j) {
      s.x += red[threadIdx.x][j].x;
      s.y += red[threadIdx.x][j].y;
    }
    partial[(size_t)blockIdx.x * kChunk + threadIdx.x] = s;
  }
}

// w[x] = beta * w[x] - sum_i c_i V_i[x]
__global__ void combine_kernel(const double2 *__restrict__ V, int64_t ld, int k, int64_t n,
                               Coeffs c, double beta, double2 *__restrict__ w) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[x];
    acc.x *= beta;
    acc.y *= beta;
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
      if (i < k) {
        const double2 v = V[i * ld + x];
        acc.x -= c.c[i].x * v.x - c.c[i].y * v.y;
        acc.y -= c.c[i].x * v.y + c.c[i].y * v.x;
      }
    w[x] = acc;
  }
}

__global__ void scale_copy_kernel(const double2 *__restrict__ x, double s, int64_t n,
                                  double2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i] = make_double2(v.x * s, v.y * s);
  }
}

__global__ void to_c64_kernel(const double2 *__restrict__ x, int64_t n, float2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void to_c128_kernel(const float2 *__restrict__ x, int64_t n, double2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    y[i] = make_double2((double)v.x, (double)v.y);
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): x += 0x9e3779b97f4a7c15, then two
// xor-shift-multiply rounds.  Entry i uses counter 2i (real) and 2i+1 (imag),
// mapped to [-1, 1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__global__ void random_start_kernel(uint64_t seed, int64_t n, double2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed + 2 * (uint64_t)i), b = splitmix64(seed + 2 * (uint64_t)i + 1);
    y[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
  }
}

struct Ctx {
  int64_t n;
  int sms;
  cudaStream_t s;
  double2 *partial_d;
  std::vector<double2> partial_h;
  unsigned grid() const {
    int64_t g = (n + 255) / 256;
    int64_t cap = (int64_t)sms * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
  }
};

// h[i] = <V_i, w> for i < k (vectors at V + i*ld)
int dots(Ctx &c, const double2 *V, int64_t ld, int k, const double2 *w, std::vector<double2> &h) {
  h.assign(k, make_double2(0.0, 0.0));
  for (int i0 = 0; i0 < k; i0 += kChunk) {
    const int kk = k - i0 < kChunk ? k - i0 : kChunk;
    dots_kernel<<<kDotBlocks, 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, w, c.partial_d);
    FOCK_CUDA_TRY(cudaGetLastError());
    FOCK_CUDA_TRY(cudaMemcpyAsync(c.partial_h.data(), c.partial_d, sizeof(double2) * kDotBlocks * kChunk,
                                  cudaMemcpyDeviceToHost, c.s));
    FOCK_CUDA_TRY(cudaStreamSynchronize(c.s));
    for (int i = 0; i < kk; ++i) {
      double2 t = make_double2(0.0, 0.0);
      for (int b = 0; b < kDotBlocks; ++b) {
        t.x += c.partial_h[(size_t)b * kChunk + i].x;
        t.y += c.partial_h[(size_t)b * kChunk + i].y;
      }
      h[i0 + i] = t;
    }
  }
  return FOCK_OK;
}

// w = beta * w - sum_i h_i V_i
int combine(Ctx &c, const double2 *V, int64_t ld, int k, const std::vector<double2> &h, double beta,
            double2 *w) {
  if (k == 0) {
    if (beta != 1.0) {
      scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, beta, c.n, w);
      FOCK_CUDA_TRY(cudaGetLastError());
    }
    return FOCK_OK;
  }
  for (int i0 = 0; i0 < k; i0 += kChunk) {
    const int kk = k - i0 < kChunk ? k - i0 : kChunk;
    Coeffs cf;
    for (int i = 0; i < kChunk; ++i) cf.c[i] = i < kk ? h[i0 + i] : make_double2(0.0, 0.0);
    combine_kernel<<<c.grid(), 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, cf, i0 == 0 ? beta : 1.0, w);
    FOCK_CUDA_TRY(cudaGetLastError());
  }
  return FOCK_OK;
}

double norm(Ctx &c, const double2 *w, int *st) {
  std::vector<double2> h;
  *st = dots(c, w, 0, 1, w, h);
  return sqrt(fmax(h[0].x, 0.0));
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm count).
int sturm_below(const std::vector<double> &a, const std::vector<double> &b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? off / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b (b[i] couples i and i+1).
void lowest_eigenpair(const std::vector<double> &a, const std::vector<double> &b, double &theta,
                      std::vector<double> &y) {
  const size_t m = a.size();
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(a, b, mid) >= 1) hi = mid; else lo = mid;
  }
  theta = 0.5 * (lo + hi);
  // inverse iteration on (T - theta I), shifted slightly below the eigenvalue
  const double shift = theta - 1e-13 * fmax(fabs(theta), 1.0);
  y.assign(m, 1.0);
  std::vector<double> dd(m), ll(m), z(m);
  for (int it = 0; it < 3; ++it) {
    // LDL^T-free Thomas algorithm on the tridiagonal system
    std::vector<double> cp(m), rhs(y);
    double den = a[0] - shift;
    if (fabs(den) < 1e-300) den = 1e-300;
    cp[0] = m > 1 ? b[0] / den : 0.0;
    rhs[0] = rhs[0] / den;
    for (size_t i = 1; i < m; ++i) {
      den = (a[i] - shift) - b[i - 1] * cp[i - 1];
      if (fabs(den) < 1e-300) den = 1e-300;
      cp[i] = i + 1 < m ? b[i] / den : 0.0;
      rhs[i] = (rhs[i] - b[i - 1] * rhs[i - 1]) / den;
    }
    for (size_t i = m - 1; i-- > 0;) rhs[i] -= cp[i] * rhs[i + 1];
    double nr = 0.0;
    for (size_t i = 0; i < m; ++i) nr += rhs[i] * rhs[i];
    nr = sqrt(nr);
    for (size_t i = 0; i < m; ++i) y[i] = rhs[i] / nr;
  }
}

}  // namespace

extern "C" int fock_lanczos_ground(const fock_space *sp, const fock_ham *ham, int32_t max_iter,
                                   int32_t restart_len, double tol, uint64_t seed, int precision,
                                   const void *start_dev, double *E0, double *residual,
                                   void *vec_dev, int32_t *iters, void *stream) {
  if (!sp || !ham || !E0 || max_iter < 1 || restart_len < 2 || restart_len > 256 || !(tol > 0.0))
    return FOCK_ERR_ARG;
  if (precision < FOCK_PREC_F64 || precision > FOCK_PREC_F32_MIXED) return FOCK_ERR_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  if (cur != sp->device) return FOCK_ERR_DEVICE;
  Ctx c;
  c.n = sp->nc;
  c.sms = fock_get_sm_count(sp->device);
  c.s = (cudaStream_t)stream;
  c.partial_h.resize((size_t)kDotBlocks * kChunk);
  const int64_t n = c.n;
  int m = restart_len;
  if ((int64_t)m > n) m = (int)n;
  if (m < 1) m = 1;

  double2 *V = nullptr, *w = nullptr;
  float2 *c64a = nullptr, *c64b = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = fock_apply_ws_bytes(sp, ham, 1, FOCK_PREC_F64);
  int st = FOCK_OK;
  auto cleanup = [&]() {
    cudaFree(V);
    cudaFree(w);
    cudaFree(c64a);
    cudaFree(c64b);
    cudaFree(ws);
    cudaFree(c.partial_d);
  };
#define TRY(x)                  \
  do {                          \
    st = (x);                   \
    if (st) { cleanup(); return st; } \
  } while (0)
  TRY(cudaMalloc(&V, sizeof(double2) * (size_t)n * (m + 1)) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&w, sizeof(double2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&c.partial_d, sizeof(double2) * kDotBlocks * kChunk) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  if (ws_bytes) TRY(cudaMalloc(&ws, ws_bytes) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  if (precision == FOCK_PREC_F32_MIXED) {
    TRY(cudaMalloc(&c64a, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
    TRY(cudaMalloc(&c64b, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  }

  // H x -> y with the requested precision (y, x complex128)
  auto apply = [&](int prec, const double2 *x, double2 *y) -> int {
    if (prec == FOCK_PREC_F32_MIXED) {
      to_c64_kernel<<<c.grid(), 256, 0, c.s>>>(x, n, c64a);
      int r = fock_apply_internal(sp, ham, c64a, c64b, 1, prec, FOCK_ARM_HASH, nullptr, 0, c.s);
      if (r) return r;
      to_c128_kernel<<<c.grid(), 256, 0, c.s>>>(c64b, n, y);
      return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
    }
    return fock_apply_internal(sp, ham, x, y, 1, prec, FOCK_ARM_HASH, ws, ws_bytes, c.s);
  };

  // start vector
  if (start_dev) {
    TRY(cudaMemcpyAsync(V, start_dev, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
            ? FOCK_OK : FOCK_ERR_CUDA);
  } else {
    random_start_kernel<<<c.grid(), 256, 0, c.s>>>(seed, n, V);
  }
  double nv = norm(c, V, &st);
  if (st) { cleanup(); return st; }
  if (!(nv > 0.0)) { cleanup(); return FOCK_ERR_ARG; }
  scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(V, 1.0 / nv, n, V);

  const double mixed_floor = 1e-5;
  int phase_prec = precision;
  int total = 0;
  double theta = 0.0;
  bool converged = false;
  std::vector<double> alpha, beta, y;
  std::vector<double2> h, h2;
  while (true) {
    alpha.clear();
    beta.clear();
    int j = 0;
    double cur_tol = phase_prec == FOCK_PREC_F32_MIXED ? fmax(tol, mixed_floor) : tol;
    bool stop_cycle = false, phase_done = false;
    for (j = 0; j < m; ++j) {
      double2 *vj = V + (size_t)j * n;
      TRY(apply(phase_prec, vj, w));
      total += 1;
      // full re-orthogonalisation against v_0..v_j (twice); its first pass
      // also removes the alpha_j and beta_{j-1} components of the recurrence
      TRY(dots(c, V, n, j + 1, w, h));
      const double a = h[j].x;
      TRY(combine(c, V, n, j + 1, h, 1.0, w));
      TRY(dots(c, V, n, j + 1, w, h2));
      TRY(combine(c, V, n, j + 1, h2, 1.0, w));
      const double b = norm(c, w, &st);
      if (st) { cleanup(); return st; }
      alpha.push_back(a + h2[j].x);
      lowest_eigenpair(alpha, beta, theta, y);
      const double est = fabs(b * y[j]);
      if (est <= cur_tol * fmax(fabs(theta), 1.0) || b <= 1e-300 * fmax(fabs(theta), 1.0)) phase_done = true;
      if (phase_done || total >= max_iter || j == m - 1) {
        stop_cycle = true;
        break;
      }
      beta.push_back(b);
      scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, 1.0 / b, n, V + (size_t)(j + 1) * n);
    }
    (void)stop_cycle;
    // Ritz vector u = sum_i y_i v_i into w, normalised, then moved to v_0
    const int kk = (int)alpha.size();
    std::vector<double2> cy(kk);
    for (int i = 0; i < kk; ++i) cy[i] = make_double2(-y[i], 0.0);
    TRY(combine(c, V, n, kk, cy, 0.0, w));
    double nu = norm(c, w, &st);
    if (st) { cleanup(); return st; }
    scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, 1.0 / nu, n, V);
    if (phase_done) {
      if (phase_prec == FOCK_PREC_F32_MIXED && tol < mixed_floor) {
        phase_prec = FOCK_PREC_F64;  // final FP64 refinement
      } else {
        converged = true;
        break;
      }
    }
    if (total >= max_iter) break;
  }
  // Rayleigh quotient and residual with an FP64-class product
  TRY(apply(FOCK_PREC_F64, V, w));
  TRY(dots(c, V, n, 1, w, h));
  const double E = h[0].x;
  std::vector<double2> e1(1, make_double2(E, 0.0));
  TRY(combine(c, V, n, 1, e1, 1.0, w));
  const double res = norm(c, w, &st);
  if (st) { cleanup(); return st; }
  if (vec_dev)
    TRY(cudaMemcpyAsync(vec_dev, V, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
            ? FOCK_OK : FOCK_ERR_CUDA);
  TRY(cudaStreamSynchronize(c.s) == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA);
  *E0 = E;
  if (residual) *residual = res;
  if (iters) *iters = total;
  cleanup();
#undef TRY
  return converged ? FOCK_OK : FOCK_ERR_NOCONV;
}
