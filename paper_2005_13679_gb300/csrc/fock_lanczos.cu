// fock_lanczos.cu -- Lanczos ground state of H (Sec. 6).
//
// Krylov vectors are complex128 in device memory.  Inside a cycle of at most
// restart_len vectors every new vector is orthogonalised against all previous
// ones of the cycle (classical Gram-Schmidt applied twice, the complete
// re-orthogonalisation of Sec. 6); a cycle ends with a thick restart that keeps
// the lowest Ritz vectors.  The small projected eigen-problem is solved on the
// host by Jacobi rotations.
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

// partial[b][i] = sum over this block's elements of conj(V_i[x]) w[x].  With
// REAL the vectors have zero imaginary parts and only real parts are combined.
template <bool REAL>
__global__ void dots_kernel(const double2 *__restrict__ V, int64_t ld, int k, int64_t n,
                            const double2 *__restrict__ w, double2 *__restrict__ partial) {
  double2 acc[kChunk];
#pragma unroll
  for (int i = 0; i < kChunk; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (REAL) {
      const double wx = w[x].x;
#pragma unroll
      for (int i = 0; i < kChunk; ++i)
        if (i < k) acc[i].x = fma(V[i * ld + x].x, wx, acc[i].x);
    } else {
      const double2 wx = w[x];
#pragma unroll
      for (int i = 0; i < kChunk; ++i)
        if (i < k) {
          const double2 v = V[i * ld + x];
          acc[i].x = fma(v.x, wx.x, fma(v.y, wx.y, acc[i].x));
          acc[i].y = fma(v.x, wx.y, fma(-v.y, wx.x, acc[i].y));
        }
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

// w[x] = beta * w[x] - sum_i c_i V_i[x]  (REAL: real parts only; imaginary
// parts stay exactly zero)
template <bool REAL>
__global__ void combine_kernel(const double2 *__restrict__ V, int64_t ld, int k, int64_t n,
                               Coeffs c, double beta, double2 *__restrict__ w) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (REAL) {
      double acc = beta == 0.0 ? 0.0 : w[x].x * beta;   // beta = 0: w is write-only
#pragma unroll
      for (int i = 0; i < kChunk; ++i)
        if (i < k) acc = fma(-c.c[i].x, V[i * ld + x].x, acc);
      w[x] = make_double2(acc, 0.0);
    } else {
      double2 acc = make_double2(0.0, 0.0);
      if (beta != 0.0) {
        acc = w[x];
        acc.x *= beta;
        acc.y *= beta;
      }
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

__global__ void random_start_kernel(uint64_t seed, int64_t n, bool real, double2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed + 2 * (uint64_t)i), b = splitmix64(seed + 2 * (uint64_t)i + 1);
    y[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, real ? 0.0 : (double)(b >> 11) * 0x1.0p-52 - 1.0);
  }
}

struct Ctx {
  int64_t n;
  bool real;
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
    if (c.real) dots_kernel<true><<<kDotBlocks, 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, w, c.partial_d);
    else dots_kernel<false><<<kDotBlocks, 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, w, c.partial_d);
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
    if (c.real) combine_kernel<true><<<c.grid(), 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, cf, i0 == 0 ? beta : 1.0, w);
    else combine_kernel<false><<<c.grid(), 256, 0, c.s>>>(V + (size_t)i0 * ld, ld, kk, c.n, cf, i0 == 0 ? beta : 1.0, w);
    FOCK_CUDA_TRY(cudaGetLastError());
  }
  return FOCK_OK;
}

double norm(Ctx &c, const double2 *w, int *st) {
  std::vector<double2> h;
  *st = dots(c, w, 0, 1, w, h);
  return sqrt(fmax(h[0].x, 0.0));
}

// Eigen-decomposition of a small dense symmetric matrix A (n x n, row-major)
// by cyclic Jacobi rotations: each rotation zeroes one off-diagonal pair,
// the sweeps repeat until the off-diagonal norm is negligible.  On return
// evals[i] ascending and evecs[i*n + k] = component k of eigenvector i.
void jacobi_eigen(std::vector<double> A, int n, std::vector<double> &evals, std::vector<double> &evecs) {
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // accumulate Q = Q R
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - sn * qkq;
          Q[(size_t)k * n + q] = sn * qkp + c * qkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && A[(size_t)order[j - 1] * n + order[j - 1]] > A[(size_t)order[j] * n + order[j]]; --j) {
      int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
    }
  evals.resize(n);
  evecs.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    evals[i] = A[(size_t)order[i] * n + order[i]];
    for (int k = 0; k < n; ++k) evecs[(size_t)i * n + k] = Q[(size_t)k * n + order[i]];
  }
}

}  // namespace

// Thick-restart Lanczos over vectors of n complex128 entries; `apply` computes
// H x -> y in the requested precision on the stream (x, y device vectors of
// the precision's storage type, ws a workspace of ws_bytes).
int fock_lanczos_run(int64_t n_vec, bool ham_real, int device, const FockApplyFn &apply_fn, size_t ws_bytes,
                     size_t ws_min, int32_t max_iter, int32_t restart_len, double tol, uint64_t seed, int precision,
                     const void *start_dev, double *E0, double *residual, void *vec_dev, int32_t *iters,
                     cudaStream_t stream) {
  if (!E0 || max_iter < 1 || restart_len < 2 || restart_len > 256 || !(tol > 0.0) || n_vec < 1)
    return FOCK_ERR_ARG;
  if (precision < FOCK_PREC_F64 || precision > FOCK_PREC_F32_MIXED) return FOCK_ERR_ARG;
  Ctx c;
  c.n = n_vec;
  // A real Hamiltonian keeps a real start vector real: every product and every
  // Gram-Schmidt step then has zero imaginary parts, which are skipped.
  c.real = ham_real && start_dev == nullptr;
  c.sms = fock_get_sm_count(device);
  c.s = stream;
  c.partial_h.resize((size_t)kDotBlocks * kChunk);
  const int64_t n = c.n;
  int m = restart_len;
  if ((int64_t)m > n) m = (int)n;
  if (m < 1) m = 1;

  double2 *V = nullptr, *w = nullptr;
  float2 *c64a = nullptr, *c64b = nullptr;
  void *ws = nullptr;
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
  TRY(cudaMalloc(&V, sizeof(double2) * (size_t)n * (m + 8)) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&w, sizeof(double2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&c.partial_d, sizeof(double2) * kDotBlocks * kChunk) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  if (precision == FOCK_PREC_F32_MIXED) {
    TRY(cudaMalloc(&c64a, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
    TRY(cudaMalloc(&c64b, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  }
  // the preferred workspace (it selects the fastest path), else the minimum
  if (ws_bytes && cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    ws = nullptr;
    ws_bytes = ws_min;
    if (ws_bytes) TRY(cudaMalloc(&ws, ws_bytes) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  }

  // H x -> y with the requested precision (y, x complex128)
  auto apply = [&](int prec, const double2 *x, double2 *y) -> int {
    if (prec == FOCK_PREC_F32_MIXED) {
      to_c64_kernel<<<c.grid(), 256, 0, c.s>>>(x, n, c64a);
      int r = apply_fn(prec, c64a, c64b, ws, ws_bytes, c.s);
      if (r) return r;
      to_c128_kernel<<<c.grid(), 256, 0, c.s>>>(c64b, n, y);
      return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
    }
    return apply_fn(prec, x, y, ws, ws_bytes, c.s);
  };

  // start vector
  if (start_dev) {
    TRY(cudaMemcpyAsync(V, start_dev, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
            ? FOCK_OK : FOCK_ERR_CUDA);
  } else {
    random_start_kernel<<<c.grid(), 256, 0, c.s>>>(seed, n, c.real, V);
  }
  double nv = norm(c, V, &st);
  if (st) { cleanup(); return st; }
  if (!(nv > 0.0)) { cleanup(); return FOCK_ERR_ARG; }
  scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(V, 1.0 / nv, n, V);

  // Thick restart (Wu and Simon): a cycle grows the basis V[0..j] of at most m
  // vectors; at restart the `keep` lowest Ritz vectors and the last residual
  // direction start the next cycle, with the projected matrix
  //     T = [ diag(theta_i)  s ;  s^T  alpha ... ]  (arrowhead, then tridiagonal).
  const double mixed_floor = 1e-5;
  const int keep = m >= 6 ? (m / 3 < 8 ? m / 3 : 8) : 1;
  int phase_prec = precision;
  int total = 0, p = 0;   // p: Ritz vectors carried into the cycle (V[0..p-1]), V[p] = residual
  double theta = 0.0;
  bool converged = false;
  std::vector<double> T((size_t)m * m, 0.0), evals, evecs;
  std::vector<double2> h, h2;
  while (true) {
    const double cur_tol = phase_prec == FOCK_PREC_F32_MIXED ? fmax(tol, mixed_floor) : tol;
    bool phase_done = false;
    int j = p, dim = 0;
    double b = 0.0;
    for (j = p; j < m; ++j) {
      double2 *vj = V + (size_t)j * n;
      TRY(apply(phase_prec, vj, w));
      total += 1;
      // full re-orthogonalisation against v_0..v_j (twice)
      TRY(dots(c, V, n, j + 1, w, h));
      TRY(combine(c, V, n, j + 1, h, 1.0, w));
      TRY(dots(c, V, n, j + 1, w, h2));
      TRY(combine(c, V, n, j + 1, h2, 1.0, w));
      b = norm(c, w, &st);
      if (st) { cleanup(); return st; }
      T[(size_t)j * m + j] = h[j].x + h2[j].x;
      dim = j + 1;
      std::vector<double> Tj((size_t)dim * dim);
      for (int r = 0; r < dim; ++r)
        for (int q = 0; q < dim; ++q) Tj[(size_t)r * dim + q] = T[(size_t)r * m + q];
      jacobi_eigen(Tj, dim, evals, evecs);
      theta = evals[0];
      const double est = fabs(b * evecs[(size_t)0 * dim + j]);
      if (est <= cur_tol * fmax(fabs(theta), 1.0) || b <= 1e-300 * fmax(fabs(theta), 1.0)) phase_done = true;
      if (phase_done || total >= max_iter || j == m - 1) break;
      T[(size_t)(j + 1) * m + j] = T[(size_t)j * m + j + 1] = b;
      scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, 1.0 / b, n, V + (size_t)(j + 1) * n);
    }
    const bool switch_phase = phase_done && phase_prec == FOCK_PREC_F32_MIXED && tol < mixed_floor;
    const int np = (phase_done || total >= max_iter || switch_phase) ? 1 : (keep < dim ? keep : dim);
    // Ritz vectors u_i = sum_k y_i[k] v_k into the spare slots V[m..], then V[0..np-1]
    for (int i = 0; i < np; ++i) {
      std::vector<double2> cy(dim);
      for (int k = 0; k < dim; ++k) cy[k] = make_double2(-evecs[(size_t)i * dim + k], 0.0);
      TRY(combine(c, V, n, dim, cy, 0.0, V + (size_t)(m + i) * n));
    }
    for (int i = 0; i < np; ++i)
      TRY(cudaMemcpyAsync(V + (size_t)i * n, V + (size_t)(m + i) * n, sizeof(double2) * n,
                          cudaMemcpyDeviceToDevice, c.s) == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA);
    if (phase_done && !switch_phase) { converged = true; break; }
    if (total >= max_iter) break;
    std::fill(T.begin(), T.end(), 0.0);
    if (switch_phase) {
      phase_prec = FOCK_PREC_F64;  // final FP64 refinement from the current Ritz vector
      p = 0;
      continue;
    }
    // keep np Ritz pairs and the residual direction w / b
    for (int i = 0; i < np; ++i) {
      T[(size_t)i * m + i] = evals[i];
      const double si = b * evecs[(size_t)i * dim + (dim - 1)];
      T[(size_t)i * m + np] = T[(size_t)np * m + i] = si;
    }
    scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, 1.0 / b, n, V + (size_t)np * n);
    p = np;
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

extern "C" int fock_lanczos_ground(const fock_space *sp, const fock_ham *ham, int32_t max_iter,
                                   int32_t restart_len, double tol, uint64_t seed, int precision,
                                   const void *start_dev, double *E0, double *residual,
                                   void *vec_dev, int32_t *iters, void *stream) {
  if (!sp || !ham || ham->sp != sp) return FOCK_ERR_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  if (cur != sp->device) return FOCK_ERR_DEVICE;
  FockApplyFn apply = [sp, ham](int prec, const void *x, void *y, void *ws, size_t ws_bytes, cudaStream_t s) {
    return fock_apply_internal(sp, ham, x, y, 1, prec, FOCK_ARM_HASH, ws, ws_bytes, s);
  };
  return fock_lanczos_run(sp->nc, ham->real, sp->device, apply, fock_apply_ws_pref(sp, ham, 1, FOCK_PREC_F64),
                          fock_apply_ws_bytes(sp, ham, 1, FOCK_PREC_F64), max_iter, restart_len, tol, seed, precision, start_dev, E0, residual, vec_dev, iters,
                          (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Short-iterative-Lanczos time step (the consumer of H C named in Sec. 2):
// C <- exp(-i H dt) C by the Krylov space of C.  With v_0 = C / ||C|| and the
// Lanczos vectors v_0 .. v_{m-1} (every new vector orthogonalised twice
// against all previous ones), T = V^H H V is tridiagonal and
//     exp(-i H dt) C ~ ||C|| V exp(-i T dt) e_0.
// exp(-i T dt) e_0 comes from the Jacobi eigen-decomposition of T.  The
// Krylov space grows until the weight of the next vector, beta_{m-1} times
// the last component of exp(-i T dt) e_0, falls below tol (relative to
// ||C||), the space is invariant, or max_krylov vectors are used.
// ---------------------------------------------------------------------------
extern "C" int fock_sil_step(const fock_space *sp, const fock_ham *ham, void *C_dev, double dt,
                             int32_t max_krylov, double tol, int precision, int32_t *krylov_used,
                             double *err_est, void *stream) {
  if (!sp || !ham || !C_dev || max_krylov < 1 || max_krylov > 128 || !(tol > 0.0) || !isfinite(dt))
    return FOCK_ERR_ARG;
  if (precision < FOCK_PREC_F64 || precision > FOCK_PREC_F32_MIXED) return FOCK_ERR_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  if (cur != sp->device) return FOCK_ERR_DEVICE;
  Ctx c;
  c.n = sp->nc;
  c.real = false;                 // exp(-i H dt) makes any vector complex
  c.sms = fock_get_sm_count(sp->device);
  c.s = (cudaStream_t)stream;
  c.partial_h.resize((size_t)kDotBlocks * kChunk);
  const int64_t n = c.n;
  int K = max_krylov;
  if ((int64_t)K > n) K = (int)n;

  double2 *V = nullptr, *w = nullptr;
  float2 *c64a = nullptr, *c64b = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = fock_apply_ws_pref(sp, ham, 1, precision);
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
  TRY(cudaMalloc(&V, sizeof(double2) * (size_t)n * K) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&w, sizeof(double2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  TRY(cudaMalloc(&c.partial_d, sizeof(double2) * kDotBlocks * kChunk) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  if (ws_bytes && cudaMalloc(&ws, ws_bytes) != cudaSuccess) {   // preferred, else minimum workspace
    cudaGetLastError();
    ws = nullptr;
    ws_bytes = fock_apply_ws_bytes(sp, ham, 1, precision);
    if (ws_bytes) TRY(cudaMalloc(&ws, ws_bytes) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  }
  if (precision == FOCK_PREC_F32_MIXED) {
    TRY(cudaMalloc(&c64a, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
    TRY(cudaMalloc(&c64b, sizeof(float2) * (size_t)n) == cudaSuccess ? FOCK_OK : FOCK_ERR_NOMEM);
  }
  auto apply = [&](const double2 *x, double2 *y) -> int {
    if (precision == FOCK_PREC_F32_MIXED) {
      to_c64_kernel<<<c.grid(), 256, 0, c.s>>>(x, n, c64a);
      int r = fock_apply_internal(sp, ham, c64a, c64b, 1, precision, FOCK_ARM_HASH, ws, ws_bytes, c.s);
      if (r) return r;
      to_c128_kernel<<<c.grid(), 256, 0, c.s>>>(c64b, n, y);
      return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
    }
    return fock_apply_internal(sp, ham, x, y, 1, precision, FOCK_ARM_HASH, ws, ws_bytes, c.s);
  };

  const double beta0 = norm(c, (const double2 *)C_dev, &st);
  if (st) { cleanup(); return st; }
  if (krylov_used) *krylov_used = 0;
  if (err_est) *err_est = 0.0;
  if (beta0 == 0.0) {
    cleanup();
    return FOCK_OK;
  }
  scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>((const double2 *)C_dev, 1.0 / beta0, n, V);
  TRY(cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA);
  std::vector<double> alpha, beta;
  std::vector<double> cre, cim;                       // exp(-i T dt) e_0
  std::vector<double2> h, h2;
  double err = 0.0;
  int m = 0;
  for (int j = 0; j < K; ++j) {
    double2 *vj = V + (size_t)j * n;
    TRY(apply(vj, w));
    TRY(dots(c, V, n, j + 1, w, h));
    TRY(combine(c, V, n, j + 1, h, 1.0, w));
    TRY(dots(c, V, n, j + 1, w, h2));                  // second Gram-Schmidt pass
    TRY(combine(c, V, n, j + 1, h2, 1.0, w));
    alpha.push_back(h[j].x + h2[j].x);
    const double b = norm(c, w, &st);
    if (st) { cleanup(); return st; }
    m = j + 1;
    // exp(-i T dt) e_0 for the current m x m tridiagonal T
    std::vector<double> T((size_t)m * m, 0.0), evals, evecs;
    for (int i = 0; i < m; ++i) T[(size_t)i * m + i] = alpha[i];
    for (int i = 0; i + 1 < m; ++i) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = beta[i];
    jacobi_eigen(T, m, evals, evecs);
    cre.assign(m, 0.0);
    cim.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
      const double ph = -evals[i] * dt, w0 = evecs[(size_t)i * m + 0];
      for (int k = 0; k < m; ++k) {
        const double q = evecs[(size_t)i * m + k] * w0;
        cre[k] += q * cos(ph);
        cim[k] += q * sin(ph);
      }
    }
    err = b * hypot(cre[m - 1], cim[m - 1]);
    if (err < tol || b <= 1e-14 * fabs(alpha[0]) || b == 0.0 || m == K) break;
    beta.push_back(b);
    scale_copy_kernel<<<c.grid(), 256, 0, c.s>>>(w, 1.0 / b, n, V + (size_t)(j + 1) * n);
    TRY(cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA);
  }
  // C = beta0 sum_k c_k v_k  (combine computes w = 0 w - sum h_k v_k)
  std::vector<double2> coef(m);
  for (int k = 0; k < m; ++k) coef[k] = make_double2(-beta0 * cre[k], -beta0 * cim[k]);
  TRY(combine(c, V, n, m, coef, 0.0, (double2 *)C_dev));
  TRY(cudaStreamSynchronize(c.s) == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA);
  if (krylov_used) *krylov_used = m;
  if (err_est) *err_est = err;
  cleanup();
#undef TRY
  return err < tol ? FOCK_OK : FOCK_ERR_NOCONV;
}
