// fock_space.cu -- configuration space, hash kernels and jump-map builders.
//
//   Eq. nc        N_c(N, M) = C(N + M - 1, M - 1)            -> fock_space_create
//   Algorithm 1   configuration -> index                      -> fock_rank
//   Algorithm 2   index -> configuration                      -> fock_unrank
//   Sec. 4        single / double jump maps (Fig. 4)          -> fock_build_jump_maps
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "fock_common.cuh"
#include "fock_device.cuh"

extern "C" const char *fock_strerror(int status) {
  switch (status) {
    case FOCK_OK: return "ok";
    case FOCK_ERR_ARG: return "invalid argument";
    case FOCK_ERR_OVERFLOW: return "configuration count does not fit in int64";
    case FOCK_ERR_INVALID_CONFIG: return "occupation vector is not a configuration of the space";
    case FOCK_ERR_RANGE: return "configuration index out of range";
    case FOCK_ERR_NOMEM: return "device memory exhausted or request does not fit";
    case FOCK_ERR_NOT_HERMITIAN: return "one- or two-body operator is not Hermitian";
    case FOCK_ERR_ALIAS: return "input and output buffers overlap";
    case FOCK_ERR_CUDA: return "CUDA runtime error";
    case FOCK_ERR_NOCONV: return "Lanczos did not reach the tolerance";
    case FOCK_ERR_UNSUPPORTED: return "unsupported combination of options";
    case FOCK_ERR_TIMEOUT: return "bounded device wait expired";
    case FOCK_ERR_NOT_BUILT: return "jump maps not built";
    case FOCK_ERR_DEVICE: return "object belongs to another device";
    case FOCK_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch of the no-allocation entry point";
    case FOCK_ERR_NOT_CONSERVING: return "operator changes the total orbital weight of the sector";
    default: return "unknown status";
  }
}

extern "C" int fock_version(void) { return 100; }

int fock_get_sm_count(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 1;
  return n;
}

// C(n + m - 1, m - 1) exactly, -1 if it does not fit in int64.
static int64_t host_count(int64_t n, int64_t m) {
  if (m <= 0 || n < 0) return 0;
  unsigned __int128 r = 1;
  for (int64_t i = 1; i <= m - 1; ++i) {
    r = r * (unsigned __int128)(n + i) / (unsigned __int128)i;
    if (r > (unsigned __int128)INT64_MAX) return -1;
  }
  return (int64_t)r;
}

static int check_device(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  return cur == dev ? FOCK_OK : FOCK_ERR_DEVICE;
}

static void free_tables(FockTables &t) {
  cudaFree(t.mod64);
  cudaFree(t.sat64);
  cudaFree(t.mod32);
  cudaFree(t.sat32);
  t.mod64 = t.sat64 = nullptr;
  t.mod32 = t.sat32 = nullptr;
}

// Pascal's rule row by row: C(x, j) = C(x-1, j-1) + C(x-1, j), wrapping (mod)
// and saturating (sat) additions.
static int build_tables(int N, int M, FockTables &t) {
  t.rows = M > 1 ? M - 1 : 1;
  t.xdim = N + M + 3;
  const int jmax = t.rows;  // largest lower index C(x, j) needed is j = M - 1
  std::vector<uint64_t> pm((size_t)(jmax + 1) * t.xdim, 0), ps((size_t)(jmax + 1) * t.xdim, 0);
  for (int x = 0; x < t.xdim; ++x) {
    pm[(size_t)x] = 1;
    ps[(size_t)x] = 1;  // C(x, 0) = 1
  }
  for (int j = 1; j <= jmax; ++j) {
    for (int x = 1; x < t.xdim; ++x) {
      size_t a = (size_t)(j - 1) * t.xdim + (x - 1), b = (size_t)j * t.xdim + (x - 1);
      pm[(size_t)j * t.xdim + x] = pm[a] + pm[b];
      uint64_t s = ps[a] + ps[b];
      ps[(size_t)j * t.xdim + x] = (s < ps[a]) ? UINT64_MAX : s;
    }
  }
  size_t n = (size_t)t.rows * t.xdim;
  std::vector<uint64_t> m64(n, 0), s64(n, 0);
  std::vector<uint32_t> m32(n, 0), s32(n, 0);
  for (int m = 0; m < t.rows; ++m)
    for (int x = 0; x < t.xdim; ++x) {
      size_t src = (size_t)(m + 1) * t.xdim + x, dst = (size_t)m * t.xdim + x;
      if (M == 1) {
        m64[dst] = s64[dst] = 0;
      } else {
        m64[dst] = pm[src];
        s64[dst] = ps[src];
      }
      m32[dst] = (uint32_t)(m64[dst] & 0xffffffffu);
      s32[dst] = s64[dst] > 0xffffffffull ? 0xffffffffu : (uint32_t)s64[dst];
    }
  FOCK_CUDA_TRY(cudaMalloc(&t.mod64, n * 8));
  FOCK_CUDA_TRY(cudaMalloc(&t.sat64, n * 8));
  FOCK_CUDA_TRY(cudaMalloc(&t.mod32, n * 4));
  FOCK_CUDA_TRY(cudaMalloc(&t.sat32, n * 4));
  FOCK_CUDA_TRY(cudaMemcpy(t.mod64, m64.data(), n * 8, cudaMemcpyHostToDevice));
  FOCK_CUDA_TRY(cudaMemcpy(t.sat64, s64.data(), n * 8, cudaMemcpyHostToDevice));
  FOCK_CUDA_TRY(cudaMemcpy(t.mod32, m32.data(), n * 4, cudaMemcpyHostToDevice));
  FOCK_CUDA_TRY(cudaMemcpy(t.sat32, s32.data(), n * 4, cudaMemcpyHostToDevice));
  return FOCK_OK;
}

extern "C" int fock_space_create(int32_t N, int32_t M, fock_space **out) {
  if (!out || N < 1 || M < 1 || M > FOCK_MAXM) return FOCK_ERR_ARG;
  int64_t nc = host_count(N, M);
  if (nc < 0) return FOCK_ERR_OVERFLOW;
  fock_space *sp = (fock_space *)calloc(1, sizeof(fock_space));
  if (!sp) return FOCK_ERR_NOMEM;
  sp->N = N;
  sp->M = M;
  sp->nc = nc;
  if (cudaGetDevice(&sp->device) != cudaSuccess) {
    free(sp);
    return FOCK_ERR_CUDA;
  }
  sp->idx32 = nc < (int64_t)0xffffffffll;
  int st;
  try {                                  // no C++ exception crosses the C ABI
    st = build_tables(N, M, sp->tab);
  } catch (const std::bad_alloc &) {
    st = FOCK_ERR_NOMEM;
  }
  if (st == FOCK_OK && cudaMalloc(&sp->d_flag, 256) != cudaSuccess) st = FOCK_ERR_NOMEM;
  if (st != FOCK_OK) {
    free_tables(sp->tab);
    cudaFree(sp->d_flag);
    free(sp);
    return st;
  }
  // Resolve the no-alloc scratch array on this device now (loading its module
  // under lazy loading), so that fock_apply_H_noalloc never has to.  A failure
  // here is not an error of the space; that entry point retries and reports it.
  void *scratch = nullptr;
  fock_noalloc_scratch(sp->device, &scratch);
  *out = sp;
  return FOCK_OK;
}

extern "C" int fock_jump_maps_free(fock_space *sp) {
  if (!sp) return FOCK_ERR_ARG;
  cudaFree(sp->d_j1);
  cudaFree(sp->d_j2);
  sp->d_j1 = sp->d_j2 = nullptr;
  sp->j1_bytes = sp->j2_bytes = 0;
  return FOCK_OK;
}

extern "C" int fock_space_destroy(fock_space *sp) {
  if (!sp) return FOCK_OK;
  fock_jump_maps_free(sp);
  cudaFree(sp->dm_ws);
  cudaFree(sp->dm_part);
  free_tables(sp->tab);
  cudaFree(sp->d_flag);
  free(sp);
  return FOCK_OK;
}

extern "C" int fock_space_size(const fock_space *sp, int64_t *nc) {
  if (!sp || !nc) return FOCK_ERR_ARG;
  *nc = sp->nc;
  return FOCK_OK;
}

// ---------------------------------------------------------------------------
// rank / unrank
// ---------------------------------------------------------------------------
__global__ void fock_rank_kernel(int N, int M, int64_t nc, const uint64_t *__restrict__ mod,
                                 int xdim, const int32_t *__restrict__ occ, int64_t count,
                                 int64_t *__restrict__ idx, uint32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *o = occ + i * M;
    int S[FOCK_MAXM];
    int run = 0;
    bool ok = true;
#pragma unroll
    for (int m = 0; m < FOCK_MAXM; ++m) {
      if (m < M) {
        int v = o[m];
        ok = ok && v >= 0 && v <= N;
        run += (v >= 0 && v <= N) ? v : 0;
        S[m] = run > N ? N : run;
      } else {
        S[m] = N;
      }
    }
    ok = ok && run == N;
    if (!ok) {
      idx[i] = -1;
      atomicOr(flag, FOCK_DEVFLAG_INVALID);
      continue;
    }
    idx[i] = (int64_t)fock_rank_prefix<uint64_t, FOCK_MAXM>(S, M, (uint64_t)nc, mod, xdim);
  }
}

__global__ void fock_unrank_kernel(int N, int M, int64_t nc, const uint64_t *__restrict__ sat,
                                   int xdim, const int64_t *__restrict__ idx, int64_t count,
                                   int32_t *__restrict__ occ, uint32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = idx[i];
    int32_t *o = occ + i * M;
    if (g < 0 || g >= nc) {
      for (int m = 0; m < M; ++m) o[m] = -1;
      atomicOr(flag, FOCK_DEVFLAG_RANGE);
      continue;
    }
    int S[FOCK_MAXM];
    fock_decode_prefix<uint64_t, FOCK_MAXM>((uint64_t)g, N, M, (uint64_t)nc, sat, xdim, S);
    int prev = 0;
#pragma unroll
    for (int m = 0; m < FOCK_MAXM; ++m)
      if (m < M) {
        o[m] = S[m] - prev;
        prev = S[m];
      }
  }
}

static unsigned grid_for(int64_t count, int threads, int device) {
  int64_t blocks = (count + threads - 1) / threads;
  int64_t cap = (int64_t)fock_get_sm_count(device) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

static int run_checked(const fock_space *sp, cudaStream_t st, uint32_t mask, int err) {
  uint32_t flag = 0;
  FOCK_CUDA_TRY(cudaGetLastError());
  FOCK_CUDA_TRY(cudaMemcpyAsync(&flag, sp->d_flag, 4, cudaMemcpyDeviceToHost, st));
  FOCK_CUDA_TRY(cudaStreamSynchronize(st));
  return (flag & mask) ? err : FOCK_OK;
}

extern "C" int fock_rank(const fock_space *sp, const int32_t *occ_dev, int64_t count,
                         int64_t *idx_dev, void *stream) {
  if (!sp || count < 0 || (count > 0 && (!occ_dev || !idx_dev))) return FOCK_ERR_ARG;
  int st = check_device(sp->device);
  if (st) return st;
  if (count == 0) return FOCK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  FOCK_CUDA_TRY(cudaMemsetAsync(sp->d_flag, 0, 4, s));
  fock_rank_kernel<<<grid_for(count, 256, sp->device), 256, 0, s>>>(
      sp->N, sp->M, sp->nc, sp->tab.mod64, sp->tab.xdim, occ_dev, count, idx_dev, sp->d_flag);
  return run_checked(sp, s, FOCK_DEVFLAG_INVALID, FOCK_ERR_INVALID_CONFIG);
}

extern "C" int fock_unrank(const fock_space *sp, const int64_t *idx_dev, int64_t count,
                           int32_t *occ_dev, void *stream) {
  if (!sp || count < 0 || (count > 0 && (!occ_dev || !idx_dev))) return FOCK_ERR_ARG;
  int st = check_device(sp->device);
  if (st) return st;
  if (count == 0) return FOCK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  FOCK_CUDA_TRY(cudaMemsetAsync(sp->d_flag, 0, 4, s));
  fock_unrank_kernel<<<grid_for(count, 256, sp->device), 256, 0, s>>>(
      sp->N, sp->M, sp->nc, sp->tab.sat64, sp->tab.xdim, idx_dev, count, occ_dev, sp->d_flag);
  return run_checked(sp, s, FOCK_DEVFLAG_RANGE, FOCK_ERR_RANGE);
}

// ---------------------------------------------------------------------------
// Jump maps (Sec. 4).  One thread per configuration; every slot is written
// for every configuration, so consecutive threads write consecutive words.
// ---------------------------------------------------------------------------
__global__ void fock_single_map_kernel(int N, int M, int64_t nc, const uint64_t *__restrict__ sat,
                                       const uint64_t *__restrict__ mod, int xdim,
                                       int32_t *__restrict__ J1) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
       g += (int64_t)gridDim.x * blockDim.x) {
    int S[FOCK_MAXM];
    fock_decode_prefix<uint64_t, FOCK_MAXM>((uint64_t)g, N, M, (uint64_t)nc, sat, xdim, S);
    for (int k = 0; k < M; ++k) {
      int nk = S[k] - (k > 0 ? S[k - 1] : 0);
      for (int l = 0; l < M; ++l) {
        int32_t v = -1;
        if (nk >= 1) {
          int T[FOCK_MAXM];
#pragma unroll
          for (int m = 0; m < FOCK_MAXM; ++m) T[m] = S[m] - (k <= m) + (l <= m);
          v = (int32_t)fock_rank_prefix<uint64_t, FOCK_MAXM>(T, M, (uint64_t)nc, mod, xdim);
        }
        J1[(size_t)(k * M + l) * nc + g] = v;
      }
    }
  }
}

__global__ void fock_double_map_kernel(int N, int M, int64_t nc, const uint64_t *__restrict__ sat,
                                       const uint64_t *__restrict__ mod, int xdim,
                                       int32_t *__restrict__ J2) {
  const int P = M * (M + 1) / 2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
       g += (int64_t)gridDim.x * blockDim.x) {
    int S[FOCK_MAXM];
    fock_decode_prefix<uint64_t, FOCK_MAXM>((uint64_t)g, N, M, (uint64_t)nc, sat, xdim, S);
    int r = 0;
    for (int k = 0; k < M; ++k) {
      int nk = S[k] - (k > 0 ? S[k - 1] : 0);
      for (int q = k; q < M; ++q, ++r) {
        int nq = S[q] - (q > 0 ? S[q - 1] : 0);
        bool ok = (k == q) ? nk >= 2 : (nk >= 1 && nq >= 1);
        int a = 0;
        for (int s = 0; s < M; ++s) {
          for (int l = s; l < M; ++l, ++a) {
            int32_t v = -1;
            if (ok) {
              int T[FOCK_MAXM];
#pragma unroll
              for (int m = 0; m < FOCK_MAXM; ++m)
                T[m] = S[m] - (k <= m) - (q <= m) + (s <= m) + (l <= m);
              v = (int32_t)fock_rank_prefix<uint64_t, FOCK_MAXM>(T, M, (uint64_t)nc, mod, xdim);
            }
            J2[(size_t)(r * P + a) * nc + g] = v;
          }
        }
      }
    }
  }
}

extern "C" int fock_build_jump_maps(fock_space *sp, int which, int dry_run, size_t *bytes,
                                    void *stream) {
  if (!sp || which < 1 || which > 3) return FOCK_ERR_ARG;
  int st = check_device(sp->device);
  if (st) return st;
  const int M = sp->M, P = fock_pair_count(M);
  size_t b1 = (which & FOCK_MAP_SINGLE) ? (size_t)4 * M * M * (size_t)sp->nc : 0;
  size_t b2 = (which & FOCK_MAP_DOUBLE) ? (size_t)4 * P * P * (size_t)sp->nc : 0;
  if (dry_run) {
    if (!bytes) return FOCK_ERR_ARG;
    *bytes = b1 + b2;
    return FOCK_OK;
  }
  if (sp->nc >= ((int64_t)1 << 31)) return FOCK_ERR_UNSUPPORTED;
  if ((which & FOCK_MAP_DOUBLE) && sp->N < 2) b2 = 0;  // no pair can be removed
  size_t need = (sp->d_j1 ? 0 : b1) + (sp->d_j2 ? 0 : b2);
  size_t fr = 0, tot = 0;
  FOCK_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  if (need + ((size_t)256 << 20) > fr) return FOCK_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 128;
  unsigned grid = grid_for(sp->nc, threads, sp->device);
  if ((which & FOCK_MAP_SINGLE) && !sp->d_j1) {
    FOCK_CUDA_TRY(cudaMalloc(&sp->d_j1, b1));
    sp->j1_bytes = b1;
    fock_single_map_kernel<<<grid, threads, 0, s>>>(sp->N, M, sp->nc, sp->tab.sat64, sp->tab.mod64,
                                                    sp->tab.xdim, sp->d_j1);
    FOCK_CUDA_TRY(cudaGetLastError());
  }
  if ((which & FOCK_MAP_DOUBLE) && !sp->d_j2 && b2 > 0) {
    FOCK_CUDA_TRY(cudaMalloc(&sp->d_j2, b2));
    sp->j2_bytes = b2;
    fock_double_map_kernel<<<grid, threads, 0, s>>>(sp->N, M, sp->nc, sp->tab.sat64, sp->tab.mod64,
                                                    sp->tab.xdim, sp->d_j2);
    FOCK_CUDA_TRY(cudaGetLastError());
  }
  if (bytes) *bytes = sp->j1_bytes + sp->j2_bytes;
  return FOCK_OK;
}

extern "C" int fock_jump_map_get(const fock_space *sp, int which, const int32_t **map_dev,
                                 int64_t *slots, int64_t *slot_stride) {
  if (!sp || !map_dev || (which != FOCK_MAP_SINGLE && which != FOCK_MAP_DOUBLE)) return FOCK_ERR_ARG;
  const int M = sp->M, P = fock_pair_count(M);
  const int32_t *p = which == FOCK_MAP_SINGLE ? sp->d_j1 : sp->d_j2;
  if (!p) return FOCK_ERR_NOT_BUILT;
  *map_dev = p;
  if (slots) *slots = which == FOCK_MAP_SINGLE ? (int64_t)M * M : (int64_t)P * P;
  if (slot_stride) *slot_stride = sp->nc;
  return FOCK_OK;
}
