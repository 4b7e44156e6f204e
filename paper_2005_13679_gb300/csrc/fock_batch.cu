// fock_batch.cu -- uneven batches of independent problems: one persistent
// launch applies every instance's H, and a batched thick-restart Lanczos runs
// each restart cycle of every instance as one CUDA graph replay.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "fock_apply_sparse.cuh"

int fock_make_terms(const fock_ham *ham, int maxm, FockTerm *out);
int fock_apply_internal(const fock_space *sp, const fock_ham *ham, const void *C, void *sigma, int nrhs, int precision,
                        int arm, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t fock_apply_ws_pref(const fock_space *sp, const fock_ham *ham, int nrhs, int precision);
int fock_prepare_df_ranges(const void *C, const int64_t *src, const int64_t *dst, const int64_t *len, int nr,
                           void *ws, int device, cudaStream_t stream);

namespace {

// ---------------------------------------------------------------------------
// Device descriptors
// ---------------------------------------------------------------------------
struct BatchInst {
  int N, M, xdim, rows, nrem, nadd, nsq, real;
  uint32_t nc, pad;
  long long off;                  // offset of the instance in concatenated vectors
  long long soff;                 // offset of its FP32-pair split copy in the batch workspace
  const uint32_t *mod, *sat;
  const FockRemoval *rem;
  const FockTerm *terms;
  const void *coef_df, *sq_df, *coef32, *sq32;
  double coef_scale;
};

struct BatchItem {
  int inst;
  uint32_t g0, g1;                // configuration range of one work item
};

struct BatchArgs {
  const BatchInst *inst;
  const BatchItem *items;
  int nitems;
  unsigned *queue;                // work counter, zeroed before every launch
  const int *active;              // per-instance mask, or NULL
  const void *C;
  void *sigma;
  const int *in_exp;              // FP32-pair input scale, or NULL
  SparseSmemLayout L;
};

const int kBatchMaxM = 12;
const uint32_t kOwnMinNc = 1u << 18;   // smaller instances stay in the shared persistent launch

// One persistent launch over every instance.  A block claims items from the
// queue; items are ordered largest instance first and are whole tiles of 128
// configurations, so the ragged ends of small instances fill the tail.
template <class P, bool REAL>
__global__ void __launch_bounds__(FOCK_APPLY_THREADS, 4) fock_batch_apply_kernel(const BatchArgs b) {
  constexpr int MAXM = kBatchMaxM;
  constexpr bool DF = std::is_same<P, PolDFP>::value;
  using vec_t = typename P::vec_t;
  using out_t = decltype(P::finish(typename P::acc_t{}, 1.0, REAL));
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const int tid = threadIdx.x, nt = blockDim.x;
  uint32_t *pd = (uint32_t *)(smem + b.L.off_pd) + tid;
  int *nn = (int *)(smem + b.L.off_n) + tid;
#pragma unroll
  for (int j = 0; j < MAXM; ++j) pd[(2 * MAXM + j) * nt] = 0u;
  const double in_scale = b.in_exp ? fock_pow2(__ldg(b.in_exp)) : 1.0;
  int staged = -1;
  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(b.queue, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= b.nitems) break;
    const BatchItem item = b.items[it];
    const BatchInst I = b.inst[item.inst];
    if (item.inst != staged) {
      sparse_stage<P>(smem, b.L, I.rows, I.xdim, I.mod, I.sat, I.nsq, DF ? I.sq_df : I.sq32, I.nadd, I.terms,
                      DF ? I.coef_df : I.coef32);
      __syncthreads();
      staged = item.inst;
    }
    if (!b.active || b.active[item.inst]) {
      SparseView v;
      v.N = I.N; v.M = I.M; v.nrem = I.nrem; v.xs = I.xdim + 2; v.xdim = I.xdim; v.nrhs = 1; v.nc = I.nc;
      v.mod = (const uint32_t *)(smem + b.L.off_mod);
      v.sat = (const uint32_t *)(smem + b.L.off_sat);
      v.sq = smem + b.L.off_sq;
      v.terms = (const FockTerm *)(smem + b.L.off_terms);
      v.coef = smem + b.L.off_coef;
      v.rem = I.rem;
      v.C = (const vec_t *)b.C + (DF ? I.soff : I.off);
      v.sigma = (out_t *)b.sigma + I.off;
      v.map = nullptr;
      v.slots = nullptr;
      v.out_scale = DF ? I.coef_scale * in_scale : 1.0;
      for (uint32_t tile = item.g0; tile < item.g1; tile += nt)
        sparse_config<MAXM, P, REAL, 1, false>(v, tile + tid, pd, nn, nt);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Segmented FP64 vector kernels for the batched Lanczos.  Concatenated vectors
// are cut into chunks that never straddle an instance.
// ---------------------------------------------------------------------------
const int kVec = 8;           // vectors per fused pass
const int64_t kChunkLen = 16384;

struct Chunk {
  int inst;
  int pad;
  long long b, e;
};

// partial[c][i] = sum over chunk c of conj(V_{i0+i}[x]) w[x], i < kk
template <bool REAL>
__global__ void bdots_kernel(const double2 *__restrict__ V, long long ld, int kk, const double2 *__restrict__ w,
                             const Chunk *__restrict__ chunks, int nchunks, double2 *__restrict__ partial) {
  __shared__ double2 red[kVec][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk ch = chunks[c];
    double2 acc[kVec];
#pragma unroll
    for (int i = 0; i < kVec; ++i) acc[i] = make_double2(0.0, 0.0);
    for (long long x = ch.b + threadIdx.x; x < ch.e; x += blockDim.x) {
      if (REAL) {
        const double wx = w[x].x;
#pragma unroll
        for (int i = 0; i < kVec; ++i)
          if (i < kk) acc[i].x = fma(V[i * ld + x].x, wx, acc[i].x);
      } else {
        const double2 wx = w[x];
#pragma unroll
        for (int i = 0; i < kVec; ++i)
          if (i < kk) {
            const double2 v = V[i * ld + x];
            acc[i].x = fma(v.x, wx.x, fma(v.y, wx.y, acc[i].x));
            acc[i].y = fma(v.x, wx.y, fma(-v.y, wx.x, acc[i].y));
          }
      }
    }
#pragma unroll
    for (int i = 0; i < kVec; ++i) {
      double2 a = acc[i];
      for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
      }
      if (lane == 0) red[i][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < kVec) {
      double2 s = make_double2(0.0, 0.0);
      for (int j = 0; j < nw; ++j) {
        s.x += red[threadIdx.x][j].x;
        s.y += red[threadIdx.x][j].y;
      }
      partial[(size_t)c * kVec + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// out[inst * ldo + i0 + i] = sum of the instance's chunk partials, i < kk
__global__ void breduce_kernel(const double2 *__restrict__ partial, const int *__restrict__ cbeg, int count, int kk,
                               int i0, double2 *__restrict__ out, int ldo) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  const int i = threadIdx.x;
  if (i >= kk) return;
  double2 s = make_double2(0.0, 0.0);
  for (int c = cbeg[inst]; c < cbeg[inst + 1]; ++c) {
    s.x += partial[(size_t)c * kVec + i].x;
    s.y += partial[(size_t)c * kVec + i].y;
  }
  out[(size_t)inst * ldo + i0 + i] = s;
}

// w[x] = (beta ? w[x] : 0) - sum_i coef[inst][i0 + i] V_{i0+i}[x]
template <bool REAL>
__global__ void bcombine_kernel(const double2 *__restrict__ V, long long ld, int kk, int i0,
                                const double2 *__restrict__ coef, int ldc, bool keep_w, double2 *__restrict__ w,
                                const Chunk *__restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk ch = chunks[c];
    double2 cf[kVec];
#pragma unroll
    for (int i = 0; i < kVec; ++i) cf[i] = i < kk ? coef[(size_t)ch.inst * ldc + i0 + i] : make_double2(0.0, 0.0);
    for (long long x = ch.b + threadIdx.x; x < ch.e; x += blockDim.x) {
      double2 acc = keep_w ? w[x] : make_double2(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < kVec; ++i)
        if (i < kk) {
          const double2 v = V[i * ld + x];
          if (REAL) {
            acc.x = fma(-cf[i].x, v.x, acc.x);
          } else {
            acc.x -= cf[i].x * v.x - cf[i].y * v.y;
            acc.y -= cf[i].x * v.y + cf[i].y * v.x;
          }
        }
      w[x] = acc;
    }
  }
}

// dst[x] = w[x] * f(inst), f = 1/sqrt(nrm2) for active instances with nrm2 > 0, else 0
__global__ void bscale_kernel(const double2 *__restrict__ w, const double2 *__restrict__ nrm2, int ldn,
                              const int *__restrict__ active, double2 *__restrict__ dst,
                              const Chunk *__restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk ch = chunks[c];
    const double n2 = nrm2[(size_t)ch.inst * ldn].x;
    const double f = (active[ch.inst] && n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
    for (long long x = ch.b + threadIdx.x; x < ch.e; x += blockDim.x) {
      const double2 v = w[x];
      dst[x] = make_double2(v.x * f, v.y * f);
    }
  }
}

// alpha[j][inst] = Re h1[inst][j] + Re h2[inst][j];  beta[j][inst] = sqrt(nrm2[inst])
__global__ void bstore_kernel(const double2 *__restrict__ h1, const double2 *__restrict__ h2, int ldh, int j,
                              const double2 *__restrict__ nrm2, int ldn, int count, double *__restrict__ alpha,
                              double *__restrict__ beta) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= count) return;
  alpha[(size_t)j * count + inst] = h1[(size_t)inst * ldh + j].x + h2[(size_t)inst * ldh + j].x;
  beta[(size_t)j * count + inst] = sqrt(fmax(nrm2[(size_t)inst * ldn].x, 0.0));
}

__device__ __forceinline__ uint64_t bsplitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// start vectors from SplitMix64 (same counters as the single-problem solver,
// offset by each instance's position)
__global__ void brandom_kernel(uint64_t seed, long long n, bool real, double2 *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t a = bsplitmix64(seed + 2 * (uint64_t)i), b = bsplitmix64(seed + 2 * (uint64_t)i + 1);
    y[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, real ? 0.0 : (double)(b >> 11) * 0x1.0p-52 - 1.0);
  }
}

void jacobi_small(std::vector<double> A, int n, std::vector<double> &evals, std::vector<double> &evecs) {
  // cyclic Jacobi rotations (see fock_lanczos.cu for the single-problem twin)
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
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - sn * qkq;
          Q[(size_t)k * n + q] = sn * qkp + c * qkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  evals.resize(n);
  evecs.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    evals[i] = A[(size_t)order[i] * n + order[i]];
    for (int k = 0; k < n; ++k) evecs[(size_t)i * n + k] = Q[(size_t)k * n + order[i]];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host object
// ---------------------------------------------------------------------------
struct fock_batch {
  int count = 0, device = 0;
  std::vector<fock_space *> sp;
  std::vector<fock_ham *> ham;
  std::vector<FockTerm *> d_terms;   // per instance, encoded for kBatchMaxM
  std::vector<int64_t> off;      // count + 1
  int64_t total = 0, terms = 0;
  bool real = true;
  BatchInst *d_inst = nullptr;
  std::vector<BatchInst> h_inst;
  // work items
  int tiles_per_item = 8, blocks_per_sm = 0;
  int nitems = 0;
  BatchItem *d_items = nullptr;
  unsigned *d_queue = nullptr;
  int *d_active = nullptr;       // all ones unless a solver masks instances
  // FP32-pair scratch: status words + split copy of the instances the
  // persistent launch serves (split_total configurations, ranges pr_*)
  void *ws = nullptr;
  size_t ws_bytes = 0;
  int64_t split_total = 0;
  std::vector<int64_t> pr_src, pr_dst, pr_len;
  // instances large enough for their own two-phase apply (one after another
  // on the stream, sharing one workspace)
  std::vector<char> own;
  int nown = 0;
  void *own_ws = nullptr;
  size_t own_ws_bytes = 0, own_ws_need = 0;
  int max_nadd = 0, max_rows = 1, max_xdim = 0, max_nsq = 0;
};

static int build_items(fock_batch *b, int tiles) {
  std::vector<int> order(b->count);
  for (int i = 0; i < b->count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->h_inst[x].nc > b->h_inst[y].nc; });
  std::vector<BatchItem> items;
  const uint32_t span = (uint32_t)tiles * FOCK_APPLY_THREADS;
  for (int i : order) {
    if (b->own[i]) continue;
    const uint32_t nc = b->h_inst[i].nc;
    for (uint32_t g0 = 0; g0 < nc; g0 += span) {
      BatchItem it;
      it.inst = i;
      it.g0 = g0;
      it.g1 = g0 + span < nc ? g0 + span : nc;
      items.push_back(it);
    }
  }
  cudaFree(b->d_items);
  b->d_items = nullptr;
  b->nitems = 0;
  b->tiles_per_item = tiles;
  if (items.empty()) return FOCK_OK;
  FOCK_CUDA_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()));
  FOCK_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
  b->nitems = (int)items.size();
  b->tiles_per_item = tiles;
  return FOCK_OK;
}

extern "C" int fock_batch_destroy(fock_batch *b) {
  if (!b) return FOCK_OK;
  for (auto *t : b->d_terms) cudaFree(t);
  for (auto *h : b->ham) fock_hamiltonian_destroy(h);
  for (auto *s : b->sp) fock_space_destroy(s);
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_queue);
  cudaFree(b->d_active);
  cudaFree(b->ws);
  cudaFree(b->own_ws);
  delete b;
  return FOCK_OK;
}

extern "C" int fock_batch_create(int32_t count, const int32_t *N, const int32_t *M, const double *const *h_host,
                                 const double *const *W_host, double tol, fock_batch **out) {
  if (count < 1 || !N || !M || !h_host || !out) return FOCK_ERR_ARG;
  fock_batch *b = new fock_batch();
  b->count = count;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return FOCK_ERR_CUDA;
  }
  b->off.assign(count + 1, 0);
  int st = FOCK_OK;
  for (int i = 0; i < count && !st; ++i) {
    fock_space *s = nullptr;
    fock_ham *h = nullptr;
    st = fock_space_create(N[i], M[i], &s);
    if (!st && !s->idx32) st = FOCK_ERR_UNSUPPORTED;
    if (!st) st = fock_hamiltonian_create(s, h_host[i], W_host ? W_host[i] : nullptr, tol, &h);
    if (s) b->sp.push_back(s);
    if (h) b->ham.push_back(h);
    if (!st && (size_t)h->nadd * 48 > (size_t)64 * 1024) st = FOCK_ERR_UNSUPPORTED;
    FockTerm *dt = nullptr;
    if (!st) {
      std::vector<FockTerm> tt(h->nadd > 0 ? h->nadd : 1);
      st = fock_make_terms(h, kBatchMaxM, tt.data());
      if (!st && cudaMalloc(&dt, sizeof(FockTerm) * tt.size()) != cudaSuccess) st = FOCK_ERR_NOMEM;
      if (!st && cudaMemcpy(dt, tt.data(), sizeof(FockTerm) * tt.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = FOCK_ERR_CUDA;
      if (dt) b->d_terms.push_back(dt);
    }
    if (st) break;
    b->off[i + 1] = b->off[i] + s->nc;
    // its own apply when the instance is large and its default path is a two-phase one
    int32_t path = FOCK_PATH_LIST;
    const size_t pref = fock_apply_ws_pref(s, h, 1, FOCK_PREC_F64);
    const bool own = s->nc >= kOwnMinNc && fock_apply_path(s, h, 1, FOCK_PREC_F64, FOCK_ARM_HASH, pref, &path) == FOCK_OK &&
                     (path == FOCK_PATH_TWOPHASE_TC || path == FOCK_PATH_TWOPHASE || path == FOCK_PATH_TWOPHASE_BLOCK);
    b->own.push_back(own ? 1 : 0);
    if (own) {
      b->nown++;
      b->own_ws_need = std::max(b->own_ws_need, std::max(pref, fock_apply_ws_pref(s, h, 1, FOCK_PREC_F32_MIXED)));
    }
    b->terms += h->config_terms;
    b->real = b->real && h->real;
    BatchInst I;
    memset(&I, 0, sizeof(I));
    I.N = s->N; I.M = s->M; I.xdim = s->tab.xdim; I.rows = s->tab.rows; I.nrem = h->nrem; I.nadd = h->nadd;
    I.nsq = s->N + 4; I.real = h->real; I.nc = (uint32_t)s->nc; I.off = b->off[i];
    I.soff = b->split_total;
    if (!own) {
      b->pr_src.push_back(b->off[i]);
      b->pr_dst.push_back(b->split_total);
      b->pr_len.push_back(s->nc);
      b->split_total += s->nc;
    }
    I.mod = s->tab.mod32; I.sat = s->tab.sat32; I.rem = h->d_rem; I.terms = dt;
    I.coef_df = h->d_coefdf; I.sq_df = h->d_sqrtdf; I.coef32 = h->d_coef32; I.sq32 = h->d_sqrt32;
    I.coef_scale = h->coef_scale;
    b->h_inst.push_back(I);
    if (!own) {
      b->max_nadd = std::max(b->max_nadd, h->nadd);
      b->max_rows = std::max(b->max_rows, s->tab.rows);
      b->max_xdim = std::max(b->max_xdim, s->tab.xdim);
      b->max_nsq = std::max(b->max_nsq, s->N + 4);
    }
  }
  if (!st) {
    b->total = b->off[count];
    if (cudaMalloc(&b->d_inst, sizeof(BatchInst) * count) != cudaSuccess ||
        cudaMalloc(&b->d_queue, 256) != cudaSuccess || cudaMalloc(&b->d_active, sizeof(int) * count) != cudaSuccess)
      st = FOCK_ERR_NOMEM;
  }
  if (!st) {
    std::vector<int> ones(count, 1);
    if (cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_active, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      st = FOCK_ERR_CUDA;
  }
  if (!st) st = build_items(b, 8);
  if (st) {
    fock_batch_destroy(b);
    return st;
  }
  *out = b;
  return FOCK_OK;
}

extern "C" int fock_batch_offsets(const fock_batch *b, int64_t *offsets) {
  if (!b || !offsets) return FOCK_ERR_ARG;
  for (int i = 0; i <= b->count; ++i) offsets[i] = b->off[i];
  return FOCK_OK;
}

extern "C" int fock_batch_own_apply(const fock_batch *b, int32_t *own) {
  if (!b || !own) return FOCK_ERR_ARG;
  for (int i = 0; i < b->count; ++i) own[i] = b->own[i];
  return FOCK_OK;
}

extern "C" int fock_batch_terms(const fock_batch *b, int64_t *config_terms) {
  if (!b || !config_terms) return FOCK_ERR_ARG;
  *config_terms = b->terms;
  return FOCK_OK;
}

template <class P, bool REAL>
static int launch_batch(fock_batch *b, const void *C, void *sigma, const int *in_exp, const int *active,
                        cudaStream_t s) {
  auto kern = fock_batch_apply_kernel<P, REAL>;
  BatchArgs a;
  a.inst = b->d_inst;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.queue = b->d_queue;
  a.active = active;
  a.C = C;
  a.sigma = sigma;
  a.in_exp = in_exp;
  a.L = sparse_layout<kBatchMaxM>(b->max_nadd, sizeof(typename P::coef_t), b->max_rows, b->max_xdim, b->max_nsq,
                                  sizeof(typename P::amp_t), FOCK_APPLY_THREADS);
  const size_t smem = a.L.total;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fock_cuda_status(e);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FOCK_APPLY_THREADS, smem);
  if (e != cudaSuccess) return fock_cuda_status(e);
  if (per_sm < 1) return FOCK_ERR_UNSUPPORTED;
  if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
  int grid = per_sm * fock_get_sm_count(b->device);
  if (grid > b->nitems) grid = b->nitems;
  FOCK_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), s));
  kern<<<grid, FOCK_APPLY_THREADS, smem, s>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FOCK_OK : fock_cuda_status(e);
}

// The persistent launch over the instances without an apply of their own.
static int batch_apply_shared(fock_batch *b, const void *C, void *sigma, int precision, const int *active,
                              cudaStream_t s) {
  if (b->nitems == 0) return FOCK_OK;
  if (precision == FOCK_PREC_F64) {
    const size_t need = 256 + (size_t)b->split_total * sizeof(float4);
    if (b->ws_bytes < need) return FOCK_ERR_NOMEM;
    int st = fock_prepare_df_ranges(C, b->pr_src.data(), b->pr_dst.data(), b->pr_len.data(), (int)b->pr_src.size(),
                                    b->ws, b->device, s);
    if (st) return st;
    const void *Cin = (const char *)b->ws + 256;
    const int *in_exp = (const int *)b->ws + 1;
    return b->real ? launch_batch<PolDFP, true>(b, Cin, sigma, in_exp, active, s)
                   : launch_batch<PolDFP, false>(b, Cin, sigma, in_exp, active, s);
  }
  if (precision == FOCK_PREC_F32_MIXED)
    return b->real ? launch_batch<PolMixedP, true>(b, C, sigma, nullptr, active, s)
                   : launch_batch<PolMixedP, false>(b, C, sigma, nullptr, active, s);
  return FOCK_ERR_UNSUPPORTED;
}

// Every instance: the shared launch, then the instances with an apply of
// their own (skipped where host_active is given and 0).
static int batch_apply_internal(fock_batch *b, const void *C, void *sigma, int precision, const int *active,
                                cudaStream_t s, const int *host_active = nullptr) {
  int st = batch_apply_shared(b, C, sigma, precision, active, s);
  if (st || b->nown == 0) return st;
  if (b->own_ws_bytes < b->own_ws_need) return FOCK_ERR_NOMEM;
  const size_t elem = precision == FOCK_PREC_F64 ? 16 : 8;
  for (int i = 0; i < b->count && !st; ++i) {
    if (!b->own[i] || (host_active && !host_active[i])) continue;
    st = fock_apply_internal(b->sp[i], b->ham[i], (const char *)C + (size_t)b->off[i] * elem,
                             (char *)sigma + (size_t)b->off[i] * elem, 1, precision, FOCK_ARM_HASH, b->own_ws,
                             b->own_ws_bytes, s);
  }
  return st;
}

static int ensure_ws(fock_batch *b) {
  const size_t need = 256 + (size_t)b->split_total * sizeof(float4);
  if (b->ws_bytes < need) {
    cudaFree(b->ws);
    b->ws = nullptr;
    b->ws_bytes = 0;
    FOCK_CUDA_TRY(cudaMalloc(&b->ws, need));
    b->ws_bytes = need;
  }
  if (b->own_ws_bytes < b->own_ws_need) {
    cudaFree(b->own_ws);
    b->own_ws = nullptr;
    b->own_ws_bytes = 0;
    FOCK_CUDA_TRY(cudaMalloc(&b->own_ws, b->own_ws_need));
    b->own_ws_bytes = b->own_ws_need;
  }
  return FOCK_OK;
}

static int check_batch(const fock_batch *b) {
  if (!b) return FOCK_ERR_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return FOCK_ERR_CUDA;
  return cur == b->device ? FOCK_OK : FOCK_ERR_DEVICE;
}

extern "C" int fock_batch_apply(fock_batch *b, const void *C_dev, void *sigma_dev, int precision, void *stream) {
  int st = check_batch(b);
  if (st) return st;
  if (!C_dev || !sigma_dev) return FOCK_ERR_ARG;
  if (precision != FOCK_PREC_F64 && precision != FOCK_PREC_F32_MIXED) return FOCK_ERR_UNSUPPORTED;
  const size_t bytes = (size_t)b->total * (precision == FOCK_PREC_F64 ? 16 : 8);
  const char *c0 = (const char *)C_dev, *s0 = (const char *)sigma_dev;
  if (c0 < s0 + bytes && s0 < c0 + bytes) return FOCK_ERR_ALIAS;
  st = ensure_ws(b);
  if (st) return st;
  return batch_apply_internal(b, C_dev, sigma_dev, precision, nullptr, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
static std::string tune_key(const fock_batch *b, int precision) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the instance shapes
  for (const BatchInst &I : b->h_inst) {
    const uint64_t v[3] = {(uint64_t)I.N, (uint64_t)I.M, (uint64_t)I.nadd};
    for (uint64_t x : v) {
      h ^= x;
      h *= 1099511628211ull;
    }
  }
  char buf[96];
  snprintf(buf, sizeof(buf), "batch %016llx count %d prec %d sms %d", (unsigned long long)h, b->count, precision,
           fock_get_sm_count(b->device));
  return std::string(buf);
}

extern "C" int fock_batch_autotune(fock_batch *b, const void *C_dev, void *sigma_dev, int precision,
                                   const char *cache_path, int32_t *tiles_per_item, int32_t *blocks_per_sm,
                                   void *stream) {
  int st = check_batch(b);
  if (st) return st;
  if (!C_dev || !sigma_dev) return FOCK_ERR_ARG;
  if (precision != FOCK_PREC_F64 && precision != FOCK_PREC_F32_MIXED) return FOCK_ERR_UNSUPPORTED;
  const std::string key = tune_key(b, precision);
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "r")) {
      char line[256];
      int t = 0, bp = -1;
      while (fgets(line, sizeof(line), f)) {
        int tt, bb;
        char k[160];
        if (sscanf(line, "%159[^|]| tiles %d blocks %d", k, &tt, &bb) == 3 && key + " " == std::string(k)) {
          t = tt;
          bp = bb;
        }
      }
      fclose(f);
      if (t > 0) {
        b->blocks_per_sm = bp;
        st = build_items(b, t);
        if (tiles_per_item) *tiles_per_item = t;
        if (blocks_per_sm) *blocks_per_sm = bp;
        return st;
      }
    }
  }
  st = ensure_ws(b);
  if (st) return st;
  if (b->nown == b->count) {             // no instance in the shared launch: nothing to tune
    if (tiles_per_item) *tiles_per_item = b->tiles_per_item;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    return FOCK_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  FOCK_CUDA_TRY(cudaEventCreate(&e0));
  FOCK_CUDA_TRY(cudaEventCreate(&e1));
  const int tiles_c[] = {1, 2, 4, 8, 16, 32};
  const int blocks_c[] = {0, 3, 2, 1};   // 0: occupancy maximum
  float best = 1e30f;
  int bt = 8, bb = 0;
  for (int t : tiles_c) {
    st = build_items(b, t);
    if (st) break;
    for (int bp : blocks_c) {
      b->blocks_per_sm = bp;
      st = batch_apply_shared(b, C_dev, sigma_dev, precision, nullptr, s);  // warm-up
      if (st) break;
      FOCK_CUDA_TRY(cudaEventRecord(e0, s));
      for (int r = 0; r < 3 && !st; ++r) st = batch_apply_shared(b, C_dev, sigma_dev, precision, nullptr, s);
      FOCK_CUDA_TRY(cudaEventRecord(e1, s));
      FOCK_CUDA_TRY(cudaEventSynchronize(e1));
      if (st) break;
      float ms = 0.f;
      FOCK_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bt = t;
        bb = bp;
      }
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  b->blocks_per_sm = bb;
  st = build_items(b, bt);
  if (st) return st;
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "a")) {
      fprintf(f, "%s | tiles %d blocks %d | %.4f ms\n", key.c_str(), bt, bb, best / 3.0f);
      fclose(f);
    }
  }
  if (tiles_per_item) *tiles_per_item = bt;
  if (blocks_per_sm) *blocks_per_sm = bb;
  return FOCK_OK;
}

// ---------------------------------------------------------------------------
// Batched thick-restart Lanczos
// ---------------------------------------------------------------------------
namespace {

struct BLanczos {
  fock_batch *b;
  cudaStream_t s;
  int m, keep, count, nchunks;
  bool real;
  long long n;
  double2 *V = nullptr, *W = nullptr, *G = nullptr;       // basis [m+1+keep][n], work, ground vectors
  double2 *partial = nullptr, *H1 = nullptr, *H2 = nullptr, *NR = nullptr, *Y = nullptr;
  double *alpha = nullptr, *beta = nullptr;
  Chunk *chunks = nullptr;
  int *cbeg = nullptr;
  int ldh;
  int grid;
  const int *hact = nullptr;     // host activity of the instances (their own applies are skipped at 0)

  int dots(const double2 *Vb, int k, const double2 *w, double2 *out) {
    for (int i0 = 0; i0 < k; i0 += kVec) {
      const int kk = k - i0 < kVec ? k - i0 : kVec;
      if (real) bdots_kernel<true><<<grid, 256, 0, s>>>(Vb + (size_t)i0 * n, n, kk, w, chunks, nchunks, partial);
      else bdots_kernel<false><<<grid, 256, 0, s>>>(Vb + (size_t)i0 * n, n, kk, w, chunks, nchunks, partial);
      breduce_kernel<<<count, kVec, 0, s>>>(partial, cbeg, count, kk, i0, out, ldh);
    }
    return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
  }
  // w = (keep_w ? w : 0) - sum_i coef[inst][i] V_i
  int combine(const double2 *Vb, int k, const double2 *coef, bool keep_w, double2 *w) {
    for (int i0 = 0; i0 < k; i0 += kVec) {
      const int kk = k - i0 < kVec ? k - i0 : kVec;
      const bool kw = keep_w || i0 > 0;
      if (real) bcombine_kernel<true><<<grid, 256, 0, s>>>(Vb + (size_t)i0 * n, n, kk, i0, coef, ldh, kw, w, chunks, nchunks);
      else bcombine_kernel<false><<<grid, 256, 0, s>>>(Vb + (size_t)i0 * n, n, kk, i0, coef, ldh, kw, w, chunks, nchunks);
    }
    return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
  }
  // one Lanczos step j (apply, two Gram-Schmidt passes, alpha, beta, next vector)
  int step(int j) {
    double2 *vj = V + (size_t)j * n;
    int st = batch_apply_internal(b, vj, W, FOCK_PREC_F64, b->d_active, s, hact);
    if (st) return st;
    if ((st = dots(V, j + 1, W, H1))) return st;
    if ((st = combine(V, j + 1, H1, true, W))) return st;
    if ((st = dots(V, j + 1, W, H2))) return st;
    if ((st = combine(V, j + 1, H2, true, W))) return st;
    if ((st = dots(W, 1, W, NR))) return st;
    bstore_kernel<<<(count + 127) / 128, 128, 0, s>>>(H1, H2, ldh, j, NR, ldh, count, alpha, beta);
    bscale_kernel<<<grid, 256, 0, s>>>(W, NR, ldh, b->d_active, V + (size_t)(j + 1) * n, chunks, nchunks);
    return cudaGetLastError() == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
  }
};

}  // namespace

extern "C" int fock_batch_lanczos_ground(fock_batch *b, int32_t max_iter, int32_t restart_len, double tol,
                                         uint64_t seed, double *E0_out, double *residual_out, int32_t *iters_out,
                                         void *stream) {
  int st = check_batch(b);
  if (st) return st;
  if (!E0_out || max_iter < 1 || restart_len < 4 || restart_len > 64 || !(tol > 0.0)) return FOCK_ERR_ARG;
  st = ensure_ws(b);
  if (st) return st;
  // The solver runs on a stream of its own (the legacy default stream cannot be
  // captured into a graph), ordered after the caller's stream.
  cudaStream_t own = nullptr;
  cudaEvent_t ready = nullptr;
  if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) return FOCK_ERR_CUDA;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ready, (cudaStream_t)stream) != cudaSuccess || cudaStreamWaitEvent(own, ready, 0) != cudaSuccess) {
    cudaStreamDestroy(own);
    if (ready) cudaEventDestroy(ready);
    return FOCK_ERR_CUDA;
  }
  BLanczos L;
  L.b = b;
  L.s = own;
  L.count = b->count;
  L.n = b->total;
  L.real = b->real;
  L.m = restart_len;
  L.keep = std::max(1, std::min(L.m / 3, 8));
  L.ldh = L.m + 2;
  L.grid = fock_get_sm_count(b->device) * 4;
  const int count = b->count, m = L.m, keep = L.keep;
  const long long n = L.n;

  // chunks that never straddle an instance
  std::vector<Chunk> ch;
  std::vector<int> cb(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    cb[i] = (int)ch.size();
    for (long long x = b->off[i]; x < b->off[i + 1]; x += kChunkLen) {
      Chunk c;
      c.inst = i;
      c.pad = 0;
      c.b = x;
      c.e = std::min<long long>(x + kChunkLen, b->off[i + 1]);
      ch.push_back(c);
    }
  }
  cb[count] = (int)ch.size();
  L.nchunks = (int)ch.size();

  cudaGraphExec_t graphs[2] = {nullptr, nullptr};
  auto cleanup = [&]() {
    for (auto &g : graphs)
      if (g) cudaGraphExecDestroy(g);
    cudaFree(L.V); cudaFree(L.W); cudaFree(L.G); cudaFree(L.partial); cudaFree(L.H1); cudaFree(L.H2);
    cudaFree(L.NR); cudaFree(L.Y); cudaFree(L.alpha); cudaFree(L.beta); cudaFree(L.chunks); cudaFree(L.cbeg);
    std::vector<int> ones(count, 1);
    cudaStreamSynchronize(own);
    cudaMemcpy(b->d_active, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    cudaEventDestroy(ready);
    cudaStreamDestroy(own);
  };
#define BTRY(x)                       \
  do {                                \
    st = (x);                         \
    if (st) { cleanup(); return st; } \
  } while (0)
#define BCUDA(x)                                   \
  do {                                             \
    cudaError_t e_ = (x);                          \
    BTRY(e_ == cudaSuccess ? FOCK_OK : fock_cuda_status(e_)); \
  } while (0)
  BCUDA(cudaMalloc(&L.V, sizeof(double2) * (size_t)n * (m + 1 + keep)));
  BCUDA(cudaMalloc(&L.W, sizeof(double2) * (size_t)n));
  BCUDA(cudaMalloc(&L.G, sizeof(double2) * (size_t)n));
  BCUDA(cudaMalloc(&L.partial, sizeof(double2) * (size_t)L.nchunks * kVec));
  BCUDA(cudaMalloc(&L.H1, sizeof(double2) * (size_t)count * L.ldh));
  BCUDA(cudaMalloc(&L.H2, sizeof(double2) * (size_t)count * L.ldh));
  BCUDA(cudaMalloc(&L.NR, sizeof(double2) * (size_t)count * L.ldh));
  BCUDA(cudaMalloc(&L.Y, sizeof(double2) * (size_t)count * L.ldh));
  BCUDA(cudaMalloc(&L.alpha, sizeof(double) * (size_t)m * count));
  BCUDA(cudaMalloc(&L.beta, sizeof(double) * (size_t)m * count));
  BCUDA(cudaMalloc(&L.chunks, sizeof(Chunk) * ch.size()));
  BCUDA(cudaMalloc(&L.cbeg, sizeof(int) * (count + 1)));
  BCUDA(cudaMemcpy(L.chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice));
  BCUDA(cudaMemcpy(L.cbeg, cb.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice));
  cudaStream_t s = L.s;

  // start vectors: SplitMix64, normalised per instance
  brandom_kernel<<<L.grid, 256, 0, s>>>(seed, n, L.real, L.W);
  BTRY(L.dots(L.W, 1, L.W, L.NR));
  bscale_kernel<<<L.grid, 256, 0, s>>>(L.W, L.NR, L.ldh, b->d_active, L.V, L.chunks, L.nchunks);

  // one product outside any capture (first launch of each kernel variant)
  BTRY(batch_apply_internal(b, L.V, L.W, FOCK_PREC_F64, b->d_active, s));

  // host state per instance
  std::vector<int> active(count, 1), iters(count, 0), pcur(count, 0);
  std::vector<int> cap_active(count, 1);   // activity the graphs were captured with
  L.hact = active.data();
  std::vector<std::vector<double>> theta(count), coup(count);   // kept Ritz values and couplings
  std::vector<double> ha((size_t)m * count), hb((size_t)m * count);
  std::vector<double2> Yh((size_t)count * L.ldh);
  bool any_noconv = false;
  int total = 0, p = 0;
  while (true) {
    // one restart cycle: steps p..m-1 as one graph
    const int gi = p == 0 ? 0 : 1;
    // an instance with its own apply that stopped: capture again without it
    bool recapture = false;
    for (int i = 0; i < count; ++i) recapture = recapture || (b->own[i] && active[i] != cap_active[i]);
    if (recapture) {
      for (auto &g : graphs)
        if (g) cudaGraphExecDestroy(g);
      graphs[0] = graphs[1] = nullptr;
      cap_active = active;
    }
    if (!graphs[gi]) {
      cudaGraph_t g;
      BCUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
      for (int j = p; j < m && !st; ++j) st = L.step(j);
      cudaError_t ce = cudaStreamEndCapture(s, &g);
      if (st) { cleanup(); return st; }
      BCUDA(ce);
      BCUDA(cudaGraphInstantiate(&graphs[gi], g, 0));
      cudaGraphDestroy(g);
    }
    BCUDA(cudaGraphLaunch(graphs[gi], s));
    total += m - p;
    BCUDA(cudaMemcpyAsync(ha.data(), L.alpha, sizeof(double) * m * count, cudaMemcpyDeviceToHost, s));
    BCUDA(cudaMemcpyAsync(hb.data(), L.beta, sizeof(double) * m * count, cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    // projected problems, convergence, restart coefficients (Ritz vector i -> row i of Y)
    const bool last = total >= max_iter;
    std::fill(Yh.begin(), Yh.end(), make_double2(0.0, 0.0));
    std::vector<std::vector<double>> Ys(keep, std::vector<double>((size_t)count * L.ldh, 0.0));
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      iters[i] += m - p;
      const int dim = m;
      std::vector<double> T((size_t)dim * dim, 0.0);
      for (int r = 0; r < p; ++r) {
        T[(size_t)r * dim + r] = theta[i][r];
        T[(size_t)r * dim + p] = T[(size_t)p * dim + r] = coup[i][r];
      }
      for (int j = p; j < m; ++j) {
        T[(size_t)j * dim + j] = ha[(size_t)j * count + i];
        if (j + 1 < m) T[(size_t)(j + 1) * dim + j] = T[(size_t)j * dim + j + 1] = hb[(size_t)j * count + i];
      }
      std::vector<double> ev, vec;
      jacobi_small(T, dim, ev, vec);
      const double bl = hb[(size_t)(m - 1) * count + i];
      const double est = fabs(bl * vec[(size_t)0 * dim + (dim - 1)]);
      const bool conv = est <= tol * fmax(fabs(ev[0]), 1.0) || bl == 0.0;
      const int np = (conv || last) ? 1 : keep;
      for (int r = 0; r < np; ++r)
        for (int k = 0; k < dim; ++k) Ys[r][(size_t)i * L.ldh + k] = vec[(size_t)r * dim + k];
      theta[i].assign(ev.begin(), ev.begin() + np);
      coup[i].resize(np);
      for (int r = 0; r < np; ++r) coup[i][r] = bl * vec[(size_t)r * dim + (dim - 1)];
      if (conv || last) {
        if (!conv) any_noconv = true;
        active[i] = 2;   // finished this cycle: its ground vector is formed below
      }
    }
    // Ritz vectors into the spare slots V[m+1 .. m+keep]
    for (int r = 0; r < keep; ++r) {
      for (size_t z = 0; z < Yh.size(); ++z) Yh[z] = make_double2(-Ys[r][z], 0.0);
      BCUDA(cudaMemcpyAsync(L.Y, Yh.data(), sizeof(double2) * Yh.size(), cudaMemcpyHostToDevice, s));
      BTRY(L.combine(L.V, m, L.Y, false, L.V + (size_t)(m + 1 + r) * n));
      BCUDA(cudaStreamSynchronize(s));
    }
    // finished instances: ground vector out of spare slot 0
    bool any_active = false;
    for (int i = 0; i < count; ++i) {
      if (active[i] == 2) {
        BCUDA(cudaMemcpyAsync(L.G + b->off[i], L.V + (size_t)(m + 1) * n + b->off[i],
                              sizeof(double2) * (b->off[i + 1] - b->off[i]), cudaMemcpyDeviceToDevice, s));
        active[i] = 0;
      }
      any_active = any_active || active[i] == 1;
    }
    BCUDA(cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    if (!any_active) break;
    // thick restart: V[0..keep-1] <- Ritz vectors, V[keep] <- V[m] (residual direction)
    for (int r = 0; r < keep; ++r)
      BCUDA(cudaMemcpyAsync(L.V + (size_t)r * n, L.V + (size_t)(m + 1 + r) * n, sizeof(double2) * n,
                            cudaMemcpyDeviceToDevice, s));
    BCUDA(cudaMemcpyAsync(L.V + (size_t)keep * n, L.V + (size_t)m * n, sizeof(double2) * n,
                          cudaMemcpyDeviceToDevice, s));
    p = keep;
  }
  // FP64-class Rayleigh quotients and residuals of every instance's vector
  std::vector<int> ones(count, 1);
  BCUDA(cudaMemcpyAsync(b->d_active, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
  BTRY(batch_apply_internal(b, L.G, L.W, FOCK_PREC_F64, nullptr, s));
  BTRY(L.dots(L.G, 1, L.W, L.H1));
  std::vector<double2> e1((size_t)count * L.ldh);
  BCUDA(cudaMemcpyAsync(e1.data(), L.H1, sizeof(double2) * e1.size(), cudaMemcpyDeviceToHost, s));
  BCUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) Yh[(size_t)i * L.ldh] = make_double2(e1[(size_t)i * L.ldh].x, 0.0);
  BCUDA(cudaMemcpyAsync(L.Y, Yh.data(), sizeof(double2) * Yh.size(), cudaMemcpyHostToDevice, s));
  BTRY(L.combine(L.G, 1, L.Y, true, L.W));
  BTRY(L.dots(L.W, 1, L.W, L.NR));
  std::vector<double2> r2((size_t)count * L.ldh);
  BCUDA(cudaMemcpyAsync(r2.data(), L.NR, sizeof(double2) * r2.size(), cudaMemcpyDeviceToHost, s));
  BCUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) {
    E0_out[i] = e1[(size_t)i * L.ldh].x;
    if (residual_out) residual_out[i] = sqrt(fmax(r2[(size_t)i * L.ldh].x, 0.0));
    if (iters_out) iters_out[i] = iters[i];
  }
  cleanup();
#undef BTRY
#undef BCUDA
  return any_noconv ? FOCK_ERR_NOCONV : FOCK_OK;
}
