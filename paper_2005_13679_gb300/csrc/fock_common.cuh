// fock_common.cuh -- internal types shared by the translation units of libfock.
//
// Nothing here is part of the C ABI (include/fock.h).  The hash used on the
// device is the closed form of Eq. TotalCost summed with the hockey-stick
// identity:
//
//     rank(n) = N_c - 1 - sum_{m=0}^{M-2} C(S_m + m, m + 1),   S_m = n_0 + ... + n_m,
//
// i.e. N_c - 1 - rank(n) is the combinatorial-number-system code of the strictly
// increasing sequence x_m = S_m + m.  It equals Algorithm 1's index (the cost of
// the particles placed in orbital m, summed over the basket sizes, telescopes to
// C(S_m + m, m) - C(S_{m-1} + m, m)).  Unranking (Algorithm 2) is the greedy
// decoding of that code, top orbital first.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <functional>

#include "../../include/fock.h"

#define FOCK_MAXM 12
#define FOCK_MAX_NRHS 16
#define FOCK_WS_HEADER 256   // bytes before the FP32-pair copy of C in an apply workspace

// Device-side status word bits (written with atomicOr by kernels that validate
// their inputs; read back by the host after the launch).
#define FOCK_DEVFLAG_INVALID 1u
#define FOCK_DEVFLAG_RANGE 2u

#define FOCK_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return fock_cuda_status(_e);      \
  } while (0)

static inline int fock_cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return FOCK_ERR_NOMEM;
  return FOCK_ERR_CUDA;
}

static inline int fock_pair_count(int M) { return M * (M + 1) / 2; }
__host__ __device__ static inline int fock_pair_index(int M, int k, int q) {
  // k <= q, lexicographic order of (k, q)
  return k * M - (k * (k - 1)) / 2 + (q - k);
}

// Binomial tables of one space.  Row m (0 <= m <= M-2) holds C(x, m+1) for
// x in [0, xdim).  `mod` entries are exact modulo 2^64 (wrapping Pascal sums),
// `sat` entries saturate at UINT64_MAX; 32-bit copies keep the low word (mod)
// or min(value, 2^32-1) (sat).  Target indices are sums and differences of
// `mod` entries, exact modulo the word size and therefore exact whenever the
// true index fits; searches compare against `sat` entries.
struct FockTables {
  int rows;   // M - 1 (at least 1 so that pointers are valid)
  int xdim;   // N + M + 3
  uint64_t *mod64, *sat64;  // device
  uint32_t *mod32, *sat32;  // device
};

struct fock_space {
  int32_t N, M;
  int64_t nc;
  int device;
  bool idx32;            // nc < 2^32 - 1: 32-bit index arithmetic
  FockTables tab;
  uint32_t *d_flag;      // one status word for validating kernels
  int32_t *d_j1;         // single-jump map or NULL
  int32_t *d_j2;         // double-jump map or NULL
  size_t j1_bytes, j2_bytes;
  // workspace of fock_density_matrices, kept between calls (grown on demand)
  void *dm_ws, *dm_part;
  size_t dm_ws_bytes, dm_part_bytes;
};

// One removal (one or two annihilated orbitals) and its slice of additions.
struct FockRemoval {
  int8_t k, q;        // q = -1 for a one-particle removal
  int8_t size;        // 1 or 2
  int8_t pad;
  int32_t a_beg, a_end;   // range in the addition arrays
  int32_t slot_base;      // r * P (two-body) or k * M (one-body) for the maps arm
};

// One addition (one or two created orbitals) with its coefficient index.
struct FockAddition {
  int8_t s, l;        // s = -1 for a one-particle addition
  int16_t a_index;    // pair index of (s, l) (two-body) or l (one-body)
};

struct FockTerm;

struct fock_ham {
  const fock_space *sp;
  int device;
  int nrem;                 // number of removal entries
  int nadd;                 // number of addition entries (total)
  bool real;                // all coefficients real
  bool dense;               // every (pair, pair) coefficient present (two-body only)
  int64_t config_terms;
  double coef_scale;        // coefficients stored divided by this power of two
  double max_abs_coef;
  // host copies
  FockRemoval *h_rem;
  FockAddition *h_add;
  double *h_coef;           // [nadd] complex, unscaled
  // device copies
  FockRemoval *d_rem;
  FockAddition *d_add;
  double2 *d_coef64;        // complex double, unscaled
  float4 *d_coefdf;         // (re_hi, im_hi, re_lo, im_lo) of coef / coef_scale
  float2 *d_coef32;         // complex float of coef / coef_scale
  double *d_sqrt64;         // sqrt(i), i in [0, N+3]
  float2 *d_sqrtdf;         // (hi, lo) split of sqrt(i)
  float *d_sqrt32;
  FockTerm *d_terms;        // [nadd] prefix-table offsets/corrections of each (removal, addition)
  float4 *d_gauss1;         // dense only: [P*P] (Re R, Re R + Im R) as FP32 pairs, scaled
  float4 *d_gauss2;         // dense only: [ceil(P/2)*P] (Im R - Re R) of rows 2i, 2i+1, scaled
  unsigned char *d_tc_a;    // dense, 2 <= M <= 6: digit image of R for the tensor-core phase 1
  int *d_tc_er;             // its row exponents
  unsigned char *d_tc_ma;   // the same for the FP32-mixed form (fp16 hi/lo split of R)
  int *d_tc_mer;
  // operators that conserve the pair weight k + q = s + l (reduced coefficients
  // block diagonal by the pair sum; fock_twophase_block.cu)
  bool pairsum;
  float4 *d_blk_df;         // block tables, (re_hi, im_hi, re_lo, im_lo) of coef / coef_scale
  float2 *d_blk_32;         // block tables, complex float, unscaled
  // ... whose blocks are rank one off the diagonal (contact interactions;
  // fock_twophase_pairs.cu): c_K, 2 c_K and D_r as pairs (scaled) and floats
  bool ps1;
  float2 *d_ps1_df;
  float *d_ps1_32;
  // nearest-neighbour operators (h on sites and bonds k, k + 1 mod M, W only
  // on-site): per-bond and per-site coefficients, indexed by the precision
  bool nn;
  int nn_nb;                // bonds: M - 1, or M for a ring
  double nn_scale;          // FOCK_PREC_F64 arrays stored divided by this power of two
  void *d_nn_bond[3];       // [2 nb] h_kl, h_lk of bond (k, k + 1 mod M)
  void *d_nn_e[3];          // [M][N + 1] site energies E_k(n) = h_kk n + W_kkkk n (n - 1) / 2
  void *d_nn_t[3];          // [N + 1][N + 1] hop amplitudes sqrt(a (b + 1)) (native FP64 only; null for large N)
  int32_t *d_slots;         // [nadd] jump-map slot of each term
  // workspace owned by the Hamiltonian (used when the caller passes none)
  void *ws;
  size_t ws_bytes;
  // kernel path and arm chosen by fock_autotune / fock_apply_set_path, per
  // precision and right-hand-side class (one, several); FOCK_PATH_AUTO = none
  int8_t tuned_path[3][2];
  int8_t tuned_arm[3][2];
  // profiling hook (fock_apply_set_events)
  cudaEvent_t ev_start, ev_stop;
  // buffers for fock_apply_H_host, and the stream and events that copy sigma
  // out by chunks while phase 2 of the two-phase path runs
  void *hb_in, *hb_out;
  size_t hb_bytes;
  cudaStream_t hb_copy;
  cudaEvent_t hb_ev[8];
  cudaStream_t hb_copy_in;  // chunked copy of C into hb_in, with hb_in_ev[0..7] after the chunks
  cudaEvent_t hb_in_ev[9];  // (and hb_in_ev[8] ordering that stream after the caller's)
};

// Launch helpers implemented in fock_apply.cu and used by fock_lanczos.cu.
// Device address of the fixed scratch array of fock_apply_H_noalloc on `dev`
// (looked up once per device with that device current, then cached).
int fock_noalloc_scratch(int dev, void **addr);
int fock_apply_internal(const fock_space *sp, const fock_ham *ham, const void *C, void *sigma,
                        int nrhs, int precision, int arm, void *ws, size_t ws_bytes,
                        cudaStream_t stream);
size_t fock_apply_ws_bytes(const fock_space *sp, const fock_ham *ham, int nrhs, int precision);
size_t fock_apply_ws_pref(const fock_space *sp, const fock_ham *ham, int nrhs, int precision);
int fock_prepare_df(const void *C, int64_t n, void *ws, int device, cudaStream_t stream);
int fock_get_sm_count(int device);

// H x -> y for the Lanczos driver: (precision, x, y, workspace, its bytes, stream).
typedef std::function<int(int, const void *, void *, void *, size_t, cudaStream_t)> FockApplyFn;
int fock_lanczos_run(int64_t n_vec, bool ham_real, int device, const FockApplyFn &apply_fn, size_t ws_bytes,
                     size_t ws_min,
                     int32_t max_iter, int32_t restart_len, double tol, uint64_t seed, int precision,
                     const void *start_dev, double *E0, double *residual, void *vec_dev, int32_t *iters,
                     cudaStream_t stream);
