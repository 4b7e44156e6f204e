/*
 * fock.h -- C ABI of the GB300 library for the bosonic Fock-space hot path of
 * Andriati & Gammal, "Hashing algorithms, optimized mappings and massive
 * parallelization of multiconfigurational methods for bosons"
 * (arXiv:2005.13679).
 *
 * The library computes, on one GPU, the action sigma = H C of the many-body
 * Hamiltonian (Eq. Haction)
 *
 *     H = sum_{kl} h_kl a^dag_k a_l + 1/2 sum_{kqsl} W_kqsl a^dag_k a^dag_q a_s a_l
 *
 * on coefficient vectors over the Fock basis of N bosons in M orbitals
 * (Eq. nc, N_c(N, M) = C(N+M-1, M-1) configurations), together with the
 * configuration hash (Eq. TotalCost, Algorithms 1 and 2), the single- and
 * double-jump index maps of Sec. 4, and a Lanczos ground-state driver (Sec. 6).
 *
 * Conventions used by every entry point:
 *   - orbitals are numbered 0..M-1, an occupation vector is int32 n[0..M-1]
 *     with sum N;
 *   - configuration indices are int64 and follow Algorithm 1: index 0 has all
 *     particles in orbital 0, index N_c - 1 has them all in orbital M - 1;
 *   - complex numbers are interleaved (re, im); h is row-major [M][M]
 *     (h[k*M+l] multiplies a^dag_k a_l), W is row-major [M][M][M][M]
 *     (W[((k*M+q)*M+s)*M+l] multiplies 1/2 a^dag_k a^dag_q a_s a_l);
 *   - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *     pointers are host pointers owned by the caller;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     calls are asynchronous on it unless stated otherwise;
 *   - every call returns an int status: FOCK_OK (0) or a negative FOCK_ERR_*
 *     code; fock_strerror() names it.  No call aborts the process, and on error
 *     no output is guaranteed unless the call says so.
 *
 * Ownership: fock_space and fock_ham objects are created and destroyed by the
 * library and bound to the CUDA device that was current at creation; they may
 * be shared by threads for read-only calls (rank, unrank, apply) but not
 * destroyed while a call on them is running.
 */
#ifndef FOCK_H
#define FOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------- */
/* Status codes                                                              */
/* ------------------------------------------------------------------------- */
#define FOCK_OK                  0
#define FOCK_ERR_ARG            -1   /* null pointer, size or enum out of range  */
#define FOCK_ERR_OVERFLOW       -2   /* N_c(N, M) >= 2^63                         */
#define FOCK_ERR_INVALID_CONFIG -3   /* an occupation vector is not in H(N, M)   */
#define FOCK_ERR_RANGE          -4   /* an index is outside [0, N_c)             */
#define FOCK_ERR_NOMEM          -5   /* a device allocation failed / won't fit   */
#define FOCK_ERR_NOT_HERMITIAN  -6   /* h or the two-body operator not Hermitian */
#define FOCK_ERR_ALIAS          -7   /* input and output buffers overlap         */
#define FOCK_ERR_CUDA           -8   /* a CUDA runtime call failed               */
#define FOCK_ERR_NOCONV         -9   /* Lanczos stopped before the tolerance     */
#define FOCK_ERR_UNSUPPORTED   -10   /* combination the library does not provide  */
#define FOCK_ERR_TIMEOUT       -11   /* a bounded device wait gave up            */
#define FOCK_ERR_NOT_BUILT     -12   /* jump maps requested but not built        */
#define FOCK_ERR_DEVICE        -13   /* object used on another device            */
#define FOCK_ERR_SCRATCH_LIMIT -14   /* request exceeds the fixed no-alloc scratch */
#define FOCK_ERR_NOT_CONSERVING -15  /* operator changes a sector's total weight  */

/* Human-readable name of a status code (static storage, never NULL). */
const char *fock_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int fock_version(void);

/* ------------------------------------------------------------------------- */
/* Configuration space H(N, M)  (Eq. nc; Sec. 3)                             */
/* ------------------------------------------------------------------------- */
typedef struct fock_space fock_space;

/* Create the space of N >= 1 bosons in 1 <= M <= 12 orbitals on the current
 * device: computes N_c(N, M) (Eq. nc) exactly and uploads the binomial tables
 * used by the hash (Eq. TotalCost).  Fails with FOCK_ERR_OVERFLOW when
 * N_c >= 2^63, FOCK_ERR_ARG for N < 1, M < 1 or M > 12, FOCK_ERR_CUDA or
 * FOCK_ERR_NOMEM on device errors.  *out is set only on success. */
int fock_space_create(int32_t N, int32_t M, fock_space **out);

/* Release the space, its tables and any jump maps.  NULL is accepted. */
int fock_space_destroy(fock_space *sp);

/* N_c(N, M), the number of configurations. */
int fock_space_size(const fock_space *sp, int64_t *nc);

/* Rank a batch of occupation vectors (Algorithm 1).  occ_dev is
 * [count][M] int32, idx_dev receives count int64 indices.  Rows that are not
 * valid configurations (a negative entry or a sum other than N) receive -1
 * and the call returns FOCK_ERR_INVALID_CONFIG after the whole batch ran.
 * Synchronous: waits on `stream` to read the validity flag. */
int fock_rank(const fock_space *sp, const int32_t *occ_dev, int64_t count,
              int64_t *idx_dev, void *stream);

/* Unrank a batch of indices (Algorithm 2).  idx_dev has count int64 entries,
 * occ_dev receives [count][M] int32.  An index outside [0, N_c) gives a row
 * of -1 and FOCK_ERR_RANGE after the whole batch ran.  Synchronous. */
int fock_unrank(const fock_space *sp, const int64_t *idx_dev, int64_t count,
                int32_t *occ_dev, void *stream);

/* ------------------------------------------------------------------------- */
/* Jump maps  (Sec. 4, "Mapping routines"; Fig. 4)                          */
/* ------------------------------------------------------------------------- */
#define FOCK_MAP_SINGLE 1   /* one particle k -> l                           */
#define FOCK_MAP_DOUBLE 2   /* two particles {k, q} -> {s, l}                */

/* Build the jump maps selected by `which` (a mask of FOCK_MAP_*) on the
 * device, owned by the space.  Layouts, chosen so that consecutive
 * configurations are consecutive in memory:
 *   single: int32 J1[(k*M + l) * N_c + gamma] = index of n(gamma) - e_k + e_l,
 *           or -1 when n_k = 0 (k == l gives gamma itself when n_k >= 1);
 *   double: int32 J2[(r*P + a) * N_c + gamma], P = M(M+1)/2, where r and a
 *           number the pairs k <= q in lexicographic order
 *           (pair(k, q) = k*M - k(k-1)/2 + (q - k)); the entry is the index of
 *           n(gamma) - e_k - e_q + e_s + e_l for r = (k, q) and a = (s, l), or
 *           -1 when r cannot be removed (n_k, n_q >= 1, and n_k >= 2 if k == q).
 * Memory: 4*M*M*N_c bytes (single) and 4*P*P*N_c bytes (double); both need
 * N_c < 2^31.  With dry_run != 0 nothing is built and *bytes receives the
 * total; otherwise *bytes (may be NULL) receives the bytes now held.
 * FOCK_ERR_NOMEM when the maps do not fit in free device memory. */
int fock_build_jump_maps(fock_space *sp, int which, int dry_run, size_t *bytes, void *stream);

/* Read-only device pointer to a built map (see layouts above), its number of
 * slots (M*M or P*P) and the slot stride in elements (N_c).
 * FOCK_ERR_NOT_BUILT if that map is not built. */
int fock_jump_map_get(const fock_space *sp, int which, const int32_t **map_dev,
                      int64_t *slots, int64_t *slot_stride);

/* Free the jump maps (the space stays valid). */
int fock_jump_maps_free(fock_space *sp);

/* ------------------------------------------------------------------------- */
/* Hamiltonian  (Eqs. noninteracting, interacting; Sec. 2)                   */
/* ------------------------------------------------------------------------- */
typedef struct fock_ham fock_ham;

/* Stage h ([M][M] complex, interleaved) and W ([M]^4 complex, or NULL for a
 * one-body operator) for the space.  The two-body operator depends only on the
 * multisets {k, q} and {s, l}, so W is reduced to one coefficient per pair of
 * multisets (summing the orderings); for N >= 2 the one-body term is folded
 * into that reduced two-body form through sum_x a^dag_k a^dag_x a_x a_l =
 * (N - 1) a^dag_k a_l on H(N, M).  When tol >= 0 the call checks that h and
 * the reduced two-body operator are Hermitian to within tol times the largest
 * coefficient and returns FOCK_ERR_NOT_HERMITIAN otherwise; tol < 0 skips the
 * check (the apply is defined for any coefficients).  Host buffers are
 * copied; the caller keeps ownership. */
int fock_hamiltonian_create(const fock_space *sp, const double *h_host,
                            const double *W_host, double tol, fock_ham **out);

/* Release a Hamiltonian and its device workspace.  NULL is accepted. */
int fock_hamiltonian_destroy(fock_ham *ham);

/* Operation count of one apply, in "configuration terms": the number of
 * (configuration, operator-string) pairs with a nonzero coefficient,
 *   N_c + N_c(N-1, M) * #{k != l : h_kl != 0}
 *       + N_c(N-2, M) * #{(r, a) : reduced two-body coefficient != 0},
 * independent of the implementation (the throughput metric's numerator). */
int fock_hamiltonian_terms(const fock_ham *ham, int64_t *config_terms);

/* Nonzero 1 if every coefficient is real (imaginary parts all zero). */
int fock_hamiltonian_is_real(const fock_ham *ham, int *is_real);

/* Structure found in the operator when it was created, as FOCK_FORM_* bits:
 * DENSE every reduced two-body coefficient present; PAIR_WEIGHT reduced
 * coefficients only between pairs of equal orbital sum (k + q = s + l);
 * PAIR_MOMENTUM additionally rank one off the diagonal inside every pair-sum
 * block with real entries (contact interactions, Sec. 6): the two-phase
 * pair-weight path then runs through the 2M - 1 pair-momentum amplitudes;
 * NEAREST_NEIGHBOUR the Bose-Hubbard class served by FOCK_PATH_NN. */
#define FOCK_FORM_DENSE 1
#define FOCK_FORM_PAIR_WEIGHT 2
#define FOCK_FORM_PAIR_MOMENTUM 4
#define FOCK_FORM_NEAREST_NEIGHBOUR 8
int fock_hamiltonian_forms(const fock_ham *ham, int32_t *forms);

/* ------------------------------------------------------------------------- */
/* sigma = H C  (Eq. Haction)                                                */
/* ------------------------------------------------------------------------- */
/* precision */
#define FOCK_PREC_F64        0  /* complex128 in/out; FP32-pair arithmetic
                                   (48-bit significands); on the tensor-core
                                   path each entry is within 2^-39.9 B of the
                                   exact sigma, B = sum_r |A_r| ||R_r||_1
                                   max|X| (the bound in fock_apply_tc.cuh),
                                   measured 9e-14 normwise on random states */
#define FOCK_PREC_F64_NATIVE 1  /* complex128 in/out; native FP64 arithmetic */
#define FOCK_PREC_F32_MIXED  2  /* complex64 in/out; FP32 products, FP32-pair
                                   accumulation per configuration             */
/* arm */
#define FOCK_ARM_AUTO 0         /* library's choice                            */
#define FOCK_ARM_HASH 1         /* target indices from the hash on the fly    */
#define FOCK_ARM_MAPS 2         /* target indices from the built jump maps    */

/* Kernel paths of the apply (fock_apply_path, fock_apply_set_path,
 * fock_autotune).  AUTO takes the first that can serve the call in the order
 * listed: the two-phase evaluation through the (N-2)-particle space with its
 * first phase on the tensor cores (dense reduced coefficients, 2 <= M <= 6,
 * FOCK_PREC_F64 or FOCK_PREC_F32_MIXED, hash arm, the preferred workspace),
 * the same with FP32 phase 1 (M <= 8), the nearest-neighbour kernel (h only on
 * sites and bonds k, k+1, a ring when h_{0,M-1} != 0, W only on-site; hash
 * arm), the register-resident dense kernel (dense coefficients, M <= 10), the
 * sparse kernel (at most 2048 reduced coefficients), the list kernel (always;
 * the only path for N_c >= 2^32 - 1).  The two-phase evaluation for operators
 * that conserve the pair weight (FOCK_PATH_TWOPHASE_BLOCK: every reduced
 * coefficient links pairs {k, q} and {s, l} with k + q = s + l, as the
 * Lieb-Liniger ring in plane waves, Sec. 6, where k + q is the pair's
 * momentum; 2 <= M <= 12, FOCK_PREC_F64 or FOCK_PREC_F32_MIXED, hash arm, the
 * preferred workspace) comes after the dense two-phase paths: its reduced
 * coefficients are block diagonal by the pair sum, so phase 1 evaluates
 * sum_K |block K|^2 products per (N-2)-particle configuration. */
#define FOCK_PATH_AUTO        0
#define FOCK_PATH_TWOPHASE_TC 1
#define FOCK_PATH_TWOPHASE    2
#define FOCK_PATH_NN          3
#define FOCK_PATH_DENSE       4
#define FOCK_PATH_SPARSE      5
#define FOCK_PATH_LIST        6
#define FOCK_PATH_TWOPHASE_BLOCK 7

/* The path an apply with these options takes (a workspace of
 * workspace_bytes, 0 for none), honouring a path set by fock_autotune or
 * fock_apply_set_path.  FOCK_ERR_NOT_BUILT for FOCK_ARM_MAPS without maps. */
int fock_apply_path(const fock_space *sp, const fock_ham *ham, int32_t nrhs, int precision, int arm,
                    size_t workspace_bytes, int32_t *path);

/* Pin the path (and arm) later applies with this precision and right-hand-
 * side class (nrhs == 1 or > 1) take when the caller passes FOCK_ARM_AUTO
 * (or the same arm).  A path that cannot serve a call falls back to the
 * built-in order for that call; a choice on FOCK_ARM_MAPS lapses while the
 * jump maps are not built (freed, or never built).  FOCK_PATH_AUTO clears
 * the choice. */
int fock_apply_set_path(fock_ham *ham, int32_t nrhs, int precision, int path, int arm);

typedef struct fock_tuning {
  int32_t path;        /* FOCK_PATH_* chosen                                  */
  int32_t arm;         /* FOCK_ARM_HASH or FOCK_ARM_MAPS                      */
  int32_t candidates;  /* (path, arm) pairs timed; 0 when read from the cache */
  int32_t from_cache;  /* 1 when the choice came from cache_path              */
  double ms;           /* mean time of one apply with the choice              */
} fock_tuning;

/* Autotuner: times every (path, arm) that can serve applies with these
 * options (the maps arm only if maps are built) on device buffers it
 * allocates (a deterministic test vector, the preferred workspace): one
 * warm-up apply and three timed ones each, CUDA events on `stream`.  The
 * fastest becomes this Hamiltonian's choice (fock_apply_set_path).  With
 * cache_path not NULL a line keyed by (N, M, reduced coefficients, removal
 * lists, realness, nrhs, precision, SM count) is looked up first and the
 * measured choice appended after tuning.  Synchronous; FOCK_ERR_NOMEM when
 * the tuning buffers do not fit. */
int fock_autotune(const fock_space *sp, fock_ham *ham, int32_t nrhs, int precision, const char *cache_path,
                  fock_tuning *out, void *stream);

/* Profiling hook: when set, every apply with this Hamiltonian records
 * start_event immediately before and stop_event immediately after its main
 * H C kernel, on the apply's stream (the input preparation of FOCK_PREC_F64 is
 * outside the pair).  For the two-phase evaluation of dense coefficients the
 * main kernel is the first phase (the product with the reduced coefficients
 * over the (N-2)-particle space); the second phase follows the stop event.
 * Sector applies (fock_sector_apply_H) with this Hamiltonian record the pair
 * the same way.  Events are cudaEvent_t passed as void*, owned by the caller; NULL, NULL
 * clears the hook.  Not thread-safe with concurrent applies on the same
 * Hamiltonian. */
int fock_apply_set_events(fock_ham *ham, void *start_event, void *stop_event);

/* Device workspace (bytes) an apply with these options needs; 0 if none. */
int fock_apply_workspace_size(const fock_space *sp, const fock_ham *ham, int32_t nrhs,
                              int precision, size_t *bytes);

/* sigma = H C for nrhs vectors stored [N_c][nrhs] (configuration-major, the
 * nrhs values of one configuration adjacent), complex128 for FOCK_PREC_F64*
 * and complex64 for FOCK_PREC_F32_MIXED.  1 <= nrhs <= 16.  C_dev and
 * sigma_dev must not overlap (FOCK_ERR_ALIAS).  Each sigma_gamma is computed
 * by one thread from the configurations reached by removing one or two
 * particles from gamma and adding them back (pull form), so no atomics are
 * used and results are deterministic.  workspace_dev may be NULL, in which
 * case a buffer owned by `ham` is allocated on first use (grown when needed);
 * otherwise it must hold fock_apply_workspace_size() bytes.  Asynchronous on
 * `stream`.  FOCK_ERR_NOT_BUILT for FOCK_ARM_MAPS without the maps. */
int fock_apply_H(const fock_space *sp, const fock_ham *ham, const void *C_dev,
                 void *sigma_dev, int32_t nrhs, int precision, int arm,
                 void *workspace_dev, size_t workspace_bytes, void *stream);

/* Status of the last apply that ran the tensor-core phase 1 (the first path
 * of the list above) with this workspace.  Its bounded device waits give up
 * after about a second; phase 2 then writes NaN to sigma.  fock_apply_H and
 * fock_apply_H_noalloc return before the device work ends, so they report
 * FOCK_OK in that case; this call waits on `stream` and returns
 * FOCK_ERR_TIMEOUT if that apply's wait gave up, FOCK_OK otherwise.
 * workspace_dev is the workspace passed to fock_apply_H (NULL: the
 * Hamiltonian's own workspace, the one fock_apply_H with a NULL workspace and
 * fock_apply_H_host use); with noalloc != 0 the fixed array of
 * fock_apply_H_noalloc on the space's device is read instead.  Reads 4 bytes
 * from the device; allocates nothing.  fock_apply_H_host checks this itself. */
int fock_apply_check(const fock_space *sp, const fock_ham *ham, const void *workspace_dev, int noalloc,
                     void *stream);

/* Test hook, process-wide: poll budget of the bounded waits inside the
 * tensor-core phase 1 (its producer, MMA-issue and epilogue roles).
 * polls < 0 restores the default (2^20 polls, about a second); 0 makes every
 * such wait give up at once, so that the abort path (status word, NaN sigma,
 * FOCK_ERR_TIMEOUT) runs without a fault or a hang.  The wait that lets the
 * MMAs already issued finish before tensor memory is released always keeps
 * the default.  FOCK_ERR_ARG for polls above the default. */
int fock_debug_set_wait_polls(int64_t polls);

/* Same as fock_apply_H with host buffers: copies C_host to the device, applies
 * and copies sigma back into sigma_host, then waits on `stream`.  Device
 * buffers are owned by `ham` and reused across calls.  For pinned (page-locked)
 * host memory the copies run at full link speed. */
int fock_apply_H_host(const fock_space *sp, const fock_ham *ham, const void *C_host,
                      void *sigma_host, int32_t nrhs, int precision, int arm, void *stream);

/* sigma = H C with FOCK_PREC_F64 for callers that must not allocate device
 * memory.  The paper has no counterpart; this is an interface convenience.
 * Some callers cannot let a library allocate: their device memory belongs to
 * another allocator (a caching allocator or a fixed pool that must not be
 * bypassed), or they call in a loop where a cudaMalloc/cudaFree would
 * synchronise the device and stall their other streams.  This call takes its
 * scratch (status words plus a hi/lo split copy of C, 256 + 16*N_c*nrhs bytes)
 * from a fixed array of FOCK_NOALLOC_SCRATCH_BYTES (64 MiB) compiled into the
 * library; every GPU that loads the library keeps that array until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 * The caller still owns C_dev and sigma_dev (layouts as for fock_apply_H).
 *   - Requests needing more scratch than the array holds (N_c * nrhs above
 *     4,194,288) fail with FOCK_ERR_SCRATCH_LIMIT before any device work.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - All calls on a device share the one array and each call rewrites the
 *     parts it reads, so results do not depend on earlier calls; but calls
 *     whose work overlaps on the GPU (different streams, or host threads
 *     without ordering) race on the array and must be serialised.
 * Asynchronous on `stream`; other errors as for fock_apply_H. */
#define FOCK_NOALLOC_SCRATCH_BYTES (64u << 20)
int fock_apply_H_noalloc(const fock_space *sp, const fock_ham *ham, const void *C_dev,
                         void *sigma_dev, int32_t nrhs, int arm, void *stream);

/* ------------------------------------------------------------------------- */
/* Lanczos ground state  (Sec. 6)                                            */
/* ------------------------------------------------------------------------- */
/* Lowest eigenvalue of H by Lanczos with full re-orthogonalisation inside
 * restart cycles of restart_len vectors.  A cycle ends with a thick restart
 * (Wu and Simon): the next cycle starts from the lowest Ritz vectors of the
 * cycle (min(restart_len / 3, 8) of them, at least one) and the last residual
 * direction.  With FOCK_PREC_F32_MIXED products the solver first converges to
 * the mixed apply's own floor (1e-5 relative residual), then continues with
 * FOCK_PREC_F64 products from the current Ritz vector (final FP64
 * refinement).  Krylov vectors and all orthogonalisation are FP64 (real when
 * the Hamiltonian is real, complex otherwise); the H C products use
 * `precision`; the returned E0 is the FP64 Rayleigh quotient of the final
 * unit vector with a FOCK_PREC_F64 apply, and *residual (may be NULL) is
 * ||H v - E0 v|| for it.  Stops when the residual estimate is below
 * tol * max(|E0|, 1) or after max_iter products.  start_dev (may be NULL) is
 * an N_c complex128 start vector; otherwise one is drawn from `seed` with the
 * SplitMix64 generator.  vec_dev (may be NULL) receives the unit ground vector
 * as N_c complex128.  Synchronous.  Returns FOCK_ERR_NOCONV with the best E0
 * when max_iter is reached first. */
int fock_lanczos_ground(const fock_space *sp, const fock_ham *ham, int32_t max_iter,
                        int32_t restart_len, double tol, uint64_t seed, int precision,
                        const void *start_dev, double *E0, double *residual,
                        void *vec_dev, int32_t *iters, void *stream);

/* Short-iterative-Lanczos time step C <- exp(-i H dt) C (the SIL integrator
 * the paper names as a consumer of H C, Sec. 2).  C_dev: N_c complex128 on
 * the space's device, overwritten.  The Krylov space of C (Lanczos vectors
 * orthogonalised twice against all previous ones) grows until the weight of
 * the next vector in exp(-i T dt) e_0 is below tol (relative to ||C||), the
 * space is invariant, or max_krylov (1..128) vectors are used; T is the
 * tridiagonal projection of H, exponentiated by its eigen-decomposition on
 * the host.  Products use `precision` (FOCK_PREC_F64, _F64_NATIVE or
 * _F32_MIXED).  *krylov_used and *err_est (may be NULL) receive the Krylov
 * dimension and the final weight.  Allocates max_krylov + 1 vectors and the
 * apply workspace.  Synchronous.  Returns FOCK_ERR_NOCONV (C still updated
 * with the best estimate) when max_krylov vectors were not enough. */
int fock_sil_step(const fock_space *sp, const fock_ham *ham, void *C_dev, double dt,
                  int32_t max_krylov, double tol, int precision, int32_t *krylov_used,
                  double *err_est, void *stream);

/* ------------------------------------------------------------------------- */
/* Density matrices                                                          */
/* ------------------------------------------------------------------------- */
/* One- and two-body density matrices of the state C (Eqs. rho1 and rho2):
 *     rho1_host[2 (k M + l) + {0,1}]             = <C| a^dag_k a_l |C>,
 *     rho2_host[2 (((k M + l) M + q) M + s) + {0,1}] = <C| a^dag_k a^dag_l a_q a_s |C>,
 * complex128 interleaved, host memory of M^2 and M^4 complex values; either
 * may be NULL (not both).  C_dev holds N_c complex128 values on the space's
 * device (not required to be normalised).  rho2 is the Gram matrix of the
 * vectors a_q a_s C over the (N-2)-particle configurations; when both are
 * asked for (N >= 2), rho1 is its partial trace (sum_x rho2[k][x][x][l] =
 * (N - 1) rho1[k][l]); asked for alone, rho1 is the Gram matrix of the
 * vectors a_l C over the (N-1)-particle configurations.  Each warp reduces
 * tiles of 32 configurations: FP32-pair products within a tile, FP64 sums
 * across tiles, the warps' sums added in a fixed order (deterministic).
 * rho2 is zero for N < 2.  Allocates its device workspace (16 B per
 * configuration plus the partial sums) on the first call and keeps it with the
 * space, grown when a call needs more; fock_space_destroy releases it.  Calls
 * on one space share that workspace and must not overlap.  Synchronous on
 * `stream`.
 * FOCK_ERR_UNSUPPORTED for M > 12 or N_c >= 2^32 - 1; FOCK_ERR_DEVICE when
 * the current device is not the space's. */
int fock_density_matrices(const fock_space *sp, const void *C_dev, double *rho1_host, double *rho2_host,
                          void *stream);

/* ------------------------------------------------------------------------- */
/* Sectors of fixed total orbital weight Q = sum_i i n_i                     */
/* ------------------------------------------------------------------------- */
/* With the plane-wave orbitals of Sec. 6 (orbital i of momentum
 * (i - floor(M/2)) 2 pi / L) a sector is a total-momentum sector,
 * P = (Q - N floor(M/2)) 2 pi / L.  An operator with diagonal h and
 * W_kqsl = 0 unless k + q = s + l (Lieb-Liniger, Sec. 6) maps each sector into
 * itself (total momentum is conserved), so its eigenproblem and its dynamics
 * restrict to one sector, about N (M - 1) + 1 times smaller than H(N, M).
 * This restriction is not in the paper; it follows from the conservation law.
 * Sector vectors are ordered as H(N, M) orders its configurations (Algorithm
 * 1), restricted to the sector, and stored [N_sec][nrhs] like full vectors. */
typedef struct fock_sector fock_sector;

/* The sector of weight Q of the space (0 <= Q <= N (M - 1), FOCK_ERR_ARG
 * otherwise).  Builds the counting tables D_m(s, q) (configurations of s
 * particles in orbitals 0..m-1 of weight q; host uint64 and device mod 2^32,
 * (2M - 3)(N + 1)(Q + 1) words on the device).  FOCK_ERR_OVERFLOW when the
 * sector holds 2^31 configurations or more; FOCK_ERR_UNSUPPORTED when
 * M (N + 1)(Q + 1) exceeds 2^28 table entries.  The sector refers to `sp`,
 * which must outlive it. */
int fock_sector_create(const fock_space *sp, int64_t Q, fock_sector **out);
int fock_sector_destroy(fock_sector *sec);
int fock_sector_size(const fock_sector *sec, int64_t *n_sector);

/* Sector indices of `count` occupation vectors (int32 [count][M], device).
 * Vectors that are not configurations of the sector (negative entries, sum
 * != N, weight != Q) get -1 and the call returns FOCK_ERR_INVALID_CONFIG
 * after the whole batch ran.  Synchronous on `stream`. */
int fock_sector_rank(const fock_sector *sec, const int32_t *occ_dev, int64_t count, int64_t *idx_dev,
                     void *stream);

/* Occupation vectors of `count` sector indices; indices outside [0, N_sec)
 * give rows of -1 and FOCK_ERR_RANGE.  Synchronous on `stream`. */
int fock_sector_unrank(const fock_sector *sec, const int64_t *idx_dev, int64_t count, int32_t *occ_dev,
                       void *stream);

/* Terms one sector apply evaluates: sum over the operator's removal lists of
 * (additions) x (sector configurations in which the removal is possible).
 * FOCK_ERR_NOT_CONSERVING if a term changes the weight; FOCK_ERR_ARG if `ham`
 * was built on another space. */
int fock_sector_terms(const fock_sector *sec, const fock_ham *ham, int64_t *terms);

/* Device workspace fock_sector_apply_H wants (FOCK_PREC_F64: 256 B + 16 B per
 * configuration per right-hand side; 0 otherwise). */
int fock_sector_workspace_size(const fock_sector *sec, int32_t nrhs, int precision, size_t *bytes);

/* sigma = H C within the sector (Eq. Haction restricted), precisions and
 * buffer rules as fock_apply_H (complex128 or complex64, [N_sec][nrhs],
 * 1 <= nrhs <= 16, no aliasing).  `ham` must have been created on the
 * sector's space and conserve the weight (FOCK_ERR_NOT_CONSERVING otherwise,
 * checked on the host before any launch).  A NULL or short workspace makes
 * the sector allocate and keep its own.  Asynchronous on `stream`. */
int fock_sector_apply_H(const fock_sector *sec, const fock_ham *ham, const void *C_dev, void *sigma_dev,
                        int32_t nrhs, int precision, void *workspace_dev, size_t workspace_bytes,
                        void *stream);

/* Lanczos ground state within the sector: fock_lanczos_ground's algorithm,
 * arguments and statuses, over vectors of N_sec entries (vec_dev, if not
 * NULL, receives N_sec complex128 entries). */
int fock_sector_lanczos_ground(const fock_sector *sec, const fock_ham *ham, int32_t max_iter,
                               int32_t restart_len, double tol, uint64_t seed, int precision,
                               const void *start_dev, double *E0, double *residual, void *vec_dev,
                               int32_t *iters, void *stream);

/* ------------------------------------------------------------------------- */
/* Uneven batches of independent problems                                    */
/* ------------------------------------------------------------------------- */
typedef struct fock_batch fock_batch;

/* Stage `count` independent problems (N[i] bosons in M[i] orbitals with h[i],
 * W[i] as for fock_hamiltonian_create; W[i] may be NULL) on the current
 * device.  Their coefficient vectors are concatenated in instance order
 * (instance i at offsets[i]..offsets[i+1], see fock_batch_offsets), complex
 * interleaved.  An instance with at least 2^18 configurations whose default
 * single-vector FP64-class path is a two-phase one (FOCK_PATH_TWOPHASE_TC,
 * FOCK_PATH_TWOPHASE, FOCK_PATH_TWOPHASE_BLOCK) gets an apply of its own, one
 * after another on the stream with one shared workspace.  Every other
 * instance is served by one persistent launch: a block takes work items (a
 * range of configurations of one instance, largest instances first) from an
 * atomic queue and stages that instance's tables in shared memory when the
 * instance changes.  Requires N_c < 2^32 - 1 per instance.  Hermiticity is
 * checked as in fock_hamiltonian_create with tol. */
int fock_batch_create(int32_t count, const int32_t *N, const int32_t *M, const double *const *h_host,
                      const double *const *W_host, double tol, fock_batch **out);
int fock_batch_destroy(fock_batch *b);

/* offsets[0..count] of the instances in concatenated vectors (host array). */
int fock_batch_offsets(const fock_batch *b, int64_t *offsets);

/* own[0..count-1]: 1 where the instance has an apply of its own (see
 * fock_batch_create), 0 where the persistent launch serves it (host array). */
int fock_batch_own_apply(const fock_batch *b, int32_t *own);

/* Sum of the instances' configuration terms (see fock_hamiltonian_terms). */
int fock_batch_terms(const fock_batch *b, int64_t *config_terms);

/* sigma = H_i C_i for every instance i, precision FOCK_PREC_F64 (complex128,
 * FP32-pair arithmetic; one scale for the instances of the persistent launch,
 * so their vectors should lie within 2^100 of each other in magnitude; an
 * instance with its own apply is scaled by itself) or FOCK_PREC_F32_MIXED
 * (complex64).  Buffers as for fock_apply_H, concatenated.  Device scratch
 * (queue counter, FP32-pair split copy of the instances of the persistent
 * launch, the shared workspace of the others) is owned by the batch and
 * allocated by the first call.  Asynchronous on `stream`. */
int fock_batch_apply(fock_batch *b, const void *C_dev, void *sigma_dev, int precision, void *stream);

/* Autotuner: times the persistent launch of fock_batch_apply on the caller's
 * buffers (contents are overwritten in sigma only; nothing is timed when every
 * instance has its own apply) for work items of 1..32 tiles of 128
 * configurations and 1..4 resident blocks per SM, keeps the fastest for this
 * batch and precision, and reports it.  If cache_path is not NULL the choice
 * is read from / appended to that text file, keyed by the instance sizes, the
 * precision and the SM count.  Synchronous. */
int fock_batch_autotune(fock_batch *b, const void *C_dev, void *sigma_dev, int precision,
                        const char *cache_path, int32_t *tiles_per_item, int32_t *blocks_per_sm,
                        void *stream);

/* Lanczos ground state of every instance (as fock_lanczos_ground, FP64 Krylov
 * vectors, FP64-class products, thick restart with restart_len vectors).  Each
 * restart cycle of every instance runs as one CUDA graph replay: the batched
 * apply, the segmented re-orthogonalisation, the norms and the scalings stay
 * on the device; the host only solves the small projected problems between
 * cycles.  E0_out, residual_out and iters_out have `count` entries.  Returns
 * FOCK_ERR_NOCONV if any instance stopped at max_iter.  Synchronous. */
int fock_batch_lanczos_ground(fock_batch *b, int32_t max_iter, int32_t restart_len, double tol,
                              uint64_t seed, double *E0_out, double *residual_out, int32_t *iters_out,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FOCK_H */
