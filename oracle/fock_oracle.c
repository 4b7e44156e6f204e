/*
 * fock_oracle.c -- plain, slow CPU oracle for the bosonic Fock-space hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, table or helper with the CUDA
 * library: every quantity here is computed the long way, in the order the
 * paper states it, in IEEE double precision with a fixed loop order.
 *
 * Conventions (Andriati & Gammal, arXiv:2005.13679):
 *   - orbitals are numbered 0..M-1 (Sec. 3, "Mapping Fock states to integers");
 *   - an occupation vector n[0..M-1] holds N particles in total (Eq. constraint);
 *   - complex numbers are stored interleaved (re, im);
 *   - h[k*M + l] multiplies a^dag_k a_l;
 *   - W[((k*M + q)*M + s)*M + l] multiplies (1/2) a^dag_k a^dag_q a_s a_l.
 *
 * Parity status of each entry point is stated in its comment ("pinned by").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Eq. nc: number of configurations N_c(n, m) = C(n + m - 1, m - 1).        */
/* Eq. TotalCost adds the convention N_c(n, 0) = 0.  Returns -1 when the    */
/* count does not fit in a signed 64-bit integer.                          */
/* Pinned by: brute-force enumeration counts (tests).                      */
/* ------------------------------------------------------------------------ */
int64_t oracle_nc(int64_t n, int64_t m)
{
    if (m <= 0) return 0;
    if (n < 0) return 0;
    /* C(n+m-1, m-1) built as prod_{i=1}^{m-1} (n+i)/i; every partial product
     * C(n+i, i) is an integer, so the division is exact. */
    __int128 r = 1;
    for (int64_t i = 1; i <= m - 1; ++i) {
        r = r * (n + i) / i;
        if (r > (__int128)INT64_MAX) return -1;
    }
    return (int64_t)r;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Get index from a configuration), Sec. 3.  The index is the  */
/* total cost of Eq. TotalCost: going from the highest orbital down to      */
/* orbital 1, each particle placed in orbital m adds N_c(s, m), where s is  */
/* the number of particles still in the basket.                            */
/* Pinned by: Fig. 2 worked example (index 17) and brute-force ordering.   */
/* ------------------------------------------------------------------------ */
int64_t oracle_rank(int N, int M, const int32_t *n)
{
    int64_t k = 0;
    int64_t s = N;
    for (int m = M - 1; m >= 1; --m) {
        int32_t j = n[m];
        while (j > 0) {
            k += oracle_nc(s, m);
            s -= 1;
            j -= 1;
        }
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (Build configuration from index), Sec. 3.  Starting from the */
/* top orbital with all N particles in the basket, a particle is put in     */
/* orbital m whenever the remaining index is at least its cost N_c(s, m);  */
/* otherwise the search moves one orbital down.  What is left in the basket */
/* at the end goes to orbital 0.                                            */
/* Pinned by: round trip with Algorithm 1 and brute-force ordering.        */
/* ------------------------------------------------------------------------ */
void oracle_unrank(int N, int M, int64_t beta, int32_t *n)
{
    for (int i = 0; i < M; ++i) n[i] = 0;
    int64_t k = beta;
    int m = M - 1;
    int64_t s = N;
    while (k > 0) {
        while (k - oracle_nc(s, m) < 0) m -= 1;
        k -= oracle_nc(s, m);
        n[m] += 1;
        s -= 1;
    }
    if (s > 0) n[0] += (int32_t)s;
}

void oracle_rank_batch(int N, int M, const int32_t *occ, int64_t count, int64_t *idx)
{
    for (int64_t i = 0; i < count; ++i) idx[i] = oracle_rank(N, M, occ + i * M);
}

void oracle_unrank_batch(int N, int M, const int64_t *idx, int64_t count, int32_t *occ)
{
    for (int64_t i = 0; i < count; ++i) oracle_unrank(N, M, idx[i], occ + i * M);
}

/* ------------------------------------------------------------------------ */
/* Single-jump map (Sec. 4, "Mapping routines"): for every configuration    */
/* gamma and every pair (k, l), the index of the configuration reached by   */
/* removing one particle from k and placing it in l, or -1 when orbital k   */
/* is empty.  Layout [Nc][M][M].  Built by definition: Alg. 2, edit, Alg. 1.*/
/* Pinned by: brute-force index dictionary (tests).                        */
/* ------------------------------------------------------------------------ */
void oracle_single_jump_map(int N, int M, int32_t *out)
{
    int64_t nc = oracle_nc(N, M);
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    for (int64_t g = 0; g < nc; ++g) {
        oracle_unrank(N, M, g, n);
        for (int k = 0; k < M; ++k) {
            for (int l = 0; l < M; ++l) {
                int32_t *dst = out + (g * M + k) * M + l;
                if (n[k] < 1) { *dst = -1; continue; }
                n[k] -= 1; n[l] += 1;
                *dst = (int32_t)oracle_rank(N, M, n);
                n[l] -= 1; n[k] += 1;
            }
        }
    }
    free(n);
}

/* A pair of annihilations a_q a_k (k <= q) can act on n iff both orbitals   */
/* hold a particle, and, when k == q, the orbital holds at least two        */
/* (a_k a_k on a single particle gives zero).  Sec. 4 and Fig. 4.           */
static int removal_allowed(const int32_t *n, int k, int q)
{
    if (k == q) return n[k] >= 2;
    return n[k] >= 1 && n[q] >= 1;
}

/* Number of allowed removal pairs (k <= q) of one configuration. */
int32_t oracle_removal_count(int M, const int32_t *n)
{
    int32_t c = 0;
    for (int k = 0; k < M; ++k)
        for (int q = k; q < M; ++q)
            if (removal_allowed(n, k, q)) c += 1;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Double-jump map with variable-length rows (Sec. 4 and Fig. 4).  Row gamma */
/* lists, for every allowed removal pair (k <= q) in lexicographic order, a */
/* stride of M*M entries: entry s*M + l is the index of the configuration   */
/* after removing one particle from k and one from q and adding one to s    */
/* and one to l.  row_off has Nc+1 entries (offsets in int32 elements).     */
/* Call with out == NULL to obtain only the offsets.                        */
/* Pinned by: brute-force index dictionary, Fig. 4 counts (4 strides of    */
/* 5*5 for M=5, N=4 versus 5^4 = 625, and 3 strides skipped).              */
/* ------------------------------------------------------------------------ */
void oracle_double_jump_map(int N, int M, int64_t *row_off, int32_t *out)
{
    int64_t nc = oracle_nc(N, M);
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int64_t off = 0;
    for (int64_t g = 0; g < nc; ++g) {
        oracle_unrank(N, M, g, n);
        row_off[g] = off;
        for (int k = 0; k < M; ++k) {
            for (int q = k; q < M; ++q) {
                if (!removal_allowed(n, k, q)) continue;
                if (out) {
                    n[k] -= 1; n[q] -= 1;
                    for (int s = 0; s < M; ++s) {
                        for (int l = 0; l < M; ++l) {
                            n[s] += 1; n[l] += 1;
                            out[off + s * M + l] = (int32_t)oracle_rank(N, M, n);
                            n[l] -= 1; n[s] -= 1;
                        }
                    }
                    n[q] += 1; n[k] += 1;
                }
                off += (int64_t)M * M;
            }
        }
    }
    row_off[nc] = off;
    free(n);
}

/* ------------------------------------------------------------------------ */
/* Bosonic ladder operators on an occupation vector (Sec. 2 commutation     */
/* relation): a_k |..n_k..> = sqrt(n_k) |..n_k - 1..> (zero if n_k = 0) and  */
/* a^dag_k |..n_k..> = sqrt(n_k + 1) |..n_k + 1..>.  *amp accumulates the   */
/* square-root factors; the return value is 0 when the state vanishes.     */
/* ------------------------------------------------------------------------ */
static int op_annihilate(int32_t *n, int k, double *amp)
{
    if (n[k] == 0) return 0;
    *amp *= sqrt((double)n[k]);
    n[k] -= 1;
    return 1;
}

static void op_create(int32_t *n, int k, double *amp)
{
    *amp *= sqrt((double)(n[k] + 1));
    n[k] += 1;
}

/* Visit every basis state reached from configuration n by the Hamiltonian */
/* (Eqs. noninteracting, interacting and Haction), i.e. the column H|n>.    */
/* For each term the callback receives the target index and the complex    */
/* matrix element <target| term |n> (coefficient times operator amplitude). */
/* Operators act right to left: a^dag_k a_l applies a_l first; the          */
/* two-body string a^dag_k a^dag_q a_s a_l applies a_l, a_s, a^dag_q,       */
/* a^dag_k in that order.  No symmetry of h or W is used.                   */
typedef void (*column_visitor)(void *ctx, int64_t target, double re, double im);

static void visit_column(int N, int M, const double *h, const double *W,
                         const int32_t *n0, int32_t *work, column_visitor fn, void *ctx)
{
    for (int k = 0; k < M; ++k) {
        for (int l = 0; l < M; ++l) {
            double hre = h[2 * (k * M + l)], him = h[2 * (k * M + l) + 1];
            if (hre == 0.0 && him == 0.0) continue;
            memcpy(work, n0, sizeof(int32_t) * (size_t)M);
            double amp = 1.0;
            if (!op_annihilate(work, l, &amp)) continue;
            op_create(work, k, &amp);
            int64_t t = oracle_rank(N, M, work);
            fn(ctx, t, hre * amp, him * amp);
        }
    }
    if (!W) return;
    for (int k = 0; k < M; ++k)
        for (int q = 0; q < M; ++q)
            for (int s = 0; s < M; ++s)
                for (int l = 0; l < M; ++l) {
                    size_t w = (((size_t)k * M + q) * M + s) * M + l;
                    double wre = W[2 * w], wim = W[2 * w + 1];
                    if (wre == 0.0 && wim == 0.0) continue;
                    memcpy(work, n0, sizeof(int32_t) * (size_t)M);
                    double amp = 1.0;
                    if (!op_annihilate(work, l, &amp)) continue;
                    if (!op_annihilate(work, s, &amp)) continue;
                    op_create(work, q, &amp);
                    op_create(work, k, &amp);
                    int64_t t = oracle_rank(N, M, work);
                    fn(ctx, t, 0.5 * wre * amp, 0.5 * wim * amp);
                }
}

struct push_ctx { double *sigma; double cre, cim; };

static void push_visit(void *vctx, int64_t t, double re, double im)
{
    struct push_ctx *c = (struct push_ctx *)vctx;
    c->sigma[2 * t] += re * c->cre - im * c->cim;
    c->sigma[2 * t + 1] += re * c->cim + im * c->cre;
}

/* ------------------------------------------------------------------------ */
/* sigma = H C in push form (Eq. Haction): every source configuration beta  */
/* scatters H_{gamma beta} C_beta into every gamma it reaches.  sigma is    */
/* overwritten.  Pinned by: textbook matrix construction of H, Hermiticity, */
/* the g = 0 and Lieb-Liniger diagonal closed forms, Appendix B rules.     */
/* ------------------------------------------------------------------------ */
void oracle_apply_push(int N, int M, const double *h, const double *W,
                       const double *C, double *sigma)
{
    int64_t nc = oracle_nc(N, M);
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    memset(sigma, 0, sizeof(double) * 2 * (size_t)nc);
    struct push_ctx ctx;
    ctx.sigma = sigma;
    for (int64_t b = 0; b < nc; ++b) {
        oracle_unrank(N, M, b, n);
        ctx.cre = C[2 * b];
        ctx.cim = C[2 * b + 1];
        visit_column(N, M, h, W, n, work, push_visit, &ctx);
    }
    free(work);
    free(n);
}

struct row_ctx { const double *C; double re, im; };

static void row_visit(void *vctx, int64_t t, double re, double im)
{
    /* conj(H_{t gamma}) C_t */
    struct row_ctx *c = (struct row_ctx *)vctx;
    double cre = c->C[2 * t], cim = c->C[2 * t + 1];
    c->re += re * cre + im * cim;
    c->im += re * cim - im * cre;
}

/* ------------------------------------------------------------------------ */
/* Selected rows of sigma = H C for spaces too large for the push form.     */
/* Row gamma of H equals the conjugate of column gamma because H is         */
/* Hermitian (h = h^dag and W_kqsl = conj(W_lsqk)); the column is H|gamma>  */
/* built by the same operator strings as the push form.  Pinned by          */
/* agreement with oracle_apply_push on every row of small spaces (tests).  */
/* ------------------------------------------------------------------------ */
void oracle_apply_rows(int N, int M, const double *h, const double *W,
                       const double *C, const int64_t *rows, int64_t nrows, double *out)
{
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    for (int64_t i = 0; i < nrows; ++i) {
        struct row_ctx ctx;
        ctx.C = C; ctx.re = 0.0; ctx.im = 0.0;
        oracle_unrank(N, M, rows[i], n);
        visit_column(N, M, h, W, n, work, row_visit, &ctx);
        out[2 * i] = ctx.re;
        out[2 * i + 1] = ctx.im;
    }
    free(work);
    free(n);
}

struct dense_ctx { double *H; int64_t nc; int64_t col; };

static void dense_visit(void *vctx, int64_t t, double re, double im)
{
    struct dense_ctx *c = (struct dense_ctx *)vctx;
    c->H[2 * (t * c->nc + c->col)] += re;
    c->H[2 * (t * c->nc + c->col) + 1] += im;
}

/* Dense matrix H[gamma][beta] = <gamma|H|beta> (complex, row-major), built */
/* column by column from the operator strings.  For tiny spaces only.       */
void oracle_dense_hamiltonian(int N, int M, const double *h, const double *W, double *H)
{
    int64_t nc = oracle_nc(N, M);
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    memset(H, 0, sizeof(double) * 2 * (size_t)(nc * nc));
    struct dense_ctx ctx;
    ctx.H = H; ctx.nc = nc;
    for (int64_t b = 0; b < nc; ++b) {
        oracle_unrank(N, M, b, n);
        ctx.col = b;
        visit_column(N, M, h, W, n, work, dense_visit, &ctx);
    }
    free(work);
    free(n);
}

struct count_ctx { int64_t *targets; int64_t count; };

static void count_visit(void *vctx, int64_t t, double re, double im)
{
    (void)re; (void)im;
    struct count_ctx *c = (struct count_ctx *)vctx;
    c->targets[c->count++] = t;
}

/* Number of operator strings with a nonzero coefficient that act without   */
/* vanishing on configuration gamma (the column's term count, before equal  */
/* targets are merged).  Used only to cross-check operation counts.         */
int64_t oracle_column_terms(int N, int M, const double *h, const double *W, int64_t gamma)
{
    int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int64_t cap = (int64_t)M * M + (W ? (int64_t)M * M * M * M : 0);
    struct count_ctx ctx;
    ctx.targets = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    ctx.count = 0;
    oracle_unrank(N, M, gamma, n);
    visit_column(N, M, h, W, n, work, count_visit, &ctx);
    int64_t r = ctx.count;
    free(ctx.targets);
    free(work);
    free(n);
    return r;
}
