/*
 * ORACLE — test infrastructure only.
 *
 * Plain, slow CPU implementations of the loop hafnian used to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * this library; the product library never links, loads or calls it, and it shares no
 * code, header or table with the product's kernels.
 *
 * Three independent evaluators:
 *   orc_lhaf_brute   the definition: a sum over all partitions of the vertices into
 *                    loops (weight A_ii) and edges (weight A_ij). Sec. II: hafnian over
 *                    perfect matchings (Eq. defhaf); the loop hafnian replaces perfect
 *                    matchings by single-pair matchings (text after Eq. lhaf).
 *   orc_lhaf_dp      the same definition as a memoised recursion over vertex subsets
 *                    (remove the lowest vertex either as a loop or with a partner).
 *   orc_lhaf_subset  the subset formula of the algorithm the paper cites for loop
 *                    hafnians (Sec. II, O(N^3 2^{N/2})), with power traces from
 *                    explicit repeated matrix products; see lhaf_subset_body.h.
 *
 * Matrices are row-major N x N arrays of interleaved (re, im) doubles, i.e. the memory
 * layout of C99 double complex and of numpy complex128.
 *
 * Odd N: the subset formula needs an even size. The paper is silent on odd sizes; the
 * reading used here (and by the product) pads one extra vertex with loop weight 1 and
 * no edges, which leaves the loop hafnian unchanged (the extra vertex can only be a
 * loop). N = 0 gives 1 (the empty matching).
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------- brute force over single-pair matchings ---------------- */

static cplx brute_rec(const cplx *A, int N, uint64_t used, int with_loops) {
    int i = 0;
    while (i < N && ((used >> i) & 1u)) i++;
    if (i == N) return 1.0;
    used |= (uint64_t)1 << i;
    cplx s = 0.0;
    if (with_loops) s += A[(size_t)i * N + i] * brute_rec(A, N, used, with_loops);
    for (int j = i + 1; j < N; j++)
        if (!((used >> j) & 1u))
            s += A[(size_t)i * N + j] * brute_rec(A, N, used | ((uint64_t)1 << j), with_loops);
    return s;
}

/* lhaf (with_loops = 1) or haf (with_loops = 0) by enumerating every matching. */
int orc_lhaf_brute(const double *A, int N, int with_loops, double *out) {
    if (N < 0 || N > 20) return 1;
    cplx r = brute_rec((const cplx *)A, N, 0, with_loops);
    out[0] = creal(r);
    out[1] = cimag(r);
    return 0;
}

/* ---------------- memoised recursion over vertex subsets ---------------- */

/* f(S) = A_ii f(S\{i}) + sum_{j in S, j > i} A_ij f(S\{i,j}),  i = min S,  f({}) = 1. */
int orc_lhaf_dp(const double *A_, int N, int with_loops, double *out) {
    if (N < 0 || N > 24) return 1;
    const cplx *A = (const cplx *)A_;
    const uint64_t full = ((uint64_t)1 << N);
    cplx *f = (cplx *)malloc(sizeof(cplx) * full);
    if (!f) return 2;
    f[0] = 1.0;
    for (uint64_t S = 1; S < full; S++) {
        int i = __builtin_ctzll(S);
        uint64_t rest = S & ~((uint64_t)1 << i);
        cplx s = with_loops ? A[(size_t)i * N + i] * f[rest] : 0.0;
        for (uint64_t t = rest; t; t &= t - 1) {
            int j = __builtin_ctzll(t);
            s += A[(size_t)i * N + j] * f[rest & ~((uint64_t)1 << j)];
        }
        f[S] = s;
    }
    out[0] = creal(f[full - 1]);
    out[1] = cimag(f[full - 1]);
    free(f);
    return 0;
}

/* ---------------- subset formula, double and long double ---------------- */

#define REAL double
#define SUF _d
#define RSUF
#include "lhaf_subset_body.h"
#undef REAL
#undef SUF
#undef RSUF

#define REAL long double
#define SUF _ld
#define RSUF l
#include "lhaf_subset_body.h"
#undef REAL
#undef SUF
#undef RSUF

/* Pad to even size: one extra vertex with loop weight 1 and no edges. */
static cplx_t_d *pad_even_d(const cplx *A, int N, int *Np) {
    int Ne = N + (N & 1);
    cplx_t_d *P = (cplx_t_d *)calloc((size_t)(Ne > 0 ? Ne * Ne : 1), sizeof(cplx_t_d));
    for (int r = 0; r < N; r++)
        for (int c = 0; c < N; c++) P[(size_t)r * Ne + c] = A[(size_t)r * N + c];
    if (N & 1) P[(size_t)N * Ne + N] = 1.0;
    *Np = Ne;
    return P;
}

/* lhaf by the subset formula in double. out = (re, im); abs_sum = sum_Z |p_Z|;
 * sq_sum = sum_Z |p_Z|^2 (either may be NULL). */
int orc_lhaf_subset_stats(const double *A, int N, int nthreads, double *out, double *abs_sum,
                          double *sq_sum) {
    if (N < 0 || N > 64) return 1;
    if (N == 0) {
        out[0] = 1; out[1] = 0;
        if (abs_sum) *abs_sum = 1;
        if (sq_sum) *sq_sum = 1;
        return 0;
    }
    int Ne;
    cplx_t_d *P = pad_even_d((const cplx *)A, N, &Ne);
    cplx_t_d r;
    double as, sq;
    lhaf_subset_even_d(P, Ne, nthreads, &r, &as, &sq);
    free(P);
    out[0] = creal(r);
    out[1] = cimag(r);
    if (abs_sum) *abs_sum = as;
    if (sq_sum) *sq_sum = sq;
    return 0;
}

int orc_lhaf_subset(const double *A, int N, int nthreads, double *out, double *abs_sum) {
    return orc_lhaf_subset_stats(A, N, nthreads, out, abs_sum, NULL);
}

/* Same formula in long double (80-bit on x86-64, binary128 on aarch64). */
int orc_lhaf_subset_ld(const double *A, int N, int nthreads, double *out, double *abs_sum) {
    if (N < 0 || N > 64) return 1;
    if (N == 0) { out[0] = 1; out[1] = 0; if (abs_sum) *abs_sum = 1; return 0; }
    int Ne = N + (N & 1);
    cplx_t_ld *P = (cplx_t_ld *)calloc((size_t)Ne * Ne, sizeof(cplx_t_ld));
    const cplx *Ac = (const cplx *)A;
    for (int r = 0; r < N; r++)
        for (int c = 0; c < N; c++) P[(size_t)r * Ne + c] = Ac[(size_t)r * N + c];
    if (N & 1) P[(size_t)N * Ne + N] = 1.0L;
    cplx_t_ld r;
    long double as, sq;
    lhaf_subset_even_ld(P, Ne, nthreads, &r, &as, &sq);
    free(P);
    out[0] = (double)creall(r);
    out[1] = (double)cimagl(r);
    if (abs_sum) *abs_sum = (double)as;
    return 0;
}

/* p_Z for a list of subsets z (bit j set <=> pair (j, j+n) in Z) of the padded matrix. */
int orc_subset_terms(const double *A, int N, const uint64_t *zs, int count, int nthreads,
                     double *out) {
    if (N < 0 || N > 64) return 1;
    int Ne;
    cplx_t_d *P = pad_even_d((const cplx *)A, N, &Ne);
    const int mm = Ne > 0 ? Ne : 1, n = Ne / 2;
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
        cplx_t_d *buf = (cplx_t_d *)malloc(sizeof(cplx_t_d) *
                                           (size_t)(3 * mm * mm + 5 * mm + 2 * (n + 1)));
        int *idx = (int *)malloc(sizeof(int) * (size_t)mm);
        cplx_t_d *M = buf, *Pw = M + mm * mm, *Pt = Pw + mm * mm;
        cplx_t_d *v = Pt + mm * mm, *w = v + mm, *u = w + mm, *ut = u + mm;
        cplx_t_d *c = ut + mm, *p = c + (n + 1);
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < count; q++) {
            cplx_t_d pz = subset_pz_d(P, Ne, zs[q], M, Pw, Pt, v, w, u, ut, c, p, idx);
            out[2 * q] = creal(pz);
            out[2 * q + 1] = cimag(pz);
        }
        free(buf);
        free(idx);
    }
    free(P);
    return 0;
}
