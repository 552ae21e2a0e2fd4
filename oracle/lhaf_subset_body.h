/*
 * ORACLE — test infrastructure only. Included twice by lhaf_oracle.c, once with
 * REAL = double and once with REAL = long double, to give the subset formula in two
 * precisions (the long double copy estimates the double copy's own rounding error).
 *
 * The subset formula for the loop hafnian (the algorithm the paper cites for its
 * O(N^3 2^{N/2}) loop hafnian, Sec. II after Eq. lhaf-pure, and benchmarks in Sec. IV),
 * written out step by step with no reordering:
 *
 *   N = 2n (odd N is padded by one extra vertex with loop weight 1 and no edges).
 *   For every subset Z of the n index pairs (j, j+n), with k = |Z| and m = 2k:
 *     idx   = [j for j in Z (ascending)] + [j+n for j in Z (ascending)]
 *     M_Z   = X_Z * A0[idx, idx]           (A0 = A with zero diagonal,
 *                                           X_Z swaps the two halves of the rows)
 *     v     = diag(A)[idx],   w = X_Z v
 *     T_j   = tr(M_Z^j)                    by explicit repeated matrix products
 *     l_j   = v^T M_Z^{j-1} w              by repeated matrix-vector products
 *     c_j   = T_j / (2j) + l_j / 2,        j = 1..n
 *     p_Z   = [lambda^n] exp(sum_j c_j lambda^j)
 *             via p_0 = 1,  j p_j = sum_{i=1..j} i c_i p_{j-i}
 *   lhaf(A) = sum_Z (-1)^{n-k} p_Z
 *
 * The cross-subset sum is compensated (TwoSum, "double-double") and runs over fixed
 * contiguous blocks of z whose partials are combined in block order, so the result is
 * independent of the number of threads.
 */

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SUF)

typedef _Complex REAL FN(cplx_t);

/* p_Z for one subset z of the n pairs of the (even-size, padded) matrix A (N = 2n). */
static FN(cplx_t) FN(subset_pz)(const FN(cplx_t) *A, int N, uint64_t z,
                                FN(cplx_t) *M, FN(cplx_t) *P, FN(cplx_t) *Ptmp,
                                FN(cplx_t) *v, FN(cplx_t) *w, FN(cplx_t) *u,
                                FN(cplx_t) *utmp, FN(cplx_t) *c, FN(cplx_t) *p,
                                int *idx) {
    const int n = N / 2;
    int k = 0;
    for (int j = 0; j < n; j++)
        if ((z >> j) & 1u) idx[k++] = j;
    for (int a = 0; a < k; a++) idx[k + a] = idx[a] + n;
    const int m = 2 * k;
    if (m == 0) return (n == 0) ? 1.0 : 0.0;

    /* M_Z = X_Z A0_Z : row r of M_Z is row (r + k) mod m of A0_Z. */
    for (int r = 0; r < m; r++) {
        int rs = idx[(r + k) % m];
        for (int cc = 0; cc < m; cc++) {
            int cs = idx[cc];
            M[r * m + cc] = (rs == cs) ? 0.0 : A[(size_t)rs * N + cs];
        }
    }
    for (int a = 0; a < m; a++) v[a] = A[(size_t)idx[a] * N + idx[a]];
    for (int a = 0; a < m; a++) w[a] = v[(a + k) % m];

    /* P = M^0 = I ; u = M^0 w = w */
    for (int a = 0; a < m * m; a++) P[a] = 0.0;
    for (int a = 0; a < m; a++) P[a * m + a] = 1.0;
    for (int a = 0; a < m; a++) u[a] = w[a];

    for (int j = 1; j <= n; j++) {
        /* loop term l_j = v^T M^{j-1} w, with u = M^{j-1} w */
        FN(cplx_t) lj = 0.0;
        for (int a = 0; a < m; a++) lj += v[a] * u[a];
        /* P <- P M  (so P = M^j), trace T_j */
        for (int r = 0; r < m; r++)
            for (int cc = 0; cc < m; cc++) {
                FN(cplx_t) s = 0.0;
                for (int t = 0; t < m; t++) s += P[r * m + t] * M[t * m + cc];
                Ptmp[r * m + cc] = s;
            }
        memcpy(P, Ptmp, sizeof(FN(cplx_t)) * (size_t)m * m);
        FN(cplx_t) Tj = 0.0;
        for (int a = 0; a < m; a++) Tj += P[a * m + a];
        /* u <- M u */
        for (int r = 0; r < m; r++) {
            FN(cplx_t) s = 0.0;
            for (int t = 0; t < m; t++) s += M[r * m + t] * u[t];
            utmp[r] = s;
        }
        memcpy(u, utmp, sizeof(FN(cplx_t)) * (size_t)m);
        c[j] = Tj / (REAL)(2 * j) + lj / (REAL)2;
    }
    /* coefficient of lambda^n in exp(sum_j c_j lambda^j) */
    p[0] = 1.0;
    for (int j = 1; j <= n; j++) {
        FN(cplx_t) s = 0.0;
        for (int i = 1; i <= j; i++) s += (REAL)i * c[i] * p[j - i];
        p[j] = s / (REAL)j;
    }
    return p[n];
}

/* TwoSum error-free addition: s + e == a + b exactly. */
static inline void FN(two_sum)(REAL a, REAL b, REAL *s, REAL *e) {
    REAL x = a + b;
    REAL bb = x - a;
    *e = (a - (x - bb)) + (b - bb);
    *s = x;
}

/* Compensated accumulator (hi, lo) += x. */
static inline void FN(acc_add)(REAL *hi, REAL *lo, REAL x) {
    REAL s, e;
    FN(two_sum)(*hi, x, &s, &e);
    *hi = s;
    *lo += e;
}

/* Sum over z in [z0, z1) of sign * p_Z, with compensated re/im, sum |p_Z| and
 * sum |p_Z|^2 (the last two describe the cancellation of the signed sum). */
static void FN(subset_range)(const FN(cplx_t) *A, int N, uint64_t z0, uint64_t z1,
                             REAL out[6]) {
    const int n = N / 2;
    const int mm = N > 0 ? N : 1;
    FN(cplx_t) *buf = (FN(cplx_t) *)malloc(sizeof(FN(cplx_t)) *
                                           (size_t)(3 * mm * mm + 5 * mm + 2 * (n + 1)));
    int *idx = (int *)malloc(sizeof(int) * (size_t)mm);
    FN(cplx_t) *M = buf, *P = M + mm * mm, *Ptmp = P + mm * mm;
    FN(cplx_t) *v = Ptmp + mm * mm, *w = v + mm, *u = w + mm, *utmp = u + mm;
    FN(cplx_t) *c = utmp + mm, *p = c + (n + 1);
    REAL re_hi = 0, re_lo = 0, im_hi = 0, im_lo = 0, abs_sum = 0, sq_sum = 0;
    for (uint64_t z = z0; z < z1; z++) {
        int k = __builtin_popcountll(z);
        FN(cplx_t) pz = FN(subset_pz)(A, N, z, M, P, Ptmp, v, w, u, utmp, c, p, idx);
        REAL sgn = ((n - k) & 1) ? -1 : 1;
        FN(acc_add)(&re_hi, &re_lo, sgn * CAT(creal, RSUF)(pz));
        FN(acc_add)(&im_hi, &im_lo, sgn * CAT(cimag, RSUF)(pz));
        REAL a = CAT(cabs, RSUF)(pz);
        abs_sum += a;
        sq_sum += a * a;
    }
    out[0] = re_hi; out[1] = re_lo; out[2] = im_hi; out[3] = im_lo; out[4] = abs_sum;
    out[5] = sq_sum;
    free(buf);
    free(idx);
}

/* Full loop hafnian by the subset formula. A is row-major N x N (N already even).
 * out = lhaf, *abs_sum = sum_Z |p_Z| (the cancellation scale of the signed sum),
 * *sq_sum = sum_Z |p_Z|^2.  */
static void FN(lhaf_subset_even)(const FN(cplx_t) *A, int N, int nthreads,
                                 FN(cplx_t) *out, REAL *abs_sum, REAL *sq_sum) {
    const int n = N / 2;
    const uint64_t total = (uint64_t)1 << n;
    /* fixed block decomposition: the partial sums do not depend on nthreads */
    const uint64_t nblk = total < 4096 ? total : 4096;
    REAL *part = (REAL *)calloc((size_t)nblk * 6, sizeof(REAL));
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (long long b = 0; b < (long long)nblk; b++) {
        uint64_t z0 = total * (uint64_t)b / nblk, z1 = total * (uint64_t)(b + 1) / nblk;
        FN(subset_range)(A, N, z0, z1, part + 6 * b);
    }
    REAL re_hi = 0, re_lo = 0, im_hi = 0, im_lo = 0, as = 0, sq = 0;
    for (uint64_t b = 0; b < nblk; b++) {
        FN(acc_add)(&re_hi, &re_lo, part[6 * b + 0]);
        re_lo += part[6 * b + 1];
        FN(acc_add)(&im_hi, &im_lo, part[6 * b + 2]);
        im_lo += part[6 * b + 3];
        as += part[6 * b + 4];
        sq += part[6 * b + 5];
    }
    free(part);
    *out = (re_hi + re_lo) + (im_hi + im_lo) * (FN(cplx_t))_Complex_I;
    *abs_sum = as;
    *sq_sum = sq;
}

#undef FN
#undef CAT
#undef CAT_
