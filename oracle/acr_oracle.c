/*
 * acr_oracle.c -- CPU oracle for block cyclic reduction (BCR).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library, its
 * Python binding, the serving loop) may call, link or load this file; only the
 * test-suite, the package's smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or table with the GPU implementation.
 *
 * What it computes: the exact FP64 solution of A u = f for a block
 * tridiagonal A = tridiag(A_i, D_i, C_i) (Section 3, the block tridiagonal
 * form; the paper writes E_i, D_i, F_i) by *dense* block cyclic reduction, the
 * method that Accelerated Cyclic Reduction approximates (Section 3: BCR is
 * block Gaussian elimination without pivoting on the even/odd permuted system,
 * followed by back-substitution).  Steps, in the order of Section 3:
 *
 *   reduction, while m > m_stop:
 *     eliminated set E = {0, 2, 4, ...}, kept set K = {1, 3, ...} (0-based),
 *     the even/odd permutation of the n = 8 illustration;
 *     LU-factor every D_j, j in E (the block-diagonal H11 is inverted block
 *     by block);
 *     Schur complement (Eq. "fund": H22 - H21 H11^-1 H12 and
 *     f^(1) = f_odd - H21 H11^-1 f_even), which is again block tridiagonal:
 *       D'_k = D_i - A_i D_{i-1}^-1 C_{i-1} - C_i D_{i+1}^-1 A_{i+1}
 *       A'_k = -A_i D_{i-1}^-1 A_{i-1}
 *       C'_k = -C_i D_{i+1}^-1 C_{i+1}
 *       f'_k = f_i - A_i D_{i-1}^-1 f_{i-1} - C_i D_{i+1}^-1 f_{i+1}
 *     with k = (i-1)/2 and every term whose block does not exist dropped;
 *   top: dense LU solve of the remaining m <= m_stop blocks;
 *   back-substitution, levels in reverse:
 *       u_j = D_j^-1 (f_j - A_j u_{j-1} - C_j u_{j+1}),  j in E.
 *
 * Readings where the paper is silent: n need not be a power of two (E is all
 * even indices, the last block is eliminated when m is odd, m' = floor(m/2));
 * partial pivoting by rows *inside* each dense D_j with the lowest row index
 * winning ties; a pivot with |u_kk| <= 1e3 * eps * max|D_j| is reported as
 * singular (status -3, level and block returned).
 *
 * Layout: a block is b x b column-major (element (r, c) at r + c*b); the n
 * blocks of A, D and C are contiguous.  A_0 and C_{n-1} are ignored.  Right
 * hand sides and solutions are N x nrhs column-major, N = n*b.
 *
 * Everything is FP64, plain loops, OpenMP across the independent blocks of a
 * level.  Parity pins live in the test-suite.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_OOM (-2)
#define ORACLE_ERR_SINGULAR (-3)

#define EL(M, ld, r, c) ((M)[(size_t)(r) + (size_t)(c) * (size_t)(ld)])

/* ORACLE_MUTANT plants one deliberate mistake; only the test-suite's mutation
 * test compiles it (to show that the pins catch each kind of slip).  The
 * default build is 0: no mutation. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- dense LU */

/* Right-looking LU with partial (row) pivoting, in place.  piv[k] is the row
 * swapped with row k at step k.  Returns 0, or -1 on a (near) zero pivot. */
static int lu_factor(int b, double *M, size_t ld, int *piv) {
    double amax = 0.0;
    for (int c = 0; c < b; ++c)
        for (int r = 0; r < b; ++r) {
            double v = fabs(EL(M, ld, r, c));
            if (v > amax) amax = v;
        }
    double tiny = 1e3 * DBL_EPSILON * amax;
    for (int k = 0; k < b; ++k) {
        int p = k;
        double best = fabs(EL(M, ld, k, k));
        for (int r = k + 1; r < b && ORACLE_MUTANT != 7; ++r) {  /* mutant 7: no interchange */
            double v = fabs(EL(M, ld, r, k));
            if (v > best) { best = v; p = r; }
        }
        piv[k] = p;
        if (!(best > tiny)) return -1;  /* also catches NaN */
        if (p != k)
            for (int c = 0; c < b; ++c) {
                double t = EL(M, ld, k, c);
                EL(M, ld, k, c) = EL(M, ld, p, c);
                EL(M, ld, p, c) = t;
            }
        double inv = 1.0 / EL(M, ld, k, k);
        for (int r = k + 1; r < b; ++r) EL(M, ld, r, k) *= inv;
        for (int c = k + 1; c < b; ++c) {
            double ukc = EL(M, ld, k, c);
            if (ukc == 0.0) continue;
            for (int r = k + 1; r < b; ++r) EL(M, ld, r, c) -= EL(M, ld, r, k) * ukc;
        }
    }
    return 0;
}

/* Overwrite X (b x ncols, leading dim ldx) with M^-1 X, M = P^T L U. */
static void lu_solve(int b, const double *LU, size_t ld, const int *piv,
                     double *X, size_t ldx, int ncols) {
    for (int q = 0; q < ncols; ++q) {
        double *x = X + (size_t)q * ldx;
        for (int k = 0; k < b; ++k)
            if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
        for (int c = 0; c < b; ++c) {          /* L y = P x, unit lower */
            double xc = x[c];
            if (xc != 0.0)
                for (int r = c + 1; r < b; ++r) x[r] -= EL(LU, ld, r, c) * xc;
        }
        for (int c = b - 1; c >= 0; --c) {     /* U z = y */
            x[c] /= EL(LU, ld, c, c);
            double xc = x[c];
            if (xc != 0.0)
                for (int r = 0; r < c; ++r) x[r] -= EL(LU, ld, r, c) * xc;
        }
    }
}

/* Y -= M X with M b x b (ld b), X and Y b x ncols (leading dims ldx, ldy). */
static void gemm_sub(int b, const double *M, const double *X, size_t ldx,
                     double *Y, size_t ldy, int ncols) {
    for (int q = 0; q < ncols; ++q)
        for (int k = 0; k < b; ++k) {
            double xk = X[(size_t)k + (size_t)q * ldx];
            if (xk == 0.0) continue;
            const double *mc = M + (size_t)k * b;
            double *y = Y + (size_t)q * ldy;
#if ORACLE_MUTANT == 4 /* transposed operand */
            for (int r = 0; r < b; ++r) y[r] -= M[(size_t)r * b + k] * xk;
#else
            for (int r = 0; r < b; ++r) y[r] -= mc[r] * xk;
#endif
        }
}

/* ------------------------------------------------------- dense direct solve */

/* Solve the assembled N x N system (column-major) by partial-pivoted LU.
 * M and F are not modified.  Returns 0 or ORACLE_ERR_SINGULAR. */
int oracle_dense_solve(int N, const double *M, const double *F, int nrhs, double *X) {
    if (N <= 0 || nrhs < 0) return ORACLE_ERR_ARG;
    double *W = (double *)malloc(sizeof(double) * (size_t)N * N);
    int *piv = (int *)malloc(sizeof(int) * (size_t)N);
    if (!W || !piv) { free(W); free(piv); return ORACLE_ERR_OOM; }
    memcpy(W, M, sizeof(double) * (size_t)N * N);
    memcpy(X, F, sizeof(double) * (size_t)N * nrhs);
    int st = lu_factor(N, W, N, piv);
    if (st == 0) lu_solve(N, W, N, piv, X, N, nrhs);
    free(W); free(piv);
    return st == 0 ? ORACLE_OK : ORACLE_ERR_SINGULAR;
}

/* -------------------------------------------------------- block cyclic red. */

typedef struct {
    int m;        /* blocks at this level */
    double *D;    /* m blocks; even slots hold LU(D_j) after factoring */
    double *A;    /* m blocks (A_0 = 0) */
    double *C;    /* m blocks (C_{m-1} = 0) */
    int *piv;     /* m * b pivots (even slots used) */
    double *F;    /* (m*b) x nrhs column-major level right-hand side */
} level_t;

static void free_level(level_t *L) {
    free(L->D); free(L->A); free(L->C); free(L->piv); free(L->F);
    memset(L, 0, sizeof(*L));
}

static int alloc_level(level_t *L, int m, int b, int nrhs) {
    size_t bb = (size_t)b * b;
    L->m = m;
    L->D = (double *)calloc((size_t)m * bb, sizeof(double));
    L->A = (double *)calloc((size_t)m * bb, sizeof(double));
    L->C = (double *)calloc((size_t)m * bb, sizeof(double));
    L->piv = (int *)calloc((size_t)m * b, sizeof(int));
    L->F = (double *)calloc((size_t)m * b * (nrhs > 0 ? nrhs : 1), sizeof(double));
    if (!L->D || !L->A || !L->C || !L->piv || !L->F) { free_level(L); return -1; }
    return 0;
}

/* One reduction step: factor the even blocks of `cur` and form `nxt`.
 * If nrhs > 0 the level right-hand side is reduced too.  On a singular block
 * *bad is set to its index at this level. */
static int reduce_level(level_t *cur, level_t *nxt, int b, int nrhs, int *bad) {
    const int m = cur->m;
    const size_t bb = (size_t)b * b;
    const int ne = (m + 1) / 2, nk = m / 2;
    const size_t ldF = (size_t)m * b, ldFn = (size_t)nk * b;
    double *XA = (double *)calloc((size_t)ne * bb, sizeof(double));
    double *XC = (double *)calloc((size_t)ne * bb, sizeof(double));
    double *G = (double *)calloc((size_t)ne * b * (nrhs > 0 ? nrhs : 1), sizeof(double));
    if (!XA || !XC || !G) { free(XA); free(XC); free(G); return ORACLE_ERR_OOM; }
    if (alloc_level(nxt, nk, b, nrhs)) { free(XA); free(XC); free(G); return ORACLE_ERR_OOM; }
    int status = ORACLE_OK;
    *bad = -1;

    /* LU of the eliminated blocks, then D_j^-1 A_j, D_j^-1 C_j, D_j^-1 f_j. */
#pragma omp parallel for schedule(dynamic)
    for (int e = 0; e < ne; ++e) {
        const int j = 2 * e;
        double *Dj = cur->D + (size_t)j * bb;
        int *pj = cur->piv + (size_t)j * b;
        if (lu_factor(b, Dj, b, pj)) {
#pragma omp critical
            { if (*bad < 0 || j < *bad) *bad = j; status = ORACLE_ERR_SINGULAR; }
            continue;
        }
        if (j > 0) {
            memcpy(XA + (size_t)e * bb, cur->A + (size_t)j * bb, bb * sizeof(double));
            lu_solve(b, Dj, b, pj, XA + (size_t)e * bb, b, b);
        }
        if (j + 1 < m) {
            memcpy(XC + (size_t)e * bb, cur->C + (size_t)j * bb, bb * sizeof(double));
            lu_solve(b, Dj, b, pj, XC + (size_t)e * bb, b, b);
        }
        for (int q = 0; q < nrhs; ++q)
            memcpy(G + (size_t)e * b + (size_t)q * ne * b,
                   cur->F + (size_t)j * b + (size_t)q * ldF, b * sizeof(double));
        if (nrhs > 0) lu_solve(b, Dj, b, pj, G + (size_t)e * b, (size_t)ne * b, nrhs);
    }
    if (status != ORACLE_OK) { free(XA); free(XC); free(G); free_level(nxt); return status; }

    /* Schur complement on the kept blocks (i odd, new index k = (i-1)/2). */
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nk; ++k) {
        const int i = 2 * k + 1;
        const double *Ai = cur->A + (size_t)i * bb, *Ci = cur->C + (size_t)i * bb;
        double *Dn = nxt->D + (size_t)k * bb, *An = nxt->A + (size_t)k * bb,
               *Cn = nxt->C + (size_t)k * bb;
        const int em = (i - 1) / 2, ep = (i + 1) / 2; /* slots of i-1 and i+1 in XA/XC/G */
        memcpy(Dn, cur->D + (size_t)i * bb, bb * sizeof(double));
        gemm_sub(b, Ai, XC + (size_t)em * bb, b, Dn, b, b);           /* - A_i D^-1 C_{i-1} */
        if (i + 1 < m && ORACLE_MUTANT != 1)                                /* mutant 1: dropped term */
            gemm_sub(b, Ci, XA + (size_t)ep * bb, b, Dn, b, b);            /* - C_i D^-1 A_{i+1} */
        if (i >= 3) gemm_sub(b, Ai, XA + (size_t)(ORACLE_MUTANT == 3 && ep < ne ? ep : em) * bb, b, An, b, b);
                                                  /* A' = -A_i D^-1 A_{i-1}; mutant 3: wrong index */
#if ORACLE_MUTANT == 2 /* wrong sign */
        for (size_t e2 = 0; e2 < bb; ++e2) An[e2] = -An[e2];
#endif
        if (i + 2 < m) gemm_sub(b, Ci, XC + (size_t)ep * bb, b, Cn, b, b); /* C' = -C_i D^-1 C_{i+1} */
        for (int q = 0; q < nrhs; ++q)
            memcpy(nxt->F + (size_t)k * b + (size_t)q * ldFn,
                   cur->F + (size_t)i * b + (size_t)q * ldF, b * sizeof(double));
        if (nrhs > 0) {
            gemm_sub(b, Ai, G + (size_t)em * b, (size_t)ne * b, nxt->F + (size_t)k * b, ldFn, nrhs);
            if (i + 1 < m && ORACLE_MUTANT != 5)                       /* mutant 5: dropped term */
                gemm_sub(b, Ci, G + (size_t)ep * b, (size_t)ne * b, nxt->F + (size_t)k * b, ldFn, nrhs);
        }
    }
    free(XA); free(XC); free(G);
    return ORACLE_OK;
}

static int init_level0(level_t *L, int n, int b, const double *A, const double *D,
                       const double *C, const double *F, int nrhs) {
    size_t bb = (size_t)b * b;
    if (alloc_level(L, n, b, nrhs)) return ORACLE_ERR_OOM;
    memcpy(L->D, D, (size_t)n * bb * sizeof(double));
    if (n > 1) {
        memcpy(L->A + bb, A + bb, (size_t)(n - 1) * bb * sizeof(double));
        memcpy(L->C, C, (size_t)(n - 1) * bb * sizeof(double));
    }
    if (nrhs > 0) memcpy(L->F, F, (size_t)n * b * nrhs * sizeof(double));
    return ORACLE_OK;
}

/* Dense BCR solve.  On ORACLE_ERR_SINGULAR, err_level/err_block (if non-NULL)
 * receive the level and the block index at that level. */
int oracle_bcr_solve(int n, int b, const double *A, const double *D, const double *C,
                     const double *F, int nrhs, double *X, int m_stop,
                     int *err_level, int *err_block) {
    if (n <= 0 || b <= 0 || nrhs < 0 || !A || !D || !C || (nrhs > 0 && (!F || !X)))
        return ORACLE_ERR_ARG;
    if (m_stop < 1) m_stop = 1;
    int maxlev = 1;
    for (int m = n; m > 1; m /= 2) ++maxlev;
    level_t *lev = (level_t *)calloc((size_t)maxlev + 1, sizeof(level_t));
    if (!lev) return ORACLE_ERR_OOM;
    int st = init_level0(&lev[0], n, b, A, D, C, F, nrhs);
    int t = 0;
    while (st == ORACLE_OK && lev[t].m > m_stop) {
        int bad;
        st = reduce_level(&lev[t], &lev[t + 1], b, nrhs, &bad);
        if (st == ORACLE_ERR_SINGULAR) {
            if (err_level) *err_level = t;
            if (err_block) *err_block = bad;
        }
        if (st == ORACLE_OK) ++t;
    }
    if (st == ORACLE_OK) {
        /* top: assemble the remaining m-block system densely and solve it */
        level_t *T = &lev[t];
        const int m = T->m, Nt = m * b;
        const size_t bb = (size_t)b * b;
        double *M = (double *)calloc((size_t)Nt * Nt, sizeof(double));
        double *U = (double *)malloc(sizeof(double) * (size_t)Nt * (nrhs > 0 ? nrhs : 1));
        if (!M || !U) st = ORACLE_ERR_OOM;
        for (int i = 0; st == ORACLE_OK && i < m; ++i)
            for (int c = 0; c < b; ++c)
                for (int r = 0; r < b; ++r) {
                    EL(M, Nt, i * b + r, i * b + c) = T->D[i * bb + r + (size_t)c * b];
                    if (i > 0) EL(M, Nt, i * b + r, (i - 1) * b + c) = T->A[i * bb + r + (size_t)c * b];
                    if (i + 1 < m) EL(M, Nt, i * b + r, (i + 1) * b + c) = T->C[i * bb + r + (size_t)c * b];
                }
        if (st == ORACLE_OK && nrhs > 0) {
            st = oracle_dense_solve(Nt, M, T->F, nrhs, U);
            if (st == ORACLE_ERR_SINGULAR) { if (err_level) *err_level = t; if (err_block) *err_block = 0; }
        }
        free(M);
        /* back-substitution: U holds the solution of level t */
        for (int s = t - 1; st == ORACLE_OK && nrhs > 0 && s >= 0; --s) {
            level_t *L = &lev[s];
            const int ml = L->m, nk = ml / 2;
            const size_t ld = (size_t)ml * b, ldc = (size_t)nk * b;
            double *Ul = (double *)malloc(sizeof(double) * ld * nrhs);
            if (!Ul) { st = ORACLE_ERR_OOM; break; }
            for (int k = 0; k < nk; ++k)                 /* kept blocks: known */
                for (int q = 0; q < nrhs; ++q)
                    memcpy(Ul + (size_t)(2 * k + 1) * b + q * ld, U + (size_t)k * b + q * ldc,
                           b * sizeof(double));
#pragma omp parallel for schedule(dynamic)
            for (int j = 0; j < ml; j += 2) {            /* eliminated blocks */
                double *uj = Ul + (size_t)j * b;
                for (int q = 0; q < nrhs; ++q)
                    memcpy(uj + q * ld, L->F + (size_t)j * b + q * ld, b * sizeof(double));
                if (j > 0) gemm_sub(b, L->A + (size_t)j * bb, Ul + (size_t)(j - 1) * b, ld, uj, ld, nrhs);
                if (j + 1 < ml)                                /* mutant 6: wrong neighbour */
                    gemm_sub(b, L->C + (size_t)j * bb, Ul + (size_t)(ORACLE_MUTANT == 6 && j > 0 ? j - 1 : j + 1) * b,
                             ld, uj, ld, nrhs);
                lu_solve(b, L->D + (size_t)j * bb, b, L->piv + (size_t)j * b, uj, ld, nrhs);
            }
            free(U);
            U = Ul;
        }
        if (st == ORACLE_OK && nrhs > 0) memcpy(X, U, sizeof(double) * (size_t)n * b * nrhs);
        free(U);
    }
    for (int s = 0; s <= maxlev; ++s) free_level(&lev[s]);
    free(lev);
    return st;
}

/* Run `nlev` reduction levels (no right-hand side) and return the reduced
 * blocks.  outD/outA/outC must hold n blocks each; *m_out receives the number
 * of blocks of the reduced system (its A_0 and C_{m-1} are zero). */
int oracle_bcr_reduce(int n, int b, const double *A, const double *D, const double *C,
                      int nlev, double *outD, double *outA, double *outC, int *m_out) {
    if (n <= 0 || b <= 0 || nlev < 0) return ORACLE_ERR_ARG;
    level_t cur, nxt;
    memset(&nxt, 0, sizeof(nxt));
    int st = init_level0(&cur, n, b, A, D, C, NULL, 0);
    for (int t = 0; st == ORACLE_OK && t < nlev && cur.m > 1; ++t) {
        int bad;
        st = reduce_level(&cur, &nxt, b, 0, &bad);
        if (st == ORACLE_OK) { free_level(&cur); cur = nxt; memset(&nxt, 0, sizeof(nxt)); }
    }
    if (st == ORACLE_OK) {
        size_t sz = (size_t)cur.m * b * b * sizeof(double);
        memcpy(outD, cur.D, sz); memcpy(outA, cur.A, sz); memcpy(outC, cur.C, sz);
        *m_out = cur.m;
    }
    free_level(&cur);
    return st;
}

/* The elimination schedule in original block indices: for each level, the
 * original indices of the blocks it eliminates.  Writes, per level, the count
 * followed by the indices into out (capacity cap ints).  Returns the number of
 * levels, or -1 if cap is too small.  The final block (top solve) is reported
 * as the last level. */
int oracle_bcr_schedule(int n, int m_stop, int *out, int cap) {
    if (m_stop < 1) m_stop = 1;
    int *ids = (int *)malloc(sizeof(int) * (size_t)n);
    if (!ids) return -1;
    for (int i = 0; i < n; ++i) ids[i] = i;
    int m = n, pos = 0, nlev = 0;
    while (1) {
        int last = m <= m_stop;
        int cnt = last ? m : (m + 1) / 2;
        if (pos + 1 + cnt > cap) { free(ids); return -1; }
        out[pos++] = cnt;
        for (int j = 0; j < m; j += last ? 1 : 2) out[pos++] = ids[j];
        ++nlev;
        if (last) break;
        for (int k = 0; k < m / 2; ++k) ids[k] = ids[2 * k + 1];
        m /= 2;
    }
    free(ids);
    return nlev;
}

/* Per-column relative residual ||f - M x||_2 / ||f||_2 for the block
 * tridiagonal M (dense blocks), FP64. */
int oracle_residual(int n, int b, const double *A, const double *D, const double *C,
                    const double *X, const double *F, int nrhs, double *rel) {
    const size_t bb = (size_t)b * b, N = (size_t)n * b;
    double *R = (double *)malloc(sizeof(double) * N * (nrhs > 0 ? nrhs : 1));
    if (!R) return ORACLE_ERR_OOM;
    memcpy(R, F, sizeof(double) * N * nrhs);
    for (int i = 0; i < n; ++i) {
        gemm_sub(b, D + i * bb, X + (size_t)i * b, N, R + (size_t)i * b, N, nrhs);
        if (i > 0) gemm_sub(b, A + i * bb, X + (size_t)(i - 1) * b, N, R + (size_t)i * b, N, nrhs);
        if (i + 1 < n) gemm_sub(b, C + i * bb, X + (size_t)(i + 1) * b, N, R + (size_t)i * b, N, nrhs);
    }
    for (int q = 0; q < nrhs; ++q) {
        double rn = 0, fn = 0;
        for (size_t r = 0; r < N; ++r) {
            rn += R[r + q * N] * R[r + q * N];
            fn += F[r + q * N] * F[r + q * N];
        }
        rel[q] = fn > 0 ? sqrt(rn / fn) : sqrt(rn);
    }
    free(R);
    return ORACLE_OK;
}
