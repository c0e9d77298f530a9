// acr_internal.h -- internal launchers and descriptors shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace acr {

// One batched block product: out = beta * cin + alpha * sum_t a[t] * bm[t],
// every operand a blksz x blksz column-major block (leading dimension blksz).
// A NULL a[t] drops term t; a NULL cin means beta is ignored.
template <class T>
struct GemmProb {
    T* out;
    const T* cin;
    const T* a[2];
    const T* bm[2];
    T alpha, beta;
};

// One batched block x multi-vector product of the solve sweeps:
//   out[:, q] = cin[:, q] + alpha * sum_t m[t] x[t][:, q],   q < nrhs,
// m[t] a blksz x blksz block (leading dimension blksz), or, when bit t of
// diag_mask is set, the blksz diagonal of a diagonal block;  x[t], cin, out
// blksz-row panels with leading dimensions ldx, ldc, ldo.  cin may be NULL
// (treated as zero).  A NULL m[t] drops term t.
template <class T>
struct SweepProb {
    T* out;
    const T* cin;
    const T* m[3];
    const T* x[3];
    long long ldo, ldc, ldx;
    T alpha;
    int diag_mask;
};

// --- batched Gauss-Jordan inversion with partial pivoting (in place) -------
// mats: count blocks of b x b (stride b*b).  info[e] is set to k+1 for the
// first pivot k that is zero or not finite (0: fine).  ws_piv: count*b ints.
template <class T>
cudaError_t gj_inverse(T* mats, int b, int count, int* info, int* ws_piv, cudaStream_t s);

// --- batched multi-term block product ---------------------------------------
template <class T>
cudaError_t gemm_batched(const GemmProb<T>* d_probs, int nprob, int b, int use_tc, cudaStream_t s);

// --- batched block x multi-vector (solve sweeps, dense FP64 residual) ----
template <class T>
cudaError_t sweep_batched(const SweepProb<T>* d_probs, int nprob, int b, int nrhs, cudaStream_t s);

// --- level-0 staging --------------------------------------------------------
// Expand/route the input blocks into the level-0 arrays of the factor:
// even D_j -> dinv[j/2], odd D_i -> dodd[i/2], even A_j -> aev[j/2],
// odd A_i -> ak[i/2], likewise C.  in_kind 0: dense column-major blocks;
// 1: banded (D: 3b per block, A/C: b per block).  bad: set to 1 if any input
// value that is read is not finite.
template <class T>
cudaError_t stage_level0(int in_kind, int n, int b, const double* A, const double* D,
                         const double* C, T* dinv, T* dodd, T* aev, T* ak, T* cev, T* ck,
                         int* bad, cudaStream_t s);

// --- iterative refinement (FP64) -------------------------------------------
// r = f - M x for the banded operator (5 diagonals in FP64).
cudaError_t resid_banded(int n, int b, const double* Dl, const double* Dd, const double* Du,
                         const double* a, const double* c, const double* x, const double* f,
                         double* r, int nrhs, cudaStream_t s);
// sumsq[q] = sum_r v[r, q]^2 for q < nrhs (deterministic two-pass), ws holds
// nrhs * 1024 doubles.
cudaError_t col_sumsq(const double* v, long long N, int nrhs, double* ws, double* sumsq,
                      cudaStream_t s);
// dst = (float) src
cudaError_t convert_d2f(const double* src, float* dst, long long n, cudaStream_t s);
// x += (double) d
cudaError_t add_f2d(double* x, const float* d, long long n, cudaStream_t s);
// x += d
cudaError_t add_d2d(double* x, const double* d, long long n, cudaStream_t s);

}  // namespace acr
