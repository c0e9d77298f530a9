// k_level0.cu -- the first reduction level of a 5-point operator.
//
// For the 2D discretisations of Section 3 the level-0 blocks have exact
// structure: D_i is tridiagonal and A_i, C_i (E_i, F_i in the paper) are
// diagonal.  Then D_j^-1 costs O(b^2) (two bidiagonal solves per row of the
// inverse) instead of O(b^3), D_j^-1 A_j is a column scaling of D_j^-1, and
// the Schur complement of Eq. "fund" is an elementwise expression -- level 0
// becomes memory-bound work instead of half of all block products.
#include <atomic>
#include <cmath>

#include "acr_internal.h"

namespace acr {

// One CTA per eliminated block (up to 512 threads), thread t handling rows
// t, t + blockDim, ... of D_j^-1.  The three diagonals are staged
// in shared memory with coalesced loads; thread 0 then runs the LU recurrence
// (b sequential FP64 steps, all operands in shared memory).
// Row r of X = T^-1 solves T^T y = e_r, i.e. U^T z = e_r (forward, z_c = 0
// for c < r) then L^T y = z (backward).  z is written to X in the first pass
// and overwritten by y in the second; both passes are coalesced across rows.
template <class T>
__global__ void __launch_bounds__(512) k_tridiag_inv(const double* __restrict__ Dband, int n, int b,
                                                     T* __restrict__ dinv, int* __restrict__ info) {
    extern __shared__ double sh[];
    double* l = sh;       // l[k] = D[k,k-1] / u[k-1]; holds D[k,k-1] until the recurrence
    double* u = sh + b;   // pivots; holds D[k,k] until the recurrence
    double* du = sh + 2 * b;
    T* lt = reinterpret_cast<T*>(sh + 3 * b);  // l[k] in T
    T* rt = lt + b;                            // du[k-1] / u[k] in T
    __shared__ double s_red[32];
    const int e = blockIdx.y, j = 2 * e;
    const double* Dl = Dband + (size_t)j * 3 * b;
    const double* Dd = Dl + b;
    const double* Du = Dd + b;
    double amax = 0.0;
    for (int k = threadIdx.x; k < b; k += blockDim.x) {
        l[k] = Dl[k];
        u[k] = Dd[k];
        du[k] = (k + 1 < b) ? Du[k] : 0.0;
        amax = fmax(amax, fabs(u[k]));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) amax = fmax(amax, s_red[w]);
        const double tiny = 16.0 * 2.220446049250313e-16 * amax;
        int bad = 0;
        double up = u[0];
        l[0] = 0.0;
        if (!(fabs(up) > tiny)) bad = 1;
        for (int k = 1; k < b; ++k) {
            const double lk = (up != 0.0) ? l[k] / up : 0.0;
            up = u[k] - lk * du[k - 1];
            l[k] = lk;
            u[k] = up;
            if (!bad && !(fabs(up) > tiny)) bad = k + 1;
        }
        info[e] = bad;
    }
    __syncthreads();
    // per-element recurrences in the factor's precision, divisions hoisted
    for (int k = threadIdx.x; k < b; k += blockDim.x) {
        lt[k] = (T)l[k];
        rt[k] = (k > 0 && u[k] != 0.0) ? (T)(du[k - 1] / u[k]) : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
        T* X = dinv + (size_t)e * b * b + r;
        // forward: z_c for c >= r (the entries c < r are written by the backward pass)
        T z = (u[r] != 0.0) ? (T)(1.0 / u[r]) : T(0);
        X[(size_t)r * b] = z;
        for (int c = r + 1; c < b; ++c) {
            z = -rt[c] * z;
            X[(size_t)c * b] = z;
        }
        // backward: y_c = z_c - l_{c+1} y_{c+1}.  The z_c are read back 32 at a
        // time before the chunk's stores, so that one memory latency is paid per
        // chunk rather than per column.
        T y = X[(size_t)(b - 1) * b];
        for (int c0 = b - 2; c0 >= 0; c0 -= 32) {
            T zc[32];
#pragma unroll
            for (int u2 = 0; u2 < 32; ++u2) {
                const int c = c0 - u2;
                zc[u2] = (c >= 0 && c >= r) ? X[(size_t)c * b] : T(0);
            }
#pragma unroll
            for (int u2 = 0; u2 < 32; ++u2) {
                const int c = c0 - u2;
                if (c >= 0) {
                    y = zc[u2] - lt[c + 1] * y;
                    X[(size_t)c * b] = y;
                }
            }
        }
    }
}

template <class T>
cudaError_t tridiag_inverse(const double* Dband, int n, int b, T* dinv, int* info, cudaStream_t s) {
    const int ne = (n + 1) / 2;
    if (ne <= 0) return cudaSuccess;
    const int nt = b >= 512 ? 512 : ((b + 31) / 32) * 32;
    const size_t sm = 3 * (size_t)b * sizeof(double) + 2 * (size_t)b * sizeof(T);
    if (sm > 48 * 1024) ensure_smem((const void*)k_tridiag_inv<T>, sm);
    k_tridiag_inv<T><<<dim3(1, ne), nt, sm, s>>>(Dband, n, b, dinv, info);
    count_launches(1);
    return cudaGetLastError();
}

// grid (tiles, nk); every thread handles elements of the b x b outputs of one
// kept block, column-major (consecutive threads, consecutive rows).
template <class T>
__global__ void k_schur_level0(const double* __restrict__ Dband, const double* __restrict__ a,
                               const double* __restrict__ c, int n, int b, const T* __restrict__ dinv,
                               T* nd_even, T* nd_odd, T* na_even, T* na_odd, T* nc_even, T* nc_odd) {
    const int k = blockIdx.y, i = 2 * k + 1;
    const size_t bb = (size_t)b * b;
    const bool kev = (k & 1) == 0;
    const int ks = k >> 1;
    T* oD = (kev ? nd_even : nd_odd) + ks * bb;
    T* oA = (i >= 3) ? (kev ? na_even : na_odd) + ks * bb : nullptr;
    T* oC = (i + 2 < n) ? (kev ? nc_even : nc_odd) + ks * bb : nullptr;
    const bool hasR = (i + 1 < n);
    const T* Xm = dinv + (size_t)(k) * bb;       // D_{i-1}^-1 (slot (i-1)/2 = k)
    const T* Xp = dinv + (size_t)(k + 1) * bb;   // D_{i+1}^-1 (slot (i+1)/2)
    const double* ai = a + (size_t)i * b;
    const double* ci = c + (size_t)i * b;
    const double* am = a + (size_t)(i - 1) * b;
    const double* cm = c + (size_t)(i - 1) * b;
    const double* ap = hasR ? a + (size_t)(i + 1) * b : nullptr;
    const double* cp = hasR ? c + (size_t)(i + 1) * b : nullptr;
    const double* Dl = Dband + (size_t)i * 3 * b;
    const double* Dd = Dl + b;
    const double* Du = Dd + b;
    // columns split over blockIdx.x, rows over threads (no integer division)
    for (int col = blockIdx.x; col < b; col += gridDim.x) {
        const T cmc = (T)cm[col], amc = (T)am[col];
        const T apc = hasR ? (T)ap[col] : T(0), cpc = hasR ? (T)cp[col] : T(0);
        const size_t o0 = (size_t)col * b;
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            const size_t t = o0 + r;
            T d = T(0);
            if (r == col) d = (T)Dd[r];
            else if (r == col + 1) d = (T)Dl[r];
            else if (col == r + 1) d = (T)Du[r];
            const T air = (T)ai[r], cir = (T)ci[r];
            const T xm = Xm[t];
            d -= air * xm * cmc;
            T xp = T(0);
            if (hasR) {
                xp = Xp[t];
                d -= cir * xp * apc;
            }
            oD[t] = d;
            if (oA) oA[t] = -air * xm * amc;
            if (oC) oC[t] = -cir * xp * cpc;
        }
    }
}

template <class T>
cudaError_t schur_level0(const double* Dband, const double* a, const double* c, int n, int b, const T* dinv,
                         T* nd_even, T* nd_odd, T* na_even, T* na_odd, T* nc_even, T* nc_odd, cudaStream_t s) {
    const int nk = n / 2;
    if (nk <= 0) return cudaSuccess;
    int gx = b < 16 ? b : 16;
    dim3 g(gx, nk);
    k_schur_level0<T><<<g, 256, 0, s>>>(Dband, a, c, n, b, dinv, nd_even, nd_odd, na_even, na_odd, nc_even,
                                        nc_odd);
    count_launches(1);
    return cudaGetLastError();
}

template <class T>
__global__ void k_stage_diag(const double* __restrict__ a, const double* __restrict__ c, int n, int b, T* aev,
                             T* cev, T* ak, T* ck, int* bad, const double* __restrict__ Dband) {
    const int j = blockIdx.y;
    const int slot = j >> 1;
    T* da = (j & 1) ? ak + (size_t)slot * b : aev + (size_t)slot * b;
    T* dc = (j & 1) ? ck + (size_t)slot * b : cev + (size_t)slot * b;
    bool fin = true;
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
        const double av = (j > 0) ? a[(size_t)j * b + r] : 0.0;
        const double cv = (j + 1 < n) ? c[(size_t)j * b + r] : 0.0;
        fin &= isfinite(av) && isfinite(cv);
        for (int d = 0; d < 3; ++d) fin &= isfinite(Dband[(size_t)j * 3 * b + d * b + r]);
        da[r] = (T)av;
        dc[r] = (T)cv;
    }
    if (!fin) atomicExch(bad, 1);
}

template <class T>
cudaError_t stage_diagonals(const double* a, const double* c, int n, int b, T* aev, T* cev, T* ak, T* ck,
                            int* bad, const double* Dband, cudaStream_t s) {
    k_stage_diag<T><<<dim3(1, n), 256, 0, s>>>(a, c, n, b, aev, cev, ak, ck, bad, Dband);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t tridiag_inverse<float>(const double*, int, int, float*, int*, cudaStream_t);
template cudaError_t tridiag_inverse<double>(const double*, int, int, double*, int*, cudaStream_t);
template cudaError_t schur_level0<float>(const double*, const double*, const double*, int, int, const float*,
                                         float*, float*, float*, float*, float*, float*, cudaStream_t);
template cudaError_t schur_level0<double>(const double*, const double*, const double*, int, int, const double*,
                                          double*, double*, double*, double*, double*, double*, cudaStream_t);
template cudaError_t stage_diagonals<float>(const double*, const double*, int, int, float*, float*, float*, float*,
                                            int*, const double*, cudaStream_t);
template cudaError_t stage_diagonals<double>(const double*, const double*, int, int, double*, double*, double*,
                                             double*, int*, const double*, cudaStream_t);

}  // namespace acr
