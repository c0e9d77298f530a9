// k_harith.cu -- batched kernels of the hierarchical (HODLR) arithmetic that
// reduces the low levels of block cyclic reduction with every block held in
// compressed form (Section 3: the inverses, products and sums of the
// reduction are carried out in H-matrix arithmetic, with truncation to the
// tolerance after each sum).
//
// The block format these kernels serve ("stacked" HODLR): a b x b block with
// L tree levels keeps
//   - its 2^L diagonal leaves (leaf x leaf, column-major, contiguous);
//   - per tree level l, two b x K_l column-major panels U_l and V_l (leading
//     dimension b).  Node i of level l (node size s = b >> l) covers rows
//     [i s, (i+1) s) and the columns of its sibling i^1; its block is
//     U_l[rows of i] V_l[rows of i^1]^T.  Columns beyond a node's rank are 0.
// Restricting a panel to a node's (or a diagonal block's) rows is then a
// pointer offset, which turns every step of the arithmetic into batches of
// small dense products over row ranges of these panels.
//
// Kernels (list form: one descriptor per problem; _t form: one address
// template per launch, problems found from the block and node index):
//   k_vgemm(_t)  batched products of different sizes: C = beta Cin + sum_t alpha_t op(A_t) op(B_t)
//   k_vgemm_w    the same with at most 8 output columns, one warp per problem
//   k_hrecomp(_t) truncation of one low-rank sum U V^T per node: Householder QR of U,
//              Y = V R_U^T, Householder QR of Y, one-sided Jacobi SVD of R_Y,
//              V' = Q_Y W (the leading right singular vectors of U V^T, rank by
//              sigma_k > tol sigma_1); U' = U (V^T V') follows by k_vgemm.  A
//              randomized mode works on the range of U (V^T Omega) instead
//   k_hcopy(_t)  scaled (optionally row-scaled) copies of panels between blocks
//   k_tri_leaf_inv, k_gj_reg  FP64 inverses of the leaves (tridiagonal level-0
//              leaves in O(leaf^2); pivoted Gauss-Jordan in registers) and of
//              the capacitance matrices
//   k_hkmat    the (2K x 2K) capacitance matrices [[I, T_b], [T_a, I]] of the
//              Woodbury steps of the inverse, in FP64
//   k_hband    the level-0 blocks of a 5-point operator in this format
//   k_hpack    nodes of finished blocks into the solve's pool (U, then V^T)
//   k_lr_w, k_lr_u  U' = U (V^T V') for the stand-alone truncation entry
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <cstdint>

#include "acr_internal.h"

namespace acr {

// ---------------------------------------------------------------- k_vgemm
// 64 x 32 output tile per CTA of 256 threads; thread (tx, ty) = (tid & 15,
// tid >> 4) owns rows tx + 16 i (i < 4) and columns 2 ty + j (j < 2).  Each
// term's op(A) and op(B) tiles are staged in shared memory 16 k at a time,
// with the loads ordered along the stored (contiguous) dimension of each
// operand; alpha is folded into the staged A values.
constexpr int VG_BM = 64, VG_BN = 32, VG_BK = 16;

template <class T>
__global__ void __launch_bounds__(256) k_vgemm(const VProb<T>* __restrict__ probs, const VTerm<T>* __restrict__ terms,
                                               const int2* __restrict__ tiles) {
    __shared__ T As[VG_BK][VG_BM + 1];
    __shared__ T Bs[VG_BK][VG_BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int2 tl = tiles[blockIdx.x];
    const VProb<T> P = probs[tl.x];
    const int m0 = (tl.y >> 16) * VG_BM, n0 = (tl.y & 0xffff) * VG_BN;
    T acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = T(0);
    for (int t = 0; t < P.nt; ++t) {
        const VTerm<T> Tm = terms[P.t0 + t];
        const bool ta = Tm.flags & 1, tb = Tm.flags & 2;
        for (int k0 = 0; k0 < Tm.K; k0 += VG_BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                int mm, kk;
                if (!ta) { mm = e & 63; kk = e >> 6; }
                else { mm = e >> 4; kk = e & 15; }
                const int m = m0 + mm, k = k0 + kk;
                T v = T(0);
                if (m < P.M && k < Tm.K)
                    v = ta ? Tm.A[(size_t)k + (size_t)m * Tm.lda] : Tm.A[(size_t)m + (size_t)k * Tm.lda];
                As[kk][mm] = v * Tm.alpha;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = tid + 256 * q;
                int nn, kk;
                if (!tb) { kk = e & 15; nn = e >> 4; }
                else { nn = e & 31; kk = e >> 5; }
                const int n = n0 + nn, k = k0 + kk;
                T v = T(0);
                if (n < P.N && k < Tm.K)
                    v = tb ? Tm.B[(size_t)n + (size_t)k * Tm.ldb] : Tm.B[(size_t)k + (size_t)n * Tm.ldb];
                Bs[kk][nn] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < VG_BK; ++kk) {
                T a[4], bb[2];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
                bb[0] = Bs[kk][2 * ty];
                bb[1] = Bs[kk][2 * ty + 1];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[i][0] = fma(a[i], bb[0], acc[i][0]);
                    acc[i][1] = fma(a[i], bb[1], acc[i][1]);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int n = n0 + 2 * ty + j;
        if (n >= P.N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + tx + 16 * i;
            if (m >= P.M) continue;
            T v = acc[i][j];
            if (P.Cin) v += P.beta * P.Cin[(size_t)m + (size_t)n * P.ldcin];
            P.C[(size_t)m + (size_t)n * P.ldc] = v;
        }
    }
}

// Narrow outputs (N <= 8, the ranks of most nodes): 64 x 8 tiles, thread
// (tx, ty) = (tid & 63, tid >> 6) owns row tx and columns 2 ty, 2 ty + 1, so no
// multiply-add is spent on columns beyond 8.
constexpr int VN_BN = 8;

template <class T>
__global__ void __launch_bounds__(256) k_vgemm_n8(const VProb<T>* __restrict__ probs,
                                                  const VTerm<T>* __restrict__ terms, const int2* __restrict__ tiles) {
    __shared__ T As[VG_BK][VG_BM + 1];
    __shared__ T Bs[VG_BK][VN_BN];
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    const int2 tl = tiles[blockIdx.x];
    const VProb<T> P = probs[tl.x];
    const int m0 = (tl.y >> 16) * VG_BM, n0 = (tl.y & 0xffff) * VN_BN;
    T acc0 = T(0), acc1 = T(0);
    for (int t = 0; t < P.nt; ++t) {
        const VTerm<T> Tm = terms[P.t0 + t];
        const bool ta = Tm.flags & 1, tb = Tm.flags & 2;
        for (int k0 = 0; k0 < Tm.K; k0 += VG_BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                int mm, kk;
                if (!ta) { mm = e & 63; kk = e >> 6; }
                else { mm = e >> 4; kk = e & 15; }
                const int m = m0 + mm, k = k0 + kk;
                T v = T(0);
                if (m < P.M && k < Tm.K)
                    v = ta ? Tm.A[(size_t)k + (size_t)m * Tm.lda] : Tm.A[(size_t)m + (size_t)k * Tm.lda];
                As[kk][mm] = v * Tm.alpha;
            }
            if (tid < VG_BK * VN_BN) {
                int nn, kk;
                if (!tb) { kk = tid & 15; nn = tid >> 4; }
                else { nn = tid & 7; kk = tid >> 3; }
                const int n = n0 + nn, k = k0 + kk;
                T v = T(0);
                if (n < P.N && k < Tm.K)
                    v = tb ? Tm.B[(size_t)n + (size_t)k * Tm.ldb] : Tm.B[(size_t)k + (size_t)n * Tm.ldb];
                Bs[kk][nn] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < VG_BK; ++kk) {
                const T a = As[kk][tx];
                acc0 = fma(a, Bs[kk][2 * ty], acc0);
                acc1 = fma(a, Bs[kk][2 * ty + 1], acc1);
            }
            __syncthreads();
        }
    }
    const int m = m0 + tx;
    if (m >= P.M) return;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int n = n0 + 2 * ty + j;
        if (n >= P.N) continue;
        T v = j ? acc1 : acc0;
        if (P.Cin) v += P.beta * P.Cin[(size_t)m + (size_t)n * P.ldcin];
        P.C[(size_t)m + (size_t)n * P.ldc] = v;
    }
}

template <class T>
cudaError_t vgemm(const VProb<T>* probs, const VTerm<T>* terms, const int2* tiles, long long ntiles, int narrow,
                  cudaStream_t s) {
    long long done = 0;
    while (done < ntiles) {
        const int cnt = (int)std::min<long long>(ntiles - done, 1 << 30);
        if (narrow) k_vgemm_n8<T><<<cnt, 256, 0, s>>>(probs, terms, tiles + done);
        else k_vgemm<T><<<cnt, 256, 0, s>>>(probs, terms, tiles + done);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

void vgemm_tiles(int prob, int M, int N, bool narrow, std::vector<int2>& tiles) {
    const int bn = narrow ? VN_BN : VG_BN;
    const int tm = (M + VG_BM - 1) / VG_BM, tn = (N + bn - 1) / bn;
    for (int i = 0; i < tm; ++i)
        for (int j = 0; j < tn; ++j) tiles.push_back(make_int2(prob, (i << 16) | j));
}

// ---------------------------------------------------------------- k_hrecomp
template <class T>
__device__ __forceinline__ T hwarp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Householder QR of the s x c panel P (ld s) in place, LAPACK convention
// (H_j = I - tau_j v_j v_j^T, v_j[j] = 1 stored over the diagonal): the first
// min(s, c) reflectors; rdiag receives R's diagonal, the strict upper part of
// R stays in P.  Called by all 256 threads.
template <class T>
__device__ void hh_qr(T* P, int s, int c, T* tau, T* rdiag, T* red, int* flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nr = min(s, c);
    for (int j = 0; j < nr; ++j) {
        T* col = P + (size_t)j * s;
        T part = T(0);
        for (int r = j + 1 + tid; r < s; r += 256) part += col[r] * col[r];
        part = hwarp_sum(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            T xn2 = T(0);
            for (int w = 0; w < 8; ++w) xn2 += red[w];
            const T alpha = col[j];
            if (xn2 == T(0)) {
                tau[j] = T(0);
                rdiag[j] = alpha;
                red[8] = T(0);
                *flag = 0;
            } else {
                T beta = sqrt(alpha * alpha + xn2);
                if (alpha > T(0)) beta = -beta;
                tau[j] = (beta - alpha) / beta;
                rdiag[j] = beta;
                red[8] = T(1) / (alpha - beta);
                *flag = 1;
            }
        }
        __syncthreads();
        const T scl = red[8];
        if (*flag)
            for (int r = j + 1 + tid; r < s; r += 256) col[r] *= scl;
        __syncthreads();
        if (tid == 0) col[j] = T(1);
        __syncthreads();
        const T tj = tau[j];
        if (tj != T(0))
            for (int cc = j + 1 + warp; cc < c; cc += 8) {
                T* pc = P + (size_t)cc * s;
                T d = T(0);
                for (int r = j + lane; r < s; r += 32) d += col[r] * pc[r];
                d = hwarp_sum(d) * tj;
                for (int r = j + lane; r < s; r += 32) pc[r] -= d * col[r];
            }
        __syncthreads();
    }
}

// One CTA per node.  Shared memory: panel s x R | RU r0 x R | RY ke x ke |
// Z s x HR_KZ | tau, rdiag, sv (ke each) | ord (ke ints); ke = r0 rounded up
// to even.
constexpr int HR_KZ = 8;

template <class T>
size_t hrecomp_smem(int s, int R) {
    const int r0 = std::min(s, R), ke = r0 + (r0 & 1);
    return ((size_t)s * R + (size_t)r0 * R + (size_t)ke * ke + (size_t)s * HR_KZ + 3 * (size_t)ke) * sizeof(T) +
           (size_t)ke * sizeof(int) + 16;
}

// Sketch mode (ks > 0): the range of U V^T is first captured by the sketch
// Y = U (V^T Omega) with ks Rademacher columns (a fixed hash of row and
// column), Y = Q R; then B^T = V (U^T Q) (s x ks) plays the part of Y below,
// so every QR and the Jacobi run at width ks instead of min(s, R).  A node
// whose kept rank exceeds ks - 6 is not resolved by the sketch: its rank is
// reported as -1 and nothing is written (the exact mode is run on it).

template <class T>
size_t hrecomp_sk_smem(int s, int R, int ks) {
    return ((size_t)s * R + (size_t)R * ks + 2 * (size_t)s * ks + (size_t)ks * ks + (size_t)s * HR_KZ +
            3 * (size_t)ks) * sizeof(T) + (size_t)ks * sizeof(int) + 16;
}

__device__ __forceinline__ float rademacher(int r, int c) {
    uint32_t h = (uint32_t)r * 0x9E3779B1u + (uint32_t)c * 0x7FEB352Du + 0x165667B1u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return (h & 1u) ? 1.f : -1.f;
}

template <class T>
__device__ void hrecomp_body(const RProb<T>& Pr, int* __restrict__ rank_out, T tol, int kcap, int ks = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[9];
    __shared__ int s_flag;
    const bool sk = ks > 0;
    const int s = Pr.s, R = Pr.R, r0 = sk ? min(ks, min(s, R)) : min(s, R), ke = r0 + (r0 & 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* Pn = reinterpret_cast<T*>(smem_raw);
    T *RU, *Wk = nullptr, *Yp = nullptr, *Qp = nullptr, *RY;
    if (!sk) {
        RU = Pn + (size_t)s * R;
        RY = RU + (size_t)r0 * R;
    } else {
        RU = nullptr;
        Wk = Pn + (size_t)s * R;
        Yp = Wk + (size_t)R * ks;
        Qp = Yp + (size_t)s * ks;
        RY = Qp + (size_t)s * ks;
    }
    T* Z = RY + (size_t)ke * ke;
    T* tau = Z + (size_t)s * HR_KZ;
    T* rdg = tau + ke;
    T* sv = rdg + ke;
    int* ord = reinterpret_cast<int*>(sv + ke);
    T* Yr = sk ? Yp : Pn;  // the panel whose QR feeds the Jacobi step
    const int wout = Pr.wout;
    if (r0 == 0) {
        for (int e = tid; e < s * wout; e += 256) Pr.Vout[(size_t)(e % s) + (size_t)(e / s) * Pr.ldvo] = T(0);
        if (tid == 0) *rank_out = 0;
        return;
    }
    if (sk) {
        const int k = r0;
        for (int e = tid; e < s * R; e += 256) Pn[e] = Pr.V[(size_t)(e % s) + (size_t)(e / s) * Pr.ldv];
        __syncthreads();
        // (the row index starts at j in the loops below, so that the threads
        // of a warp, which hold different j, read different banks)
        for (int e = tid; e < R * k; e += 256) {  // Wk = V^T Omega
            const int j = e % R, c = e / R;
            T acc = T(0);
            for (int t = 0; t < s; ++t) {
                const int r = (t + j) % s;
                acc = fma(Pn[r + (size_t)j * s], (T)rademacher(r, c), acc);
            }
            Wk[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < s * R; e += 256) Pn[e] = Pr.U[(size_t)(e % s) + (size_t)(e / s) * Pr.ldu];
        __syncthreads();
        for (int e = tid; e < s * k; e += 256) {  // Y = U Wk
            const int r = e % s, c = e / s;
            T acc = T(0);
            for (int j = 0; j < R; ++j) acc = fma(Pn[r + (size_t)j * s], Wk[j + (size_t)c * R], acc);
            Yp[e] = acc;
        }
        __syncthreads();
        hh_qr<T>(Yp, s, k, tau, rdg, red, &s_flag);
        for (int e = tid; e < s * k; e += 256) Qp[e] = ((e % s) == (e / s)) ? T(1) : T(0);
        __syncthreads();
        for (int j = k - 1; j >= 0; --j) {  // Q = H_0 .. H_{k-1} [I; 0]
            const T tj = tau[j];
            if (tj == T(0)) continue;
            const T* v = Yp + (size_t)j * s;
            for (int c = warp; c < k; c += 8) {
                T* qc = Qp + (size_t)c * s;
                T d = T(0);
                for (int r = j + lane; r < s; r += 32) d += v[r] * qc[r];
                d = hwarp_sum(d) * tj;
                for (int r = j + lane; r < s; r += 32) qc[r] -= d * v[r];
            }
            __syncthreads();
        }
        for (int e = tid; e < R * k; e += 256) {  // Wk = U^T Q
            const int j = e % R, c = e / R;
            T acc = T(0);
            for (int t = 0; t < s; ++t) {
                const int r = (t + j) % s;
                acc = fma(Pn[r + (size_t)j * s], Qp[r + (size_t)c * s], acc);
            }
            Wk[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < s * R; e += 256) Pn[e] = Pr.V[(size_t)(e % s) + (size_t)(e / s) * Pr.ldv];
        __syncthreads();
        for (int e = tid; e < s * k; e += 256) {  // B^T = V Wk
            const int r = e % s, c = e / s;
            T acc = T(0);
            for (int j = 0; j < R; ++j) acc = fma(Pn[r + (size_t)j * s], Wk[j + (size_t)c * R], acc);
            Yp[e] = acc;
        }
        __syncthreads();
    } else if (R >= s) {
        // ---- as wide as the node: Y = V U^T (s x s) directly -------------------
        // (U V^T = Y^T; Y's left singular vectors are those wanted), one QR
        // instead of two
        for (int e = tid; e < s * s; e += 256) {
            const int r = e % s, c = e / s;
            T y = T(0);
            for (int j = 0; j < R; ++j)
                y = fma(Pr.V[(size_t)r + (size_t)j * Pr.ldv], Pr.U[(size_t)c + (size_t)j * Pr.ldu], y);
            Pn[e] = y;
        }
        __syncthreads();
    } else {
        // ---- QR of U: keep R_U (r0 x R, upper trapezoidal) -------------------
        for (int e = tid; e < s * R; e += 256) Pn[e] = Pr.U[(size_t)(e % s) + (size_t)(e / s) * Pr.ldu];
        __syncthreads();
        hh_qr<T>(Pn, s, R, tau, rdg, red, &s_flag);
        for (int e = tid; e < r0 * R; e += 256) {
            const int i = e % r0, j = e / r0;
            RU[e] = (i < j) ? Pn[i + (size_t)j * s] : (i == j ? rdg[i] : T(0));
        }
        __syncthreads();
        // ---- Y = V R_U^T in the panel (column c reads V's columns >= c only,
        // so increasing c may overwrite column c in place; each thread owns its
        // rows)
        for (int e = tid; e < s * R; e += 256) Pn[e] = Pr.V[(size_t)(e % s) + (size_t)(e / s) * Pr.ldv];
        __syncthreads();
        for (int r = tid; r < s; r += 256)
            for (int c = 0; c < r0; ++c) {
                T y = T(0);
                for (int j = c; j < R; ++j) y = fma(Pn[r + (size_t)j * s], RU[c + (size_t)j * r0], y);
                Pn[r + (size_t)c * s] = y;
            }
        __syncthreads();
    }
    // ---- QR of Y (s x r0): R_Y into RY (ke x ke, zero padded) ----------------
    hh_qr<T>(Yr, s, r0, tau, rdg, red, &s_flag);
    for (int e = tid; e < ke * ke; e += 256) {
        const int i = e % ke, j = e / ke;
        T v = T(0);
        if (i < r0 && j < r0) v = (i < j) ? Yr[i + (size_t)j * s] : (i == j ? rdg[i] : T(0));
        RY[e] = v;
    }
    __syncthreads();
    // ---- one-sided Jacobi on the columns of R_Y (round-robin pairs) ----------
    // a pair counts as orthogonal when |a.b| <= ke u |a| |b|: the rounding of
    // a dot product of ke terms is about that size, so a tighter test would
    // keep rotating columns at the noise level (FP32) without converging
    const T eps = T(ke) * (sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-7));
    {
        T part = T(0);
        for (int e = tid; e < ke * ke; e += 256) part += RY[e] * RY[e];
        part = hwarp_sum(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            T f = T(0);
            for (int w = 0; w < 8; ++w) f += red[w];
            red[8] = f;
        }
        __syncthreads();
    }
    const T negl = red[8] * (sizeof(T) == 8 ? T(1e-28) : T(1e-13));
    __syncthreads();
    // Squared column norms are kept in sv (recomputed each sweep, updated by
    // every rotation: ||a'||^2 = ||a||^2 - t g, ||b'||^2 = ||b||^2 + t g) for
    // the skip test only: a pair whose two columns are both below 1e-2 tol
    // times the largest initial column norm (a lower bound of sigma_1) is
    // left alone: whatever the rotations do, those columns stay far below the
    // truncation level, so they cannot change the kept singular values or
    // the rank.
    T* cn = sv;
    for (int c = warp; c < ke; c += 8) {
        T n2 = T(0);
        for (int r = lane; r < ke; r += 32) n2 += RY[r + (size_t)c * ke] * RY[r + (size_t)c * ke];
        n2 = hwarp_sum(n2);
        if (lane == 0) cn[c] = n2;
    }
    __syncthreads();
    if (tid == 0) {
        T mx = T(0);
        for (int c = 0; c < ke; ++c) mx = fmax(mx, cn[c]);
        red[8] = fmax(negl, mx * (T(1e-2) * tol) * (T(1e-2) * tol));
    }
    __syncthreads();
    const T skip2 = red[8];
    __syncthreads();
    if (ke >= 2) {
        for (int sweep = 0; sweep < 16; ++sweep) {
            if (tid == 0) s_flag = 0;
            if (sweep > 0) {
                for (int c = warp; c < ke; c += 8) {
                    T n2 = T(0);
                    for (int r = lane; r < ke; r += 32) n2 += RY[r + (size_t)c * ke] * RY[r + (size_t)c * ke];
                    n2 = hwarp_sum(n2);
                    if (lane == 0) cn[c] = n2;
                }
            }
            __syncthreads();
            for (int rnd = 0; rnd < ke - 1; ++rnd) {
                for (int q = warp; q < ke / 2; q += 8) {
                    int a, bc;
                    if (q == 0) { a = ke - 1; bc = rnd; }
                    else { a = (rnd + q) % (ke - 1); bc = (rnd - q + (ke - 1)) % (ke - 1); }
                    if (!(cn[a] + cn[bc] > skip2)) continue;  // uniform over the warp
                    T* ca = RY + (size_t)a * ke;
                    T* cb = RY + (size_t)bc * ke;
                    // the rotation from the pair's own norms (norms carried
                    // over from earlier rotations drift at the noise level,
                    // and a rotation from drifted norms need not orthogonalise)
                    T ga = T(0), al = T(0), be = T(0);
                    for (int r = lane; r < ke; r += 32) {
                        const T x = ca[r], y = cb[r];
                        ga = fma(x, y, ga);
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                    }
                    ga = hwarp_sum(ga);
                    al = hwarp_sum(al);
                    be = hwarp_sum(be);
                    if (jacobi_needs(al, be, ga, eps)) {
                        const T zeta = (be - al) / (T(2) * ga);
                        const T t = jacobi_tan(zeta);
                        const T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
                        for (int r = lane; r < ke; r += 32) {
                            const T x = ca[r], y = cb[r];
                            ca[r] = cs * x - sn * y;
                            cb[r] = sn * x + cs * y;
                        }
                        __syncwarp();
                        if (lane == 0) {
                            cn[a] = fmax(T(0), al - t * ga);
                            cn[bc] = be + t * ga;
                            s_flag = 1;
                        }
                    }
                }
                __syncthreads();
            }
            const bool converged = !s_flag;
            __syncthreads();
            if (converged) break;
        }
    }
    // ---- singular values, order, rank ------------------------------------------
    for (int c = warp; c < ke; c += 8) {
        T n2 = T(0);
        for (int r = lane; r < ke; r += 32) n2 += RY[r + (size_t)c * ke] * RY[r + (size_t)c * ke];
        n2 = hwarp_sum(n2);
        if (lane == 0) sv[c] = sqrt(n2);
    }
    __syncthreads();
    for (int c = tid; c < ke; c += 256) {  // decreasing, ties by index, NaN last
        const T vc = isnan(sv[c]) ? T(-1) : sv[c];
        int pos = 0;
        for (int j = 0; j < ke; ++j) {
            const T vj = isnan(sv[j]) ? T(-1) : sv[j];
            pos += (vj > vc) || (vj == vc && j < c);
        }
        ord[pos] = c;
    }
    __syncthreads();
    if (tid == 0) {
        const T s1 = sv[ord[0]];
        int r = 0;
        if (s1 > T(0) && !isnan(s1))
            while (r < ke && r < wout && r < kcap && sv[ord[r]] > tol * s1) ++r;
        if (sk && r > r0 - 6 && r < kcap && r0 < min(s, R)) r = -1;  // the sketch saturated
        s_flag = r;
        *rank_out = r;
    }
    __syncthreads();
    const int rk = s_flag;
    if (rk < 0) return;
    // ---- V' = Q_Y [W; 0] for the kept columns, HR_KZ at a time -----------------
    for (int c0 = 0; c0 < wout; c0 += HR_KZ) {
        const int nc = min(HR_KZ, wout - c0);
        for (int e = tid; e < s * nc; e += 256) {
            const int r = e % s, c = e / s, cg = c0 + c;
            T v = T(0);
            if (cg < rk && r < r0) {
                const int src = ord[cg];
                const T nv = sv[src];
                v = nv > T(0) ? RY[r + (size_t)src * ke] / nv : T(0);
            }
            Z[r + (size_t)c * s] = v;
        }
        __syncthreads();
        if (c0 < rk)
            for (int j = r0 - 1; j >= 0; --j) {
                const T tj = tau[j];
                if (tj == T(0)) continue;
                const T* v = Yr + (size_t)j * s;
                for (int c = warp; c < nc; c += 8) {
                    T* zc = Z + (size_t)c * s;
                    T d = T(0);
                    for (int r = j + lane; r < s; r += 32) d += v[r] * zc[r];
                    d = hwarp_sum(d) * tj;
                    for (int r = j + lane; r < s; r += 32) zc[r] -= d * v[r];
                }
                __syncthreads();
            }
        for (int e = tid; e < s * nc; e += 256) {
            const int r = e % s, c = e / s;
            Pr.Vout[(size_t)r + (size_t)(c0 + c) * Pr.ldvo] = (c0 + c < rk) ? Z[r + (size_t)c * s] : T(0);
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_hrecomp(const RProb<T>* __restrict__ probs, int* __restrict__ ranks, T tol,
                                                 int kcap) {
    hrecomp_body<T>(probs[blockIdx.x], ranks + blockIdx.x, tol, kcap);
}

template <class T>
cudaError_t hrecomp(const RProb<T>* probs, int nprob, int smax, int Rmax, int* ranks, double tol, int kcap,
                    cudaStream_t st) {
    if (nprob <= 0) return cudaSuccess;
    const size_t sm = hrecomp_smem<T>(smax, Rmax);
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem((const void*)k_hrecomp<T>, sm);
    if (e != cudaSuccess) return e;
    int done = 0;
    while (done < nprob) {
        const int cnt = std::min(nprob - done, 1 << 30);
        k_hrecomp<T><<<cnt, 256, sm, st>>>(probs + done, ranks + done, (T)tol, kcap);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

size_t hrecomp_smem_bytes(int s, int R, int es) {
    return es == 8 ? hrecomp_smem<double>(s, R) : hrecomp_smem<float>(s, R);
}

// U'_i = U_i (V_i^T V'_i) for count nodes of s x R (node stride s R):
// W_i = V_i^T V'_i (R x R, in W), then U'_i = U_i W_i.  One thread per output
// element, sums in index order.
template <class T>
__global__ void k_lr_w(const T* __restrict__ V, const T* __restrict__ Vp, T* __restrict__ W, int count, int s, int R) {
    const long long n = (long long)count * R * R;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long node = e / ((long long)R * R);
        const int ab = (int)(e % ((long long)R * R)), a = ab % R, b2 = ab / R;
        const T* v = V + node * s * R + (long long)a * s;
        const T* vp = Vp + node * s * R + (long long)b2 * s;
        T acc = T(0);
        for (int r = 0; r < s; ++r) acc = fma(v[r], vp[r], acc);
        W[e] = acc;
    }
}
template <class T>
__global__ void k_lr_u(const T* __restrict__ U, const T* __restrict__ W, T* __restrict__ Uo, int count, int s, int R) {
    const long long n = (long long)count * s * R;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long node = e / ((long long)s * R);
        const int rb = (int)(e % ((long long)s * R)), r = rb % s, b2 = rb / s;
        const T* u = U + node * s * R + r;
        const T* w = W + node * R * R + (long long)b2 * R;
        T acc = T(0);
        for (int a = 0; a < R; ++a) acc = fma(u[(long long)a * s], w[a], acc);
        Uo[e] = acc;
    }
}
template <class T>
cudaError_t lowrank_apply(const T* U, const T* V, const T* Vp, T* W, T* Uo, int count, int s, int R, cudaStream_t st) {
    if (count <= 0 || s <= 0 || R <= 0) return cudaSuccess;
    k_lr_w<T><<<1024, 256, 0, st>>>(V, Vp, W, count, s, R);
    k_lr_u<T><<<1024, 256, 0, st>>>(U, W, Uo, count, s, R);
    count_launches(2);
    return cudaGetLastError();
}
template cudaError_t lowrank_apply<float>(const float*, const float*, const float*, float*, float*, int, int, int,
                                          cudaStream_t);
template cudaError_t lowrank_apply<double>(const double*, const double*, const double*, double*, double*, int, int,
                                           int, cudaStream_t);

size_t hrecomp_sketch_smem_bytes(int s, int R, int ks, int es) {
    return es == 8 ? hrecomp_sk_smem<double>(s, R, ks) : hrecomp_sk_smem<float>(s, R, ks);
}

// ---------------------------------------------------------------- k_hcopy
// dst[r, c] = beta * dst[r, c] + alpha * dv[r] * dc[c] * src[r, c] (dv, dc
// optional; a NULL src contributes 0; beta == 0 does not read dst), rows x
// cols per problem.  One CTA per chunk of 2048 consecutive elements (column
// after column) of one problem: chunks[i] = (problem, first element / 2048).
template <class T>
__global__ void __launch_bounds__(256) k_hcopy(const CProb<T>* __restrict__ probs, const int2* __restrict__ chunks) {
    const int2 ch = chunks[blockIdx.x];
    const CProb<T> P = probs[ch.x];
    const int n = P.rows * P.cols;
    const int e0 = ch.y * 2048;
    const int e1 = min(n, e0 + 2048);
    for (int e = e0 + (int)threadIdx.x; e < e1; e += 256) {
        const int c = e / P.rows, r = e - c * P.rows;
        T v = T(0);
        if (P.src) {
            v = P.alpha * P.src[(size_t)r + (size_t)c * P.lds];
            if (P.dv) v *= P.dv[r];
            if (P.dc) v *= P.dc[c];
        }
        T* d = P.dst + (size_t)r + (size_t)c * P.ldd;
        if (P.beta != T(0)) v += P.beta * *d;
        *d = v;
    }
}

template <class T>
cudaError_t hcopy(const CProb<T>* probs, const int2* chunks, long long nchunks, cudaStream_t s) {
    long long done = 0;
    while (done < nchunks) {
        const int cnt = (int)std::min<long long>(nchunks - done, 1 << 30);
        k_hcopy<T><<<cnt, 256, 0, s>>>(probs, chunks + done);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

void hcopy_chunks(int prob, long long elems, std::vector<int2>& chunks) {
    for (long long e = 0; e < elems; e += 2048) chunks.push_back(make_int2(prob, (int)(e / 2048)));
}

// ---------------------------------------------------------------- leaf inverses
// FP64 inverse of every leaf of a tridiagonal block (level 0 of a 5-point
// operator): leaf (g, lam) covers rows [lam leaf, (lam+1) leaf) of D_{sel[g]}
// (Dband: [sub, diag, super] per block, rounded to T first).  The leaf's LU factors (no pivoting:
// used only for strictly diagonally dominant rows, where they are stable) are
// formed once; thread c solves L y = e_c forward (y kept in shared memory,
// ld leaf + 1) and U x = y backward, writing x over y; the leaf's inverse is
// then stored column after column with coalesced writes.  O(leaf^2) per leaf.
template <class T>
__global__ void __launch_bounds__(128) k_tri_leaf_inv(const double* __restrict__ Dband, const int* __restrict__ sel,
                                                      int b, int leaf, T* __restrict__ out) {
    extern __shared__ double tl_sm[];
    double* lo = tl_sm;        // multipliers l_r (r >= 1)
    double* dg = lo + leaf;    // pivots u_r
    double* up = dg + leaf;    // super-diagonal
    double* Y = up + leaf;     // leaf x leaf, ld leaf + 1
    const int ld = leaf + 1;
    const int nl = b / leaf;
    const int g = blockIdx.x / nl, lam = blockIdx.x % nl;
    const double* sub = Dband + (size_t)sel[g] * 3 * b + (size_t)lam * leaf;
    const double* dia = sub + b;
    const double* sup = dia + b;
    // the entries as the factor's precision holds them (the off-diagonal
    // nodes of the same blocks are stored in T): the leaf inverses are those
    // of exactly the rounded blocks the rest of the arithmetic sees
    auto rd = [](double v) { return (double)(T)v; };
    for (int r = threadIdx.x; r < leaf; r += blockDim.x) up[r] = rd(sup[r]);
    if (threadIdx.x == 0) {
        double u = rd(dia[0]);
        dg[0] = u;
        lo[0] = 0.0;
        for (int r = 1; r < leaf; ++r) {
            const double l = rd(sub[r]) / u;
            lo[r] = l;
            u = rd(dia[r]) - l * rd(sup[r - 1]);
            dg[r] = u;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < leaf; c += blockDim.x) {
        double* y = Y + (size_t)c * ld;
        double v = 1.0;
        y[c] = 1.0;
        for (int r = c + 1; r < leaf; ++r) {
            v = -lo[r] * v;
            y[r] = v;
        }
        double xn = 0.0;
        for (int r = leaf - 1; r >= 0; --r) {
            const double yr = r >= c ? y[r] : 0.0;
            const double xr = (yr - (r + 1 < leaf ? up[r] * xn : 0.0)) / dg[r];
            y[r] = xr;
            xn = xr;
        }
    }
    __syncthreads();
    T* o = out + (size_t)blockIdx.x * leaf * leaf;
    for (int e = threadIdx.x; e < leaf * leaf; e += blockDim.x) {
        const int c = e / leaf, r = e - c * leaf;
        o[e] = (T)Y[(size_t)c * ld + r];
    }
}

template <class T>
cudaError_t tri_leaf_inverse(const double* Dband, const int* sel, int nsel, int b, int leaf, T* out, cudaStream_t s) {
    if (nsel <= 0) return cudaSuccess;
    const long long nb = (long long)nsel * (b / leaf);
    if (nb > (1LL << 30)) return cudaErrorInvalidValue;
    long long done = 0;
    while (done < nb) {
        const int cnt = (int)std::min<long long>(nb - done, 1 << 30);
        const size_t sm = (3 * (size_t)leaf + (size_t)leaf * (leaf + 1)) * sizeof(double);
        ensure_smem((const void*)k_tri_leaf_inv<T>, sm);
        k_tri_leaf_inv<T><<<cnt, 128, sm, s>>>(Dband, sel, b, leaf, out + (size_t)done * leaf * leaf);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- k_hkmat
// Kd[p] (2K x 2K, FP64, column-major) = [[I, T_{2p+1}], [T_{2p}, I]] from the
// K x K cores Tc (column-major, node after node); one CTA per parent.
template <class T>
__global__ void k_hkmat(const T* __restrict__ Tc, double* __restrict__ Kd, int K) {
    const size_t p = blockIdx.x;
    const T* Ta = Tc + (2 * p) * (size_t)K * K;
    const T* Tb = Ta + (size_t)K * K;
    double* out = Kd + p * (size_t)4 * K * K;
    const int K2 = 2 * K;
    for (int e = threadIdx.x; e < K2 * K2; e += blockDim.x) {
        const int r = e % K2, c = e / K2;
        double v;
        if (r < K && c >= K) v = (double)Tb[r + (size_t)(c - K) * K];
        else if (r >= K && c < K) v = (double)Ta[(r - K) + (size_t)c * K];
        else v = (r == c) ? 1.0 : 0.0;
        out[e] = v;
    }
}

template <class T>
cudaError_t hkmat(const T* Tc, double* Kd, int nparent, int K, cudaStream_t s) {
    if (nparent <= 0 || K <= 0) return cudaSuccess;
    int done = 0;
    while (done < nparent) {
        const int cnt = std::min(nparent - done, 1 << 30);
        k_hkmat<T><<<cnt, 256, 0, s>>>(Tc + (size_t)done * 2 * K * K, Kd + (size_t)done * 4 * K * K, K);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- k_hband
// Level-0 block D_g of a 5-point operator (tridiagonal: Dband = [sub, diag,
// super] per block) in the stacked format with one column per tree level:
// leaves hold the tridiagonal's diagonal blocks, the upper node 2p of level
// l is the single entry super[(2p+1)s - 1] at (last row of 2p, first column of
// 2p+1), the lower node 2p+1 the entry sub[(2p+1)s] at (first row of 2p+1,
// last column of 2p).  U_l, V_l of block g at Ul[l-1] + g*b, Vl[l-1] + g*b.
template <class T>
__global__ void k_hband(const double* __restrict__ Dband, int b, int L, T* __restrict__ leaves, HBandOut<T> o) {
    const int g = blockIdx.x;
    const int leaf = b >> L;
    const double* sub = Dband + (size_t)g * 3 * b;
    const double* dg = sub + b;
    const double* sup = dg + b;
    T* lv = leaves + (size_t)g * b * leaf;
    for (int e = threadIdx.x; e < b * leaf; e += blockDim.x) {
        const int lam = e / (leaf * leaf), w = e % (leaf * leaf);
        const int r = w % leaf, c = w / leaf, gr = lam * leaf + r, gc = lam * leaf + c;
        double v = 0.0;
        if (r == c) v = dg[gr];
        else if (c == r + 1) v = sup[gr];
        else if (r == c + 1) v = sub[gr];
        (void)gc;
        lv[e] = (T)v;
    }
    for (int l = 1; l <= L; ++l) {
        const int s = b >> l;
        T* U = o.U[l] + (size_t)g * b;
        T* V = o.V[l] + (size_t)g * b;
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            const int i = r / s, w = r % s;
            T u = T(0), v = T(0);
            if ((i & 1) == 0) {       // upper node i: its U row (last of i), and node i+1's V row (last of i)
                if (w == s - 1) { u = (T)sup[r]; v = T(1); }
            } else {                  // lower node i: its U row (first of i), and node i-1's V row (first of i)
                if (w == 0) { u = (T)sub[r]; v = T(1); }
            }
            U[r] = u;
            V[r] = v;
        }
    }
}

template <class T>
cudaError_t hband(const double* Dband, int nblk, int b, int L, T* leaves, const HBandOut<T>& o, cudaStream_t s) {
    if (nblk <= 0) return cudaSuccess;
    k_hband<T><<<nblk, 256, 0, s>>>(Dband, b, L, leaves, o);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- k_hpack
// One node into the solve's pool: U (s x rank, column-major), then V stored
// transposed (rank x s), the layout the compressed sweeps read.
template <class T>
__global__ void __launch_bounds__(256) k_hpack(const PProb<T>* __restrict__ probs) {
    const PProb<T> P = probs[blockIdx.x];
    const int n = P.s * P.rank;
    for (int e = threadIdx.x; e < n; e += 256) {
        P.dst[e] = P.U[(size_t)(e % P.s) + (size_t)(e / P.s) * P.ldu];
        const int ii = e % P.rank, j = e / P.rank;
        P.dst[n + e] = P.V[(size_t)j + (size_t)ii * P.ldv];
    }
}

template <class T>
cudaError_t hpack(const PProb<T>* probs, int nprob, cudaStream_t s) {
    int done = 0;
    while (done < nprob) {
        const int cnt = std::min(nprob - done, 1 << 30);
        k_hpack<T><<<cnt, 256, 0, s>>>(probs + done);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

template cudaError_t vgemm<float>(const VProb<float>*, const VTerm<float>*, const int2*, long long, int, cudaStream_t);
template cudaError_t vgemm<double>(const VProb<double>*, const VTerm<double>*, const int2*, long long, int,
                                   cudaStream_t);
template cudaError_t hrecomp<float>(const RProb<float>*, int, int, int, int*, double, int, cudaStream_t);
template cudaError_t hrecomp<double>(const RProb<double>*, int, int, int, int*, double, int, cudaStream_t);
template cudaError_t hcopy<float>(const CProb<float>*, const int2*, long long, cudaStream_t);
template cudaError_t hcopy<double>(const CProb<double>*, const int2*, long long, cudaStream_t);
template cudaError_t tri_leaf_inverse<float>(const double*, const int*, int, int, int, float*, cudaStream_t);
template cudaError_t tri_leaf_inverse<double>(const double*, const int*, int, int, int, double*, cudaStream_t);
template cudaError_t hkmat<float>(const float*, double*, int, int, cudaStream_t);
template cudaError_t hkmat<double>(const double*, double*, int, int, cudaStream_t);
template cudaError_t hband<float>(const double*, int, int, int, float*, const HBandOut<float>&, cudaStream_t);
template cudaError_t hband<double>(const double*, int, int, int, double*, const HBandOut<double>&, cudaStream_t);
template cudaError_t hpack<float>(const PProb<float>*, int, cudaStream_t);
template cudaError_t hpack<double>(const PProb<double>*, int, cudaStream_t);

}  // namespace acr

// =============================================================================
// Template batches: the problem (g, i) of a batch is derived from blockIdx and
// its operands' addresses from the batch's strides (see HAddr).
// =============================================================================
namespace acr {

template <class T>
__device__ __forceinline__ const T* haddr(const HAddr<T>& a, int g, int i) {
    if (!a.base) return nullptr;
    const long long gg = a.gmap ? (long long)a.gmap[g] : (long long)g;
    if (gg < 0) return nullptr;
    return a.base + gg * a.gs + (long long)((i >> a.ishift) ^ a.ixor) * a.is;
}

template <class T, bool NARROW>
__global__ void __launch_bounds__(256) k_vgemm_t(const __grid_constant__ VPT<T> P, int tpm, int tpn) {
    constexpr int BN = NARROW ? VN_BN : VG_BN;
    __shared__ T As[VG_BK][VG_BM + 1];
    __shared__ T Bs[VG_BK][BN + (NARROW ? 0 : 1)];
    const int tid = threadIdx.x;
    const long long tpp = (long long)tpm * tpn;
    const long long p = blockIdx.x / tpp;
    const int tt = (int)(blockIdx.x - p * tpp);
    const int g = (int)(p / P.ni), i = (int)(p - (long long)g * P.ni);
    T* C = const_cast<T*>(haddr(P.C, g, i));
    if (!C) return;
    const T* Cin = haddr(P.Cin, g, i);
    const int m0 = (tt / tpn) * VG_BM, n0 = (tt % tpn) * BN;
    // thread layout: wide tiles as k_vgemm (4 rows x 2 columns), narrow tiles
    // as k_vgemm_n8 (1 row x 2 columns)
    const int tx = NARROW ? (tid & 63) : (tid & 15), ty = NARROW ? (tid >> 6) : (tid >> 4);
    constexpr int RI = NARROW ? 1 : 4;
    T acc[RI][2];
#pragma unroll
    for (int r = 0; r < RI; ++r) acc[r][0] = acc[r][1] = T(0);
    for (int t = 0; t < P.nt; ++t) {
        const VTT<T>& Tm = P.t[t];
        const T* A = haddr(Tm.A, g, i);
        const T* B = haddr(Tm.B, g, i);
        if (!A || !B) continue;  // uniform over the CTA
        const bool ta = Tm.flags & 1, tb = Tm.flags & 2;
        const int lda = Tm.A.ld, ldb = Tm.B.ld;
        for (int k0 = 0; k0 < Tm.K; k0 += VG_BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!ta && 4 * q >= Tm.K - k0) break;  // columns the multiply loop does not read
                const int e = tid + 256 * q;
                int mm, kk;
                if (!ta) { mm = e & 63; kk = e >> 6; }
                else { mm = e >> 4; kk = e & 15; }
                const int m = m0 + mm, k = k0 + kk;
                T v = T(0);
                if (m < P.M && k < Tm.K) v = ta ? A[(size_t)k + (size_t)m * lda] : A[(size_t)m + (size_t)k * lda];
                As[kk][mm] = v * Tm.alpha;
            }
            for (int e = tid; e < VG_BK * BN; e += 256) {
                int nn, kk;
                if (!tb) { kk = e & 15; nn = e >> 4; }
                else { nn = e % BN; kk = e / BN; }
                const int n = n0 + nn, k = k0 + kk;
                T v = T(0);
                if (n < P.N && k < Tm.K) v = tb ? B[(size_t)n + (size_t)k * ldb] : B[(size_t)k + (size_t)n * ldb];
                Bs[kk][nn] = v;
            }
            __syncthreads();
            // terms of small inner dimension (node ranks) use only the first
            // K - k0 staged columns: stop after them, in steps of 4
            const int kn = min(VG_BK, Tm.K - k0);
#pragma unroll
            for (int k4 = 0; k4 < VG_BK; k4 += 4) {
                if (k4 >= kn) break;
#pragma unroll
                for (int kq = 0; kq < 4; ++kq) {
                    const int kk = k4 + kq;
                    const T b0 = Bs[kk][2 * ty], b1 = Bs[kk][2 * ty + 1];
#pragma unroll
                    for (int r = 0; r < RI; ++r) {
                        const T a = As[kk][tx + (NARROW ? 0 : 16 * r)];
                        acc[r][0] = fma(a, b0, acc[r][0]);
                        acc[r][1] = fma(a, b1, acc[r][1]);
                    }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int n = n0 + 2 * ty + j;
        if (n >= P.N) continue;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int m = m0 + tx + (NARROW ? 0 : 16 * r);
            if (m >= P.M) continue;
            T v = acc[r][j];
            if (Cin) v += P.beta * Cin[(size_t)m + (size_t)n * P.Cin.ld];
            C[(size_t)m + (size_t)n * P.C.ld] = v;
        }
    }
}

// Products with at most 8 output columns, one warp per (problem, row tile),
// 8 warps per CTA, no shared memory and no barrier.
//   KL (M <= 8): lane l computes the outputs l and l + 32 of the M x N
//     block (column-major order): the rank x rank products V^T U of the
//     HODLR arithmetic, a handful of outputs over a long inner dimension.
//   !KL: lane l owns rows r0 + l and r0 + l + 32 of a 64-row tile.
// Every output is summed exactly as the tile kernel sums it (terms in order,
// k ascending, acc = fma(alpha op(A)[m, k], op(B)[k, n], acc), then
// + beta Cin), so the two give bitwise the same results.  A lane split of the
// inner dimension, more accurate per product, was measured to change the
// rounding of the HODLR inverses enough to raise the FGMRES iterations of the
// 1024^2 Helmholtz solve from 21 to 25; the order is kept.
template <class T, int NN, bool KL>
__global__ void __launch_bounds__(256) k_vgemm_w(const __grid_constant__ VPT<T> P, int tpm, long long nwork) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * 8 + warp;
    if (w >= nwork) return;
    const long long p = w / tpm;
    const int tile = (int)(w - p * tpm);
    const int g = (int)(p / P.ni), i = (int)(p - (long long)g * P.ni);
    T* C = const_cast<T*>(haddr(P.C, g, i));
    if (!C) return;
    const T* Cin = haddr(P.Cin, g, i);
    const int M = P.M, N = P.N;
    if (KL) {
        const int o0 = lane, o1 = lane + 32;
        const bool ok0 = o0 < M * N, ok1 = o1 < M * N;
        const int m0 = ok0 ? o0 % M : 0, n0 = ok0 ? o0 / M : 0;
        const int m1 = ok1 ? o1 % M : 0, n1 = ok1 ? o1 / M : 0;
        if (!ok0) return;  // no output for this lane (lanes are not synchronised below)
        T acc0 = T(0), acc1 = T(0);
        for (int t = 0; t < P.nt; ++t) {
            const VTT<T>& Tm = P.t[t];
            const T* A = haddr(Tm.A, g, i);
            const T* B = haddr(Tm.B, g, i);
            if (!A || !B) continue;
            const bool ta = Tm.flags & 1, tb = Tm.flags & 2;
            const long long lda = Tm.A.ld, ldb = Tm.B.ld;
            // element (m, k) of op(A) at A + m * sam + k * sak, (k, n) of op(B) at B + k * sbk + n * sbn
            const long long sam = ta ? lda : 1, sak = ta ? 1 : lda, sbk = tb ? ldb : 1, sbn = tb ? 1 : ldb;
            const T* a0 = A + m0 * sam;
            const T* b0 = B + n0 * sbn;
            const T* a1 = A + m1 * sam;
            const T* b1 = B + n1 * sbn;
            const T al = Tm.alpha;
            if (ok1) {
#pragma unroll 4
                for (int k = 0; k < Tm.K; ++k) {
                    acc0 = fma(al * a0[k * sak], b0[k * sbk], acc0);
                    acc1 = fma(al * a1[k * sak], b1[k * sbk], acc1);
                }
            } else {
#pragma unroll 8
                for (int k = 0; k < Tm.K; ++k) acc0 = fma(al * a0[k * sak], b0[k * sbk], acc0);
            }
        }
        {
            T v = acc0;
            if (Cin) v += P.beta * Cin[(size_t)m0 + (size_t)n0 * P.Cin.ld];
            C[(size_t)m0 + (size_t)n0 * P.C.ld] = v;
        }
        if (ok1) {
            T v = acc1;
            if (Cin) v += P.beta * Cin[(size_t)m1 + (size_t)n1 * P.Cin.ld];
            C[(size_t)m1 + (size_t)n1 * P.C.ld] = v;
        }
    } else {
        const int r0 = tile * 64 + lane, r1 = r0 + 32;
        const bool ok0 = r0 < M, ok1 = r1 < M;
        T acc0[NN], acc1[NN];
#pragma unroll
        for (int n = 0; n < NN; ++n) acc0[n] = acc1[n] = T(0);
        for (int t = 0; t < P.nt; ++t) {
            const VTT<T>& Tm = P.t[t];
            const T* A = haddr(Tm.A, g, i);
            const T* B = haddr(Tm.B, g, i);
            if (!A || !B) continue;
            const bool ta = Tm.flags & 1, tb = Tm.flags & 2;
            const int lda = Tm.A.ld, ldb = Tm.B.ld;
            const T al = Tm.alpha;
#pragma unroll 4
            for (int k = 0; k < Tm.K; ++k) {
                const T a0 = ok0 ? al * (ta ? A[(size_t)k + (size_t)r0 * lda] : A[(size_t)r0 + (size_t)k * lda]) : T(0);
                const T a1 = ok1 ? al * (ta ? A[(size_t)k + (size_t)r1 * lda] : A[(size_t)r1 + (size_t)k * lda]) : T(0);
#pragma unroll
                for (int n = 0; n < NN; ++n) {
                    const T bv = n < N ? (tb ? B[(size_t)n + (size_t)k * ldb] : B[(size_t)k + (size_t)n * ldb]) : T(0);
                    acc0[n] = fma(a0, bv, acc0[n]);
                    acc1[n] = fma(a1, bv, acc1[n]);
                }
            }
        }
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            if (n >= N) continue;
            if (ok0) {
                T v = acc0[n];
                if (Cin) v += P.beta * Cin[(size_t)r0 + (size_t)n * P.Cin.ld];
                C[(size_t)r0 + (size_t)n * P.C.ld] = v;
            }
            if (ok1) {
                T v = acc1[n];
                if (Cin) v += P.beta * Cin[(size_t)r1 + (size_t)n * P.Cin.ld];
                C[(size_t)r1 + (size_t)n * P.C.ld] = v;
            }
        }
    }
}

template <class T, int NN>
cudaError_t vgemm_w_launch(const VPT<T>& P, bool kl, cudaStream_t s) {
    const int tpm = kl ? 1 : (P.M + 63) / 64;
    const long long nwork = (long long)P.ng * P.ni * tpm;
    const long long nb = (nwork + 7) / 8;
    if (nb >= (1LL << 31)) return cudaErrorInvalidValue;
    if (kl) k_vgemm_w<T, NN, true><<<(unsigned)nb, 256, 0, s>>>(P, tpm, nwork);
    else k_vgemm_w<T, NN, false><<<(unsigned)nb, 256, 0, s>>>(P, tpm, nwork);
    count_launches(1);
    return cudaGetLastError();
}

template <class T>
cudaError_t vgemm_tile_launch(const VPT<T>& P, cudaStream_t s) {
    const bool narrow = P.N <= VN_BN;
    const int tpm = (P.M + VG_BM - 1) / VG_BM, tpn = (P.N + (narrow ? VN_BN : VG_BN) - 1) / (narrow ? VN_BN : VG_BN);
    const long long n = (long long)P.ng * P.ni * tpm * tpn;
    if (n >= (1LL << 31)) return cudaErrorInvalidValue;
    if (narrow) k_vgemm_t<T, true><<<(unsigned)n, 256, 0, s>>>(P, tpm, tpn);
    else k_vgemm_t<T, false><<<(unsigned)n, 256, 0, s>>>(P, tpm, tpn);
    count_launches(1);
    return cudaGetLastError();
}

// Products with at most 8 output columns have three kernels that sum every
// output in the same order (bitwise the same results): 0 the warp kernel
// with lanes over outputs (M <= 8), 1 the warp kernel with lanes over rows,
// 2 the tile kernel.
template <class T>
cudaError_t vgemm_small_launch(const VPT<T>& P, int cand, cudaStream_t s) {
    if (cand == 2) return vgemm_tile_launch<T>(P, s);
    const bool kl = cand == 0;
    if (P.N <= 1) return vgemm_w_launch<T, 1>(P, kl, s);
    if (P.N <= 2) return vgemm_w_launch<T, 2>(P, kl, s);
    if (P.N <= 4) return vgemm_w_launch<T, 4>(P, kl, s);
    return vgemm_w_launch<T, 8>(P, kl, s);
}

// Online tile autotuner for those products: per shape (element size, M, N,
// the terms' inner dimensions, the number of problems) each candidate runs
// on one of the shape's first launches between CUDA events, and once every
// candidate's time is in, the fastest serves the shape from then on.  Since
// the candidates give the same bits, the choice changes timing only.  No
// candidate is timed inside a stream capture (the default runs there).
struct VgKey {
    int es, M, N, nt;
    long long nprob;
    int K[VT_MAXT];
    bool operator<(const VgKey& o) const {
        if (es != o.es) return es < o.es;
        if (M != o.M) return M < o.M;
        if (N != o.N) return N < o.N;
        if (nt != o.nt) return nt < o.nt;
        if (nprob != o.nprob) return nprob < o.nprob;
        for (int i = 0; i < nt; ++i)
            if (K[i] != o.K[i]) return K[i] < o.K[i];
        return false;
    }
};
struct VgTune {
    int ncand = 0, next = 0, best = -1;
    int cand[3] = {0, 0, 0};
    cudaEvent_t ev[3][2] = {};
    bool recorded[3] = {false, false, false};  // both events of candidate c are on a stream
    bool timed[3] = {false, false, false};
    float ms[3] = {0.f, 0.f, 0.f};
};
static std::mutex g_vg_mu;
static std::map<VgKey, VgTune> g_vg;
static std::atomic<long long> g_vg_tuned{0};  // shapes whose choice is made

template <class T>
cudaError_t vgemm_t(const VPT<T>& P, cudaStream_t s) {
    if (P.M <= 0 || P.N <= 0 || P.ni <= 0 || P.ng <= 0) return cudaSuccess;
    if (P.N <= 8) {
        VgKey key;
        memset(&key, 0, sizeof(key));
        key.es = (int)sizeof(T); key.M = P.M; key.N = P.N; key.nt = P.nt; key.nprob = (long long)P.ng * P.ni;
        for (int i = 0; i < P.nt && i < VT_MAXT; ++i) key.K[i] = P.t[i].K;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) {
            cudaGetLastError();
            cst = cudaStreamCaptureStatusActive;
        }
        int cand = P.M <= 8 ? 0 : 1;  // the default
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_vg_mu);
            VgTune& st = g_vg[key];
            if (st.ncand == 0) {
                if (P.M <= 8) st.cand[st.ncand++] = 0;
                st.cand[st.ncand++] = 1;
                st.cand[st.ncand++] = 2;
            }
            if (st.best < 0) {
                bool all = true;
                for (int c = 0; c < st.ncand; ++c) {
                    if (!st.timed[c] && st.recorded[c] && cudaEventQuery(st.ev[c][1]) == cudaSuccess) {
                        if (cudaEventElapsedTime(&st.ms[c], st.ev[c][0], st.ev[c][1]) != cudaSuccess)
                            st.ms[c] = 3.0e38f;  // no usable time: never the fastest
                        st.timed[c] = true;
                    }
                    all = all && st.timed[c];
                }
                cudaGetLastError();  // a pending event query is not an error
                if (all) {
                    int b = 0;
                    for (int c = 1; c < st.ncand; ++c)
                        if (st.ms[c] < st.ms[b]) b = c;
                    st.best = b;
                    g_vg_tuned.fetch_add(1);
                }
            }
            if (st.best >= 0) {
                cand = st.cand[st.best];
            } else if (cst == cudaStreamCaptureStatusNone && st.next < st.ncand) {
                const int c = st.next++;
                if (cudaEventCreate(&st.ev[c][0]) == cudaSuccess && cudaEventCreate(&st.ev[c][1]) == cudaSuccess) {
                    cand = st.cand[c];
                    e0 = st.ev[c][0];
                    e1 = st.ev[c][1];
                } else {
                    cudaGetLastError();
                    st.ncand = c;  // time no further candidate
                    st.best = c > 0 ? 0 : -1;
                }
            }
        }
        if (e0) cudaEventRecord(e0, s);
        const cudaError_t e = vgemm_small_launch<T>(P, cand, s);
        if (e1) {
            cudaEventRecord(e1, s);
            std::lock_guard<std::mutex> lk(g_vg_mu);
            VgTune& st = g_vg[key];
            for (int c = 0; c < st.ncand; ++c)
                if (st.ev[c][1] == e1) st.recorded[c] = true;
        }
        return e;
    }
    const bool narrow = P.N <= VN_BN;
    const int tpm = (P.M + VG_BM - 1) / VG_BM, tpn = (P.N + (narrow ? VN_BN : VG_BN) - 1) / (narrow ? VN_BN : VG_BN);
    const long long n = (long long)P.ng * P.ni * tpm * tpn;
    if (n >= (1LL << 31)) return cudaErrorInvalidValue;
    if (narrow) k_vgemm_t<T, true><<<(unsigned)n, 256, 0, s>>>(P, tpm, tpn);
    else k_vgemm_t<T, false><<<(unsigned)n, 256, 0, s>>>(P, tpm, tpn);
    count_launches(1);
    return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(256) k_hcopy_t(const __grid_constant__ CPT<T> P, int cpp) {
    const long long p = blockIdx.x / cpp;
    const int ch = (int)(blockIdx.x - p * cpp);
    const int g = (int)(p / P.ni), i = (int)(p - (long long)g * P.ni);
    T* dst = const_cast<T*>(haddr(P.dst, g, i));
    if (!dst) return;
    const T* src = haddr(P.src, g, i);
    const T* dv = haddr(P.dv, g, i);
    const T* dc = haddr(P.dc, g, i);
    const int n = P.rows * P.cols;
    const int e1 = min(n, (ch + 1) * 2048);
    for (int e = ch * 2048 + (int)threadIdx.x; e < e1; e += 256) {
        const int c = e / P.rows, r = e - c * P.rows;
        T v = T(0);
        if (src) {
            v = P.alpha * src[(size_t)r + (size_t)c * P.src.ld];
            if (dv) v *= dv[r];
            if (dc) v *= dc[c];
        }
        T* d = dst + (size_t)r + (size_t)c * P.dst.ld;
        if (P.beta != T(0)) v += P.beta * *d;
        *d = v;
    }
}

template <class T>
cudaError_t hcopy_t(const CPT<T>& P, cudaStream_t s) {
    const long long el = (long long)P.rows * P.cols;
    if (el <= 0 || P.ni <= 0 || P.ng <= 0) return cudaSuccess;
    if (el >= (1LL << 31)) return cudaErrorInvalidValue;
    const int cpp = (int)((el + 2047) / 2048);
    const long long n = (long long)P.ng * P.ni * cpp;
    if (n >= (1LL << 31)) return cudaErrorInvalidValue;
    k_hcopy_t<T><<<(unsigned)n, 256, 0, s>>>(P, cpp);
    count_launches(1);
    return cudaGetLastError();
}

// one node per CTA; the body is k_hrecomp's
template <class T>
__global__ void __launch_bounds__(256) k_hrecomp_t(const __grid_constant__ RPT<T> P, int* __restrict__ ranks, T tol,
                                                   int kcap, int ks) {
    const int node = blockIdx.x;
    const int g = node / P.ni, i = node - g * P.ni;
    RProb<T> q;
    q.U = haddr(P.U, g, i);
    q.V = haddr(P.V, g, i);
    q.Vout = const_cast<T*>(haddr(P.Vout, g, i));
    q.ldu = P.U.ld;
    q.ldv = P.V.ld;
    q.ldvo = P.Vout.ld;
    q.s = P.s;
    q.R = P.R;
    q.wout = P.wout;
    hrecomp_body<T>(q, ranks + node, tol, kcap, ks);
}

template <class T>
cudaError_t hrecomp_t(const RPT<T>& P, int* ranks, double tol, int kcap, int ks_, cudaStream_t st) {
    const long long n = (long long)P.ng * P.ni;
    if (n <= 0) return cudaSuccess;
    if (n >= (1LL << 31)) return cudaErrorInvalidValue;
    const int ks = (ks_ > 0 && ks_ < std::min(P.s, P.R)) ? ks_ : 0;
    const size_t sm = ks ? hrecomp_sk_smem<T>(P.s, P.R, ks) : hrecomp_smem<T>(P.s, P.R);
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem((const void*)k_hrecomp_t<T>, sm);
    if (e != cudaSuccess) return e;
    k_hrecomp_t<T><<<(unsigned)n, 256, sm, st>>>(P, ranks, (T)tol, kcap, ks);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t vgemm_t<float>(const VPT<float>&, cudaStream_t);
template cudaError_t vgemm_t<double>(const VPT<double>&, cudaStream_t);
template cudaError_t hcopy_t<float>(const CPT<float>&, cudaStream_t);
template cudaError_t hcopy_t<double>(const CPT<double>&, cudaStream_t);
template cudaError_t hrecomp_t<float>(const RPT<float>&, int*, double, int, int, cudaStream_t);
template cudaError_t hrecomp_t<double>(const RPT<double>&, int*, double, int, int, cudaStream_t);

}  // namespace acr

// =============================================================================
// Batched inversion of small blocks (b <= 64) by Gauss-Jordan with partial
// pivoting, register resident: 256 threads per block, thread (r, g) = (tid &
// 63, tid >> 6) holds row r, columns [16 g, 16 g + 16) of the 64 x 64 working
// matrix (a b x b block is embedded in the identity).  Each pivot step finds
// the pivot in column k (lowest row index on ties), swaps rows k and p, and
// broadcasts the scaled pivot row and column k through shared memory for the
// rank-1 update; column k of the result is -column k / pivot and the pivot
// position its reciprocal.  The composed row interchanges are undone on the
// columns at the end.  info[e] = k + 1 for the first pivot k that is not
// finite or at most 16 eps(T) max |block| in magnitude (0: none).
// =============================================================================
namespace acr {

// (4 CTAs per SM: the matrices are latency-bound, one pivot step several
// barriers, so more of them in flight keep the FP64 pipes busier)
template <class T>
__global__ void __launch_bounds__(256, 4) k_gj_reg(T* __restrict__ mats, int b, int* __restrict__ info) {
    constexpr int B = 64, G = 16;
    __shared__ T rowk[B], colk[B], rowp[B];
    __shared__ T wv[8];
    __shared__ int wi[8];
    __shared__ int piv[B], srcpos[B], dstpos[B];
    __shared__ int s_info, s_p;
    __shared__ T s_amax;
    const int tid = threadIdx.x, r = tid & 63, g = tid >> 6, lane = tid & 31, warp = tid >> 5;
    T* Gm = mats + (size_t)blockIdx.x * b * b;
    T m[G];
    T amax = T(0);
    bool fin = true;
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const int c = g * G + j;
        T v;
        if (r < b && c < b) {
            v = Gm[(size_t)r + (size_t)c * b];
            fin &= isfinite(v);
            amax = fmax(amax, fabs(v));
        } else {
            v = (r == c) ? T(1) : T(0);
        }
        m[j] = v;
    }
    if (!fin) amax = T(INFINITY);
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) wv[warp] = amax;
    if (tid == 0) s_info = 0;
    __syncthreads();
    if (tid == 0) {
        T a = T(0);
        for (int w = 0; w < 8; ++w) a = fmax(a, wv[w]);
        s_amax = a;
    }
    __syncthreads();
    const T tiny = T(16) * (sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-7)) * s_amax;
    for (int k = 0; k < b; ++k) {
        const int gk = k >> 4, jk = k & 15;
        // ---- pivot: the two warps holding column k reduce over rows >= k ----
        if (g == gk) {
            T v = T(-1);
            int idx = 0x7fffffff;
            T mk = T(0);
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (j == jk) mk = m[j];  // register select (no dynamic index)
            if (r >= k && r < b) {
                v = fabs(mk);
                if (!isfinite(mk)) v = T(INFINITY);
                idx = r;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
                if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
            }
            if (lane == 0) { wv[warp & 1] = v; wi[warp & 1] = idx; }
        }
        __syncthreads();
        if (tid == 0) {
            T v = wv[0];
            int idx = wi[0];
            if (wv[1] > v || (wv[1] == v && wi[1] < idx)) { v = wv[1]; idx = wi[1]; }
            const int p = (idx < b) ? idx : k;
            s_p = p;
            piv[k] = p;
            if ((!(v > tiny) || !isfinite(v)) && s_info == 0) s_info = k + 1;
        }
        __syncthreads();
        const int p = s_p;
        // ---- interchange rows k and p ----
        if (p != k) {
            if (r == k) {
#pragma unroll
                for (int j = 0; j < G; ++j) rowk[g * G + j] = m[j];
            } else if (r == p) {
#pragma unroll
                for (int j = 0; j < G; ++j) rowp[g * G + j] = m[j];
            }
            __syncthreads();
            if (r == k) {
#pragma unroll
                for (int j = 0; j < G; ++j) m[j] = rowp[g * G + j];
            } else if (r == p) {
#pragma unroll
                for (int j = 0; j < G; ++j) m[j] = rowk[g * G + j];
            }
            __syncthreads();
        }
        // ---- pivot row and column to shared memory ----
        if (g == gk) {
            T mk = T(0);
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (j == jk) mk = m[j];
            colk[r] = mk;
        }
        if (r == k) {
#pragma unroll
            for (int j = 0; j < G; ++j) rowk[g * G + j] = m[j];
        }
        __syncthreads();
        const T pv = rowk[k];
        const bool bad = !(fabs(pv) > tiny) || !isfinite(pv);
        const T inv = bad ? T(1) : T(1) / pv;
        // ---- update ----
        if (r == k) {
#pragma unroll
            for (int j = 0; j < G; ++j) m[j] = (g * G + j == k) ? inv : m[j] * inv;
        } else {
            const T ck = colk[r];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int c = g * G + j;
                m[j] = (c == k) ? -ck * inv : fma(-ck * inv, rowk[c], m[j]);
            }
        }
        __syncthreads();
    }
    // ---- undo the interchanges on the columns (composed from the pivots in
    // reverse order) ----
    if (tid == 0) {
        for (int c = 0; c < B; ++c) srcpos[c] = c;
        for (int k = b - 1; k >= 0; --k) {
            const int pk = piv[k];
            const int t = srcpos[k]; srcpos[k] = srcpos[pk]; srcpos[pk] = t;
        }
        // srcpos[c]: the working column that holds output column c
        for (int c = 0; c < B; ++c) dstpos[srcpos[c]] = c;
        info[blockIdx.x] = s_info;
    }
    __syncthreads();
    if (r < b) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int src = g * G + j;
            if (src < b) Gm[(size_t)r + (size_t)dstpos[src] * b] = m[j];
        }
    }
}

// The same inversion for b > 64 falls back to gj_inverse.
template <class T>
cudaError_t gj_inverse_small(T* mats, int b, int count, int* info, int* ws_piv, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (b > 64) return gj_inverse<T>(mats, b, count, info, ws_piv, s);
    long long done = 0;
    while (done < count) {
        const int cnt = (int)std::min<long long>(count - done, 1 << 30);
        k_gj_reg<T><<<cnt, 256, 0, s>>>(mats + (size_t)done * b * b, b, info + done);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

template cudaError_t gj_inverse_small<float>(float*, int, int, int*, int*, cudaStream_t);
template cudaError_t gj_inverse_small<double>(double*, int, int, int*, int*, cudaStream_t);

}  // namespace acr
