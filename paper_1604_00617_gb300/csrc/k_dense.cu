// k_dense.cu -- dense block kernels of the block cyclic reduction path.
//
//  * batched Gauss-Jordan inversion with partial pivoting: the block-diagonal
//    H11 of the even/odd permuted system is inverted block by block
//    (Section 3, "its inverse can be computed as the inverse of each
//    individual block");
//  * batched multi-term block products for D_j^-1 A_j, D_j^-1 C_j and the
//    Schur complement H22 - H21 H11^-1 H12 (Section 3, Eq. "fund");
//  * batched block x multi-vector products for the right-hand-side reduction
//    f^(1) = f_odd - H21 H11^-1 f_even and the back-substitution;
//  * FP64 refinement helpers (residual with the original 5-point operator,
//    column norms, conversions).
//
// All blocks are column-major with leading dimension b.
#include <algorithm>
#include <cfloat>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "acr_internal.h"

namespace acr {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int k) { g_launches.fetch_add(k); }

cudaError_t ensure_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

template <class T> struct Lim;
template <> struct Lim<float> { static __device__ __forceinline__ float eps() { return FLT_EPSILON; } };
template <> struct Lim<double> { static __device__ __forceinline__ double eps() { return DBL_EPSILON; } };

template <class T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
template <class T> __device__ __forceinline__ bool tfinite(T x) { return isfinite(x); }

// 16-byte vectors of T
template <class T, int V> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 2> { using type = double2; };
template <class VT, class T> __device__ __forceinline__ T vget(const VT& v, int i);
template <> __device__ __forceinline__ float vget<float4, float>(const float4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double vget<double2, double>(const double2& v, int i) {
    return i == 0 ? v.x : v.y;
}

// Block-wide reduction helpers (blockDim.x multiple of 32, <= 1024).
template <class T>
__device__ __forceinline__ T block_max(T v, T* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = (l < nw) ? red[l] : T(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;  // valid in every thread
}

// Arg-max of |value| with the lowest index winning ties.  Every thread passes
// its candidate (val >= 0, idx; idx = INT_MAX for none).  Returns in all threads.
template <class T>
__device__ __forceinline__ void block_argmax(T& val, int& idx, T* rv, int* ri) {
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, val, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) { rv[w] = val; ri[w] = idx; }
    __syncthreads();
    if (l < nw) { val = rv[l]; idx = ri[l]; } else { val = T(-1); idx = 0x7fffffff; }
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, val, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
}

// ===========================================================================
// Gauss-Jordan inversion, one CTA per block, whole block in shared memory.
// In-place GJ with row interchanges; the inverse is unscrambled by applying
// the column interchanges in reverse order.  Singular test: a pivot that is
// not finite or |p| <= 16 eps max|D| records info = k+1 (the factor still
// runs to completion on a pivot of 1 so that nothing downstream faults).
// ===========================================================================
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_gj_small(T* __restrict__ mats, int b, int* __restrict__ info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = b + 1;
    T* M = reinterpret_cast<T*>(smem_raw);
    int* piv = reinterpret_cast<int*>(M + (size_t)ld * b);
    int* csrc = piv + b;
    __shared__ T rv[32];
    __shared__ int ri[32];
    __shared__ int s_info;
    T* G = mats + (size_t)blockIdx.x * b * b;
    const int tid = threadIdx.x;

    T amax = T(0);
    bool fin = true;
    for (int i = tid; i < b * b; i += NT) {
        const int r = i % b, c = i / b;
        const T v = G[i];
        M[r + c * ld] = v;
        fin &= tfinite(v);
        amax = fmax(amax, tabs(v));
    }
    if (!fin) amax = T(INFINITY);
    if (tid == 0) s_info = 0;
    amax = block_max(amax, rv);
    const T tiny = T(16) * Lim<T>::eps() * amax;

    for (int k = 0; k < b; ++k) {
        T val = T(-1);
        int idx = 0x7fffffff;
        for (int r = k + tid; r < b; r += NT) {
            const T v = tabs(M[r + k * ld]);
            if (v > val || (v == val && r < idx)) { val = v; idx = r; }
        }
        block_argmax(val, idx, rv, ri);
        const int p = (idx < b) ? idx : k;
        const bool bad = !(val > tiny) || !tfinite(val);
        if (tid == 0) {
            piv[k] = p;
            if (bad && s_info == 0) s_info = k + 1;
        }
        if (p != k)
            for (int c = tid; c < b; c += NT) {
                const T t = M[k + c * ld];
                M[k + c * ld] = M[p + c * ld];
                M[p + c * ld] = t;
            }
        __syncthreads();
        const T pv = M[k + k * ld];
        const T inv = bad ? T(1) : T(1) / pv;
        __syncthreads();
        for (int c = tid; c < b; c += NT)
            if (c != k) M[k + c * ld] *= inv;
        __syncthreads();
        for (int i = tid; i < b * b; i += NT) {
            const int r = i % b, c = i / b;
            if (r != k && c != k) M[r + c * ld] -= M[r + k * ld] * M[k + c * ld];
        }
        __syncthreads();
        for (int r = tid; r < b; r += NT)
            M[r + k * ld] = (r == k) ? inv : -M[r + k * ld] * inv;
        __syncthreads();
    }
    if (tid == 0) {
        for (int c = 0; c < b; ++c) csrc[c] = c;
        for (int k = b - 1; k >= 0; --k) {
            const int p = piv[k];
            const int t = csrc[k]; csrc[k] = csrc[p]; csrc[p] = t;
        }
        info[blockIdx.x] = s_info;
    }
    __syncthreads();
    for (int i = tid; i < b * b; i += NT) {
        const int r = i % b, c = i / b;
        G[i] = M[r + csrc[c] * ld];
    }
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan for blocks too large for shared memory.  Panel step:
// one CTA per block runs the GJ steps of pivots k0..k0+kb-1 on the b x kb
// panel of columns [k0, k0+kb) held in shared memory, recording the row
// interchanges.  Update step: every other column j gets
//     M[:, j] <- (P M)[:, j] with rows K zeroed + Panel * (P M)[K, j]
// (P: the panel's row interchanges), which is exactly the effect of the same
// GJ steps on that column.
// ---------------------------------------------------------------------------
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_gj_panel(T* __restrict__ mats, int b, int k0, int kb,
                                                 int* __restrict__ pivs, int* __restrict__ info,
                                                 const T* __restrict__ amax_in) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* P = reinterpret_cast<T*>(smem_raw);  // b x kb, leading dim b
    __shared__ T rv[32];
    __shared__ int ri[32];
    T* G = mats + (size_t)blockIdx.x * b * b;
    int* piv = pivs + (size_t)blockIdx.x * b;
    const int tid = threadIdx.x;
    for (int i = tid; i < b * kb; i += NT) P[i] = G[(size_t)k0 * b + i];
    const T tiny = T(16) * Lim<T>::eps() * amax_in[blockIdx.x];
    int first_bad = 0;
    __syncthreads();
    for (int kk = 0; kk < kb; ++kk) {
        const int k = k0 + kk;
        T val = T(-1);
        int idx = 0x7fffffff;
        for (int r = k + tid; r < b; r += NT) {
            const T v = tabs(P[r + kk * b]);
            if (v > val || (v == val && r < idx)) { val = v; idx = r; }
        }
        block_argmax(val, idx, rv, ri);
        const int p = (idx < b) ? idx : k;
        const bool bad = !(val > tiny) || !tfinite(val);
        if (bad && first_bad == 0) first_bad = k + 1;
        if (tid == 0) piv[k] = p;
        if (p != k)
            for (int c = tid; c < kb; c += NT) {
                const T t = P[k + c * b];
                P[k + c * b] = P[p + c * b];
                P[p + c * b] = t;
            }
        __syncthreads();
        const T inv = bad ? T(1) : T(1) / P[k + kk * b];
        __syncthreads();
        for (int c = tid; c < kb; c += NT)
            if (c != kk) P[k + c * b] *= inv;
        __syncthreads();
        for (int i = tid; i < b * kb; i += NT) {
            const int r = i % b, c = i / b;
            if (r != k && c != kk) P[r + c * b] -= P[r + kk * b] * P[k + c * b];
        }
        __syncthreads();
        for (int r = tid; r < b; r += NT)
            P[r + kk * b] = (r == k) ? inv : -P[r + kk * b] * inv;
        __syncthreads();
    }
    for (int i = tid; i < b * kb; i += NT) G[(size_t)k0 * b + i] = P[i];
    if (tid == 0 && first_bad && info[blockIdx.x] == 0) info[blockIdx.x] = first_bad;
}

// Register-resident panel step: thread t owns panel rows t, t+NT, ... (RPT of
// them, KB values each, in registers).  Per pivot, one barrier: every warp
// reduces its rows to its best candidate (largest |value| in the pivot
// column, lowest row on ties) and the owner of that row publishes the whole
// row in the warp's slot, as the owner of row k publishes row k; after the
// barrier every warp reduces the warps' candidates (the same total order, so
// the same pivot as a block-wide arg-max) and reads the pivot row from the
// winner's slot.  In FP32 the order is that of gj_pivot_key (the same order
// as the float comparison), reduced by redux.sync maxima and minima.  Slots
// alternate between two buffers by step parity: a buffer is rewritten two
// steps later, after a barrier that every reader of its previous contents has
// passed.  A row is stored with element 0 at VE - 1 and elements 1.. as
// 16-byte vectors from VE on.  Same pivots and the same arithmetic as
// k_gj_panel.  The pivot loop is not unrolled (a straight-line copy of all KB
// steps does not fit the instruction cache): instead every step leaves each
// row rotated left by one column, so the pivot column is always v[.][0] and
// register indices stay static; after KB steps the columns are back in order.
// With a stash (non-NULL), the kernel ends with the work of k_gj_gather for
// the columns [colA, colB) outside its panel (the only ones the update reads):
// those columns are not written here, and the pivots are at hand.
template <class T, int NT, int RPT, int KB>
__global__ void __launch_bounds__(NT) k_gj_panel_reg(T* __restrict__ mats, int b, int k0,
                                                     int* __restrict__ pivs, int* __restrict__ info,
                                                     const T* __restrict__ amax_in, int colA, int colB,
                                                     T* __restrict__ stash, int* __restrict__ slotmap) {
    constexpr int NW = NT / 32;
    constexpr int VE = 16 / (int)sizeof(T);  // elements per 16-byte vector
    constexpr int SH = VE - 1;               // row element c is stored at c + SH
    constexpr int RL = KB + VE;              // stored row length, a multiple of VE
    constexpr bool F32 = sizeof(T) == 4;
    static_assert(KB % VE == 0 && NW <= 32, "panel layout");
    using V16 = typename std::conditional<F32, float4, double2>::type;
    __shared__ T rv[2][NW];
    __shared__ unsigned rkey[2][NW];
    __shared__ int ri[2][NW];
    __shared__ __align__(16) T srow[2][NW][RL];  // each warp's candidate row
    __shared__ __align__(16) T skr[2][RL];       // row k
    __shared__ int s_piv[KB];
    T* G = mats + (size_t)blockIdx.x * b * b;
    int* piv = pivs + (size_t)blockIdx.x * b;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T v[RPT][KB];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int r = tid + i * NT;
#pragma unroll
        for (int c = 0; c < KB; ++c) v[i][c] = (r < b) ? G[r + (size_t)(k0 + c) * b] : T(0);
    }
    const T tiny = T(16) * Lim<T>::eps() * amax_in[blockIdx.x];
    int first_bad = 0;
#pragma unroll 1
    for (int kk = 0; kk < KB; ++kk) {
        const int k = k0 + kk, par = kk & 1;
        T val = T(-1);
        int idx = 0x7fffffff;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = tid + i * NT;
            if (r >= k && r < b) {
                const T a = tabs(v[i][0]);
                if (a > val) { val = a; idx = r; }
            }
        }
        unsigned wkey = 0;
        if constexpr (F32) {
            const unsigned key = gj_pivot_key((float)val, idx != 0x7fffffff);
            wkey = __reduce_max_sync(0xffffffffu, key);
            idx = (int)__reduce_min_sync(0xffffffffu, key == wkey ? (unsigned)idx : 0xffffffffu);
        } else {
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, val, o);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
                if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
            }
        }
        // the warp's candidate row and row k: element 0, then 16-byte vectors
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = tid + i * NT;
            const bool cand = r == idx, rowk = r == k;
            if (cand || rowk) {
#pragma unroll
                for (int m = 0; m < KB / VE; ++m) {
                    V16 w;
                    T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
                    for (int e = 0; e < VE; ++e) wp[e] = (m * VE + e + 1 < KB) ? v[i][m * VE + e + 1] : T(0);
                    if (cand) *reinterpret_cast<V16*>(&srow[par][warp][VE * (m + 1)]) = w;
                    if (rowk) *reinterpret_cast<V16*>(&skr[par][VE * (m + 1)]) = w;
                }
                if (cand) srow[par][warp][SH] = v[i][0];
                if (rowk) skr[par][SH] = v[i][0];
            }
        }
        if (lane == 0) {
            rv[par][warp] = val;
            rkey[par][warp] = wkey;
            ri[par][warp] = idx;
        }
        __syncthreads();
        if constexpr (F32) {
            const unsigned k0v = lane < NW ? rkey[par][lane] : 0u;
            const unsigned i0v = lane < NW ? (unsigned)ri[par][lane] : 0xffffffffu;
            const unsigned bk = __reduce_max_sync(0xffffffffu, k0v);
            idx = (int)__reduce_min_sync(0xffffffffu, k0v == bk ? i0v : 0xffffffffu);
            val = bk ? (T)gj_pivot_mag(bk) : T(-1);
        } else {
            val = lane < NW ? rv[par][lane] : T(-1);
            idx = lane < NW ? ri[par][lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, val, o);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
                if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
            }
        }
        const int p = (idx < b) ? idx : k;
        const bool bad = !(val > tiny) || !tfinite(val);
        if (bad && first_bad == 0) first_bad = k + 1;
        if (tid == 0) {
            piv[k] = p;
            s_piv[kk] = p;
        }
        // the pivot row: the winning warp's slot (row k itself when p == k)
        const T* spr = (p == k) ? skr[par] : srow[par][(p % NT) >> 5];
        const T inv = bad ? T(1) : T(1) / spr[SH];
        // row p takes row k's values; fi: each row's multiplier
        T fi[RPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = tid + i * NT;
            if (r == p && r != k) {
                v[i][0] = skr[par][SH];
#pragma unroll
                for (int m = 0; m < KB / VE; ++m) {
                    const V16 w = *reinterpret_cast<const V16*>(&skr[par][VE * (m + 1)]);
                    const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
                    for (int e = 0; e < VE; ++e)
                        if (m * VE + e + 1 < KB) v[i][m * VE + e + 1] = wp[e];
                }
            }
            fi[i] = v[i][0] * inv;
        }
        // column c of this step is stored at c - 1 afterwards (the pivot
        // column, c = 0, moves to KB - 1); the pivot row's elements 1.. are
        // read a 16-byte vector at a time.  Row k is redone below.
#pragma unroll
        for (int m = 0; m < KB / VE; ++m) {
            const V16 w = *reinterpret_cast<const V16*>(spr + VE * (m + 1));
            const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                const int c = m * VE + e;
                if (c < KB - 1) {
#pragma unroll
                    for (int i = 0; i < RPT; ++i) v[i][c] = v[i][c + 1] - fi[i] * wp[e];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = tid + i * NT;
            if (r == k) {
#pragma unroll
                for (int m = 0; m < KB / VE; ++m) {
                    const V16 w = *reinterpret_cast<const V16*>(spr + VE * (m + 1));
                    const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
                    for (int e = 0; e < VE; ++e)
                        if (m * VE + e < KB - 1) v[i][m * VE + e] = wp[e] * inv;
                }
                v[i][KB - 1] = inv;
            } else {
                v[i][KB - 1] = -fi[i];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int r = tid + i * NT;
        if (r < b) {
#pragma unroll
            for (int c = 0; c < KB; ++c) G[r + (size_t)(k0 + c) * b] = v[i][c];
        }
    }
    if (tid == 0 && first_bad && info[blockIdx.x] == 0) info[blockIdx.x] = first_bad;
    if (!stash) return;
    // gather (see k_gj_gather): composed interchanges of the panel, slot map,
    // and the moved rows of the other columns of [colA, colB) into the stash
    extern __shared__ int gsh[];
    int* perm = gsh;          // b
    int* slot = perm + b;     // b
    int* list = slot + b;     // KB
    __shared__ int s_cnt;
    for (int r = tid; r < b; r += NT) { perm[r] = r; slot[r] = -1; }
    __syncthreads();  // also orders every s_piv write before the reads below
    if (tid == 0) {
        for (int kk = 0; kk < KB; ++kk) {
            const int k = k0 + kk, p = s_piv[kk];
            const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
            slot[k] = kk;
        }
        int cnt = 0;
        for (int kk = 0; kk < KB; ++kk) {
            const int p = s_piv[kk];
            if (p >= k0 + KB && slot[p] < 0) { slot[p] = KB + cnt; list[cnt++] = p; }
        }
        s_cnt = cnt;
    }
    __syncthreads();
    const int ns = KB + s_cnt;
    for (int r = tid; r < b; r += NT) slotmap[(size_t)blockIdx.x * b + r] = slot[r];
    T* st = stash + (size_t)blockIdx.x * 2 * KB * b;
    const int nJ = (colB - colA) - KB;
    for (int i = tid; i < ns * nJ; i += NT) {
        const int sl = i % ns, jc = i / ns;
        const int c = colA + jc < k0 ? colA + jc : colA + jc + KB;
        const int r = sl < KB ? k0 + sl : list[sl - KB];
        st[(size_t)sl * b + c] = G[perm[r] + (size_t)c * b];
    }
}

// Two-kernel update for full parallelism over (row tile, column tile, block).
// gather: the rows that the panel's interchanges move (the kb pivot rows K
// and the rows they were swapped with) are copied, after interchange, to a
// stash (slot s, all b columns); slot map: -1 (row unchanged), s < kb (row in
// K: base 0, stash row s is (P M)[K]), s >= kb (displaced row: base = stash).
template <class T>
__global__ void k_gj_gather(const T* __restrict__ mats, int b, int k0, int kb, int colA, int colB,
                            const int* __restrict__ pivs, T* __restrict__ stash, int* __restrict__ slotmap) {
    extern __shared__ int sh_i[];
    int* perm = sh_i;        // b
    int* slot = perm + b;    // b
    int* list = slot + b;    // kb
    __shared__ int s_cnt;
    const T* G = mats + (size_t)blockIdx.y * b * b;
    const int* piv = pivs + (size_t)blockIdx.y * b;
    T* st = stash + (size_t)blockIdx.y * 2 * kb * b;
    for (int r = threadIdx.x; r < b; r += blockDim.x) { perm[r] = r; slot[r] = -1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int kk = 0; kk < kb; ++kk) {
            const int k = k0 + kk, p = piv[k];
            const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
            slot[k] = kk;
        }
        int cnt = 0;
        for (int kk = 0; kk < kb; ++kk) {
            const int p = piv[k0 + kk];
            if (p >= k0 + kb && slot[p] < 0) { slot[p] = kb + cnt; list[cnt++] = p; }
        }
        s_cnt = cnt;
    }
    __syncthreads();
    const int ns = kb + s_cnt;
    if (blockIdx.x == 0)
        for (int r = threadIdx.x; r < b; r += blockDim.x) slotmap[(size_t)blockIdx.y * b + r] = slot[r];
    const int c0 = colA + blockIdx.x * 64;  // this CTA's columns of [colA, colB)
    for (int i = threadIdx.x; i < ns * 64; i += blockDim.x) {
        const int s = i % ns, j = i / ns, c = c0 + j;
        if (c >= colB) continue;
        const int r = s < kb ? k0 + s : list[s - kb];
        st[(size_t)s * b + c] = G[perm[r] + (size_t)c * b];
    }
}

// update: acc = Panel[rows, K] * stash[0:kb, cols] over the columns outside K.
template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gj_update_par(T* __restrict__ mats, int b, int k0, int kb, int colA, int colB, const T* __restrict__ stash,
                const int* __restrict__ slotmap, int tiles_m) {
    constexpr int RY = BM / TM, RX = BN / TN, NT = RY * RX;
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN + 1];
    T* G = mats + (size_t)blockIdx.y * b * b;
    const T* st = stash + (size_t)blockIdx.y * 2 * kb * b;
    const int* slot = slotmap + (size_t)blockIdx.y * b;
    const int nJ = (colB - colA) - kb;  // columns of [colA, colB) outside the panel
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int row0 = tm * BM, j0 = tn * BN;
    const int tid = threadIdx.x, ty = tid % RY, tx = tid / RY;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int kq = 0; kq < kb; kq += BK) {
        for (int i = tid; i < BM * BK; i += NT) {
            const int r = i % BM, k = i / BM;
            const int gr = row0 + r;
            As[k][r] = (gr < b && kq + k < kb) ? G[gr + (size_t)(k0 + kq + k) * b] : T(0);
        }
        for (int i = tid; i < BK * BN; i += NT) {
            const int j = i % BN, k = i / BN;
            const int jc = j0 + j;
            const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
            Bs[k][j] = (jc < nJ && kq + k < kb) ? st[(size_t)(kq + k) * b + c] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T af[TM], bf[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) af[i] = As[k][ty + i * RY];
#pragma unroll
            for (int j = 0; j < TN; ++j) bf[j] = Bs[k][tx + j * RX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int jc = j0 + tx + j * RX;
        if (jc >= nJ) continue;
        const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = row0 + ty + i * RY;
            if (r >= b) continue;
            const int sl = slot[r];
            const size_t o = r + (size_t)c * b;
            const T base = (sl < 0) ? G[o] : (sl < kb ? T(0) : st[(size_t)sl * b + c]);
            G[o] = base + acc[i][j];
        }
    }
}

// Same update with V consecutive rows per thread (16-byte vector access of
// the b x b block in the epilogue; a warp covers 32*V consecutive rows of one
// column).  Tile BM x BN, TN columns per thread.
template <class T, int V, int BM, int BN, int BK, int TN>
__global__ void __launch_bounds__((BM / V) * (BN / TN))
k_gj_update_vec(T* __restrict__ mats, int b, int k0, int kb, int colA, int colB, const T* __restrict__ stash,
                const int* __restrict__ slotmap, int tiles_m) {
    using VT = typename VecT<T, V>::type;
    constexpr int RY = BM / V, RX = BN / TN, NT = RY * RX;
    __shared__ __align__(16) T As[BK][BM];
    __shared__ T Bs[BK][BN + 1];
    T* G = mats + (size_t)blockIdx.y * b * b;
    const T* st = stash + (size_t)blockIdx.y * 2 * kb * b;
    const int* slot = slotmap + (size_t)blockIdx.y * b;
    const int nJ = (colB - colA) - kb;  // columns of [colA, colB) outside the panel
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int row0 = tm * BM, j0 = tn * BN;
    const int tid = threadIdx.x, ty = tid % RY, tx = tid / RY;
    const int rbase = row0 + ty * V;
    T acc[V][TN];
#pragma unroll
    for (int i = 0; i < V; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    // the operands of a K chunk go through registers: all of a chunk's loads
    // are issued at once, and the next chunk's while this one is multiplied
    constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
    static_assert(LA * NT == BM * BK && LB * NT == BK * BN, "tile loads");
    T ra[LA], rb[LB];
    auto fetch = [&](int kq) {
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            const int i = tid + u * NT, r = i % BM, k = i / BM;
            const int gr = row0 + r;
            ra[u] = (gr < b && kq + k < kb) ? G[gr + (size_t)(k0 + kq + k) * b] : T(0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = tid + u * NT, j = i % BN, k = i / BN;
            const int jc = j0 + j;
            const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
            rb[u] = (jc < nJ && kq + k < kb) ? st[(size_t)(kq + k) * b + c] : T(0);
        }
    };
    fetch(0);
    for (int kq = 0; kq < kb; kq += BK) {
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            const int i = tid + u * NT;
            As[i / BM][i % BM] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = tid + u * NT;
            Bs[i / BN][i % BN] = rb[u];
        }
        __syncthreads();
        if (kq + BK < kb) fetch(kq + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const VT av = *reinterpret_cast<const VT*>(&As[k][ty * V]);
            T bf[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) bf[j] = Bs[k][tx + j * RX];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const T a = vget<VT, T>(av, i);
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a, bf[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    if (rbase >= b) return;
    int sl[V];
    bool plain = true;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        sl[i] = slot[rbase + i];
        plain &= sl[i] < 0;
    }
    if (plain) {
        // loads of a group of columns before its stores (the stores could
        // alias later loads, so interleaving them serialises the round trips)
        constexpr int JG = TN < 8 ? TN : 8;
#pragma unroll
        for (int jg = 0; jg < TN; jg += JG) {
            VT v[JG];
#pragma unroll
            for (int jj = 0; jj < JG; ++jj) {
                const int jc = j0 + tx + (jg + jj) * RX;
                const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
                if (jc < nJ) v[jj] = *reinterpret_cast<const VT*>(G + rbase + (size_t)c * b);
            }
#pragma unroll
            for (int jj = 0; jj < JG; ++jj) {
                const int jc = j0 + tx + (jg + jj) * RX;
                if (jc >= nJ) continue;
                const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
                T* pv = reinterpret_cast<T*>(&v[jj]);
#pragma unroll
                for (int i = 0; i < V; ++i) pv[i] += acc[i][jg + jj];
                *reinterpret_cast<VT*>(G + rbase + (size_t)c * b) = v[jj];
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int jc = j0 + tx + j * RX;
        if (jc >= nJ) continue;
        const int c = colA + jc < k0 ? colA + jc : colA + jc + kb;
        T* gp = G + rbase + (size_t)c * b;
        {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const T base = (sl[i] < 0) ? gp[i] : (sl[i] < kb ? T(0) : st[(size_t)sl[i] * b + c]);
                gp[i] = base + acc[i][j];
            }
        }
    }
}

// Gather of the tensor-core form of the rank-kb update of panel [k0, k0+kb):
// the pivot rows' values at every column go, transposed (k fastest), to stT
// (b x kb per matrix: the K-major right operand), and the rows the update
// treats specially get their base value in place at every column outside the
// panel: 0 at the pivot positions, and at a row that received an interchanged
// row, that row's values.  The product G[:, c] += G[:, panel] stT[c, :]^T
// then completes the same update as k_gj_update_* (for columns outside the
// panel).  Each CTA owns 32 columns: it reads all its values before writing.
template <class T>
__global__ void k_gj_gather_tc(T* __restrict__ mats, int b, int k0, int kb, const int* __restrict__ pivs,
                               T* __restrict__ stT) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    int* perm = reinterpret_cast<int*>(sh_raw);  // b
    int* slot = perm + b;                        // b
    int* list = slot + b;                        // kb
    T* vals = reinterpret_cast<T*>(sh_raw + (((size_t)(2 * b + kb) * sizeof(int) + 15) & ~(size_t)15));  // 2kb x 33
    __shared__ int s_cnt;
    T* G = mats + (size_t)blockIdx.y * b * b;
    const int* piv = pivs + (size_t)blockIdx.y * b;
    T* st = stT + (size_t)blockIdx.y * b * kb;
    for (int r = threadIdx.x; r < b; r += blockDim.x) { perm[r] = r; slot[r] = -1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int kk = 0; kk < kb; ++kk) {
            const int k = k0 + kk, p = piv[k];
            const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
            slot[k] = kk;
        }
        int cnt = 0;
        for (int kk = 0; kk < kb; ++kk) {
            const int p = piv[k0 + kk];
            if (p >= k0 + kb && slot[p] < 0) { slot[p] = kb + cnt; list[cnt++] = p; }
        }
        s_cnt = cnt;
    }
    __syncthreads();
    const int ns = kb + s_cnt;
    const int c0 = blockIdx.x * 32;
    // consecutive threads take consecutive slots of one column: the pivot rows
    // of a panel are mostly consecutive rows, so reads and writes coalesce
    for (int i = threadIdx.x; i < ns * 32; i += blockDim.x) {
        const int sl = i % ns, j = i / ns, c = c0 + j;
        const int r = sl < kb ? k0 + sl : list[sl - kb];
        vals[sl * 33 + j] = c < b ? G[perm[r] + (size_t)c * b] : T(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kb * 32; i += blockDim.x) {
        const int sl = i % kb, j = i / kb, c = c0 + j;
        if (c < b) st[(size_t)c * kb + sl] = vals[sl * 33 + j];
    }
    for (int i = threadIdx.x; i < ns * 32; i += blockDim.x) {
        const int sl = i % ns, j = i / ns, c = c0 + j;
        if (c >= b || (c >= k0 && c < k0 + kb)) continue;
        const int r = sl < kb ? k0 + sl : list[sl - kb];
        G[r + (size_t)c * b] = sl < kb ? T(0) : vals[sl * 33 + j];
    }
}

// Column interchanges of the blocked path as one permutation: CTA z composes
// block z's interchanges (applied in reverse pivot order, in shared memory)
// into src[c] = the column that ends at position c.
__global__ void k_gj_perm(const int* __restrict__ pivs, int b, int* __restrict__ srcs) {
    extern __shared__ int sh_p[];
    int* piv = sh_p;      // b
    int* src = sh_p + b;  // b
    const int z = blockIdx.x;
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        piv[c] = pivs[(size_t)z * b + c];
        src[c] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = b - 1; k >= 0; --k) {
            const int p = piv[k];
            if (p != k) {
                const int t = src[k];
                src[k] = src[p];
                src[p] = t;
            }
        }
    __syncthreads();
    for (int c = threadIdx.x; c < b; c += blockDim.x) srcs[(size_t)z * b + c] = src[c];
}

// Apply it: a tile of UR rows x all b columns through shared memory (each
// element read once and written once, UR consecutive rows per column).
constexpr int UR = 16;
template <class T>
__global__ void k_gj_permute(T* __restrict__ mats, int b, const int* __restrict__ srcs) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T* tile = reinterpret_cast<T*>(sh_raw);  // [b][UR]
    T* G = mats + (size_t)blockIdx.y * b * b;
    const int* src = srcs + (size_t)blockIdx.y * b;
    const int r0 = blockIdx.x * UR;
    const int nr = min(UR, b - r0);
    for (int i0 = threadIdx.x; i0 < UR * b; i0 += 8 * blockDim.x) {  // 8 loads in flight per thread
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x, r = i % UR, c = i / UR;
            v[u] = (i < UR * b && r < nr) ? G[(r0 + r) + (size_t)c * b] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < UR * b) tile[(i / UR) * UR + i % UR] = v[u];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < UR * b; i += blockDim.x) {
        const int r = i % UR, c = i / UR;
        if (r < nr) G[(r0 + r) + (size_t)c * b] = tile[src[c] * UR + r];
    }
}

// Column interchanges in reverse order, one thread per row.
template <class T>
__global__ void k_gj_unscramble(T* __restrict__ mats, int b, const int* __restrict__ pivs) {
    extern __shared__ int spiv[];
    T* G = mats + (size_t)blockIdx.y * b * b;
    const int* piv = pivs + (size_t)blockIdx.y * b;
    for (int i = threadIdx.x; i < b; i += blockDim.x) spiv[i] = piv[i];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b) return;
    for (int k = b - 1; k >= 0; --k) {
        const int p = spiv[k];
        if (p != k) {
            const T t = G[r + (size_t)k * b];
            G[r + (size_t)k * b] = G[r + (size_t)p * b];
            G[r + (size_t)p * b] = t;
        }
    }
}

// max |entry| per block; grid (chunks, count), combined with an integer
// atomicMax on the IEEE bits (order-preserving for values >= 0); a NaN or Inf
// entry gives +Inf.  out must be zeroed first.
__device__ __forceinline__ void atomic_max_pos(float* a, float v) {
    atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

template <class T>
__global__ void k_maxabs(const T* __restrict__ mats, int b, T* __restrict__ out) {
    __shared__ T red[32];
    const T* G = mats + (size_t)blockIdx.y * b * b;
    const size_t bb = (size_t)b * b;
    T m = T(0);
    bool fin = true;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bb; i += (size_t)gridDim.x * blockDim.x) {
        const T v = G[i];
        fin &= tfinite(v);
        m = fmax(m, tabs(v));
    }
    if (!fin) m = T(INFINITY);
    m = block_max(m, red);
    if (threadIdx.x == 0) atomic_max_pos(out + blockIdx.y, m);
}

template <class T>
static size_t gj_small_smem(int b) {
    return (size_t)(b + 1) * b * sizeof(T) + 2 * (size_t)b * sizeof(int);
}

// Outer panel width of the two-level blocked inversion.
template <class T>
static int gj_outer_width(int b) {
    const int KB = sizeof(T) == 8 ? 16 : 32;
    return b >= 4 * 128 ? 128 : (b >= 4 * 64 ? 64 : KB);
}

// Two-level blocked Gauss-Jordan: inner panels of KB columns (register
// kernel) update only their outer panel of KO columns; after the outer panel
// is done, one rank-KO update (the same identity with panel width KO) brings
// every other column up to date.  Each column outside the outer panel is read
// and written once per outer panel instead of once per inner panel.
// Tensor-core outer update: the transposed pivot-row buffer, its problems
// (one per matrix) and tensor maps (0: the matrices, 1: the buffer).
struct GjTc {
    float* stT;
    const TcProb* probs;
    const void* maps;
    int* err;
};

template <class T>
static cudaError_t gj_blocked(T* mats, int b, int count, int* info, int* ws_piv, T* amax, T* stash, int* slotmap,
                              cudaStream_t s, const GjTc* tco = nullptr) {
    constexpr int KB = sizeof(T) == 8 ? 16 : 32;
    const int KO = tco ? 128 : gj_outer_width<T>(b);
    cudaMemsetAsync(amax, 0, sizeof(T) * count, s);
    {
        // enough CTAs to keep every SM streaming when a level has few blocks
        // (the maximum is order-independent, so the split changes no bit)
        const long long bb = (long long)b * b;
        long long cx = std::max(16LL, (608LL + count - 1) / count);
        cx = std::min(cx, std::max(1LL, bb / 1024));
        cx = std::min(cx, 256LL);
        k_maxabs<T><<<dim3((unsigned)cx, count), 256, 0, s>>>(mats, b, amax);
    }
    count_launches(1);
    const size_t psmem = (size_t)b * KB * sizeof(T);
    auto kp = k_gj_panel<T, 512>;
    ensure_smem((const void*)kp, psmem);
    constexpr int BMU = sizeof(T) == 8 ? 64 : 128, TMU = sizeof(T) == 8 ? 4 : 8;
    // rank-kw update of the columns [cA, cB) outside [k0, k0 + kw)
    // (gathered: the panel kernel has filled the stash and the slot map)
    auto update = [&](int k0, int kw, int cA, int cB, bool gathered) {
        const int nJ = (cB - cA) - kw;
        if (nJ <= 0) return;
        if (!gathered) {
            k_gj_gather<T><<<dim3((cB - cA + 63) / 64, count), 256, (2 * (size_t)b + kw) * sizeof(int), s>>>(
                mats, b, k0, kw, cA, cB, ws_piv, stash, slotmap);
            count_launches(1);
        }
        const int tmu = (b + BMU - 1) / BMU, tnu = (nJ + BMU - 1) / BMU;
        if (b % (16 / (int)sizeof(T)) == 0) {
            constexpr int VV = 16 / sizeof(T), TNV = (BMU * BMU) / (256 * VV);
            k_gj_update_vec<T, VV, BMU, BMU, 8, TNV><<<dim3(tmu * tnu, count), 256, 0, s>>>(
                mats, b, k0, kw, cA, cB, stash, slotmap, tmu);
        } else {
            k_gj_update_par<T, BMU, BMU, 8, TMU, TMU><<<dim3(tmu * tnu, count), 256, 0, s>>>(
                mats, b, k0, kw, cA, cB, stash, slotmap, tmu);
        }
        count_launches(1);
    };
    for (int K0 = 0; K0 < b; K0 += KO) {
        const int KOi = (b - K0) < KO ? (b - K0) : KO;
        for (int k0 = K0; k0 < K0 + KOi; k0 += KB) {
            const int kbi = (K0 + KOi - k0) < KB ? (K0 + KOi - k0) : KB;
            bool gathered = false;
            if (kbi == KB && b <= 1024) {  // panel rows in registers, gather fused
                const bool g = KOi > KB;
                const size_t gsm = g ? (2 * (size_t)b + KB) * sizeof(int) : 0;
                T* sts = g ? stash : nullptr;
                if (b <= 512)
                    k_gj_panel_reg<T, 512, 1, KB><<<count, 512, gsm, s>>>(mats, b, k0, ws_piv, info, amax, K0,
                                                                          K0 + KOi, sts, slotmap);
                // blocks above 512 rows: 512 threads with two rows each (fewer warps
                // per barrier than one row per thread; the same pivots and bits)
                else
                    k_gj_panel_reg<T, 512, 2, KB><<<count, 512, gsm, s>>>(mats, b, k0, ws_piv, info, amax, K0,
                                                                          K0 + KOi, sts, slotmap);
                gathered = g;
            } else {
                kp<<<count, 512, (size_t)b * kbi * sizeof(T), s>>>(mats, b, k0, kbi, ws_piv, info, amax);
            }
            count_launches(1);
            update(k0, kbi, K0, K0 + KOi, gathered);  // inside the outer panel
        }
        // everything else, once per outer panel
        if constexpr (sizeof(T) == 4) {
            if (tco) {
                const size_t gsm = (((size_t)(2 * b + KOi) * sizeof(int) + 15) & ~(size_t)15) +
                                   (size_t)2 * KOi * 33 * sizeof(T);
                ensure_smem((const void*)k_gj_gather_tc<T>, gsm);
                k_gj_gather_tc<T><<<dim3((b + 31) / 32, count), 256, gsm, s>>>(mats, b, K0, KOi, ws_piv, tco->stT);
                count_launches(1);
                const int nt = b / 128 - KOi / 128;
                cudaError_t e =
                    gemm_tc_ex(tco->probs, count, tco->maps, b, KOi, K0, nt, K0 / 128, KOi / 128, 0, tco->err, s);
                if (e != cudaSuccess) return e;
                continue;
            }
        }
        update(K0, KOi, 0, b, false);
    }
    const size_t usm = (size_t)UR * b * sizeof(T);
    if (usm <= 160 * 1024 && 2 * (size_t)b * sizeof(int) <= 160 * 1024) {
        // the slot map is free by now: it holds the composed permutation
        ensure_smem((const void*)k_gj_perm, 2 * (size_t)b * sizeof(int));
        k_gj_perm<<<count, 256, 2 * (size_t)b * sizeof(int), s>>>(ws_piv, b, slotmap);
        count_launches(1);
        ensure_smem((const void*)k_gj_permute<T>, usm);
        k_gj_permute<T><<<dim3((b + UR - 1) / UR, count), 256, usm, s>>>(mats, b, slotmap);
        count_launches(1);
        return cudaGetLastError();
    }
    dim3 gu((b + 255) / 256, count);
    k_gj_unscramble<T><<<gu, 256, b * sizeof(int), s>>>(mats, b, ws_piv);
    count_launches(1);
    return cudaGetLastError();
}

template <class T>
cudaError_t gj_inverse(T* mats, int b, int count, int* info, int* ws_piv, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    cudaMemsetAsync(info, 0, sizeof(int) * count, s);
    const size_t small = gj_small_smem<T>(b);
    if (small <= 200 * 1024) {
        auto kern = k_gj_small<T, 256>;
        ensure_smem((const void*)kern, small);
        kern<<<count, 256, small, s>>>(mats, b, info);
        count_launches(1);
        return cudaGetLastError();
    }
    // blocked path: temporaries from the stream-ordered pool
    const int KO = gj_outer_width<T>(b);
    T* amax = nullptr;
    cudaError_t e = cudaMallocAsync(&amax, sizeof(T) * count, s);
    if (e != cudaSuccess) return e;
    T* stash = nullptr;
    e = cudaMallocAsync(&stash, sizeof(T) * (size_t)count * 2 * KO * b + sizeof(int) * (size_t)count * b, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(amax, s);
        return e;
    }
    int* slotmap = reinterpret_cast<int*>(stash + (size_t)count * 2 * KO * b);
    e = gj_blocked<T>(mats, b, count, info, ws_piv, amax, stash, slotmap, s);
    cudaFreeAsync(amax, s);
    cudaFreeAsync(stash, s);
    return e;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bool gj_tc_supported(int b) { return tc_supported(b) && b >= 256 && gj_small_smem<float>(b) > 200 * 1024; }

cudaError_t gj_inverse_tc(float* mats, int b, int count, int* info, int* ws_piv, int* d_err, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (!gj_tc_supported(b)) return cudaErrorInvalidValue;
    constexpr int KB = 32, KO = 128;
    cudaMemsetAsync(info, 0, sizeof(int) * count, s);
    const size_t mb = tc_map_bytes();
    // one allocation: amax | inner stash (2 KB rows) | slot map | stT | problems | maps
    const size_t o_stash = al256(sizeof(float) * count);
    const size_t o_slot = o_stash + al256(sizeof(float) * (size_t)count * 2 * KB * b);
    const size_t o_stT = o_slot + al256(sizeof(int) * (size_t)count * b);
    const size_t o_prob = o_stT + al256(sizeof(float) * (size_t)count * KO * b);
    const size_t o_maps = o_prob + al256(sizeof(TcProb) * count);
    const size_t total = o_maps + 2 * mb;
    unsigned char* w = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&w), total, s);
    if (e != cudaSuccess) return e;
    std::vector<unsigned char> host(total - o_prob);
    TcProb* hp = reinterpret_cast<TcProb*>(host.data());
    for (int z = 0; z < count; ++z) {
        TcProb q;
        std::memset(&q, 0, sizeof(q));
        q.out = mats + (size_t)z * b * b;
        q.cin = q.out;
        q.alpha = 1.f;
        q.beta = 1.f;
        q.nterm = 1;
        q.amap[0] = 0; q.az[0] = z;
        q.bmap[0] = 1; q.bz[0] = z;
        hp[z] = q;
    }
    unsigned char* hm = host.data() + (o_maps - o_prob);
    float* stT = reinterpret_cast<float*>(w + o_stT);
    if (tc_encode_map_dims(hm, mats, b, b, count, 0) != 0 || tc_encode_map_dims(hm + mb, stT, KO, b, count, 1) != 0) {
        cudaFreeAsync(w, s);
        return cudaErrorInvalidValue;
    }
    // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(w + o_prob, host.data(), host.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        GjTc tco{stT, reinterpret_cast<const TcProb*>(w + o_prob), w + o_maps, d_err};
        e = gj_blocked<float>(mats, b, count, info, ws_piv, reinterpret_cast<float*>(w),
                              reinterpret_cast<float*>(w + o_stash), reinterpret_cast<int*>(w + o_slot), s, &tco);
    }
    cudaFreeAsync(w, s);
    return e;
}

// Scratch layout of gj_inverse_scratch (each part 256-byte aligned):
// pivots (count*b ints), max|entry| (count T), row stash (count*2*kb*b T),
// slot map (count*b ints).  The shared-memory path needs none.

template <class T>
size_t gj_scratch_bytes(int b, int count) {
    if (count <= 0 || gj_small_smem<T>(b) <= 200 * 1024) return 0;
    const int KO = gj_outer_width<T>(b);
    return al256(sizeof(int) * (size_t)count * b) + al256(sizeof(T) * (size_t)count) +
           al256(sizeof(T) * (size_t)count * 2 * KO * b) + al256(sizeof(int) * (size_t)count * b);
}

// The same batched inversion as gj_inverse, with every temporary taken from
// the caller's scratch (no device allocation).  Kernels and launch sequence
// are those of gj_inverse's blocked path.
template <class T>
cudaError_t gj_inverse_scratch(T* mats, int b, int count, int* info, void* scratch, size_t scratch_bytes,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (scratch_bytes < gj_scratch_bytes<T>(b, count)) return cudaErrorInvalidValue;
    cudaMemsetAsync(info, 0, sizeof(int) * count, s);
    const size_t small = gj_small_smem<T>(b);
    if (small <= 200 * 1024) {
        auto kern = k_gj_small<T, 256>;
        ensure_smem((const void*)kern, small);
        kern<<<count, 256, small, s>>>(mats, b, info);
        count_launches(1);
        return cudaGetLastError();
    }
    const int KO = gj_outer_width<T>(b);
    char* p = static_cast<char*>(scratch);
    int* ws_piv = reinterpret_cast<int*>(p);
    p += al256(sizeof(int) * (size_t)count * b);
    T* amax = reinterpret_cast<T*>(p);
    p += al256(sizeof(T) * (size_t)count);
    T* stash = reinterpret_cast<T*>(p);
    p += al256(sizeof(T) * (size_t)count * 2 * KO * b);
    int* slotmap = reinterpret_cast<int*>(p);
    return gj_blocked<T>(mats, b, count, info, ws_piv, amax, stash, slotmap, s);
}
template size_t gj_scratch_bytes<double>(int, int);
template size_t gj_scratch_bytes<float>(int, int);
template cudaError_t gj_inverse_scratch<double>(double*, int, int, int*, void*, size_t, cudaStream_t);
template cudaError_t gj_inverse_scratch<float>(float*, int, int, int*, void*, size_t, cudaStream_t);

// ===========================================================================
// Batched multi-term block product on CUDA cores (SIMT).
// CTA tile BM x BN, K step BK, thread tile TM x TN (rows interleaved so that
// consecutive lanes store consecutive rows).
// ===========================================================================
template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_simt(const GemmProb<T>* __restrict__ probs, int b, int tiles_m) {
    constexpr int RY = BM / TM, RX = BN / TN, NT = RY * RX;
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN + 1];
    const GemmProb<T> P = probs[blockIdx.y];
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int row0 = tm * BM, col0 = tn * BN;
    const int tid = threadIdx.x, ty = tid % RY, tx = tid / RY;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int t = 0; t < 2; ++t) {
        const T* __restrict__ A = P.a[t];
        const T* __restrict__ B = P.bm[t];
        if (A == nullptr) continue;
        for (int k0 = 0; k0 < b; k0 += BK) {
#pragma unroll
            for (int i = tid; i < BM * BK; i += NT) {
                const int r = i % BM, k = i / BM;
                const int gr = row0 + r, gk = k0 + k;
                As[k][r] = (gr < b && gk < b) ? A[gr + (size_t)gk * b] : T(0);
            }
#pragma unroll
            for (int i = tid; i < BK * BN; i += NT) {
                const int k = i % BK, c = i / BK;
                const int gk = k0 + k, gc = col0 + c;
                Bs[k][c] = (gk < b && gc < b) ? B[gk + (size_t)gc * b] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T af[TM], bf[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) af[i] = As[kk][ty + i * RY];
#pragma unroll
                for (int j = 0; j < TN; ++j) bf[j] = Bs[kk][tx + j * RX];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    // per column: the TM loads before the TM stores (out may alias cin)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int c = col0 + tx + j * RX;
        if (c >= b) continue;
        T cv[TM];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = row0 + ty + i * RY;
            cv[i] = (P.cin && r < b) ? P.cin[r + (size_t)c * b] : T(0);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = row0 + ty + i * RY;
            if (r < b) P.out[r + (size_t)c * b] = P.alpha * acc[i][j] + P.beta * cv[i];
        }
    }
}

template <class T>
cudaError_t gemm_simt(const GemmProb<T>* d_probs, int nprob, int b, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    if (sizeof(T) == 8) {
        constexpr int BM = 64, BN = 64;
        const int tm = (b + BM - 1) / BM, tn = (b + BN - 1) / BN;
        dim3 g(tm * tn, nprob);
        k_gemm_simt<T, BM, BN, 8, 4, 4><<<g, 256, 0, s>>>(d_probs, b, tm);
        count_launches(1);
    } else if (b >= 128) {
        constexpr int BM = 128, BN = 128;
        const int tm = (b + BM - 1) / BM, tn = (b + BN - 1) / BN;
        dim3 g(tm * tn, nprob);
        k_gemm_simt<T, BM, BN, 8, 8, 8><<<g, 256, 0, s>>>(d_probs, b, tm);
        count_launches(1);
    } else {
        constexpr int BM = 64, BN = 64;
        const int tm = (b + BM - 1) / BM, tn = (b + BN - 1) / BN;
        dim3 g(tm * tn, nprob);
        k_gemm_simt<T, BM, BN, 8, 4, 4><<<g, 256, 0, s>>>(d_probs, b, tm);
        count_launches(1);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t gemm_batched(const GemmProb<T>* d_probs, int nprob, int b, int use_tc, cudaStream_t s) {
    (void)use_tc;
    return gemm_simt<T>(d_probs, nprob, b, s);
}

// ===========================================================================
// Batched block x multi-vector products (solve sweeps).  One CTA computes RT
// rows of one problem for NR right-hand sides at a time; KG thread groups
// split the columns of the block, reduced through shared memory.
// ===========================================================================
template <class T, int NR, int RT, int KG, int KC>
__global__ void __launch_bounds__(RT * KG)
k_sweep(const SweepProb<T>* __restrict__ probs, int b, int nrhs, int row_tiles) {
    constexpr int NT = RT * KG;
    __shared__ T xs[KC][NR];
    __shared__ T red[KG][RT][NR + 1];
    const SweepProb<T> P = probs[blockIdx.y];
    const int row0 = blockIdx.x * RT;
    const int tid = threadIdx.x, lr = tid % RT, g = tid / RT;
    const int row = row0 + lr;
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = (nrhs - q0) < NR ? (nrhs - q0) : NR;
        T acc[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = T(0);
        const bool comb = P.sx[0] != nullptr;
        for (int t = 0; t < (comb ? 1 : 3); ++t) {
            const T* __restrict__ Mt = P.m[t];
            if (Mt == nullptr) continue;
            const T* __restrict__ X = P.x[t];
            if ((P.diag_mask >> t) & 1) {
                if (g == 0 && row < b) {
                    const T d = Mt[row];
#pragma unroll
                    for (int q = 0; q < NR; ++q)
                        if (q < nq) acc[q] += d * X[row + (size_t)(q0 + q) * P.ldx];
                }
                continue;
            }
            for (int kc = 0; kc < b; kc += KC) {
                __syncthreads();
                for (int i = tid; i < KC * NR; i += NT) {
                    const int c = i % KC, q = i / KC;
                    T v = T(0);
                    if (kc + c < b && q < nq) {
                        const size_t o = kc + c + (size_t)(q0 + q) * P.ldx;
                        if (comb) {
                            v = P.sx[0][kc + c] * X[o];
                            if (P.x[1]) v += P.sx[1][kc + c] * P.x[1][o];
                        } else {
                            v = X[o];
                        }
                    }
                    xs[c][q] = v;
                }
                __syncthreads();
                if (row < b) {
                    const int cend = (b - kc) < KC ? (b - kc) : KC;
                    for (int c = g; c < cend; c += KG) {
                        const T mv = Mt[row + (size_t)(kc + c) * b];
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] = fma(mv, xs[c][q], acc[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) red[g][lr][q] = acc[q];
        __syncthreads();
        for (int i = tid; i < RT * NR; i += NT) {
            const int r = i % RT, q = i / RT;
            const int gr = row0 + r;
            if (gr < b && q < nq) {
                T v = T(0);
#pragma unroll
                for (int gg = 0; gg < KG; ++gg) v += red[gg][r][q];
                T o = P.alpha * v;
                if (P.cin) o += P.cin[gr + (size_t)(q0 + q) * P.ldc];
                P.out[gr + (size_t)(q0 + q) * P.ldo] = o;
            }
        }
        __syncthreads();
    }
}

// Vectorized variant for blksz a multiple of V (16-byte loads of V rows):
// thread (rg, g) owns rows row0 + V*rg .. +V-1 and the columns c = g mod KG;
// the column loop is unrolled so that several 16-byte loads are in flight.

// The multi-vector operand of each term is staged whole (b x NR) in dynamic
// shared memory, so the column loop runs without barriers.
template <class T, int V, int NR, int RG, int KG>
__global__ void __launch_bounds__(RG * KG, (sizeof(T) == 4 && NR == 8) ? 3 : 1)
k_sweep_vec(const SweepProb<T>* __restrict__ probs, int b, int nrhs, T* __restrict__ part) {
    using VT = typename VecT<T, V>::type;
    constexpr int NT = RG * KG, RT = RG * V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // split-K (part != NULL): CTA z covers columns [kbeg, kend) and writes raw
    // partial sums part[((z * nprob + p) * b + row) * nrhs + q]
    const int nsplit = gridDim.z, z = blockIdx.z;
    const int KS = ((b + nsplit - 1) / nsplit + KG - 1) / KG * KG;
    const int kbeg = z * KS, kend = (kbeg + KS) < b ? (kbeg + KS) : b;
    const int kn = kend > kbeg ? kend - kbeg : 0;
    T* xs = reinterpret_cast<T*>(smem_raw);            // [kn][NR]
    T (*red)[RT][NR + 1] = reinterpret_cast<T (*)[RT][NR + 1]>(xs + (size_t)KS * NR);
    const SweepProb<T> P = probs[blockIdx.y];
    const int row0 = blockIdx.x * RT;
    const int tid = threadIdx.x, rg = tid % RG, g = tid / RG;
    const int row = row0 + rg * V;
    const bool live = row < b;
    const bool comb = P.sx[0] != nullptr;
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = (nrhs - q0) < NR ? (nrhs - q0) : NR;
        T acc[V][NR];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[v][q] = T(0);
        for (int t = 0; t < (comb ? 1 : 3); ++t) {
            const T* __restrict__ Mt = P.m[t];
            if (Mt == nullptr) continue;
            const T* __restrict__ X = P.x[t];
            if ((P.diag_mask >> t) & 1) {
                if (g == 0 && live && z == 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const T d = Mt[row + v];
#pragma unroll
                        for (int q = 0; q < NR; ++q)
                            if (q < nq) acc[v][q] += d * X[row + v + (size_t)(q0 + q) * P.ldx];
                    }
                }
                continue;
            }
            __syncthreads();
            // 8 loads in flight per thread before their stores (a store right
            // after each load would expose one memory latency per element)
            for (int i0 = tid; i0 < kn * NR; i0 += 8 * NT) {
                T xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * NT;
                    xv[u] = T(0);
                    const int cl = i % kn, q = i / kn, c = kbeg + cl;
                    if (i < kn * NR && q < nq) {
                        const size_t o = c + (size_t)(q0 + q) * P.ldx;
                        if (comb) {
                            xv[u] = P.sx[0][c] * X[o];
                            if (P.x[1]) xv[u] += P.sx[1][c] * P.x[1][o];
                        } else {
                            xv[u] = X[o];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * NT;
                    if (i < kn * NR) xs[(i % kn) * NR + i / kn] = xv[u];
                }
            }
            __syncthreads();
            if (live) {
                const T* mp = Mt + row + (size_t)kbeg * b;
#pragma unroll 8
                for (int c = g; c < kn; c += KG) {
                    const VT mv = *reinterpret_cast<const VT*>(mp + (size_t)c * b);
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        const T xq = xs[c * NR + q];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v][q] = fma(vget<VT, T>(mv, v), xq, acc[v][q]);
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int q = 0; q < NR; ++q) red[g][rg * V + v][q] = acc[v][q];
        __syncthreads();
        constexpr int PER = (RT * NR + NT - 1) / NT;  // outputs per thread
        T cv[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {  // all cin loads before the stores
            const int i = tid + u * NT, r = i % RT, q = i / RT, gr = row0 + r;
            cv[u] = (!part && P.cin && i < RT * NR && gr < b && q < nq) ? P.cin[gr + (size_t)(q0 + q) * P.ldc] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = tid + u * NT, r = i % RT, q = i / RT, gr = row0 + r;
            if (i < RT * NR && gr < b && q < nq) {
                T sum = T(0);
#pragma unroll
                for (int gg = 0; gg < KG; ++gg) sum += red[gg][r][q];
                if (part) part[(((size_t)z * gridDim.y + blockIdx.y) * b + gr) * nrhs + q0 + q] = sum;
                else P.out[gr + (size_t)(q0 + q) * P.ldo] = P.alpha * sum + cv[u];
            }
        }
        __syncthreads();
    }
}

// out = cin + alpha * sum_z part[z], fixed summation order.
template <class T>
__global__ void k_sweep_reduce(const SweepProb<T>* __restrict__ probs, int nprob, int b, int nrhs, int nsplit,
                               const T* __restrict__ part) {
    const long long total = (long long)nprob * b * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t % nrhs);
        const long long pr = t / nrhs;
        const int row = (int)(pr % b), p = (int)(pr / b);
        T sum = T(0);
        for (int zz = 0; zz < nsplit; ++zz) sum += part[(((size_t)zz * nprob + p) * b + row) * nrhs + q];
        const SweepProb<T>& P = probs[p];
        T o = P.alpha * sum;
        if (P.cin) o += P.cin[row + (size_t)q * P.ldc];
        P.out[row + (size_t)q * P.ldo] = o;
    }
}

template <class T>
cudaError_t sweep_batched(const SweepProb<T>* d_probs, int nprob, int b, int nrhs, cudaStream_t s) {
    if (nprob <= 0 || nrhs <= 0) return cudaSuccess;
    constexpr int V = sizeof(T) == 8 ? 2 : 4;
    constexpr int RG = 64, KG = 4, RT = RG * V;
    const int NRv = nrhs == 1 ? 1 : (nrhs <= 4 ? 4 : 8);
    const int rtiles = (b + RT - 1) / RT;
    // few problems: split the columns over CTAs so that every SM streams
    int nsplit = 1;
    if ((long long)nprob * rtiles < 2 * 152) {
        nsplit = (int)((4 * 152 + (long long)nprob * rtiles - 1) / ((long long)nprob * rtiles));
        nsplit = std::min(nsplit, std::max(1, b / 64));
    }
    const int KS = ((b + nsplit - 1) / nsplit + KG - 1) / KG * KG;
    const size_t vsm = ((size_t)KS * NRv + (size_t)KG * RT * (NRv + 1)) * sizeof(T);
    if (b % V == 0 && b >= 64 && vsm <= 200 * 1024) {
        T* part = nullptr;
        if (nsplit > 1 &&
            cudaMallocAsync(&part, sizeof(T) * (size_t)nsplit * nprob * b * nrhs, s) != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorMemoryAllocation;
        }
        dim3 g(rtiles, nprob, nsplit);
        if (NRv == 1) {
            auto k = k_sweep_vec<T, V, 1, RG, KG>;
            ensure_smem((const void*)k, vsm);
            k<<<g, RG * KG, vsm, s>>>(d_probs, b, nrhs, part);
        } else if (NRv == 4) {
            auto k = k_sweep_vec<T, V, 4, RG, KG>;
            ensure_smem((const void*)k, vsm);
            k<<<g, RG * KG, vsm, s>>>(d_probs, b, nrhs, part);
        } else {
            auto k = k_sweep_vec<T, V, 8, RG, KG>;
            ensure_smem((const void*)k, vsm);
            k<<<g, RG * KG, vsm, s>>>(d_probs, b, nrhs, part);
        }
        count_launches(1);
        if (part) {
            const long long tot = (long long)nprob * b * nrhs;
            int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 8);
            k_sweep_reduce<T><<<blocks, 256, 0, s>>>(d_probs, nprob, b, nrhs, nsplit, part);
            count_launches(1);
            cudaFreeAsync(part, s);
        }
        return cudaGetLastError();
    }
    constexpr int RT1 = 64, KG1 = 4, KC = 64;
    dim3 g((b + RT1 - 1) / RT1, nprob);
    const int rt = g.x;
    if (nrhs == 1)
        k_sweep<T, 1, RT1, KG1, KC><<<g, RT1 * KG1, 0, s>>>(d_probs, b, nrhs, rt);
    else if (nrhs <= 4)
        k_sweep<T, 4, RT1, KG1, KC><<<g, RT1 * KG1, 0, s>>>(d_probs, b, nrhs, rt);
    else if (nrhs <= 8)
        k_sweep<T, 8, RT1, KG1, KC><<<g, RT1 * KG1, 0, s>>>(d_probs, b, nrhs, rt);
    else
        k_sweep<T, 16, RT1, KG1, KC><<<g, RT1 * KG1, 0, s>>>(d_probs, b, nrhs, rt);
    count_launches(1);
    return cudaGetLastError();
}

// ===========================================================================
// Level-0 staging.
// ===========================================================================
template <class T>
__global__ void k_stage_dense(int n, int b, const double* __restrict__ A, const double* __restrict__ D,
                              const double* __restrict__ C, T* dinv, T* dodd, T* aev, T* ak, T* cev,
                              T* ck, int* bad) {
    const int j = blockIdx.y;  // block index
    const size_t bb = (size_t)b * b;
    const int slot = j >> 1;
    T* dD = (j & 1) ? dodd + slot * bb : dinv + slot * bb;
    T* dA = (j & 1) ? ak + slot * bb : aev + slot * bb;
    T* dC = (j & 1) ? ck + slot * bb : cev + slot * bb;
    const bool hasA = j > 0, hasC = j + 1 < n;
    bool fin = true;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bb; i += (size_t)gridDim.x * blockDim.x) {
        const double d = D[j * bb + i];
        fin &= isfinite(d);
        dD[i] = (T)d;
        if (hasA) { const double v = A[j * bb + i]; fin &= isfinite(v); dA[i] = (T)v; }
        if (hasC) { const double v = C[j * bb + i]; fin &= isfinite(v); dC[i] = (T)v; }
    }
    if (!fin) atomicExch(bad, 1);
}

template <class T>
__global__ void k_stage_banded(int n, int b, const double* __restrict__ A, const double* __restrict__ D,
                               const double* __restrict__ C, T* dinv, T* dodd, T* aev, T* ak, T* cev,
                               T* ck, int* bad) {
    const int j = blockIdx.y;
    const size_t bb = (size_t)b * b;
    const int slot = j >> 1;
    T* dD = (j & 1) ? dodd + slot * bb : dinv + slot * bb;
    T* dA = (j & 1) ? ak + slot * bb : aev + slot * bb;
    T* dC = (j & 1) ? ck + slot * bb : cev + slot * bb;
    const bool hasA = j > 0, hasC = j + 1 < n;
    const double* Dl = D + (size_t)j * 3 * b;
    const double* Dd = Dl + b;
    const double* Du = Dd + b;
    bool fin = true;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bb; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i % b), c = (int)(i / b);
        double dv = 0.0;
        if (r == c) dv = Dd[r];
        else if (r == c + 1) dv = Dl[r];
        else if (c == r + 1) dv = Du[r];
        fin &= isfinite(dv);
        dD[i] = (T)dv;
        if (hasA) { const double v = (r == c) ? A[(size_t)j * b + r] : 0.0; fin &= isfinite(v); dA[i] = (T)v; }
        if (hasC) { const double v = (r == c) ? C[(size_t)j * b + r] : 0.0; fin &= isfinite(v); dC[i] = (T)v; }
    }
    if (!fin) atomicExch(bad, 1);
}

template <class T>
cudaError_t stage_level0(int in_kind, int n, int b, const double* A, const double* D, const double* C,
                         T* dinv, T* dodd, T* aev, T* ak, T* cev, T* ck, int* bad, cudaStream_t s) {
    const size_t bb = (size_t)b * b;
    int gx = (int)((bb + 255) / 256);
    if (gx > 64) gx = 64;
    dim3 g(gx, n);
    if (in_kind == 0)
        k_stage_dense<T><<<g, 256, 0, s>>>(n, b, A, D, C, dinv, dodd, aev, ak, cev, ck, bad);
    else
        k_stage_banded<T><<<g, 256, 0, s>>>(n, b, A, D, C, dinv, dodd, aev, ak, cev, ck, bad);
    count_launches(1);
    return cudaGetLastError();
}

// ===========================================================================
// FP64 refinement helpers.
// ===========================================================================
__global__ void k_resid_banded(int n, int b, const double* __restrict__ Dl, const double* __restrict__ Dd,
                               const double* __restrict__ Du, const double* __restrict__ a,
                               const double* __restrict__ c, const double* __restrict__ x,
                               const double* __restrict__ f, double* __restrict__ r, int nrhs) {
    const long long N = (long long)n * b;
    const long long total = N * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long g = t % N, q = t / N;
        const int i = (int)(g / b), p = (int)(g % b);
        const double* xq = x + q * N;
        double y = Dd[g] * xq[g];
        if (p > 0) y += Dl[(size_t)i * b + p] * xq[g - 1];
        if (p + 1 < b) y += Du[(size_t)i * b + p] * xq[g + 1];
        if (i > 0) y += a[g] * xq[g - b];
        if (i + 1 < n) y += c[g] * xq[g + b];
        r[t] = f ? f[t] - y : y;  // f == NULL: plain product M x
    }
}

cudaError_t resid_banded(int n, int b, const double* Dl, const double* Dd, const double* Du,
                         const double* a, const double* c, const double* x, const double* f, double* r,
                         int nrhs, cudaStream_t s) {
    const long long total = (long long)n * b * nrhs;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_resid_banded<<<(int)blocks, 256, 0, s>>>(n, b, Dl, Dd, Du, a, c, x, f, r, nrhs);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_sumsq_partial(const double* __restrict__ v, long long N, double* __restrict__ ws) {
    // grid (1024 chunks, nrhs)
    __shared__ double red[32];
    const int q = blockIdx.y;
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk;
    long long hi = lo + chunk;
    if (hi > N) hi = N;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double t = v[i + q * N];
        s += t * t;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) ws[q * (long long)gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_sumsq_final(const double* __restrict__ ws, int chunks, double* __restrict__ out) {
    __shared__ double red[32];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) s += ws[q * (long long)chunks + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[q] = s;
    }
}

cudaError_t col_sumsq(const double* v, long long N, int nrhs, double* ws, double* sumsq, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    int chunks = 1024;
    if (N < 1024 * 256) chunks = (int)((N + 255) / 256);
    if (chunks < 1) chunks = 1;
    k_sumsq_partial<<<dim3(chunks, nrhs), 256, 0, s>>>(v, N, ws);
    count_launches(1);
    k_sumsq_final<<<nrhs, 256, 0, s>>>(ws, chunks, sumsq);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void k_add_f2d(double* __restrict__ x, const float* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}
__global__ void k_add_d2d(double* __restrict__ x, const double* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += d[i];
}
static int ew_blocks(long long n) {
    long long bl = (n + 255) / 256;
    if (bl > 152 * 16) bl = 152 * 16;
    return bl < 1 ? 1 : (int)bl;
}
cudaError_t convert_d2f(const double* src, float* dst, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_d2f<<<ew_blocks(n), 256, 0, s>>>(src, dst, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t add_f2d(double* x, const float* d, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_add_f2d<<<ew_blocks(n), 256, 0, s>>>(x, d, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t add_d2d(double* x, const double* d, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_add_d2d<<<ew_blocks(n), 256, 0, s>>>(x, d, n);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}
cudaError_t convert_f2d(const float* src, double* dst, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_f2d<<<ew_blocks(n), 256, 0, s>>>(src, dst, n);
    count_launches(1);
    return cudaGetLastError();
}

// grid (chunks, nrhs, nvec); ws[(i * nrhs + q) * chunks + c]
__global__ void k_multi_dot_partial(const double* __restrict__ V, const double* __restrict__ w, long long N,
                                    int nrhs, double* __restrict__ ws) {
    __shared__ double red[32];
    const int q = blockIdx.y, i = blockIdx.z, chunks = gridDim.x;
    const long long chunk = (N + chunks - 1) / chunks;
    const long long lo = blockIdx.x * chunk;
    long long hi = lo + chunk;
    if (hi > N) hi = N;
    const double* vq = V + ((long long)i * nrhs + q) * N;
    const double* wq = w + (long long)q * N;
    double s = 0.0;
    for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) s += vq[r] * wq[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) ws[((long long)i * nrhs + q) * chunks + blockIdx.x] = s;
    }
}

// grid (chunks, nrhs): one CTA per chunk of DW = 16 x 256 rows holds its
// rows of w in registers and forms all nvec partial products from them
// (w read once, 16 independent loads of V in flight per thread, the loads of
// vector i + 1 issued before the partial sum of vector i is reduced).  Each
// warp reduces its partial by shuffles and leaves it in shared memory, with
// no barrier between vectors; the 8 warp partials of a vector are added in
// warp order at the end.  ws[(i * nrhs + q) * chunks + c] as
// k_multi_dot_partial.
constexpr int DW = 16;
constexpr int DOT_VB = 64;  // vectors per shared-memory batch
__global__ void __launch_bounds__(256) k_multi_dot_w(const double* __restrict__ V, int nvec,
                                                     const double* __restrict__ w, long long N, int nrhs,
                                                     double* __restrict__ ws, int selfdot,
                                                     const int* __restrict__ need) {
    __shared__ double red[DOT_VB * 8];
    const int q = blockIdx.y, chunks = gridDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (need && !need[q]) return;  // column q not asked for: nothing written
    const long long lo = (long long)blockIdx.x * DW * 256;
    const double* wq = w + (long long)q * N;
    double wr[DW], v[DW];
#pragma unroll
    for (int u = 0; u < DW; ++u) {
        const long long r = lo + tid + u * 256;
        wr[u] = r < N ? wq[r] : 0.0;
    }
    // selfdot: one more product after the nvec vectors, w with itself
    const int ntot = nvec + (selfdot ? 1 : 0);
    if (nvec > 0) {
        const double* vq = V + (long long)q * N;
#pragma unroll
        for (int u = 0; u < DW; ++u) {
            const long long r = lo + tid + u * 256;
            v[u] = r < N ? vq[r] : 0.0;
        }
    } else {
#pragma unroll
        for (int u = 0; u < DW; ++u) v[u] = wr[u];
    }
    for (int i0 = 0; i0 < ntot; i0 += DOT_VB) {
        const int i1 = min(ntot, i0 + DOT_VB);
        for (int i = i0; i < i1; ++i) {
            double sum = 0.0;
#pragma unroll
            for (int u = 0; u < DW; ++u) sum = fma(v[u], wr[u], sum);
            if (i + 1 < nvec) {
                const double* vq = V + ((long long)(i + 1) * nrhs + q) * N;
#pragma unroll
                for (int u = 0; u < DW; ++u) {
                    const long long r = lo + tid + u * 256;
                    v[u] = r < N ? vq[r] : 0.0;
                }
            } else if (i + 1 == nvec) {
#pragma unroll
                for (int u = 0; u < DW; ++u) v[u] = wr[u];
            }
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) red[(i - i0) * 8 + warp] = sum;
        }
        __syncthreads();
        for (int i = i0 + tid; i < i1; i += 256) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += red[(i - i0) * 8 + k];
            ws[((long long)i * nrhs + q) * chunks + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

static int dot_chunks(long long N) {
    int chunks = 256;
    if (N < 256LL * 1024) chunks = (int)((N + 1023) / 1024);
    return chunks < 1 ? 1 : chunks;
}

cudaError_t multi_dot(const double* V, int nvec, const double* w, long long N, int nrhs, double* ws, double* out,
                      cudaStream_t s) {
    if (nvec <= 0 || nrhs <= 0) return cudaSuccess;
    // the workspace holds 1024 partials per product
    const long long cw = (N + (long long)DW * 256 - 1) / ((long long)DW * 256);
    if (cw <= 1024) {
        k_multi_dot_w<<<dim3((int)cw, nrhs), 256, 0, s>>>(V, nvec, w, N, nrhs, ws, 0, nullptr);
        count_launches(1);
        k_sumsq_final<<<nvec * nrhs, 256, 0, s>>>(ws, (int)cw, out);
        count_launches(1);
        return cudaGetLastError();
    }
    const int chunks = dot_chunks(N);
    k_multi_dot_partial<<<dim3(chunks, nrhs, nvec), 256, 0, s>>>(V, w, N, nrhs, ws);
    count_launches(1);
    k_sumsq_final<<<nvec * nrhs, 256, 0, s>>>(ws, chunks, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t multi_dot_self(const double* V, int nvec, const double* w, long long N, int nrhs, double* ws, double* out,
                           cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    const long long cw = (N + (long long)DW * 256 - 1) / ((long long)DW * 256);
    if (cw <= 1024) {
        k_multi_dot_w<<<dim3((int)cw, nrhs), 256, 0, s>>>(V, nvec, w, N, nrhs, ws, 1, nullptr);
        count_launches(1);
        k_sumsq_final<<<(nvec + 1) * nrhs, 256, 0, s>>>(ws, (int)cw, out);
        count_launches(1);
        return cudaGetLastError();
    }
    cudaError_t e = multi_dot(V, nvec, w, N, nrhs, ws, out, s);
    if (e != cudaSuccess) return e;
    return col_sumsq(w, N, nrhs, ws, out + (size_t)nvec * nrhs, s);
}

// One Gram-Schmidt correction with the squared norm of its result.  Grid
// (G, nrhs); CTA (g, q) takes the 256-row tiles g, g + G, ... of column q,
// thread t row t of each: w[r] += sum_i coef[i, q] V_i[r] in order i = 0, 1,
// ..., accumulating w_new[r]^2 across its tiles; the CTA's sum (shuffles,
// then warps in order) goes to ws[q * G + g].
// need != NULL: column q is skipped unless need[q] (nothing written for it).
__global__ void __launch_bounds__(256) k_gs_upd_norm(double* __restrict__ w, const double* __restrict__ V, int nvec,
                                                     const double* __restrict__ coef, long long N, int nrhs,
                                                     const int* __restrict__ need, double* __restrict__ ws) {
    __shared__ double sc[64];
    __shared__ double red[8];
    const int q = blockIdx.y, G = gridDim.x, g = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (need && !need[q]) return;
    for (int i = tid; i < nvec; i += 256) sc[i] = coef[(size_t)i * nrhs + q];
    __syncthreads();
    double* wq = w + (long long)q * N;
    double acc = 0.0;
    const long long ntile = (N + 255) / 256;
    for (long long t = g; t < ntile; t += G) {
        const long long r = t * 256 + tid;
        const bool ok = r < N;
        if (!ok) break;
        double wn = wq[r];
        const double* vp = V + (long long)q * N + r;
        const long long vs = (long long)nrhs * N;
#pragma unroll 4
        for (int i = 0; i < nvec; ++i) wn = fma(sc[i], vp[i * vs], wn);
        wq[r] = wn;
        acc = fma(wn, wn, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        double sm = 0.0;
        for (int k = 0; k < 8; ++k) sm += red[k];
        ws[(long long)q * G + g] = sm;
    }
}

// CTAs per column of k_gs_upd_norm: a function of N only, so that a column's
// summation order does not depend on how many columns share the call
static int gs_groups(long long N) {
    const long long ntile = (N + 255) / 256;
    return (int)std::max(1LL, std::min(ntile, 304LL));
}

// out[q] = sum of column q's partials (k_sumsq_final), only where need[q]
__global__ void k_final_need(const double* __restrict__ ws, int G, const int* __restrict__ need,
                             double* __restrict__ out) {
    __shared__ double red[32];
    const int q = blockIdx.x;
    if (need && !need[q]) return;
    double sm = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) sm += ws[(long long)q * G + i];
    for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sm;
    __syncthreads();
    if (threadIdx.x < 32) {
        sm = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if (threadIdx.x == 0) out[q] = sm;
    }
}

cudaError_t gs_update_norm(double* w, const double* V, int nvec, const double* coef, long long N, int nrhs,
                           const int* need, double* ws, double* out, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    if (nvec > 64) return cudaErrorInvalidValue;
    const int G = gs_groups(N);
    k_gs_upd_norm<<<dim3(G, nrhs), 256, 0, s>>>(w, V, nvec, coef, N, nrhs, need, ws);
    k_final_need<<<nrhs, 256, 0, s>>>(ws, G, need, out);
    count_launches(2);
    return cudaGetLastError();
}

// need[q] = |w'|^2 < ratio2 |w|^2;  hs[q] = |w'|^2
__global__ void k_gs_need(const double* __restrict__ sq0, const double* __restrict__ sq1, double ratio2,
                          int* __restrict__ need, double* __restrict__ hs, int nrhs) {
    for (int q = threadIdx.x; q < nrhs; q += blockDim.x) {
        need[q] = sq1[q] < ratio2 * sq0[q] ? 1 : 0;
        hs[q] = sq1[q];
    }
}
// where need[q]: coef = -h2, hacc += h2;  elsewhere coef = 0
__global__ void k_gs_coef_need(const double* __restrict__ h2, const int* __restrict__ need,
                               double* __restrict__ coef, double* __restrict__ hacc, int n, int nrhs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool nd = need[i % nrhs] != 0;
        coef[i] = nd ? -h2[i] : 0.0;
        if (nd) hacc[i] += h2[i];
    }
}

cudaError_t gs_reorth(double* w, const double* V, int nvec, const double* sq0, const double* sq1, double ratio2,
                      double* h2, double* coef, double* hacc, int* need, double* hs, long long N, int nrhs,
                      double* ws, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    k_gs_need<<<1, 32, 0, s>>>(sq0, sq1, ratio2, need, hs, nrhs);
    count_launches(1);
    const long long cw = (N + (long long)DW * 256 - 1) / ((long long)DW * 256);
    if (cw > 1024) return cudaErrorInvalidValue;
    k_multi_dot_w<<<dim3((int)cw, nrhs), 256, 0, s>>>(V, nvec, w, N, nrhs, ws, 0, need);
    count_launches(1);
    k_sumsq_final<<<nvec * nrhs, 256, 0, s>>>(ws, (int)cw, h2);
    count_launches(1);
    k_gs_coef_need<<<(nvec * nrhs + 255) / 256, 256, 0, s>>>(h2, need, coef, hacc, nvec * nrhs, nrhs);
    count_launches(1);
    return gs_update_norm(w, V, nvec, coef, N, nrhs, need, ws, hs, s);
}

__global__ void k_multi_axpy(double* __restrict__ w, const double* __restrict__ V, int nvec,
                             const double* __restrict__ coef, long long N, int nrhs) {
    const long long total = N * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / N);
        double acc = w[t];
        for (int i = 0; i < nvec; ++i) acc += coef[i * nrhs + q] * V[(long long)i * total + t];
        w[t] = acc;
    }
}

cudaError_t multi_axpy(double* w, const double* V, int nvec, const double* coef, long long N, int nrhs,
                       cudaStream_t s) {
    if (nvec <= 0 || nrhs <= 0) return cudaSuccess;
    k_multi_axpy<<<ew_blocks(N * nrhs), 256, 0, s>>>(w, V, nvec, coef, N, nrhs);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_gs_coef(const double* __restrict__ h, double* __restrict__ coef, double* __restrict__ hacc, int n,
                          int first) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = h[i];
        coef[i] = -v;
        hacc[i] = (first ? 0.0 : hacc[i]) + v;
    }
}

cudaError_t gs_coef(const double* h, double* coef, double* hacc, int n, bool first, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gs_coef<<<(n + 255) / 256, 256, 0, s>>>(h, coef, hacc, n, first ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_col_scale(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ sc,
                            long long N, int nrhs) {
    const long long total = N * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        v[t] = w[t] * sc[t / N];
}

cudaError_t col_scale(double* v, const double* w, const double* scale, long long N, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    k_col_scale<<<ew_blocks(N * nrhs), 256, 0, s>>>(v, w, scale, N, nrhs);
    count_launches(1);
    return cudaGetLastError();
}

// explicit instantiations
template cudaError_t gj_inverse<float>(float*, int, int, int*, int*, cudaStream_t);
template cudaError_t gj_inverse<double>(double*, int, int, int*, int*, cudaStream_t);
template cudaError_t gemm_batched<float>(const GemmProb<float>*, int, int, int, cudaStream_t);
template cudaError_t gemm_batched<double>(const GemmProb<double>*, int, int, int, cudaStream_t);
template cudaError_t sweep_batched<float>(const SweepProb<float>*, int, int, int, cudaStream_t);
template cudaError_t sweep_batched<double>(const SweepProb<double>*, int, int, int, cudaStream_t);
template cudaError_t stage_level0<float>(int, int, int, const double*, const double*, const double*, float*,
                                         float*, float*, float*, float*, float*, int*, cudaStream_t);
template cudaError_t stage_level0<double>(int, int, int, const double*, const double*, const double*, double*,
                                          double*, double*, double*, double*, double*, int*, cudaStream_t);

}  // namespace acr
