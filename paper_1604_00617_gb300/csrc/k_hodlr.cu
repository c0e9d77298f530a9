// k_hodlr.cu -- HODLR (hierarchically off-diagonal low-rank) blocks.
//
// Section 3 holds every block of the reduction as an H-matrix with weak
// admissibility, i.e. a HODLR matrix: a balanced binary tree over the rows of
// a b x b block; at tree level l (1..L) every node of size s = b / 2^l has
// two off-diagonal blocks (upper: rows of its first child x columns of its
// second child, lower: the converse) stored as U V^T with a rank set by the
// tolerance; the 2^L diagonal leaves of size leaf = b / 2^L are dense.
//
// Recompression of one off-diagonal block B (s x s), batched over all blocks:
//   Y = B Omega                       (s x k sketch, Omega Gaussian, seeded)
//   Y = Q R                           (Householder QR, in shared memory)
//   R = W S Z^T                       (one-sided Jacobi SVD of the k x k R)
//   U_k = Q W,   V_k = B^T U_k         (so that U_k U_k^T B = U_k V_k^T)
//   rank r = #{ sigma_i > tol * sigma_1 }, capped;  keep U_k[:, :r], V_k[:, :r]
// A node whose rank reaches k - 4 (the sketch cannot certify it) is kept
// dense.  Then B ~= U V^T with error ~ sigma_{r+1}(B).
//
// Apply (solve sweeps): y += M x = leaves * x + sum_nodes U (V^T x), tree
// level by tree level (nodes of one level touch disjoint rows, so the sum
// order is fixed).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "acr_internal.h"

namespace acr {

// ---------------------------------------------------------------- Omega
// Counter-based Gaussian: a 64-bit mix of (seed, index) gives two uniforms,
// Box-Muller turns them into one normal deviate.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

template <class T>
__global__ void k_omega(T* __restrict__ om, long long n, uint64_t seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t h = mix64(seed ^ mix64((uint64_t)i));
        const double u1 = ((h >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
        const double u2 = (double)(mix64(h) >> 11) * (1.0 / 9007199254740992.0);
        om[i] = (T)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
}

template <class T>
cudaError_t hodlr_omega(T* om, long long n, uint64_t seed, cudaStream_t s) {
    k_omega<T><<<304, 256, 0, s>>>(om, n, seed);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- GEMM
// Batched C_p = op(A_p) B_p, uniform M, N, K and leading dimensions; op(A) =
// A (M x K, column-major) or A^T (A stored K x M).  SIMT, 64 x 32 tiles, k
// steps of 32; the next step's operands are loaded into registers while the
// current one is multiplied, so one memory latency is paid per step.
template <class T, bool TA>
__global__ void __launch_bounds__(256)
k_gemm_gen(const T* const* __restrict__ Ap, const T* const* __restrict__ Bp, T* const* __restrict__ Cp, int M, int N,
           int K, int lda, int ldb, int ldc) {
    constexpr int BM = 64, BN = 32, BK = 32, TM = 4, TN = 2, RY = BM / TM;
    constexpr int NA = BM * BK / 256, NB = BK * BN / 256;  // loads per thread per step
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const T* A = Ap[blockIdx.y];
    const T* B = Bp[blockIdx.y];
    T* C = Cp[blockIdx.y];
    const int tiles_m = (M + BM - 1) / BM;
    const int row0 = (blockIdx.x % tiles_m) * BM, col0 = (blockIdx.x / tiles_m) * BN;
    const int tid = threadIdx.x, ty = tid % RY, tx = tid / RY;
    T ra[NA], rb[NB];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int i = tid + u * 256;
            int r, k;
            if (TA) { k = i % BK; r = i / BK; } else { r = i % BM; k = i / BM; }
            const int gr = row0 + r, gk = k0 + k;
            ra[u] = (gr < M && gk < K) ? (TA ? A[gk + (size_t)gr * lda] : A[gr + (size_t)gk * lda]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int i = tid + u * 256;
            const int k = i % BK, c = i / BK;
            const int gk = k0 + k, gc = col0 + c;
            rb[u] = (gk < K && gc < N) ? B[gk + (size_t)gc * ldb] : T(0);
        }
    };
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int i = tid + u * 256;
            int r, k;
            if (TA) { k = i % BK; r = i / BK; } else { r = i % BM; k = i / BM; }
            As[k][r] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int i = tid + u * 256;
            Bs[i % BK][i / BK] = rb[u];
        }
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T af[TM], bf[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) af[i] = As[k][ty + i * RY];
#pragma unroll
            for (int j = 0; j < TN; ++j) bf[j] = Bs[k][tx + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int c = col0 + tx + j * (BN / TN);
        if (c >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = row0 + ty + i * RY;
            if (r < M) C[r + (size_t)c * ldc] = acc[i][j];
        }
    }
}

// Thin batched product for the sketch widths (FP32, N <= 32): one thread owns
// TM rows of C (rows t, t + RT, ...) and all NP >= N of its columns.  Its
// entries of op(A) come straight from global memory -- for op(A) = A a warp
// reads 32 consecutive rows of one column, for op(A) = A^T each thread reads
// runs of KU consecutive k of its own column, as float4 when aligned -- and
// B (K x N) is staged once per CTA in shared memory and read back as 16-byte
// broadcasts (chunks of 4 columns, the chunk index XOR-ed with k so that the
// staging stores spread over the banks).  Every k costs one shared load per
// 4 x TM FMAs.  For small M the CTA's threads split K into KS = 128 / RT
// ranges whose partial sums are added in range order.
constexpr int THIN_NT = 128, THIN_TM = 2, THIN_KU = 16;

template <int NP>
__device__ __forceinline__ int thin_bs(int k, int c) {
    return k * NP + ((((c >> 2) ^ k) & (NP / 4 - 1)) << 2) + (c & 3);
}

template <bool TA, int NP>
__global__ void __launch_bounds__(THIN_NT)
k_gemm_thin(const float* const* __restrict__ Ap, const float* const* __restrict__ Bp, float* const* __restrict__ Cp,
            int M, int N, int K, int lda, int ldb, int ldc, int RT) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TM = THIN_TM, KU = THIN_KU;
    const int KP = (K + 7) & ~7;                      // staged rows of B (zero beyond K)
    float* Bs = reinterpret_cast<float*>(smem_raw);  // KP x NP, swizzled
    float* red = Bs + (size_t)KP * NP;               // (KS - 1) x NP x (RT * TM) partial sums
    const float* A = Ap[blockIdx.y];
    const float* B = Bp[blockIdx.y];
    float* C = Cp[blockIdx.y];
    const int tid = threadIdx.x, KS = THIN_NT / RT, g = tid / RT, t = tid % RT;
    const int R0 = blockIdx.x * RT * TM;
    // stage B: a warp covers 8 consecutive k of 4 consecutive columns
    for (int i = tid; i < KP * NP; i += THIN_NT) {
        const int c = (i >> 3) % NP, k = ((i >> 3) / NP) * 8 + (i & 7);
        Bs[thin_bs<NP>(k, c)] = (k < K && c < N) ? B[k + (size_t)c * ldb] : 0.f;
    }
    __syncthreads();
    const int kper = (((K + KS - 1) / KS) + KU - 1) / KU * KU;
    const int kb = min(K, g * kper), ke = min(K, kb + kper);
    int row[TM];
    bool live[TM];
#pragma unroll
    for (int j = 0; j < TM; ++j) {
        row[j] = R0 + t + j * RT;
        live[j] = row[j] < M;
    }
    const bool vec = TA && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && ((lda & 3) == 0);
    float acc[TM][NP];
#pragma unroll
    for (int j = 0; j < TM; ++j)
#pragma unroll
        for (int c = 0; c < NP; ++c) acc[j][c] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += KU) {
        float a[TM][KU];
        if (TA) {
#pragma unroll
            for (int j = 0; j < TM; ++j) {
                const float* col = A + (size_t)(live[j] ? row[j] : 0) * lda + k0;
                if (vec && live[j] && k0 + KU <= ke) {
#pragma unroll
                    for (int v = 0; v < KU / 4; ++v) {
                        const float4 x = reinterpret_cast<const float4*>(col)[v];
                        a[j][4 * v] = x.x;
                        a[j][4 * v + 1] = x.y;
                        a[j][4 * v + 2] = x.z;
                        a[j][4 * v + 3] = x.w;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < KU; ++u) a[j][u] = (live[j] && k0 + u < ke) ? col[u] : 0.f;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < KU; ++u)
#pragma unroll
                for (int j = 0; j < TM; ++j)
                    a[j][u] = (live[j] && k0 + u < ke) ? A[row[j] + (size_t)(k0 + u) * lda] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int k = k0 + u;
            if (k >= ke) break;
#pragma unroll
            for (int cc = 0; cc < NP / 4; ++cc) {
                const float4 bv = *reinterpret_cast<const float4*>(Bs + k * NP + (((cc ^ k) & (NP / 4 - 1)) << 2));
#pragma unroll
                for (int j = 0; j < TM; ++j) {
                    acc[j][4 * cc] = fmaf(a[j][u], bv.x, acc[j][4 * cc]);
                    acc[j][4 * cc + 1] = fmaf(a[j][u], bv.y, acc[j][4 * cc + 1]);
                    acc[j][4 * cc + 2] = fmaf(a[j][u], bv.z, acc[j][4 * cc + 2]);
                    acc[j][4 * cc + 3] = fmaf(a[j][u], bv.w, acc[j][4 * cc + 3]);
                }
            }
        }
    }
    if (KS > 1) {
        const int RR = RT * TM;
        if (g > 0)
#pragma unroll
            for (int j = 0; j < TM; ++j)
#pragma unroll
                for (int c = 0; c < NP; ++c) red[((size_t)(g - 1) * NP + c) * RR + t + j * RT] = acc[j][c];
        __syncthreads();
        if (g == 0)
            for (int gg = 1; gg < KS; ++gg)
#pragma unroll
                for (int j = 0; j < TM; ++j)
#pragma unroll
                    for (int c = 0; c < NP; ++c) acc[j][c] += red[((size_t)(gg - 1) * NP + c) * RR + t + j * RT];
    }
    if (g == 0)
#pragma unroll
        for (int j = 0; j < TM; ++j)
            if (live[j])
#pragma unroll
                for (int c = 0; c < NP; ++c)
                    if (c < N) C[row[j] + (size_t)c * ldc] = acc[j][c];
}

// launches k_gemm_thin when it applies (FP32, N <= 32, B fits in shared
// memory); returns false otherwise
static bool gemm_thin(const float* const* A, const float* const* B, float* const* C, int nprob, int M, int N, int K,
                      int lda, int ldb, int ldc, bool transA, cudaStream_t s) {
    if (N > 32 || M < 1 || K < 1) return false;
    int RT = 32;
    while (RT < THIN_NT && RT * THIN_TM < M) RT *= 2;
    const int KS = THIN_NT / RT, NP = N <= 16 ? 16 : 32;
    const size_t sm = ((size_t)((K + 7) & ~7) * NP + (size_t)(KS - 1) * NP * RT * THIN_TM) * sizeof(float);
    if (sm > 160 * 1024) return false;
    const void* fn = transA ? (NP == 16 ? (const void*)k_gemm_thin<true, 16> : (const void*)k_gemm_thin<true, 32>)
                            : (NP == 16 ? (const void*)k_gemm_thin<false, 16> : (const void*)k_gemm_thin<false, 32>);
    if (sm > 48 * 1024) ensure_smem(fn, sm);
    const int gx = (M + RT * THIN_TM - 1) / (RT * THIN_TM);
    int done = 0;
    while (done < nprob) {  // grid.y is limited to 65535
        const int cnt = std::min(nprob - done, 65535);
        dim3 g(gx, cnt);
        if (transA) {
            if (NP == 16)
                k_gemm_thin<true, 16><<<g, THIN_NT, sm, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc, RT);
            else
                k_gemm_thin<true, 32><<<g, THIN_NT, sm, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc, RT);
        } else {
            if (NP == 16)
                k_gemm_thin<false, 16><<<g, THIN_NT, sm, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc, RT);
            else
                k_gemm_thin<false, 32><<<g, THIN_NT, sm, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc, RT);
        }
        count_launches(1);
        done += cnt;
    }
    return true;
}

template <class T>
cudaError_t gemm_gen(const T* const* A, const T* const* B, T* const* C, int nprob, int M, int N, int K, int lda,
                     int ldb, int ldc, bool transA, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        if (gemm_thin(A, B, C, nprob, M, N, K, lda, ldb, ldc, transA, s)) return cudaGetLastError();
    }
    const int tiles = ((M + 63) / 64) * ((N + 31) / 32);
    int done = 0;
    while (done < nprob) {  // grid.y is limited to 65535
        const int cnt = std::min(nprob - done, 65535);
        dim3 g(tiles, cnt);
        if (transA)
            k_gemm_gen<T, true><<<g, 256, 0, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc);
        else
            k_gemm_gen<T, false><<<g, 256, 0, s>>>(A + done, B + done, C + done, M, N, K, lda, ldb, ldc);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- node SVD
// One CTA per node: Y (s x k) -> Householder QR -> Jacobi SVD of R -> U_k = Q W
// (columns by decreasing singular value) and the singular values.
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__global__ void __launch_bounds__(256) k_node_svd(const T* __restrict__ Yall, T* __restrict__ Uall,
                                                   T* __restrict__ sig_all, int s, int k, int kz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Y = reinterpret_cast<T*>(smem_raw);   // s x k, column-major (ld s); becomes the reflectors
    T* R = Y + (size_t)s * k;                // k x k (ld k)
    T* tau = R + (size_t)k * k;              // k
    T* sv = tau + k;                         // k
    T* Z = sv + k;                           // s x kz work panel
    int* ord = reinterpret_cast<int*>(Z + (size_t)s * kz);  // k
    __shared__ T red[8];
    __shared__ int s_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t node = blockIdx.x;
    const T* Yg = Yall + node * (size_t)s * k;
    for (int i = tid; i < s * k; i += 256) Y[i] = Yg[i];
    __syncthreads();
    // ---- Householder QR (LAPACK convention: H = I - tau v v^T, v[0] = 1) ----
    for (int j = 0; j < k; ++j) {
        T* col = Y + (size_t)j * s;
        // ||x[1:]||^2
        T part = T(0);
        for (int r = j + 1 + tid; r < s; r += 256) part += col[r] * col[r];
        part = warp_sum(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            T xn2 = T(0);
            for (int w = 0; w < 8; ++w) xn2 += red[w];
            const T alpha = col[j];
            if (xn2 == T(0)) {
                tau[j] = T(0);
                R[j + j * k] = alpha;
                red[0] = T(0);  // scale for v
                s_flag = 0;
            } else {
                T beta = sqrt(alpha * alpha + xn2);
                if (alpha > T(0)) beta = -beta;
                tau[j] = (beta - alpha) / beta;
                R[j + j * k] = beta;
                red[0] = T(1) / (alpha - beta);
                s_flag = 1;
            }
        }
        __syncthreads();
        const T scl = red[0];
        const bool active = s_flag != 0;
        if (active)
            for (int r = j + 1 + tid; r < s; r += 256) col[r] *= scl;
        __syncthreads();
        if (tid == 0) col[j] = T(1);
        __syncthreads();
        // apply H_j to columns j+1..k-1: one warp per column
        const T tj = tau[j];
        for (int c = j + 1 + warp; c < k; c += 8) {
            T* cc = Y + (size_t)c * s;
            T d = T(0);
            for (int r = j + lane; r < s; r += 32) d += col[r] * cc[r];
            d = warp_sum(d) * tj;
            for (int r = j + lane; r < s; r += 32) cc[r] -= d * col[r];
        }
        __syncthreads();
    }
    // R: upper triangle (row j of column c > j is Y[j, c] after the sweep)
    for (int i = tid; i < k * k; i += 256) {
        const int r = i % k, c = i / k;
        if (r < c) R[r + c * k] = Y[r + (size_t)c * s];
        else if (r > c) R[r + c * k] = T(0);
    }
    __syncthreads();
    // ---- one-sided Jacobi on the columns of R (round-robin pairs) -----------
    // Pairs of columns that are both negligible next to ||R||_F (below the
    // precision of the data) are left alone: they cannot change the ranks.
    const T eps = sizeof(T) == 8 ? T(4e-15) : T(4e-7);
    {
        T part = T(0);
        for (int i = tid; i < k * k; i += 256) part += R[i] * R[i];
        part = warp_sum(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            T f = T(0);
            for (int w = 0; w < 8; ++w) f += red[w];
            red[0] = f;
        }
        __syncthreads();
    }
    const T negl = red[0] * (sizeof(T) == 8 ? T(1e-28) : T(1e-13));
    __syncthreads();
    // One warp runs the sweeps with R in registers: lane c holds column c.
    // Round rnd of the round-robin schedule pairs column k-1 with rnd and
    // rnd+q with rnd-q (mod k-1), q = 1 .. k/2-1; a lane exchanges its column
    // with its partner by shuffles, and both lanes of a pair compute the same
    // norms, inner product and rotation, so no barrier is needed.
    if (k <= 32) {
    if (warp == 0) {
        constexpr unsigned FULL = 0xffffffffu;
        T col[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) col[r] = (lane < k && r < k) ? R[r + lane * k] : T(0);
        T nrm = T(0);
#pragma unroll
        for (int r = 0; r < 32; ++r) nrm = fma(col[r], col[r], nrm);
        const int km1 = k - 1;
        for (int sweep = 0; sweep < 12; ++sweep) {
            bool rot = false;
            for (int rnd = 0; rnd < km1; ++rnd) {
                int partner = lane;
                bool is_a = false;
                if (lane < k) {
                    if (lane == km1) {
                        partner = rnd;
                        is_a = true;
                    } else if (lane == rnd) {
                        partner = km1;
                    } else {
                        partner = ((2 * rnd - lane) % km1 + km1) % km1;
                        const int d = ((lane - rnd) % km1 + km1) % km1;
                        is_a = d >= 1 && d <= k / 2 - 1;
                    }
                }
                T pc[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) pc[r] = __shfl_sync(FULL, col[r], partner);
                const T pn = __shfl_sync(FULL, nrm, partner);
                T ga = T(0);
#pragma unroll
                for (int r = 0; r < 32; ++r) ga = fma(col[r], pc[r], ga);
                const T al = is_a ? nrm : pn, be = is_a ? pn : nrm;
                if (partner != lane && al + be > negl && jacobi_needs(al, be, ga, eps)) {
                    const T zeta = (be - al) / (T(2) * ga);
                    const T t = jacobi_tan(zeta);
                    const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
                    T n2 = T(0);
                    if (is_a) {
#pragma unroll
                        for (int r = 0; r < 32; ++r) {
                            col[r] = c * col[r] - sn * pc[r];
                            n2 = fma(col[r], col[r], n2);
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < 32; ++r) {
                            col[r] = sn * pc[r] + c * col[r];
                            n2 = fma(col[r], col[r], n2);
                        }
                    }
                    nrm = n2;
                    rot = true;
                }
            }
            if (!__any_sync(FULL, rot)) break;
        }
        if (lane < k)
#pragma unroll
            for (int r = 0; r < 32; ++r)
                if (r < k) R[r + lane * k] = col[r];
    }
    __syncthreads();
    } else {
    // wider sketches: the pairs of a round spread over the warps
    for (int sweep = 0; sweep < 12; ++sweep) {
        if (tid == 0) s_flag = 0;
        __syncthreads();
        for (int rnd = 0; rnd < k - 1; ++rnd) {
            for (int q = warp; q < k / 2; q += 8) {
                int a, bcol;
                if (q == 0) { a = k - 1; bcol = rnd; }
                else { a = (rnd + q) % (k - 1); bcol = (rnd - q + (k - 1)) % (k - 1); }
                T* ca = R + a * k;
                T* cb = R + bcol * k;
                T al = T(0), be = T(0), ga = T(0);
                for (int r = lane; r < k; r += 32) {
                    const T x = ca[r], y = cb[r];
                    al += x * x; be += y * y; ga += x * y;
                }
                al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
                if (al + be > negl && jacobi_needs(al, be, ga, eps)) {
                    const T zeta = (be - al) / (T(2) * ga);
                    const T t = jacobi_tan(zeta);
                    const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
                    for (int r = lane; r < k; r += 32) {
                        const T x = ca[r], y = cb[r];
                        ca[r] = c * x - sn * y;
                        cb[r] = sn * x + c * y;
                    }
                    if (lane == 0) s_flag = 1;
                }
            }
            __syncthreads();
        }
        // every thread reads the flag before thread 0 may reset it for the
        // next sweep, so all threads leave the loop on the same sweep
        const bool converged = !s_flag;
        __syncthreads();
        if (converged) break;
    }
    }
    // singular values and their order (decreasing, ties by index)
    for (int c = warp; c < k; c += 8) {
        T n2 = T(0);
        for (int r = lane; r < k; r += 32) n2 += R[r + c * k] * R[r + c * k];
        n2 = warp_sum(n2);
        if (lane == 0) sv[c] = sqrt(n2);
    }
    __syncthreads();
    for (int c = tid; c < k; c += 256) {  // total order (NaN lowest, ties by index): a permutation
        const T vc = isnan(sv[c]) ? T(-1) : sv[c];
        int pos = 0;
        for (int j = 0; j < k; ++j) {
            const T vj = isnan(sv[j]) ? T(-1) : sv[j];
            pos += (vj > vc) || (vj == vc && j < c);
        }
        ord[pos] = c;
    }
    __syncthreads();
    T* sg = sig_all + node * k;
    for (int i = tid; i < k; i += 256) sg[i] = sv[ord[i]];
    // ---- U_k = Q [W; 0], W = R J normalised, in panels of kz columns --------
    T* Ug = Uall + node * (size_t)s * k;
    for (int c0 = 0; c0 < k; c0 += kz) {
        const int nc = std::min(kz, k - c0);
        for (int i = tid; i < s * nc; i += 256) {
            const int r = i % s, c = i / s;
            const int src = ord[c0 + c];
            const T nv = sv[src];
            Z[r + (size_t)c * s] = (r < k && nv > T(0)) ? R[r + src * k] / nv : T(0);
        }
        __syncthreads();
        for (int j = k - 1; j >= 0; --j) {
            const T* v = Y + (size_t)j * s;
            const T tj = tau[j];
            if (tj == T(0)) continue;
            for (int c = warp; c < nc; c += 8) {
                T* zc = Z + (size_t)c * s;
                T d = T(0);
                for (int r = j + lane; r < s; r += 32) d += v[r] * zc[r];
                d = warp_sum(d) * tj;
                for (int r = j + lane; r < s; r += 32) zc[r] -= d * v[r];
            }
            __syncthreads();
        }
        for (int i = tid; i < s * nc; i += 256) {
            const int r = i % s, c = i / s;
            Ug[r + (size_t)(c0 + c) * s] = Z[r + (size_t)c * s];
        }
        __syncthreads();
    }
}

// Small nodes (s <= 128 rows, k <= 16 sketch columns): one warp per node, the
// same steps as k_node_svd -- Householder QR of Y, one-sided Jacobi on the
// columns of R (lane c holds column c), U = Q [W; 0] with W the normalised
// rotated columns, singular values in decreasing order (ties by index) --
// with the node's panels in the warp's own slice of shared memory, so that
// no step waits for the other warps of the CTA.
template <class T>
__global__ void __launch_bounds__(128)
k_node_svd_w(const T* __restrict__ Yall, T* __restrict__ Uall, T* __restrict__ sig_all, int nnodes, int s, int k) {
    constexpr int KK = 16;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t node = (size_t)blockIdx.x * 4 + warp;
    if (node >= (size_t)nnodes) return;
    const size_t per = 2 * (size_t)s * k + (size_t)k * k + k;
    T* Y = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per;  // s x k: the panel, then the reflectors
    T* Z = Y + (size_t)s * k;                                     // s x k: [W; 0], then U (unsorted)
    T* R = Z + (size_t)s * k;                                     // k x k
    T* tau = R + (size_t)k * k;                                   // k
    const T* Yg = Yall + node * (size_t)s * k;
    for (int i0 = lane; i0 < s * k; i0 += 8 * 32) {  // 8 loads in flight per lane
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (i0 + u * 32 < s * k) ? Yg[i0 + u * 32] : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u * 32 < s * k) Y[i0 + u * 32] = v[u];
    }
    __syncwarp();
    // ---- Householder QR (H = I - tau v v^T, v[j] = 1) ----
    for (int j = 0; j < k; ++j) {
        T* col = Y + (size_t)j * s;
        T part = T(0);
        for (int r = j + 1 + lane; r < s; r += 32) part += col[r] * col[r];
        const T xn2 = warp_sum(part);
        const T alpha = col[j];
        T tj, rjj, scl;
        if (xn2 == T(0)) {
            tj = T(0); rjj = alpha; scl = T(0);
        } else {
            T beta = sqrt(alpha * alpha + xn2);
            if (alpha > T(0)) beta = -beta;
            tj = (beta - alpha) / beta; rjj = beta; scl = T(1) / (alpha - beta);
        }
        __syncwarp();
        if (xn2 != T(0))
            for (int r = j + 1 + lane; r < s; r += 32) col[r] *= scl;
        if (lane == 0) { tau[j] = tj; R[j + j * k] = rjj; col[j] = T(1); }
        __syncwarp();
        for (int c = j + 1; c < k; ++c) {
            T* cc = Y + (size_t)c * s;
            T d = T(0);
            for (int r = j + lane; r < s; r += 32) d += col[r] * cc[r];
            d = warp_sum(d) * tj;
            for (int r = j + lane; r < s; r += 32) cc[r] -= d * col[r];
        }
        __syncwarp();
    }
    for (int i = lane; i < k * k; i += 32) {
        const int r = i % k, c = i / k;
        if (r < c) R[i] = Y[(size_t)c * s + r];
        else if (r > c) R[i] = T(0);
    }
    __syncwarp();
    // ---- one-sided Jacobi on R's columns, lane c holds column c ----
    const T eps = sizeof(T) == 8 ? T(4e-15) : T(4e-7);
    T cl[KK];
#pragma unroll
    for (int r = 0; r < KK; ++r) cl[r] = (lane < k && r < k) ? R[r + lane * k] : T(0);
    T nrm = T(0);
#pragma unroll
    for (int r = 0; r < KK; ++r) nrm = fma(cl[r], cl[r], nrm);
    const T negl = warp_sum(nrm) * (sizeof(T) == 8 ? T(1e-28) : T(1e-13));
    const int km1 = k - 1;
    for (int sweep = 0; sweep < 12; ++sweep) {
        bool rot = false;
        for (int rnd = 0; rnd < km1; ++rnd) {
            int partner = lane;
            bool is_a = false;
            if (lane < k) {
                if (lane == km1) { partner = rnd; is_a = true; }
                else if (lane == rnd) { partner = km1; }
                else {
                    partner = ((2 * rnd - lane) % km1 + km1) % km1;
                    const int d = ((lane - rnd) % km1 + km1) % km1;
                    is_a = d >= 1 && d <= k / 2 - 1;
                }
            }
            T pc[KK];
#pragma unroll
            for (int r = 0; r < KK; ++r) pc[r] = __shfl_sync(FULL, cl[r], partner);
            const T pn = __shfl_sync(FULL, nrm, partner);
            T ga = T(0);
#pragma unroll
            for (int r = 0; r < KK; ++r) ga = fma(cl[r], pc[r], ga);
            const T al = is_a ? nrm : pn, be = is_a ? pn : nrm;
            if (partner != lane && al + be > negl && jacobi_needs(al, be, ga, eps)) {
                const T zeta = (be - al) / (T(2) * ga);
                const T t = jacobi_tan(zeta);
                const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
                T n2 = T(0);
                if (is_a) {
#pragma unroll
                    for (int r = 0; r < KK; ++r) { cl[r] = c * cl[r] - sn * pc[r]; n2 = fma(cl[r], cl[r], n2); }
                } else {
#pragma unroll
                    for (int r = 0; r < KK; ++r) { cl[r] = sn * pc[r] + c * cl[r]; n2 = fma(cl[r], cl[r], n2); }
                }
                nrm = n2;
                rot = true;
            }
        }
        if (!__any_sync(FULL, rot)) break;
    }
    // ---- singular values, their order, W = R J / sigma ----
    const T sv = sqrt(nrm);
    const T key = isnan(sv) ? T(-1) : sv;
    int pos = 0;
#pragma unroll
    for (int j = 0; j < KK; ++j) {
        const T kj = __shfl_sync(FULL, key, j);
        if (j < k) pos += (kj > key) || (kj == key && j < lane);
    }
    for (int i = lane; i < s * k; i += 32) Z[i] = T(0);
    __syncwarp();
    if (lane < k) {
#pragma unroll
        for (int r = 0; r < KK; ++r)
            if (r < k) Z[(size_t)lane * s + r] = sv > T(0) ? cl[r] / sv : T(0);
    }
    __syncwarp();
    // ---- U = Q [W; 0], reflectors in reverse order ----
    for (int j = k - 1; j >= 0; --j) {
        const T tj = tau[j];
        if (tj == T(0)) continue;
        const T* v = Y + (size_t)j * s;
        for (int c = 0; c < k; ++c) {
            T* zc = Z + (size_t)c * s;
            T d = T(0);
            for (int r = j + lane; r < s; r += 32) d += v[r] * zc[r];
            d = warp_sum(d) * tj;
            for (int r = j + lane; r < s; r += 32) zc[r] -= d * v[r];
        }
        __syncwarp();
    }
    T* Ug = Uall + node * (size_t)s * k;
    T* sg = sig_all + node * k;
    for (int c = 0; c < k; ++c) {
        const int p = __shfl_sync(FULL, pos, c);
        for (int r = lane; r < s; r += 32) Ug[r + (size_t)p * s] = Z[r + (size_t)c * s];
    }
    if (lane < k) sg[pos] = sv;
}

template <class T>
size_t node_svd_smem(int s, int k, int kz) {
    return ((size_t)s * k + (size_t)k * k + 2 * (size_t)k + (size_t)s * kz) * sizeof(T) + (size_t)k * sizeof(int);
}

template <class T>
int node_svd_kz(int s, int k) {  // widest work panel that fits in 200 KB
    for (int kz = k; kz >= std::min(8, k); kz /= 2)
        if (node_svd_smem<T>(s, k, kz) <= 200 * 1024) return kz;
    return 0;
}

template <class T>
cudaError_t node_svd(const T* Y, T* U, T* sig, int nnodes, int s, int k, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    if (s <= 128 && k <= 16) {  // one warp per node, four per CTA
        const size_t sm = 4 * (2 * (size_t)s * k + (size_t)k * k + k) * sizeof(T);
        ensure_smem((const void*)k_node_svd_w<T>, sm);
        k_node_svd_w<T><<<(nnodes + 3) / 4, 128, sm, st>>>(Y, U, sig, nnodes, s, k);
        count_launches(1);
        return cudaGetLastError();
    }
    const int kz = node_svd_kz<T>(s, k);
    if (kz == 0) return cudaErrorInvalidValue;
    const size_t sm = node_svd_smem<T>(s, k, kz);
    ensure_smem((const void*)k_node_svd<T>, sm);
    int done = 0;
    while (done < nnodes) {
        const int cnt = std::min(nnodes - done, 1 << 30);
        k_node_svd<T><<<cnt, 256, sm, st>>>(Y + (size_t)done * s * k, U + (size_t)done * s * k, sig + (size_t)done * k,
                                             s, k, kz);
        count_launches(1);
        done += cnt;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- packing
// node i: rank r = meta[i].rank (-1: dense), destination offset meta[i].off;
// U_k, V_k (s x k) or the dense block (src pointer, ld b); rank -2: packed by
// another launch.

template <class T>
__global__ void k_pack_nodes(const HNode* __restrict__ meta, int node0, const T* __restrict__ Uk,
                             const T* __restrict__ Vk, const T* const* __restrict__ src, int s, int k, int b,
                             T* __restrict__ pool) {
    const int i = blockIdx.x;
    const HNode m = meta[node0 + i];
    if (m.rank == -2) return;  // packed by another launch
    T* dst = pool + m.off;
    if (m.rank < 0) {
        const T* B = src[i];
        for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
            const int r = t % s, c = t / s;
            dst[t] = B[r + (size_t)c * b];
        }
    } else {
        // U column-major (s x rank); V stored transposed (rank x s, i.e. the
        // rank values of one row contiguous) for the V^T x products
        const int rk = m.rank, n = s * rk;
        const T* u = Uk + (size_t)i * s * k;
        const T* v = Vk + (size_t)i * s * k;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            dst[t] = u[t];
            const int ii = t % rk, j = t / rk;
            dst[n + t] = v[j + (size_t)ii * s];
        }
    }
}

template <class T>
cudaError_t pack_nodes(const HNode* meta, int node0, int nnodes, const T* Uk, const T* Vk, const T* const* src,
                       int s, int k, int b, T* pool, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    k_pack_nodes<T><<<nnodes, 256, 0, st>>>(meta, node0, Uk, Vk, src, s, k, b, pool);
    count_launches(1);
    return cudaGetLastError();
}

// leaves: block g's 2^L diagonal leaf x leaf blocks, contiguous
template <class T>
__global__ void k_pack_leaves(const T* const* __restrict__ blocks, const long long* __restrict__ leaf_off, int b,
                              int leaf, T* __restrict__ pool) {
    const int g = blockIdx.y, li = blockIdx.x;
    const T* B = blocks[g];
    T* dst = pool + leaf_off[g] + (size_t)li * leaf * leaf;
    const int o = li * leaf;
    for (int t = threadIdx.x; t < leaf * leaf; t += blockDim.x) {
        const int r = t % leaf, c = t / leaf;
        dst[t] = B[(o + r) + (size_t)(o + c) * b];
    }
}

template <class T>
cudaError_t pack_leaves(const T* const* blocks, const long long* leaf_off, int nblocks, int b, int leaf, T* pool,
                        cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    dim3 g(b / leaf, nblocks);
    k_pack_leaves<T><<<g, 256, 0, st>>>(blocks, leaf_off, b, leaf, pool);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- apply
// y = cin + alpha * sum_t M_t x_t for compressed M_t, in two passes:
//   (A) one CTA per (problem, term, low-rank node): t_node = V^T x[cols],
//       V stored transposed so a warp reads the rank values of a row at once;
//   (B) one CTA per (problem, row tile): leaves, then per tree level the node
//       whose rows contain the tile (U t_node, or the dense node times x).
// Every output element is summed in a fixed order (leaf, level 1..L).
template <class T>
__device__ __forceinline__ T xval(const HSweepProb<T>& P, int term, int r, int q) {
    const size_t o = r + (size_t)q * P.ldx;
    if (term == 0 && P.sx[0]) {
        T v = P.sx[0][r] * P.x[0][o];
        if (P.x[1]) v += P.sx[1][r] * P.x[1][o];
        return v;
    }
    return P.x[term][o];
}

// Programmatic dependent launch: the sweep's kernels are launched so that a
// kernel's CTAs may start while its predecessor drains; every kernel reads
// only static data (descriptors, node tables, the factor pool) before this
// wait, and reads or writes the level vectors only after it, when the
// predecessor's writes are complete and visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Pass A: t = V^T x for one low-rank node per CTA.  x[cols] is staged in
// shared memory (coalesced); lane = g * rp + i handles rank index i (rp: rank
// rounded up to a power of two, <= 32) for rows j = g, g + G, ... of its
// warp's slice (G = 32 / rp), so small ranks still keep every lane busy.
// Partial sums are combined across g by shuffles, across warps in shared
// memory, in a fixed order.
template <class T, int NR>
__global__ void __launch_bounds__(256)
k_hnode_t(const HSweepProb<T>* __restrict__ probs, const HTask* __restrict__ tasks, const int* __restrict__ alist,
          const HNode* __restrict__ nodes, const T* __restrict__ pool, int b, int nrhs, T* __restrict__ tbuf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);          // s x NR
    T* red = xs + (size_t)(b / 2) * NR;               // 8 warps x 64 ranks x NR
    const HTask tk = tasks[alist[blockIdx.x]];
    const HNode hn = nodes[tk.node];
    const int rk = hn.rank;
    const HSweepProb<T>& P = probs[tk.prob];
    const int s = b >> tk.level, c0 = (tk.ni ^ 1) * s;
    const T* Vt = pool + hn.off + (size_t)s * rk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rlo = rk < 32 ? rk : 32;
    int rp = 1;
    while (rp < rlo) rp <<= 1;
    const int G = 32 / rp, g = lane / rp, i0 = lane % rp;
    const int slice = (s + 7) / 8, j0 = warp * slice, j1 = min(s, j0 + slice);
    pdl_wait();
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = min(NR, nrhs - q0);
        __syncthreads();
        for (int i0 = tid; i0 < s * NR; i0 += 8 * 256) {  // 8 loads in flight per thread
            T xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * 256, c = i % s, q = i / s;
                xv[u] = (i < s * NR && q < nq) ? xval(P, tk.term, c0 + c, q0 + q) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * 256;
                if (i < s * NR) xs[(i % s) * NR + i / s] = xv[u];
            }
        }
        __syncthreads();
        for (int ib = 0; ib < rk; ib += 32) {  // rank indices ib + i0 (two passes when rk > 32)
            const int ii = ib + i0;
            const bool live = i0 < rp && ii < rk;
            T acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = T(0);
            if (live) {
#pragma unroll 4
                for (int j = j0 + g; j < j1; j += G) {
                    const T v = Vt[ii + (size_t)j * rk];
#pragma unroll
                    for (int q = 0; q < NR; ++q) acc[q] = fma(v, xs[j * NR + q], acc[q]);
                }
            }
            for (int o = rp; o < 32; o <<= 1)
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (g == 0 && live)
#pragma unroll
                for (int q = 0; q < NR; ++q) red[((size_t)warp * 64 + ii) * NR + q] = acc[q];
        }
        __syncthreads();
        for (int i = tid; i < rk * NR; i += 256) {
            const int ii = i % rk, q = i / rk;
            if (q < nq) {
                T sum = T(0);
#pragma unroll
                for (int w = 0; w < 8; ++w) sum += red[((size_t)w * 64 + ii) * NR + q];
                tbuf[tk.toff + ii + (size_t)(q0 + q) * rk] = sum;
            }
        }
    }
}

// Pass A, one CTA per compressed term (problem, term): t_node = V^T x[cols]
// for every low-rank node of the block.  The term's whole x (b x NR) is
// staged once; every node is cut into items of CH rows of V (one tree level
// spans b / CH items), the warps take the items round-robin and write each
// item's partial t (rank x NR) to shared memory, and the partials of a node
// are summed in item order.
template <class T, int NR, int NT>
__global__ void __launch_bounds__(NT)
k_hnodes(const HSweepProb<T>* __restrict__ probs, const int* __restrict__ terms, const HTask* __restrict__ tasks,
         const HNode* __restrict__ nodes, const T* __restrict__ pool, int b, int L, int CH, int nrhs, int rkmax,
         T* __restrict__ tbuf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);    // b x NR
    T* part = xs + (size_t)b * NR;             // items x rkmax x NR
    // the block's node table, read once: rank (<= 0: no product), pool offset,
    // offset of t in tbuf
    __shared__ int s_rk[254];
    __shared__ long long s_off[254], s_toff[254];
    const int e = terms[blockIdx.x];
    const int p = e >> 1, term = e & 1;
    const HSweepProb<T>& P = probs[p];
    const int tb = P.tbase[term];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per_level = b / CH, nitems = L * per_level;
    const int npb = (1 << (L + 1)) - 2;
    constexpr int NW = NT / 32;
    for (int i = tid; i < npb; i += NT) {
        const HTask tk = tasks[tb + i];
        const HNode hn = nodes[tk.node];
        s_toff[i] = tk.toff;
        s_rk[i] = tk.toff >= 0 ? hn.rank : 0;
        s_off[i] = hn.off;
    }
    pdl_wait();
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = min(NR, nrhs - q0);
        __syncthreads();
        for (int i0 = tid; i0 < b * NR; i0 += 8 * NT) {  // 8 loads in flight per thread
            T xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NT, c = i % b, q = i / b;
                xv[u] = (i < b * NR && q < nq) ? xval(P, term, c, q0 + q) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NT;
                if (i < b * NR) xs[(i % b) * NR + i / b] = xv[u];
            }
        }
        __syncthreads();
        for (int it = warp; it < nitems; it += NW) {
            const int l = 1 + it / per_level, u = it % per_level;
            const int sz = b >> l, cpn = sz / CH;  // items per node
            const int ni = u / cpn, cc = u % cpn;
            const int nu = (1 << l) - 2 + ni;
            const int rk = s_rk[nu];
            if (rk <= 0) continue;
            const T* Vt = pool + s_off[nu] + (size_t)sz * rk;  // rank x sz, rank values of a row contiguous
            const int c0 = (ni ^ 1) * sz;
            const int rlo = rk < 32 ? rk : 32;
            int rp = 1;
            while (rp < rlo) rp <<= 1;
            const int G = 32 / rp, g = lane / rp, i0 = lane % rp;
            const int j0 = cc * CH, j1 = j0 + CH;
            for (int ib = 0; ib < rk; ib += 32) {
                const int ii = ib + i0;
                const bool live = i0 < rp && ii < rk;
                T acc[NR];
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[q] = T(0);
                if (live) {
#pragma unroll 8
                    for (int j = j0 + g; j < j1; j += G) {
                        const T v = Vt[ii + (size_t)j * rk];
                        const T* xr = xs + (size_t)(c0 + j) * NR;
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] = fma(v, xr[q], acc[q]);
                    }
                }
                for (int o = rp; o < 32; o <<= 1)
#pragma unroll
                    for (int q = 0; q < NR; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                if (g == 0 && live)
#pragma unroll
                    for (int q = 0; q < NR; ++q) part[((size_t)it * rkmax + ii) * NR + q] = acc[q];
            }
        }
        __syncthreads();
        // node sums in item order: one warp per node, lanes over (rank index, column)
        for (int nu = warp; nu < npb; nu += NW) {
            const int rk = s_rk[nu];
            if (rk <= 0) continue;
            int l = 1;
            while (((1 << (l + 1)) - 2) <= nu) ++l;
            const int ni = nu - ((1 << l) - 2), cpn = (b >> l) / CH;
            const int it0 = (l - 1) * per_level + ni * cpn;
            for (int o = lane; o < rk * nq; o += 32) {
                const int ii = o % rk, q = o / rk;
                T sum = T(0);
                for (int cc = 0; cc < cpn; ++cc) sum += part[((size_t)(it0 + cc) * rkmax + ii) * NR + q];
                tbuf[s_toff[nu] + ii + (size_t)(q0 + q) * rk] = sum;
            }
        }
    }
}

// Pass A for launches with few compressed terms: each term's items (CH rows
// of one node's V, as in k_hnodes) are spread over gridDim.y CTAs, one warp
// per item, the warp staging the CH rows of x its item reads.  Every item's
// partial t (rank x nrhs) is computed exactly as k_hnodes computes it and
// goes to gpart[(((2 p + term) * nitems + it) * rkmax + ii) * nrhs + q]
// (p: the problem's index in the launch); pass B adds a node's items in item
// order when it stages t, as k_hnodes's node sums do, so the results are the
// same bits.
template <class T, int NR>
__global__ void __launch_bounds__(256)
k_hnodes_sp(const HSweepProb<T>* __restrict__ probs, int prob_off, const int* __restrict__ terms,
            const HTask* __restrict__ tasks, const HNode* __restrict__ nodes, const T* __restrict__ pool, int b, int L,
            int CH, int nrhs, int rkmax, T* __restrict__ gpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* xw = reinterpret_cast<T*>(smem_raw) + (size_t)warp * CH * NR;  // this warp's CH x NR
    const int e = terms[blockIdx.x];
    const int p = e >> 1, term = e & 1, ep = 2 * (p - prob_off) + term;
    const HSweepProb<T>& P = probs[p];
    const int tb = P.tbase[term];
    const int per_level = b / CH, nitems = L * per_level;
    const int ipc = (nitems + gridDim.y - 1) / gridDim.y;
    const int it0 = blockIdx.y * ipc, it1 = min(nitems, it0 + ipc);
    pdl_wait();
    for (int it = it0 + warp; it < it1; it += 8) {
        const int l = 1 + it / per_level, u = it % per_level;
        const int sz = b >> l, cpn = sz / CH;
        const int ni = u / cpn, cc = u % cpn;
        const int nu = (1 << l) - 2 + ni;
        const HTask tk = tasks[tb + nu];
        if (tk.toff < 0) continue;
        const HNode hn = nodes[tk.node];
        const int rk = hn.rank;
        if (rk <= 0) continue;
        const T* Vt = pool + hn.off + (size_t)sz * rk;
        const int c0 = (ni ^ 1) * sz;
        const int rlo = rk < 32 ? rk : 32;
        int rp = 1;
        while (rp < rlo) rp <<= 1;
        const int G = 32 / rp, g = lane / rp, i0 = lane % rp;
        const int j0 = cc * CH, j1 = j0 + CH;
        T* gp = gpart + ((size_t)ep * nitems + it) * rkmax * nrhs;
        for (int q0 = 0; q0 < nrhs; q0 += NR) {
            const int nq = min(NR, nrhs - q0);
            __syncwarp();
            for (int i = lane; i < CH * NR; i += 32) {
                const int jr = i % CH, q = i / CH;
                xw[(size_t)jr * NR + q] = q < nq ? xval(P, term, c0 + j0 + jr, q0 + q) : T(0);
            }
            __syncwarp();
            for (int ib = 0; ib < rk; ib += 32) {
                const int ii = ib + i0;
                const bool live = i0 < rp && ii < rk;
                T acc[NR];
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[q] = T(0);
                if (live) {
#pragma unroll 8
                    for (int j = j0 + g; j < j1; j += G) {
                        const T v = Vt[ii + (size_t)j * rk];
                        const T* xr = xw + (size_t)(j - j0) * NR;
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] = fma(v, xr[q], acc[q]);
                    }
                }
                for (int o = rp; o < 32; o <<= 1)
#pragma unroll
                    for (int q = 0; q < NR; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                if (g == 0 && live)
#pragma unroll
                    for (int q = 0; q < NR; ++q)
                        if (q < nq) gp[(size_t)ii * nrhs + q0 + q] = acc[q];
            }
        }
    }
}

// 16-byte vectors of T for the row streams of pass B
template <class T> struct HVec;
template <> struct HVec<float> { using type = float4; static constexpr int V = 4; };
template <> struct HVec<double> { using type = double2; static constexpr int V = 2; };

// Pass B: one CTA per (problem, row tile of RT rows).  For each compressed
// term the tile's operator is a short list of column segments -- its leaf
// (leaf columns), then per tree level the node whose rows hold the tile: U
// (rank columns, input t = V^T x from pass A) or a dense node (s columns,
// input x at the partner columns).  Lanes of warp 0 read the level nodes at
// once, all inputs are staged in one phase, then the rows of every segment
// are streamed with 16-byte loads (column j of the concatenation goes to
// column group j mod KG) and the groups are summed in a fixed order.
// Split (gridDim.z > 1, part != NULL): CTA z takes the z-th of gridDim.z
// equal chunks of each term's concatenated columns and writes raw partial
// sums part[((z * nprob + p) * b + row) * nrhs + q]; k_hrows_reduce adds them
// in z order.
template <class T, int NR, int V>
__global__ void __launch_bounds__(256)
k_hrows(const HSweepProb<T>* __restrict__ probs, const HBlk* __restrict__ blks, const HNode* __restrict__ nodes,
        const HTask* __restrict__ tasks, const T* __restrict__ tbuf, const T* __restrict__ pool, int b, int leaf,
        int L, int nrhs, int RT, T* __restrict__ part, const T* __restrict__ gpart, int gCH, int grk) {
    using VT = typename HVec<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);  // [W][NR], W <= b; reused for the group sums
    __shared__ const T* s_ptr[17];
    __shared__ long long s_src[17];
    __shared__ int s_ld[17], s_cs[18], s_kind[17], s_rk[17];
    const int RG = RT / V, KG = 256 / RG;
    const HSweepProb<T>& P = probs[blockIdx.y];
    const int R0 = blockIdx.x * RT;
    const int tid = threadIdx.x, rg = tid % RG, g = tid / RG;
    const int row = R0 + rg * V;
    const int warp = tid >> 5, lane = tid & 31;
    const int nz = gridDim.z, z = blockIdx.z;
    pdl_wait();
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = min(NR, nrhs - q0);
        // this thread's final outputs (i = tid, tid + 256 < RT * NR): cin early
        T cpre[2] = {T(0), T(0)};
        if (!part && P.cin)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                const int i = tid + k2 * 256, r = i % RT, q = i / RT;
                if (i < RT * NR && q < nq) cpre[k2] = P.cin[R0 + r + (size_t)(q0 + q) * P.ldc];
            }
        T acc[V][NR];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[v][q] = T(0);
        for (int t = 0; t < 2; ++t) {
            if (!P.x[t]) continue;
            if (P.dg[t]) {
                if (g == 0 && z == 0)
#pragma unroll
                    for (int v = 0; v < V; ++v)
#pragma unroll
                        for (int q = 0; q < NR; ++q)
                            if (q < nq) acc[v][q] += P.dg[t][row + v] * P.x[t][row + v + (size_t)(q0 + q) * P.ldx];
                continue;
            }
            if (P.blk[t] < 0) continue;
            __syncthreads();  // xs and the segment table are free
            if (warp == 0) {
                const int li = R0 / leaf;
                // lane 0: the leaf; lane l (1..L): the node of tree level l
                int kind = -1, ld = 0, ncol = 0, rk = 0;
                const T* ptr = nullptr;
                long long src = 0;
                if (lane == 0) {
                    kind = 0;
                    ptr = pool + P.leaf_off[t] + (size_t)li * leaf * leaf + (R0 - li * leaf);
                    ld = leaf;
                    ncol = leaf;
                    src = (long long)li * leaf;
                } else if (lane <= L) {
                    const int l = lane, sz = b >> l, ni = R0 / sz;
                    // both loads issued before either is used
                    const HNode hn = nodes[P.node_base[t] + (1 << l) - 2 + ni];
                    const long long toff = tasks[P.tbase[t] + (1 << l) - 2 + ni].toff;
                    const int r0 = ni * sz;
                    ld = sz;
                    ptr = pool + hn.off + (R0 - r0);
                    if (hn.rank < 0) {
                        kind = 0;
                        ncol = sz;
                        src = (long long)(ni ^ 1) * sz;
                    } else if (hn.rank > 0) {
                        kind = 1;
                        ncol = hn.rank;
                        rk = hn.rank;
                        src = toff;
                    }
                }
                // exclusive prefix of the widths over lanes 0..L, in lane order
                int cs = ncol;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, cs, o);
                    if (lane >= o) cs += y;
                }
                if (lane <= L) {
                    s_ptr[lane] = ptr;
                    s_src[lane] = src;
                    s_ld[lane] = ld;
                    s_kind[lane] = kind;
                    s_rk[lane] = rk;
                    s_cs[lane + 1] = cs;
                }
                if (lane == 0) s_cs[0] = 0;
            }
            __syncthreads();
            // this CTA's columns [J0, J1) of the concatenation
            const int Wall = s_cs[L + 1];
            const int JS = (Wall + nz - 1) / nz;
            const int J0 = min(Wall, z * JS), J1 = min(Wall, J0 + JS);
            const int W = J1 - J0;
            // stage the inputs of those columns: xs[(j - J0) * NR + q]
            for (int i0 = tid; i0 < W * NR; i0 += 4 * 256) {  // 4 loads in flight per thread
                T xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * 256;
                    xv[u] = T(0);
                    if (i < W * NR) {
                        const int j = J0 + i % W, q = i / W;
                        int sg = 0;
                        while (s_cs[sg + 1] <= j) ++sg;
                        const int c = j - s_cs[sg];
                        if (q < nq) {
                            if (s_kind[sg] == 1) {
                                if (gpart) {
                                    // t of the tile's node at level sg: its items' partials, in item order
                                    const int sz = b >> sg, nj = R0 / sz, per_level = b / gCH, cpn = sz / gCH;
                                    const int nitems = L * per_level, it0 = (sg - 1) * per_level + nj * cpn;
                                    const T* gp = gpart + (((size_t)(2 * blockIdx.y + t) * nitems + it0) * grk + c) *
                                                              nrhs + q0 + q;
                                    T v = T(0);
                                    for (int cc = 0; cc < cpn; ++cc) v += gp[(size_t)cc * grk * nrhs];
                                    xv[u] = v;
                                } else {
                                    xv[u] = tbuf[s_src[sg] + c + (size_t)(q0 + q) * s_rk[sg]];
                                }
                            } else {
                                xv[u] = xval(P, t, (int)s_src[sg] + c, q0 + q);
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * 256;
                    if (i < W * NR) xs[(i % W) * NR + i / W] = xv[u];
                }
            }
            __syncthreads();
            for (int sg = 0; sg <= L; ++sg) {
                const int cs = s_cs[sg], ce = min(s_cs[sg + 1], J1);
                const int cb = max(cs, J0);
                if (ce <= cb) continue;
                const T* __restrict__ mp = s_ptr[sg] + rg * V;
                const int ld = s_ld[sg];
                int j = cb + ((g - cb) % KG + KG) % KG;
#pragma unroll 8
                for (; j < ce; j += KG) {
                    const VT mv = *reinterpret_cast<const VT*>(mp + (size_t)(j - cs) * ld);
                    const T* mvp = reinterpret_cast<const T*>(&mv);
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        const T xq = xs[(j - J0) * NR + q];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v][q] = fma(mvp[v], xq, acc[v][q]);
                    }
                }
            }
        }
        __syncthreads();
        T* red = xs;  // [KG][RT][NR]
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int q = 0; q < NR; ++q) red[((size_t)g * RT + rg * V + v) * NR + q] = acc[v][q];
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {
            const int i = tid + k2 * 256;
            const int r = i % RT, q = i / RT;
            if (i < RT * NR && q < nq) {
                T sum = T(0);
                for (int gg = 0; gg < KG; ++gg) sum += red[((size_t)gg * RT + r) * NR + q];
                if (part) {
                    part[(((size_t)z * gridDim.y + blockIdx.y) * b + R0 + r) * nrhs + q0 + q] = sum;
                } else {
                    T o = P.alpha * sum;
                    if (P.cin) o += cpre[k2];
                    P.out[R0 + r + (size_t)(q0 + q) * P.ldo] = o;
                }
            }
        }
    }
}

// Pass B for launches whose tiles are narrow (at most wmax concatenated
// columns): one warp per row tile, independent of the other warps of its
// CTA.  Lanes = RT/V row groups x (32 / (RT/V)) column groups; the warp stages
// its inputs in its own slice of shared memory, streams the rows with 16-byte
// loads, adds the column groups by shuffles and writes the tile.
template <class T, int NR, int V>
__global__ void __launch_bounds__(256, 3)
k_hrows_w(const HSweepProb<T>* __restrict__ probs, const HNode* __restrict__ nodes, const HTask* __restrict__ tasks,
          const T* __restrict__ tbuf, const T* __restrict__ pool, int b, int leaf, int L, int nrhs, int RT,
          int wmax) {
    using VT = typename HVec<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* xs = reinterpret_cast<T*>(smem_raw) + (size_t)warp * wmax * NR;  // this warp's [wmax][NR]
    const int tiles = b / RT;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= tiles) return;
    const HSweepProb<T>& P = probs[blockIdx.y];
    const int R0 = tile * RT;
    const int RG = RT / V, KG = 32 / RG;
    const int rg = lane % RG, g = lane / RG;
    const int row = R0 + rg * V;
    pdl_wait();
    for (int q0 = 0; q0 < nrhs; q0 += NR) {
        const int nq = min(NR, nrhs - q0);
        T acc[V][NR];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[v][q] = T(0);
        for (int t = 0; t < 2; ++t) {
            if (!P.x[t]) continue;
            if (P.dg[t]) {
                if (g == 0)
#pragma unroll
                    for (int v = 0; v < V; ++v)
#pragma unroll
                        for (int q = 0; q < NR; ++q)
                            if (q < nq) acc[v][q] += P.dg[t][row + v] * P.x[t][row + v + (size_t)(q0 + q) * P.ldx];
                continue;
            }
            if (P.blk[t] < 0) continue;
            // segment table in registers of lanes 0..L: lane 0 the leaf, lane l the level-l node
            const int li = R0 / leaf;
            int kind = -1, ld = 0, ncol = 0, rk = 0;
            long long off = 0, src = 0;
            if (lane == 0) {
                kind = 0;
                off = P.leaf_off[t] + (long long)li * leaf * leaf + (R0 - li * leaf);
                ld = leaf;
                ncol = leaf;
                src = (long long)li * leaf;
            } else if (lane <= L) {
                const int l = lane, sz = b >> l, ni = R0 / sz;
                const HNode hn = nodes[P.node_base[t] + (1 << l) - 2 + ni];
                const long long toff = tasks[P.tbase[t] + (1 << l) - 2 + ni].toff;
                ld = sz;
                off = hn.off + (R0 - ni * sz);
                if (hn.rank < 0) {
                    kind = 0;
                    ncol = sz;
                    src = (long long)(ni ^ 1) * sz;
                } else if (hn.rank > 0) {
                    kind = 1;
                    ncol = hn.rank;
                    rk = hn.rank;
                    src = toff;
                }
            }
            int cs = ncol;  // inclusive prefix of the widths
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, cs, o);
                if (lane >= o) cs += y;
            }
            const int W = __shfl_sync(0xffffffffu, cs, L);
            __syncwarp();  // the previous term's reads of xs are done
            // stage: segment sg holds columns [cs_sg - ncol_sg, cs_sg)
            for (int sg = 0; sg <= L; ++sg) {
                const int e1 = __shfl_sync(0xffffffffu, cs, sg);
                const int n1 = __shfl_sync(0xffffffffu, ncol, sg);
                const int k1 = __shfl_sync(0xffffffffu, kind, sg);
                const int r1 = __shfl_sync(0xffffffffu, rk, sg);
                const long long s1 = __shfl_sync(0xffffffffu, src, sg);
                const int c0 = e1 - n1;
                for (int i0 = lane; i0 < n1 * NR; i0 += 8 * 32) {  // 8 loads in flight per lane
                    T xv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + u * 32, c = i % n1, q = i / n1;
                        xv[u] = T(0);
                        if (i < n1 * NR && q < nq)
                            xv[u] = (k1 == 1) ? tbuf[s1 + c + (size_t)(q0 + q) * r1] : xval(P, t, (int)s1 + c, q0 + q);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + u * 32;
                        if (i < n1 * NR) xs[(c0 + i % n1) * NR + i / n1] = xv[u];
                    }
                }
            }
            __syncwarp();
            for (int sg = 0; sg <= L; ++sg) {
                const int e1 = __shfl_sync(0xffffffffu, cs, sg);
                const int n1 = __shfl_sync(0xffffffffu, ncol, sg);
                const int l1 = __shfl_sync(0xffffffffu, ld, sg);
                const long long o1 = __shfl_sync(0xffffffffu, off, sg);
                if (n1 <= 0) continue;
                const int c0 = e1 - n1;
                const T* __restrict__ mp = pool + o1 + rg * V;
#pragma unroll 4
                for (int c = g; c < n1; c += KG) {
                    const VT mv = *reinterpret_cast<const VT*>(mp + (size_t)c * l1);
                    const T* mvp = reinterpret_cast<const T*>(&mv);
                    const T* xr = xs + (size_t)(c0 + c) * NR;
#pragma unroll
                    for (int q = 0; q < NR; ++q)
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v][q] = fma(mvp[v], xr[q], acc[v][q]);
                }
            }
            (void)W;
        }
        // sum the column groups (lanes rg, rg + RG, ...) in a fixed order
        for (int o = RG; o < 32; o <<= 1)
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[v][q] += __shfl_xor_sync(0xffffffffu, acc[v][q], o);
        // the tile's sums through this warp's slice (RT x NR <= wmax x NR), then
        // every lane loads its cin values before storing its outputs
        __syncwarp();
        if (g == 0)
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int q = 0; q < NR; ++q) xs[(rg * V + v) + q * RT] = acc[v][q];
        __syncwarp();
        constexpr int PER = 64 * NR / 32;  // outputs per lane at RT <= 64
        T cv[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int o = lane + u * 32, r = o % RT, q = o / RT;
            cv[u] = (P.cin && o < RT * NR && q < nq) ? P.cin[R0 + r + (size_t)(q0 + q) * P.ldc] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int o = lane + u * 32, r = o % RT, q = o / RT;
            if (o < RT * NR && q < nq) P.out[R0 + r + (size_t)(q0 + q) * P.ldo] = P.alpha * xs[o] + cv[u];
        }
        __syncwarp();
    }
}

// out = cin + alpha * sum_z part[z], fixed summation order.
template <class T>
__global__ void k_hrows_reduce(const HSweepProb<T>* __restrict__ probs, int nprob, int b, int nrhs, int nsplit,
                               const T* __restrict__ part) {
    pdl_wait();
    const long long total = (long long)nprob * b * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t % nrhs);
        const long long pr = t / nrhs;
        const int row = (int)(pr % b), p = (int)(pr / b);
        T sum = T(0);
        for (int zz = 0; zz < nsplit; ++zz) sum += part[(((size_t)zz * nprob + p) * b + row) * nrhs + q];
        const HSweepProb<T>& P = probs[p];
        T o = P.alpha * sum;
        if (P.cin) o += P.cin[row + (size_t)q * P.ldc];
        P.out[row + (size_t)q * P.ldo] = o;
    }
}

// Launch with programmatic stream serialization (the kernel may start while
// the previous kernel on the stream drains; it waits in pdl_wait()).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t sm, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

template <class T>
cudaError_t hsweep(const HSweepProb<T>* probs_all, int prob_off, int nprob, const HTask* tasks, const int* alist,
                   int a_off, int na, const int* terms, int nterms, int rkmax, int wmax, T* tbuf, const HBlk* blks,
                   const HNode* nodes, const T* pool, int b, int leaf, int L, int nrhs, cudaStream_t s) {
    if (nprob <= 0 || nrhs <= 0) return cudaSuccess;
    const int NR = nrhs == 1 ? 1 : (nrhs <= 4 ? 4 : 8);
    // row tile: the largest power of two (<= 64) dividing the leaf, so that a
    // tile lies inside one leaf and inside one node of every tree level
    int RT = 1;
    while (RT < 64 && leaf % (RT * 2) == 0) RT *= 2;
    constexpr int V = HVec<T>::V;
    if (RT % V || leaf % V || L > 16) return cudaErrorInvalidValue;
    // xs holds the staged inputs (<= b columns), then the KG x RT group sums
    const size_t sm = (size_t)std::max(b, 256 * V) * NR * sizeof(T);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    // narrow tiles (the low reduction levels): one warp per tile
    // (wmax 0: only diagonal terms or copies)
    const bool by_warp = wmax <= 256 && L <= 31 && 32 % (RT / V) == 0 && RT <= 64;
    const int wslice = std::max(wmax, RT);  // the slice also holds the tile's RT x NR sums
    const size_t smW = (size_t)8 * wslice * NR * sizeof(T);
    // few row tiles: split each tile's columns over CTAs so that every SM streams
    int nsplit = 1;
    const long long tiles = (long long)nprob * (b / RT);
    if (!by_warp && tiles < 2 * 152) {
        nsplit = (int)((4 * 152 + tiles - 1) / tiles);
        nsplit = std::min(nsplit, std::max(1, b / 64));
    }
    T* part = nullptr;
    if (nsplit > 1 && cudaMallocAsync(&part, sizeof(T) * (size_t)nsplit * nprob * b * nrhs, s) != cudaSuccess) {
        cudaGetLastError();
        return cudaErrorMemoryAllocation;
    }
    const dim3 gb(b / RT, nprob, nsplit);
    const size_t smA = ((size_t)std::max(b / 2, 1) * NR + (size_t)8 * 64 * NR) * sizeof(T);
    if (smA > 200 * 1024) return cudaErrorInvalidValue;
    // pass A per term when its partials fit: items of CH rows (CH divides every node size)
    const int CH = std::min(64, leaf);
    auto smt = [&](int nr) { return ((size_t)b * nr + (size_t)L * (b / CH) * std::max(rkmax, 1) * nr) * sizeof(T); };
    const size_t smT = smt(NR);
    // decided at the widest chunk, so that every column count takes the same
    // kernel (and summation order)
    const bool per_term = terms != nullptr && rkmax <= 64 && L <= 6 && smt(8) <= 160 * 1024;
    // few terms and the CTA-per-tile pass B: pass A's items spread over 8 CTAs
    // per term, their partials added by pass B (same bits as k_hnodes)
    const bool split_a = per_term && !by_warp && nterms > 0 && nterms < 152;
    const int nitems_a = L * (b / CH);
    T* gpart = nullptr;
    if (split_a && cudaMallocAsync(&gpart, sizeof(T) * (size_t)nprob * 2 * nitems_a * std::max(rkmax, 1) * nrhs, s) !=
                       cudaSuccess) {
        cudaGetLastError();
        if (part) cudaFreeAsync(part, s);
        return cudaErrorMemoryAllocation;
    }
#define ACR_HS_LAUNCH(NRV)                                                                                       \
    {                                                                                                            \
        cudaError_t le = cudaSuccess;                                                                            \
        if (split_a) {                                                                                           \
            le = launch_pdl(k_hnodes_sp<T, NRV>, dim3(nterms, (nitems_a + 7) / 8), dim3(256),                    \
                            (size_t)8 * CH * NRV * sizeof(T), s, probs_all, prob_off, terms, tasks, nodes, pool, b, \
                            L, CH, nrhs, std::max(rkmax, 1), gpart);                                             \
            count_launches(1);                                                                                   \
        } else if (per_term) {                                                                                   \
            if (nterms >= 152) {                                                                                 \
                ensure_smem((const void*)k_hnodes<T, NRV, 256>, smT);                                          \
                le = launch_pdl(k_hnodes<T, NRV, 256>, dim3(nterms), dim3(256), smT, s, probs_all, terms, tasks, \
                                nodes, pool, b, L, CH, nrhs, std::max(rkmax, 1), tbuf);                          \
                count_launches(1);                                                                               \
            } else if (nterms > 0) { /* less than a wave: four times the warps per term */                      \
                ensure_smem((const void*)k_hnodes<T, NRV, 1024>, smT);                                         \
                le = launch_pdl(k_hnodes<T, NRV, 1024>, dim3(nterms), dim3(1024), smT, s, probs_all, terms,      \
                                tasks, nodes, pool, b, L, CH, nrhs, std::max(rkmax, 1), tbuf);                   \
                count_launches(1);                                                                               \
            }                                                                                                    \
        } else if (na > 0) {                                                                                     \
            ensure_smem((const void*)k_hnode_t<T, NRV>, smA);                                                  \
            le = launch_pdl(k_hnode_t<T, NRV>, dim3(na), dim3(256), smA, s, probs_all, tasks, alist + a_off,     \
                            nodes, pool, b, nrhs, tbuf);                                                         \
            count_launches(1);                                                                                   \
        }                                                                                                        \
        if (le != cudaSuccess) return le;                                                                        \
        if (by_warp) {                                                                                           \
            ensure_smem((const void*)k_hrows_w<T, NRV, V>, smW);                                               \
            le = launch_pdl(k_hrows_w<T, NRV, V>, dim3((b / RT + 7) / 8, nprob), dim3(256), smW, s,            \
                            probs_all + prob_off, nodes, tasks, tbuf, pool, b, leaf, L, nrhs, RT, wslice);       \
        } else {                                                                                                 \
            ensure_smem((const void*)k_hrows<T, NRV, V>, sm);                                                  \
            le = launch_pdl(k_hrows<T, NRV, V>, gb, dim3(256), sm, s, probs_all + prob_off, blks, nodes, tasks,  \
                            tbuf, pool, b, leaf, L, nrhs, RT, part, (const T*)gpart, CH, std::max(rkmax, 1));    \
        }                                                                                                        \
        if (le != cudaSuccess) return le;                                                                        \
        count_launches(1);                                                                                       \
    }
    if (NR == 1) ACR_HS_LAUNCH(1)
    else if (NR == 4) ACR_HS_LAUNCH(4)
    else ACR_HS_LAUNCH(8)
#undef ACR_HS_LAUNCH
    if (gpart) cudaFreeAsync(gpart, s);
    if (part) {
        const long long tot = (long long)nprob * b * nrhs;
        const int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 8);
        const cudaError_t le =
            launch_pdl(k_hrows_reduce<T>, dim3(blocks), dim3(256), 0, s, probs_all + prob_off, nprob, b, nrhs, nsplit,
                       (const T*)part);
        if (le != cudaSuccess) return le;
        count_launches(1);
        cudaFreeAsync(part, s);
    }
    return cudaGetLastError();
}

#define ACR_HODLR_INST(T)                                                                                         \
    template cudaError_t hodlr_omega<T>(T*, long long, uint64_t, cudaStream_t);                                   \
    template cudaError_t gemm_gen<T>(const T* const*, const T* const*, T* const*, int, int, int, int, int, int,    \
                                     int, bool, cudaStream_t);                                                    \
    template cudaError_t node_svd<T>(const T*, T*, T*, int, int, int, cudaStream_t);                              \
    template int node_svd_kz<T>(int, int);                                                                        \
    template cudaError_t pack_nodes<T>(const HNode*, int, int, const T*, const T*, const T* const*, int, int, int, \
                                       T*, cudaStream_t);                                                         \
    template cudaError_t pack_leaves<T>(const T* const*, const long long*, int, int, int, T*, cudaStream_t);       \
    template cudaError_t hsweep<T>(const HSweepProb<T>*, int, int, const HTask*, const int*, int, int, const int*, \
                                   int, int, int, T*, const HBlk*, const HNode*, const T*, int, int, int, int,  \
                                   cudaStream_t);
ACR_HODLR_INST(float)
ACR_HODLR_INST(double)

}  // namespace acr
