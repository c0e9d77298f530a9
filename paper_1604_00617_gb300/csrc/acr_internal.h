// acr_internal.h -- internal launchers and descriptors shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <vector>

namespace acr {

// Kernel launches issued by this library (all threads); the C ABI reports
// per-call deltas.
long long launch_count();
void count_launches(int k);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The limit only ever grows, under a lock, so a launch by one
// host thread is never undercut by another thread setting a smaller limit for
// the same kernel between its call here and its launch.
cudaError_t ensure_smem(const void* func, size_t bytes);

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
//
// Combined mode (sx[0] != NULL): only m[0] is applied, to the scaled sum
//   sx[0] .* x[0] + sx[1] .* x[1]    (sx[t] blksz-vectors; x[1], sx[1] may be NULL)
// which is the level-0 back-substitution D_j^-1 (a_j .* u_{j-1} + c_j .* u_{j+1})
// when A_j, C_j are diagonal.
template <class T>
struct SweepProb {
    T* out;
    const T* cin;
    const T* m[3];
    const T* x[3];
    const T* sx[2];
    long long ldo, ldc, ldx;
    T alpha;
    int diag_mask;
};

// --- level 0 of a banded (5-point) operator -----------------------------------
// Inverse of each tridiagonal D_j, j even: rows computed by the two bidiagonal
// solves of the LU factorization (no pivoting; used only when every D_j is
// strictly diagonally dominant by rows, where that factorization is stable).
// Dband: FP64 [sub, diag, super] per block (3b), dinv: ne blocks.
template <class T>
cudaError_t tridiag_inverse(const double* Dband, int n, int b, T* dinv, int* info, cudaStream_t s);
// Schur complement of level 0 with diagonal A_i, C_i (elementwise):
//   D'_k = D_i - a_i .* Dinv_{i-1} .* c_{i-1}^T - c_i .* Dinv_{i+1} .* a_{i+1}^T
//   A'_k = -a_i .* Dinv_{i-1} .* a_{i-1}^T,   C'_k = -c_i .* Dinv_{i+1} .* c_{i+1}^T
// outputs routed like the dense path (k even -> nd/na/nc_even, k odd -> *_odd).
template <class T>
cudaError_t schur_level0(const double* Dband, const double* a, const double* c, int n, int b,
                         const T* dinv, T* nd_even, T* nd_odd, T* na_even, T* na_odd, T* nc_even,
                         T* nc_odd, cudaStream_t s);
// Route the diagonals of A_j, C_j (FP64, b per block) to T arrays:
// even j -> aev/cev[j/2], odd i -> ak/ck[i/2].
template <class T>
cudaError_t stage_diagonals(const double* a, const double* c, int n, int b, T* aev, T* cev, T* ak,
                            T* ck, int* bad, const double* Dband, cudaStream_t s);

// --- batched Gauss-Jordan inversion with partial pivoting (in place) -------
// mats: count blocks of b x b (stride b*b).  info[e] is set to k+1 for the
// first pivot k that is zero or not finite (0: fine).  ws_piv: count*b ints.
template <class T>
cudaError_t gj_inverse(T* mats, int b, int count, int* info, int* ws_piv, cudaStream_t s);

// Same inversion with every temporary in caller-provided scratch (no device
// allocation); gj_scratch_bytes gives the bytes it needs (0 when the blocks
// fit the shared-memory kernel).  Returns cudaErrorInvalidValue if the
// scratch is too small.
template <class T>
size_t gj_scratch_bytes(int b, int count);
template <class T>
cudaError_t gj_inverse_scratch(T* mats, int b, int count, int* info, void* scratch, size_t scratch_bytes,
                               cudaStream_t s);
// Record a message for acr_last_error() on this thread; returns code.
int set_last_error(int code, const char* msg);

// --- batched multi-term block product ---------------------------------------
template <class T>
cudaError_t gemm_batched(const GemmProb<T>* d_probs, int nprob, int b, int use_tc, cudaStream_t s);

// --- tensor-core block products (tcgen05, three-term TF32 split) ------------
// One problem: out = beta * cin + alpha * sum_t A_t B_t with A_t block az[t]
// of the array described by tensor map amap[t] (left-operand map) and B_t
// block bz[t] of map bmap[t] (right-operand map).  blksz a multiple of 128.
struct TcProb {
    float* out;
    const float* cin;
    float alpha, beta;
    int nterm;
    int amap[2], az[2], bmap[2], bz[2];
};
bool tc_supported(int b);
size_t tc_map_bytes();
// Encode the tensor map of `count` contiguous b x b column-major FP32 blocks
// starting at base, as left (role 0) or right (role 1) operand.  0 on success.
int tc_encode_map(void* map_out, const float* base, int b, int count, int role);
// Same for `count` matrices of d0 (contiguous) x d1 elements.
int tc_encode_map_dims(void* map_out, const float* base, int d0, int d1, int count, int role);
// d_err: set to 1 if a CTA gave up on a bounded wait (then later CTAs skip).
cudaError_t gemm_tc(const TcProb* d_probs, int nprob, const void* d_maps, int b, int* d_err, cudaStream_t s);
// General form: out[:, cols] (b rows, ld b) = alpha * A_t[:, ka0 : ka0 + kdim] B_t[0 : kdim, cols] + beta * cin,
// tiles_n column tiles of 128, tile tn at column tile (tn < nskip ? tn : tn + nshift).
// b and kdim multiples of 128 and 32; A's k coordinate offset ka0 a multiple of 32.
// lolo != 0 adds the fourth split term Alo Blo.
cudaError_t gemm_tc_ex(const TcProb* d_probs, int nprob, const void* d_maps, int b, int kdim, int ka0,
                       int tiles_n, int nskip, int nshift, int lolo, int* d_err, cudaStream_t s);

// Batched FP32 inversion whose rank-128 outer-panel updates run on the tensor
// cores (gemm_tc_ex); b a multiple of 128, b >= 256.  Same pivoting and
// results (to FP32 rounding) as gj_inverse<float>.
bool gj_tc_supported(int b);
cudaError_t gj_inverse_tc(float* mats, int b, int count, int* info, int* ws_piv, int* d_err, cudaStream_t s);

// --- HODLR blocks (k_hodlr.cu) ------------------------------------------------
// Node of a compressed block: rank >= 0: U (s x rank) then V (s x rank) at off
// (B ~= U V^T); rank -1: the dense s x s node at off.  Nodes of a block are
// stored tree level by level (level l: 2^l nodes; node 2p+0 is the upper and
// 2p+1 the lower off-diagonal block of parent p).
struct HNode {
    long long off;
    int rank;
    int pad;
};
struct HBlk {
    long long leaf_off;  // 2^L leaves of leaf x leaf, column-major, contiguous
    int node_base;       // first node of this block in the node table
    int pad;
};
// Sweep problem on compressed blocks: out = cin + alpha * sum_t term_t with
// term_t = M_{blk[t]} x[t] (combined mode as SweepProb: sx[0] set) or, when
// dg[t] is set, the diagonal product dg[t] .* x[t].
template <class T>
struct HSweepProb {
    T* out;
    const T* cin;
    long long ldo, ldc, ldx;
    const T* x[2];
    const T* sx[2];
    const T* dg[2];
    int blk[2];
    int tbase[2];  // first task (of its npb node tasks) of each compressed term
    int node_base[2];         // the blocks' first node and leaves (copies of
    long long leaf_off[2];    // their HBlk, saving the kernel a dependent load)
    T alpha;
};
// Pass A runs either per low-rank node (alist: task indices) or per compressed
// term (terms: (problem << 1) | term, rkmax: the largest node rank).  wmax:
// the widest row tile of the launch (leaf plus the node widths of every tree
// level), 0 if unknown; narrow launches run one warp per row tile.
// One node product of the apply: t = V^T x (pass A).  toff: offset of t
// (rank x nrhs, column-major) in the product buffer; -1 when the node is dense
// or of rank 0.
struct HTask {
    int node, prob, term, level, ni, pad;
    long long toff;
};
template <class T>
cudaError_t hodlr_omega(T* om, long long n, uint64_t seed, cudaStream_t s);
template <class T>
cudaError_t gemm_gen(const T* const* A, const T* const* B, T* const* C, int nprob, int M, int N, int K, int lda,
                     int ldb, int ldc, bool transA, cudaStream_t s);
template <class T>
cudaError_t node_svd(const T* Y, T* U, T* sig, int nnodes, int s, int k, cudaStream_t st);
template <class T>
int node_svd_kz(int s, int k);
template <class T>
cudaError_t pack_nodes(const HNode* meta, int node0, int nnodes, const T* Uk, const T* Vk, const T* const* src,
                       int s, int k, int b, T* pool, cudaStream_t st);
template <class T>
cudaError_t pack_leaves(const T* const* blocks, const long long* leaf_off, int nblocks, int b, int leaf, T* pool,
                        cudaStream_t st);
// Apply the problems probs_all[prob_off .. prob_off + nprob); their low-rank
// node tasks are tasks[alist[a_off .. a_off + na)]; tbuf holds the node
// products (pass A writes, pass B reads).
template <class T>
cudaError_t hsweep(const HSweepProb<T>* probs_all, int prob_off, int nprob, const HTask* tasks, const int* alist,
                   int a_off, int na, const int* terms, int nterms, int rkmax, int wmax, T* tbuf, const HBlk* blks,
                   const HNode* nodes, const T* pool, int b, int leaf, int L, int nrhs, cudaStream_t s);

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
// dst = (double) src
cudaError_t convert_f2d(const float* src, double* dst, long long n, cudaStream_t s);
// Krylov helpers on nvec column blocks V_i = V + i * N * nrhs (each N x nrhs):
//   out[i * nrhs + q] = sum_r V_i[r, q] w[r, q]        (i < nvec), deterministic
cudaError_t multi_dot(const double* V, int nvec, const double* w, long long N, int nrhs, double* ws,
                      double* out, cudaStream_t s);
//   multi_dot, and out[nvec * nrhs + q] = sum_r w[r, q]^2
cudaError_t multi_dot_self(const double* V, int nvec, const double* w, long long N, int nrhs, double* ws,
                           double* out, cudaStream_t s);
//   w[r, q] += sum_i coef[i * nrhs + q] V_i[r, q] (nvec <= 64) and
//   out[q] = |w_new[:, q]|^2, in one read of V.  need != NULL: only the columns
//   with need[q] (the others are neither read nor written).
cudaError_t gs_update_norm(double* w, const double* V, int nvec, const double* coef, long long N, int nrhs,
                           const int* need, double* ws, double* out, cudaStream_t s);
//   The second Gram-Schmidt pass where the first cancelled more than
//   1 - ratio2 of the squared norm (sq1[q] < ratio2 sq0[q]): there h2 = V^T w,
//   w -= V h2 and hacc += h2; hs[q] = |w_final|^2 for every column.  N <= 4M.
cudaError_t gs_reorth(double* w, const double* V, int nvec, const double* sq0, const double* sq1, double ratio2,
                      double* h2, double* coef, double* hacc, int* need, double* hs, long long N, int nrhs,
                      double* ws, cudaStream_t s);
//   w[r, q] += sum_i coef[i * nrhs + q] V_i[r, q]
cudaError_t multi_axpy(double* w, const double* V, int nvec, const double* coef, long long N, int nrhs,
                       cudaStream_t s);
//   coef[i] = -h[i] and hacc[i] = (first ? 0 : hacc[i]) + h[i]   (i < n): one
//   Gram-Schmidt pass's coefficients and the Hessenberg column they add to
cudaError_t gs_coef(const double* h, double* coef, double* hacc, int n, bool first, cudaStream_t s);
//   v[r, q] = w[r, q] * scale[q]
cudaError_t col_scale(double* v, const double* w, const double* scale, long long N, int nrhs,
                      cudaStream_t s);

}  // namespace acr

#ifdef __CUDACC__
namespace acr {
// Tangent of a Jacobi rotation, zeta = (beta - alpha) / (2 gamma): the root
// of t^2 + 2 zeta t - 1 = 0 of smaller magnitude.  For |zeta| > 1 the square
// root is taken as |zeta| sqrt(1 + 1/zeta^2): zeta^2 overflows once |zeta|
// passes ~1e19 in FP32 (a tiny column against a large one), and the t = 0
// that follows would leave the pair as it is while still counting it as
// rotated, so the sweeps would never end.
// Whether a Jacobi pair (squared norms al, be, product ga) needs a rotation:
// |ga| > eps |a| |b|, with the norms taken apart (al * be underflows for tiny
// columns in FP32), and never for a pair with a zero norm: a column whose
// squares underflow can still have a nonzero product with a large one, and
// its zeta is infinite, so the rotation would be the identity forever.
template <class T>
__device__ __forceinline__ bool jacobi_needs(T al, T be, T ga, T eps) {
    return al > T(0) && be > T(0) && ga != T(0) && fabs(ga) > eps * sqrt(al) * sqrt(be);
}
template <class T>
__device__ __forceinline__ T jacobi_tan(T zeta) {
    const T az = fabs(zeta);
    const T root = az > T(1) ? az * sqrt(T(1) + (T(1) / az) * (T(1) / az)) : sqrt(T(1) + az * az);
    return (zeta >= T(0) ? T(1) : T(-1)) / (az + root);
}
// Arg-max key of an FP32 pivot candidate whose magnitude a was taken as
// x < 0 ? -x : x (so -0 stays -0; a is never NaN, which no comparison
// selects): the bits of a without the sign bit, plus 1; 0 for no candidate.
// Non-negative floats are ordered as their bit patterns, so the largest key
// is the largest magnitude, -0 ties with +0 as in a float comparison, and a
// tie goes to the lowest row in both orders.  gj_pivot_mag inverts a nonzero
// key.
__host__ __device__ __forceinline__ unsigned gj_pivot_key(float a, bool valid) {
#ifdef __CUDA_ARCH__
    const unsigned u = __float_as_uint(a);
#else
    unsigned u;
    memcpy(&u, &a, sizeof(u));
#endif
    return valid ? (u & 0x7fffffffu) + 1u : 0u;
}
__host__ __device__ __forceinline__ float gj_pivot_mag(unsigned key) {
    const unsigned u = key - 1u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float a;
    memcpy(&a, &u, sizeof(a));
    return a;
#endif
}
}  // namespace acr
#endif

// --- HODLR arithmetic of the low reduction levels (k_harith.cu) -------------
// Batched products of different sizes: C[M x N] = beta * Cin + sum over the
// problem's terms t0 .. t0 + nt - 1 of alpha * op(A) op(B), op(A) M x K and
// op(B) K x N; flags bit 0: op(A) = A^T (A stored K x M), bit 1: op(B) = B^T.
// Cin may be NULL (then beta is ignored) or equal to C.  Column-major
// operands with the given leading dimensions.
namespace acr {
template <class T>
struct VTerm {
    const T* A;
    const T* B;
    int lda, ldb, K, flags;
    T alpha;
};
template <class T>
struct VProb {
    T* C;
    const T* Cin;
    int ldc, ldcin, M, N;
    T beta;
    int t0, nt;
};
// Truncation of one node's low-rank sum U V^T (U, V: s x R, leading
// dimensions ldu, ldv): Vout (s x wout, ld ldvo) receives the leading right
// singular vectors of U V^T for the kept rank (sigma_k > tol sigma_1, at most
// kcap), then zero columns.
template <class T>
struct RProb {
    const T* U;
    const T* V;
    T* Vout;
    int ldu, ldv, ldvo, s, R, wout;
};
// dst[r, c] = beta * dst[r, c] + alpha * dv[r] * dc[c] * src[r, c] over
// rows x cols (dv, dc optional; a NULL src contributes 0).
template <class T>
struct CProb {
    const T* src;
    T* dst;
    const T* dv;
    const T* dc;
    int lds, ldd, rows, cols;
    T alpha, beta;
};
// One finished node into the solve's pool at dst: U (s x rank), then V^T.
template <class T>
struct PProb {
    const T* U;
    const T* V;
    T* dst;
    int ldu, ldv, s, rank;
};
constexpr int HMAXL = 16;
template <class T>
struct HBandOut {
    T* U[HMAXL + 1];
    T* V[HMAXL + 1];
};
// narrow != 0: every problem has N <= 8 (64 x 8 output tiles instead of 64 x 32)
template <class T>
cudaError_t vgemm(const VProb<T>* probs, const VTerm<T>* terms, const int2* tiles, long long ntiles, int narrow,
                  cudaStream_t s);
// appends the output tiles of problem `prob` (M x N) to `tiles`
void vgemm_tiles(int prob, int M, int N, bool narrow, std::vector<int2>& tiles);
template <class T>
cudaError_t hrecomp(const RProb<T>* probs, int nprob, int smax, int Rmax, int* ranks, double tol, int kcap,
                    cudaStream_t st);
size_t hrecomp_smem_bytes(int s, int R, int es);
// chunks: (problem, chunk) pairs, 2048 elements per chunk (hcopy_chunks)
template <class T>
cudaError_t hcopy(const CProb<T>* probs, const int2* chunks, long long nchunks, cudaStream_t s);
void hcopy_chunks(int prob, long long elems, std::vector<int2>& chunks);
// FP64 inverses of the leaves of tridiagonal blocks sel[0 .. nsel) of Dband
// (strictly diagonally dominant rows), written leaf after leaf to out
template <class T>
cudaError_t tri_leaf_inverse(const double* Dband, const int* sel, int nsel, int b, int leaf, T* out, cudaStream_t s);
// gj_inverse for many small blocks: b <= 64 register resident (same pivoting
// and info), larger b through gj_inverse
template <class T>
cudaError_t gj_inverse_small(T* mats, int b, int count, int* info, int* ws_piv, cudaStream_t s);
template <class T>
cudaError_t hkmat(const T* Tc, double* Kd, int nparent, int K, cudaStream_t s);
template <class T>
cudaError_t hband(const double* Dband, int nblk, int b, int L, T* leaves, const HBandOut<T>& o, cudaStream_t s);
template <class T>
cudaError_t hpack(const PProb<T>* probs, int nprob, cudaStream_t s);
}  // namespace acr

// --- template batches of the HODLR arithmetic -------------------------------
// A batch of problems indexed by (g, i), g < ng (block), i < ni (node or
// leaf); every operand's address is base + map(g) * gs + f(i) * is with
// map(g) = gmap ? gmap[g] : g and f(i) = (i >> ishift) ^ ixor.  A negative
// map value drops the operand: the problem (C) or the term (A, B) is skipped
// for that block.  The whole batch is one kernel argument: no per-problem
// descriptors are built or uploaded.
namespace acr {
template <class T>
struct HAddr {
    const T* base;
    const int* gmap;
    long long gs, is;
    int ishift, ixor, ld, pad;
};
constexpr int VT_MAXT = 10;
template <class T>
struct VTT {
    HAddr<T> A, B;
    int K, flags;  // flags bit 0: op(A) = A^T, bit 1: op(B) = B^T
    T alpha;
};
template <class T>
struct VPT {
    HAddr<T> C, Cin;  // Cin.base NULL: no input term
    int M, N, ni, ng, nt, pad;
    T beta;
    VTT<T> t[VT_MAXT];
};
// dst = beta dst + alpha * dv[r] * dc[c] * src over rows x cols per problem
// (src, dv, dc optional: base NULL)
template <class T>
struct CPT {
    HAddr<T> src, dst, dv, dc;
    int rows, cols, ni, ng;
    T alpha, beta;
};
// truncation of node (g, i): U (s x R, ld), V (s x R), Vout (s x wout)
template <class T>
struct RPT {
    HAddr<T> U, V, Vout;
    int s, R, wout, ni, ng;
};
template <class T>
cudaError_t vgemm_t(const VPT<T>& P, cudaStream_t s);
template <class T>
cudaError_t hcopy_t(const CPT<T>& P, cudaStream_t s);
// ks > 0 (and below min(s, R)): the randomized first pass with ks sketch
// columns; rank -1 where it does not resolve the node, whose truncation then
// needs the exact pass (hrecomp).  ks = 0: the exact pass.
template <class T>
cudaError_t hrecomp_t(const RPT<T>& P, int* ranks, double tol, int kcap, int ks, cudaStream_t st);
size_t hrecomp_sketch_smem_bytes(int s, int R, int ks, int es);
// Uo_i = U_i (V_i^T Vp_i) for count nodes of s x R (node stride s R); W holds
// count x R x R
template <class T>
cudaError_t lowrank_apply(const T* U, const T* V, const T* Vp, T* W, T* Uo, int count, int s, int R, cudaStream_t st);
}  // namespace acr
