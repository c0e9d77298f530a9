// acr_api.cu -- the C ABI (include/acr.h): handles, the level plan, the
// reduction (factor) loop, the solve sweeps and FP64 iterative refinement.
//
// Factor (Section 3, reduction phase), per level t with m blocks:
//   1. invert the eliminated blocks D_j, j = 0, 2, 4, ... in place
//      (block-diagonal H11 inverted block by block);
//   2. XA_j = D_j^-1 A_j,  XC_j = D_j^-1 C_j;
//   3. Schur complement (Eq. "fund") on the kept blocks i = 2k+1:
//        D'_k = D_i - A_i XC_{i-1} - C_i XA_{i+1}
//        A'_k = -A_i XA_{i-1},   C'_k = -C_i XC_{i+1}
//      terms whose blocks do not exist are dropped; the result is again block
//      tridiagonal with floor(m/2) blocks.
// The recursion ends at one block, which is inverted.  Kept per level for the
// solve: D_j^-1, XA_j, XC_j (eliminated) and A_i, C_i (kept).
//
// Solve: forward, per level, g_j = D_j^-1 f_j and
//   f'_k = f_i - A_i g_{i-1} - C_i g_{i+1}   (f^(1) of Eq. "fund");
// top: u = D^-1 f; back-substitution, levels in reverse:
//   u_j = g_j - XA_j u_{j-1} - XC_j u_{j+1}  (= D_j^-1 (f_j - A_j u_{j-1} - C_j u_{j+1})).
//
// Memory layout in HBM: per level, five contiguous arrays of blksz x blksz
// column-major blocks (D^-1, XA, XC for the ceil(m/2) eliminated blocks;
// A, C for the floor(m/2) kept blocks).  Level vectors are (m*blksz) x nrhs
// column-major panels; level 0 is the caller's right-hand side.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/acr.h"
#include "acr_internal.h"
#include "hred.cuh"

using namespace acr;

namespace {
thread_local std::string g_err;
}  // namespace

int acr::set_last_error(int code, const char* msg) {
    g_err = msg;
    return code;
}

namespace {

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (e_ == cudaErrorMemoryAllocation) {                                        \
                cudaGetLastError();                                                       \
                return fail(ACR_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));        \
            }                                                                             \
            return fail(ACR_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                              \
        }                                                                                 \
    } while (0)

// Where a caller's buffer lives: host memory (pageable, pinned or unknown to
// CUDA), device memory of the given device (or managed memory, reachable from
// it), or device memory of another GPU.  Kernels here only dereference memory
// of the handle's device: a buffer on another GPU is rejected before any
// launch, since reading it without peer access would fault.
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };

PtrKind ptr_kind(const void* p, int dev) {
    if (!p) return PTR_HOST;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
    return PTR_HOST;
}

struct Level {
    int m = 0, ne = 0, nk = 0;
    size_t off_dinv = 0, off_xa = 0, off_xc = 0, off_ak = 0, off_ck = 0;  // bytes in arena
};

// Device memory owned by one call or handle; freed on scope exit.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    bool async = false;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (async) cudaFreeAsync(p, s);
            else cudaFree(p);
            p = nullptr;
        }
    }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        release();
        s = st;
        async = true;
        if (bytes == 0) bytes = 16;
        return cudaMallocAsync(&p, bytes, st);
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// CUDA events owned by one call, destroyed on every return path (an event
// still pending on a stream is released once it completes).
struct Events {
    std::vector<cudaEvent_t> all;
    Events() = default;
    Events(const Events&) = delete;
    Events& operator=(const Events&) = delete;
    ~Events() {
        for (cudaEvent_t e : all) cudaEventDestroy(e);
    }
    cudaError_t make(cudaEvent_t* e) {
        const cudaError_t r = cudaEventCreate(e);
        if (r == cudaSuccess) all.push_back(*e);
        return r;
    }
};

}  // namespace

struct acr_ctx {
    int n = 0, b = 0, prec = ACR_FP64, in_kind = ACR_DENSE;
    double tol = 0.0;
    acr_opts opts{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool band0 = false;  // level 0 stored and reduced with its exact structure
    size_t es = 8;  // factor element size
    std::vector<Level> lev;
    DevBuf arena;   // persistent factors
    DevBuf op;      // FP64 copy of the original operator (refinement / residual)
    // compressed (HODLR) storage, tol > 0: the dense arena is released
    bool compressed = false;
    int leaf = 0, hL = 0;
    double tol_eff = 0.0;
    DevBuf hpool;    // leaves of every block, then the node data of every block
    DevBuf hnodes;   // HNode table
    DevBuf hblks;    // HBlk table
    DevBuf hdiag;    // level-0 diagonals (a, c of eliminated and kept blocks) when band0
    std::vector<std::vector<std::vector<int>>> bid;  // [level][array][slot] -> block id, -1 if unused
    size_t hd_off[4] = {0, 0, 0, 0};                 // element offsets of the 4 diagonal arrays in hdiag
    std::vector<double> hblk_bytes;                  // compressed bytes of every block
    std::vector<HNode> hnodes_host;                  // host copies of the node / block tables
    std::vector<HBlk> hblks_host;
    int npb = 0;                                     // off-diagonal nodes per block
    std::mutex mu;
    acr_stats_t st{};
    ~acr_ctx() {
        // stream-ordered frees, all queued before the stream may be destroyed
        arena.release();
        op.release();
        hpool.release();
        hnodes.release();
        hblks.release();
        hdiag.release();
        if (stream) cudaStreamSynchronize(stream);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
    size_t bb() const { return (size_t)b * b; }
    template <class T> T* P(size_t off) const { return reinterpret_cast<T*>(static_cast<char*>(arena.p) + off); }
    int levels() const { return (int)lev.size(); }
};

namespace {

void default_opts(acr_opts* o) {
    memset(o, 0, sizeof(*o));
    o->precision = ACR_FP64;
    o->input_kind = ACR_DENSE;
    o->leaf = 0;
    o->max_rank = 0;
    o->m_stop = 1;
    o->ir_tol = 1e-8;
    o->ir_max_iter = 20;
    o->stream = nullptr;
    o->refine = ACR_REFINE_FGMRES;
    o->h_levels = 0;
    o->h_sketch = 1;
}

// Level plan and persistent byte offsets.  Returns the arena size.  With
// band0 (5-point operator, level-0 A_i and C_i diagonal) level 0 keeps only
// the diagonals: xa/xc hold a_j, c_j of the eliminated blocks (b values each;
// D_j^-1 A_j is applied as D_j^-1 (a_j .* u)) and ak/ck those of the kept ones.
// Levels below t0 are reduced in HODLR arithmetic and take no dense storage.
size_t plan_levels(int n, int b, size_t es, std::vector<Level>& lev, bool band0 = false, int t0 = 0) {
    lev.clear();
    const size_t blk = (size_t)b * b * es;
    size_t off = 0;
    int m = n;
    while (true) {
        Level L;
        L.m = m;
        L.ne = (m + 1) / 2;
        L.nk = m / 2;
        const bool top = (m == 1);
        const bool none = (int)lev.size() < t0;
        const size_t ob = none ? 0 : ((band0 && m == n) ? (size_t)b * es : blk);  // off-diagonal storage per block
        const size_t db = none ? 0 : blk;
        L.off_dinv = off; off += L.ne * db;
        L.off_xa = off; off += top ? 0 : L.ne * ob;
        L.off_xc = off; off += top ? 0 : L.ne * ob;
        L.off_ak = off; off += L.nk * ob;
        L.off_ck = off; off += L.nk * ob;
        off = (off + 255) & ~(size_t)255;
        lev.push_back(L);
        if (top) break;
        m = m / 2;
    }
    return off;
}

// HODLR tree of a b x b block for a requested leaf size: the largest depth L
// with b divisible by 2^L and leaves b / 2^L no smaller than the request.
void hodlr_tree(int b, int want_leaf, int& L, int& leaf) {
    const int want = std::max(1, want_leaf);
    L = 0;
    while ((b % (2 << L)) == 0 && (b >> (L + 1)) >= want && L < hred::HMAXL_TREE) ++L;
    leaf = b >> L;
}

// Algorithmic flops of block cyclic reduction from level t0 on: 2 b^3 per
// dense block inverse and per block product (D' has two).
double factor_flops(const std::vector<Level>& lev, int b, size_t t0 = 0) {
    const double b3 = (double)b * b * b;
    double f = 0.0;
    for (size_t t = t0; t < lev.size(); ++t) {
        const Level& L = lev[t];
        f += 2.0 * b3 * L.ne;
        if (L.m == 1) continue;
        int nxa = 0, nxc = 0;
        for (int e = 0; e < L.ne; ++e) {
            if (2 * e > 0) ++nxa;
            if (2 * e + 1 < L.m) ++nxc;
        }
        f += 2.0 * b3 * (nxa + nxc);
        for (int k = 0; k < L.nk; ++k) {
            const int i = 2 * k + 1;
            f += 2.0 * b3 * (1 + (i + 1 < L.m));
            if (i >= 3) f += 2.0 * b3;
            if (i + 2 < L.m) f += 2.0 * b3;
        }
    }
    return f;
}

// ---------------------------------------------------------------------------
// HODLR recompression of every stored factor block (tol > 0).  The blocks are
// formed densely by the reduction; each one is then held as a HODLR matrix:
// dense leaves plus off-diagonal U V^T with ranks truncated at
// sigma_k > tol * sigma_1 of each node (randomized sketch, Householder QR,
// Jacobi SVD; nodes the sketch cannot certify stay dense).  The dense arena
// is released afterwards; the sweeps then read the compressed blocks.
// ---------------------------------------------------------------------------
int default_leaf(int b) {
    if (b >= 512) return 64;
    if (b >= 256) return 32;
    return std::min(b, 16);
}

template <class T>
int compress_factor(acr_ctx* h, hred::Result<T>* hres = nullptr) {
    const int b = h->b;
    const size_t bb = h->bb();
    cudaStream_t s = h->stream;
    // tree depth: the largest L with b divisible by 2^L and leaves b / 2^L no
    // smaller than the requested leaf size
    int L = 0, leaf = b;
    hodlr_tree(b, h->opts.leaf > 0 ? h->opts.leaf : default_leaf(b), L, leaf);
    h->leaf = leaf;
    h->hL = L;
    const int max_rank = h->opts.max_rank > 0 ? h->opts.max_rank : 0;
    const int kmax = max_rank > 0 ? std::min(64, std::max(16, ((max_rank + 8) + 1) / 2 * 2)) : 32;
    const double tol = h->tol_eff;
    const int T_ = h->levels() - 1;
    const int th = hres ? hres->th : 0;  // levels below th were reduced in HODLR arithmetic

    // ---- the stored blocks -----------------------------------------------------
    // Global block ids: first the blocks of the HODLR-arithmetic levels
    // (already compressed, ids < NW), then the dense blocks of the later levels
    // (compressed here by sketching; dense index = id - NW).
    struct WEnt {
        const hred::HSet<T>* set;
        int idx;
    };
    std::vector<WEnt> went;
    std::vector<const T*> blocks;
    int nid = 0;
    h->bid.assign(T_ + 1, std::vector<std::vector<int>>(5));
    for (int t = 0; t <= T_; ++t) {
        const Level& Lv = h->lev[t];
        const bool diag0 = h->band0 && t == 0;
        auto add = [&](int arr, size_t off, int count, auto used) {
            h->bid[t][arr].assign(count, -1);
            for (int e = 0; e < count; ++e)
                if (used(e)) {
                    h->bid[t][arr][e] = nid++;
                    blocks.push_back(h->P<T>(off) + (size_t)e * bb);
                }
        };
        auto addw = [&](int arr, const hred::HSet<T>* set, int count, auto idx, auto used) {
            h->bid[t][arr].assign(count, -1);
            for (int e = 0; e < count; ++e)
                if (used(e)) {
                    h->bid[t][arr][e] = nid++;
                    went.push_back({set, idx(e)});
                }
        };
        if (t < th) {
            addw(0, hres->dinv[t].get(), Lv.ne, [](int e) { return e; }, [](int) { return true; });
            if (t == T_ || diag0) continue;
            addw(1, hres->x[t].get(), Lv.ne, [](int e) { return 2 * e; }, [](int e) { return 2 * e > 0; });
            addw(2, hres->x[t].get(), Lv.ne, [](int e) { return 2 * e + 1; }, [&](int e) { return 2 * e + 1 < Lv.m; });
            addw(3, hres->ac[t].get(), Lv.nk, [](int k) { return 2 * (2 * k + 1); }, [](int) { return true; });
            addw(4, hres->ac[t].get(), Lv.nk, [](int k) { return 2 * (2 * k + 1) + 1; },
                 [&](int k) { return 2 * k + 2 < Lv.m; });
            continue;
        }
        add(0, Lv.off_dinv, Lv.ne, [](int) { return true; });
        if (t == T_ || diag0) continue;
        add(1, Lv.off_xa, Lv.ne, [](int e) { return 2 * e > 0; });
        add(2, Lv.off_xc, Lv.ne, [&](int e) { return 2 * e + 1 < Lv.m; });
        add(3, Lv.off_ak, Lv.nk, [](int) { return true; });
        add(4, Lv.off_ck, Lv.nk, [&](int k) { return 2 * k + 2 < Lv.m; });
    }
    const int NW = (int)went.size();
    const int NBd = (int)blocks.size();
    const int NB = NW + NBd;
    const int npb = (1 << (L + 1)) - 2;  // off-diagonal nodes per block

    // ---- sketch, QR + SVD, V for every tree level (dense blocks) ---------------
    // Two passes per tree level: every node is sketched with k1 = 16 columns
    // (ranks at most k1 - 4 are resolved by it); only the nodes whose sketch
    // saturates are sketched again with k = kmax.  Most nodes of the low
    // reduction levels have ranks of a few units, so the QR + SVD work, which
    // grows with k^2, is paid at k = kmax only where it is needed.
    const int omr = std::max(1, b / 2);
    DevBuf om;
    CK(om.alloc((size_t)omr * kmax * sizeof(T), s));
    CK(hodlr_omega<T>(om.as<T>(), (long long)omr * kmax, 0x5eedacc0ull + (uint64_t)b, s));
    std::vector<DevBuf> Uk(L + 1), Vk(L + 1), Uk2(L + 1), Vk2(L + 1);
    std::vector<int> kl(L + 1, 0), kl2(L + 1, 0);
    std::vector<std::vector<T>> hsig(L + 1), hsig2(L + 1);
    std::vector<std::vector<int>> sat(L + 1);       // node ids (g << l | ni) of the second pass
    std::vector<std::vector<int>> sat_pos(L + 1);   // id -> position in sat, or -1
    // one pass over the nodes `ids` of tree level l with k sketch columns
    auto sketch = [&](int l, const std::vector<int>& ids, int k, DevBuf& U, DevBuf& V, std::vector<T>& sig) -> int {
        const int sz = b >> l, nn = (int)ids.size();
        if (nn == 0) return ACR_OK;
        if (node_svd_kz<T>(sz, k) == 0) return fail(ACR_ERR_INVALID_ARG, "HODLR node %d too large", sz);
        std::vector<const T*> pa(nn), pb(nn);
        std::vector<T*> pc(nn);
        DevBuf Y, Sg;
        CK(Y.alloc((size_t)nn * sz * k * sizeof(T), s));
        CK(U.alloc((size_t)nn * sz * k * sizeof(T), s));
        CK(V.alloc((size_t)nn * sz * k * sizeof(T), s));
        CK(Sg.alloc((size_t)nn * k * sizeof(T), s));
        for (int i = 0; i < nn; ++i) {
            const int g = ids[i] >> l, ni = ids[i] & ((1 << l) - 1);
            const int p = ni >> 1, lower = ni & 1;
            const int r0 = lower ? (2 * p + 1) * sz : 2 * p * sz;
            const int c0 = lower ? 2 * p * sz : (2 * p + 1) * sz;
            pa[i] = blocks[g] + r0 + (size_t)c0 * b;
            pb[i] = om.as<T>();
            pc[i] = Y.as<T>() + (size_t)i * sz * k;
        }
        DevBuf dpa, dpb, dpc;
        CK(dpa.alloc(nn * sizeof(void*), s));
        CK(dpb.alloc(nn * sizeof(void*), s));
        CK(dpc.alloc(nn * sizeof(void*), s));
        CK(cudaMemcpyAsync(dpa.p, pa.data(), nn * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dpb.p, pb.data(), nn * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dpc.p, pc.data(), nn * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(gemm_gen<T>(dpa.as<const T*>(), dpb.as<const T*>(), dpc.as<T*>(), nn, sz, k, sz, b, omr, sz, false, s));
        CK(node_svd<T>(Y.as<T>(), U.as<T>(), Sg.as<T>(), nn, sz, k, s));
        // V_k = B^T U_k
        for (int i = 0; i < nn; ++i) {
            pb[i] = U.as<T>() + (size_t)i * sz * k;
            pc[i] = V.as<T>() + (size_t)i * sz * k;
        }
        CK(cudaStreamSynchronize(s));  // host pointer tables reused below
        CK(cudaMemcpyAsync(dpb.p, pb.data(), nn * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dpc.p, pc.data(), nn * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(gemm_gen<T>(dpa.as<const T*>(), dpb.as<const T*>(), dpc.as<T*>(), nn, sz, k, sz, b, sz, sz, true, s));
        sig.resize((size_t)nn * k);
        CK(cudaMemcpyAsync(sig.data(), Sg.p, (size_t)nn * k * sizeof(T), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return ACR_OK;
    };
    auto rank_of = [&](const T* sg, int k) {
        int r = 0;
        if (sg[0] > T(0))
            while (r < k && (double)sg[r] > tol * (double)sg[0]) ++r;
        return r;
    };
    for (int l = 1; l <= L && NBd > 0; ++l) {
        const int sz = b >> l, nn = NBd << l;
        int kbig = std::min(kmax, sz);
        kbig -= kbig & 1;
        if (kbig < 2) kbig = 2;
        const int k1 = std::min(kbig, 16);
        kl[l] = k1;
        kl2[l] = kbig;
        std::vector<int> all(nn);
        for (int i = 0; i < nn; ++i) all[i] = i;
        int st = sketch(l, all, k1, Uk[l], Vk[l], hsig[l]);
        if (st) return st;
        sat_pos[l].assign(nn, -1);
        if (k1 < kbig) {
            for (int i = 0; i < nn; ++i) {
                int r = rank_of(hsig[l].data() + (size_t)i * k1, k1);
                if (max_rank > 0 && r > max_rank) r = max_rank;
                if (r > k1 - 4 && 2 * r < sz) {
                    sat_pos[l][i] = (int)sat[l].size();
                    sat[l].push_back(i);
                }
            }
            st = sketch(l, sat[l], kbig, Uk2[l], Vk2[l], hsig2[l]);
            if (st) return st;
        }
    }

    // ---- ranks, layout ------------------------------------------------------------
    std::vector<HNode> nodes((size_t)NB * npb);
    std::vector<HBlk> hb(NB);
    long long off = (long long)NB * b * leaf;  // leaves first
    for (int g = 0; g < NB; ++g) {
        hb[g].leaf_off = (long long)g * b * leaf;
        hb[g].node_base = g * npb;
        hb[g].pad = 0;
    }
    std::vector<double> rsum(h->levels(), 0.0);
    std::vector<long long> rcnt(h->levels(), 0);
    std::vector<int> rmax(h->levels(), 0);
    std::vector<int> blk_level(NB, 0);
    for (int t = 0; t <= T_; ++t)
        for (int arr = 0; arr < 5; ++arr)
            for (int id : h->bid[t][arr])
                if (id >= 0) blk_level[id] = t;
    for (int l = 1; l <= L; ++l) {
        const int sz = b >> l;
        for (int g = 0; g < NB; ++g)
            for (int ni = 0; ni < (1 << l); ++ni) {
                int r = 0;
                bool dense = false;
                if (g < NW) {
                    r = went[g].set->rk(went[g].idx, l, ni);
                } else {
                    const size_t id = ((size_t)(g - NW) << l) + ni;
                    const int sp = sat_pos[l][id];
                    const int k = sp >= 0 ? kl2[l] : kl[l];
                    const T* sg = sp >= 0 ? hsig2[l].data() + (size_t)sp * k : hsig[l].data() + id * k;
                    r = rank_of(sg, k);
                    if (max_rank > 0 && r > max_rank) r = max_rank;
                    const bool sketch_full = (k < sz) && (r > k - 4);
                    dense = sketch_full || (2 * r >= sz);
                }
                HNode& hn = nodes[(size_t)g * npb + ((1 << l) - 2) + ni];
                hn.pad = 0;
                hn.off = off;
                if (dense) {
                    hn.rank = -1;
                    off += (long long)sz * sz;
                } else {
                    hn.rank = r;
                    off += 2LL * sz * r;
                }
                const int t = blk_level[g];
                const int rr = dense ? sz : r;
                rsum[t] += rr;
                rcnt[t] += 1;
                rmax[t] = std::max(rmax[t], rr);
            }
    }
    const size_t pool_bytes = (size_t)off * sizeof(T);
    CK(h->hpool.alloc(pool_bytes, h->stream));
    CK(h->hnodes.alloc(std::max<size_t>(1, nodes.size()) * sizeof(HNode), h->stream));
    CK(h->hblks.alloc((size_t)NB * sizeof(HBlk), h->stream));
    if (!nodes.empty())
        CK(cudaMemcpyAsync(h->hnodes.p, nodes.data(), nodes.size() * sizeof(HNode), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->hblks.p, hb.data(), (size_t)NB * sizeof(HBlk), cudaMemcpyHostToDevice, s));

    // ---- pack ----------------------------------------------------------------------
    if (NW > 0) {
        // blocks of the HODLR-arithmetic levels: leaves as they are, nodes at
        // their kept ranks (U, then V^T)
        std::vector<CProb<T>> cp;
        std::vector<PProb<T>> pp;
        const size_t bl = (size_t)b * leaf;
        for (int g = 0; g < NW; ++g) {
            CProb<T> c;
            memset(&c, 0, sizeof(c));
            c.src = went[g].set->lf(went[g].idx, 0);
            c.dst = h->hpool.as<T>() + hb[g].leaf_off;
            c.lds = c.ldd = (int)bl;
            c.rows = (int)bl;
            c.cols = 1;
            c.alpha = T(1);
            cp.push_back(c);
            for (int l = 1; l <= L; ++l) {
                const int sz = b >> l;
                for (int ni = 0; ni < (1 << l); ++ni) {
                    const HNode& hn = nodes[(size_t)g * npb + ((1 << l) - 2) + ni];
                    if (hn.rank <= 0) continue;
                    PProb<T> q;
                    q.U = went[g].set->Up(went[g].idx, l) + (size_t)ni * sz;
                    q.V = went[g].set->Vp(went[g].idx, l) + (size_t)(ni ^ 1) * sz;
                    q.dst = h->hpool.as<T>() + hn.off;
                    q.ldu = q.ldv = b;
                    q.s = sz;
                    q.rank = hn.rank;
                    pp.push_back(q);
                }
            }
        }
        std::vector<int2> ch;
        for (size_t i = 0; i < cp.size(); ++i) hcopy_chunks((int)i, (long long)bl, ch);
        DevBuf dcp, dch, dpp;
        CK(dcp.alloc(cp.size() * sizeof(CProb<T>), s));
        CK(dch.alloc(ch.size() * sizeof(int2), s));
        CK(cudaMemcpyAsync(dcp.p, cp.data(), cp.size() * sizeof(CProb<T>), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dch.p, ch.data(), ch.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        CK(hcopy<T>(dcp.as<CProb<T>>(), dch.as<int2>(), (long long)ch.size(), s));
        if (!pp.empty()) {
            CK(dpp.alloc(pp.size() * sizeof(PProb<T>), s));
            CK(cudaMemcpyAsync(dpp.p, pp.data(), pp.size() * sizeof(PProb<T>), cudaMemcpyHostToDevice, s));
            CK(hpack<T>(dpp.as<PProb<T>>(), (int)pp.size(), s));
        }
        CK(cudaStreamSynchronize(s));
    }
    if (NBd > 0) {
        std::vector<long long> lo(NBd);
        for (int d = 0; d < NBd; ++d) lo[d] = hb[NW + d].leaf_off;
        DevBuf dblk, dlo;
        CK(dblk.alloc((size_t)NBd * sizeof(void*), s));
        CK(dlo.alloc((size_t)NBd * sizeof(long long), s));
        CK(cudaMemcpyAsync(dblk.p, blocks.data(), (size_t)NBd * sizeof(void*), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dlo.p, lo.data(), (size_t)NBd * sizeof(long long), cudaMemcpyHostToDevice, s));
        CK(pack_leaves<T>(dblk.as<const T*>(), dlo.as<long long>(), NBd, b, leaf, h->hpool.as<T>(), s));
        for (int l = 1; l <= L; ++l) {
            const int sz = b >> l, nn = NBd << l, ns = (int)sat[l].size();
            // first launch: every node, the second-pass ones marked to skip
            // (rank -2); second launch: the second-pass nodes
            std::vector<HNode> lv((size_t)nn + ns);
            std::vector<const T*> src((size_t)nn + ns);
            for (int d = 0; d < NBd; ++d)
                for (int ni = 0; ni < (1 << l); ++ni) {
                    const size_t id = ((size_t)d << l) + ni;
                    const HNode hn = nodes[(size_t)(NW + d) * npb + ((1 << l) - 2) + ni];
                    const int p = ni >> 1, lower = ni & 1;
                    const int r0 = lower ? (2 * p + 1) * sz : 2 * p * sz;
                    const int c0 = lower ? 2 * p * sz : (2 * p + 1) * sz;
                    const T* B = blocks[d] + r0 + (size_t)c0 * b;
                    const int sp = sat_pos[l][id];
                    lv[id] = hn;
                    src[id] = B;
                    if (sp >= 0) {
                        lv[id].rank = -2;
                        lv[(size_t)nn + sp] = hn;
                        src[(size_t)nn + sp] = B;
                    }
                }
            DevBuf dm, ds;
            CK(dm.alloc(lv.size() * sizeof(HNode), s));
            CK(ds.alloc(src.size() * sizeof(void*), s));
            CK(cudaMemcpyAsync(dm.p, lv.data(), lv.size() * sizeof(HNode), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(ds.p, src.data(), src.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
            CK(pack_nodes<T>(dm.as<HNode>(), 0, nn, Uk[l].as<T>(), Vk[l].as<T>(), ds.as<const T*>(), sz, kl[l], b,
                             h->hpool.as<T>(), s));
            if (ns > 0)
                CK(pack_nodes<T>(dm.as<HNode>(), nn, ns, Uk2[l].as<T>(), Vk2[l].as<T>(), ds.as<const T*>() + nn, sz,
                                 kl2[l], b, h->hpool.as<T>(), s));
            CK(cudaStreamSynchronize(s));  // host tables of this level
        }
        CK(cudaStreamSynchronize(s));
    }
    // ---- keep the level-0 diagonals, release the dense arena ------------------------
    // (with level 0 reduced in HODLR arithmetic they were staged into hdiag
    // before the reduction)
    if (h->band0 && T_ > 0 && th == 0) {
        const Level& L0 = h->lev[0];
        const size_t n4[4] = {(size_t)L0.ne * b, (size_t)L0.ne * b, (size_t)L0.nk * b, (size_t)L0.nk * b};
        const size_t src4[4] = {L0.off_xa, L0.off_xc, L0.off_ak, L0.off_ck};
        size_t tot = 0;
        for (int i = 0; i < 4; ++i) { h->hd_off[i] = tot; tot += n4[i]; }
        CK(h->hdiag.alloc(std::max<size_t>(tot, 1) * sizeof(T), h->stream));
        for (int i = 0; i < 4; ++i)
            CK(cudaMemcpyAsync(h->hdiag.as<T>() + h->hd_off[i], h->P<T>(src4[i]), n4[i] * sizeof(T),
                               cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    h->hblk_bytes.assign(NB, (double)b * leaf * sizeof(T));
    for (int g = 0; g < NB; ++g)
        for (int i = 0; i < npb; ++i) {
            const HNode& hn = nodes[(size_t)g * npb + i];
            int l = 1;
            while (((1 << (l + 1)) - 2) <= i) ++l;
            const int sz = b >> l;
            h->hblk_bytes[g] += (hn.rank < 0 ? (double)sz * sz : 2.0 * sz * hn.rank) * sizeof(T);
        }
    h->hnodes_host = nodes;
    h->hblks_host = hb;
    h->npb = npb;
    h->arena.release();
    h->compressed = true;
    h->st.compressed = 1;
    h->st.factor_bytes = pool_bytes + nodes.size() * sizeof(HNode) + (size_t)NB * sizeof(HBlk) +
                         (h->band0 ? (size_t)(h->lev[0].ne + h->lev[0].nk) * 2 * b * sizeof(T) : 0);
    for (int t = 0; t <= T_ && t < 32; ++t) {
        h->st.rank_max[t] = rmax[t];
        h->st.rank_mean[t] = rcnt[t] ? rsum[t] / (double)rcnt[t] : 0.0;
    }
    return ACR_OK;
}

template <class T>
int run_factor(acr_ctx* h, const double* A, const double* D, const double* C) {
    const int n = h->n, b = h->b;
    const size_t bb = h->bb(), blk = bb * sizeof(T);
    cudaStream_t s = h->stream;
    const bool banded = h->in_kind == ACR_BANDED;

    // ---- stage the input on the device (FP64) ---------------------------
    const size_t nA = banded ? (size_t)n * b : (size_t)n * bb;
    const size_t nD = banded ? (size_t)n * 3 * b : (size_t)n * bb;
    DevBuf sA, sD, sC;
    const double *dA = A, *dD = D, *dC = C;
    // A and C are never read when there is a single block
    if (n > 1 && ptr_kind(A, h->dev) != PTR_DEVICE) { CK(sA.alloc(nA * 8, s)); CK(cudaMemcpyAsync(sA.p, A, nA * 8, cudaMemcpyHostToDevice, s)); dA = sA.as<double>(); }
    if (ptr_kind(D, h->dev) != PTR_DEVICE) { CK(sD.alloc(nD * 8, s)); CK(cudaMemcpyAsync(sD.p, D, nD * 8, cudaMemcpyHostToDevice, s)); dD = sD.as<double>(); }
    if (n > 1 && ptr_kind(C, h->dev) != PTR_DEVICE) { CK(sC.alloc(nA * 8, s)); CK(cudaMemcpyAsync(sC.p, C, nA * 8, cudaMemcpyHostToDevice, s)); dC = sC.as<double>(); }
    if (n == 1) { dA = nullptr; dC = nullptr; }

    // ---- FP64 operator copy (residual of the refinement) -----------------
    if (banded) {
        const size_t N = (size_t)n * b;
        CK(h->op.alloc(5 * N * 8, h->stream));
        double* o = h->op.as<double>();
        // Dl, Dd, Du de-interleaved from [sub, diag, super] per block
        for (int d = 0; d < 3; ++d)
            CK(cudaMemcpy2DAsync(o + d * N, b * 8, dD + d * b, 3 * b * 8, b * 8, n, cudaMemcpyDeviceToDevice, s));
        if (n > 1) {
            CK(cudaMemcpyAsync(o + 3 * N, dA, N * 8, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(o + 4 * N, dC, N * 8, cudaMemcpyDeviceToDevice, s));
        }
        // A_0 and C_{n-1} do not exist: zero them in the copy
        CK(cudaMemsetAsync(o + 3 * N, 0, b * 8, s));
        CK(cudaMemsetAsync(o + 4 * N + (N - b), 0, b * 8, s));
        h->st.operator_bytes = 5 * N * 8;
    } else {
        CK(h->op.alloc(3 * (size_t)n * bb * 8, h->stream));
        double* o = h->op.as<double>();
        if (n > 1) {
            CK(cudaMemcpyAsync(o, dA, (size_t)n * bb * 8, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(o + 2 * (size_t)n * bb, dC, (size_t)n * bb * 8, cudaMemcpyDeviceToDevice, s));
        }
        CK(cudaMemcpyAsync(o + (size_t)n * bb, dD, (size_t)n * bb * 8, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(o, 0, bb * 8, s));
        CK(cudaMemsetAsync(o + 2 * (size_t)n * bb + (size_t)(n - 1) * bb, 0, bb * 8, s));
        h->st.operator_bytes = 3 * (size_t)n * bb * 8;
    }

    // ---- level-0 structure: 5-point operator with diagonally dominant D_i ---
    // (the tridiagonal inverse factors D_j without pivoting, which is stable
    // for strictly row diagonally dominant tridiagonals; otherwise level 0 runs
    // the general dense path)
    h->band0 = false;
    if (banded) {
        std::vector<double> hD(nD);
        CK(cudaMemcpyAsync(hD.data(), dD, nD * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool dom = true;
        for (int i = 0; i < n && dom; ++i)
            for (int r = 0; r < b; ++r) {
                const double* Bk = hD.data() + (size_t)i * 3 * b;
                const double off = (r > 0 ? std::fabs(Bk[r]) : 0.0) + (r + 1 < b ? std::fabs(Bk[2 * b + r]) : 0.0);
                if (!(std::fabs(Bk[b + r]) > off)) { dom = false; break; }
            }
        h->band0 = dom;
    }

    // ---- the low levels in HODLR arithmetic (tol > 0, 5-point operator) -----
    // Level 0 starts from the exact HODLR form of the input (tridiagonal D_i:
    // rank 1; diagonal A_i, C_i), and the reduction goes on in H-arithmetic
    // while the ranks stay small; the levels from th on are reduced with dense
    // blocks and compressed afterwards.
    // (declared in this order so that the block sets in hres, whose buffers
    // unregister themselves from hr's range set, are released first)
    std::unique_ptr<hred::Red<T>> hr;
    hred::Result<T> hres;
    int th = 0;
    double h_ms = 0.0;
    {
        int hL = 0, hleaf = b;
        hodlr_tree(b, h->opts.leaf > 0 ? h->opts.leaf : default_leaf(b), hL, hleaf);
        if (banded && h->tol > 0 && h->opts.h_levels >= 0 && n > 1 && hL >= 1) {
            const size_t N = (size_t)n * b;
            const double* oa = h->op.as<double>() + 3 * N;  // a with a_0 = 0
            const double* oc = oa + N;                       // c with c_{n-1} = 0
            // the level-0 diagonals, routed as the solve reads them (even
            // blocks' A_j, C_j; kept blocks' A_i, C_i), NaN / Inf checked
            const size_t ne0 = (size_t)(n + 1) / 2, nk0 = (size_t)n / 2;
            const size_t n4[4] = {ne0 * b, ne0 * b, nk0 * b, nk0 * b};
            size_t tot = 0;
            for (int i = 0; i < 4; ++i) { h->hd_off[i] = tot; tot += n4[i]; }
            CK(h->hdiag.alloc(std::max<size_t>(tot, 1) * sizeof(T), h->stream));
            DevBuf hbad;
            CK(hbad.alloc(sizeof(int), s));
            CK(cudaMemsetAsync(hbad.p, 0, sizeof(int), s));
            T* hd = h->hdiag.as<T>();
            CK(stage_diagonals<T>(oa, oc, n, b, hd + h->hd_off[0], hd + h->hd_off[1], hd + h->hd_off[2],
                                  hd + h->hd_off[3], hbad.as<int>(), dD, s));
            // contiguous copies of a, c in the factor's precision (row and
            // column scalings of the level-0 products)
            DevBuf aTb, cTb;
            const T* aT = nullptr;
            const T* cT = nullptr;
            if constexpr (sizeof(T) == 8) {
                aT = oa;
                cT = oc;
            } else {
                CK(aTb.alloc(N * sizeof(T), s));
                CK(cTb.alloc(N * sizeof(T), s));
                CK(convert_d2f(oa, aTb.as<float>(), (long long)N, s));
                CK(convert_d2f(oc, cTb.as<float>(), (long long)N, s));
                aT = aTb.as<T>();
                cT = cTb.as<T>();
            }
            hr.reset(new hred::Red<T>());
            hr->s = s;
            hr->b = b;
            hr->L = hL;
            hr->leaf = hleaf;
            // The truncation errors of every level's Schur complements add
            // up over the reduction: the HODLR arithmetic truncates at tol / 10
            // (not below a few units of the factor's rounding) to keep the
            // solve within the 10 tol bound.
            const double floor_es = sizeof(T) == 8 ? 32 * 2.220446049250313e-16 : 8 * 1.1920929e-7;
            hr->tol = std::max(h->tol / 10.0, floor_es);
            hr->kcap = h->opts.max_rank > 0 ? h->opts.max_rank : b;
            hr->sketch = h->opts.h_sketch != 0;
            hr->rs.add(dD, (size_t)n * 3 * b * 8);
            hr->rs.add(aT, N * sizeof(T));
            hr->rs.add(cT, N * sizeof(T));
            Events hev;
            cudaEvent_t he0, he1;
            CK(hev.make(&he0));
            CK(hev.make(&he1));
            CK(cudaEventRecord(he0, s));
            const long long hl0 = launch_count();
            const auto hw0 = std::chrono::steady_clock::now();
            // a level's inverses may miss the identity by at most 1e4 times the
            // truncation tolerance on random vectors
            const int hst = hred::reduce<T>(*hr, n, dD, aT, cT, h->opts.h_levels, ACR_HRANK_SWITCH, 1e4 * hr->tol, hres,
                                            h->band0);
            h->st.h_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - hw0).count() -
                              hr->wait_ms;
            CK(cudaEventRecord(he1, s));
            const cudaError_t se = cudaStreamSynchronize(s);
            if (se != cudaSuccess) CK(se);
            int bad = 0;
            CK(cudaMemcpy(&bad, hbad.p, sizeof(int), cudaMemcpyDeviceToHost));
            if (bad) return fail(ACR_ERR_INVALID_ARG, "input holds a NaN or Inf");
            if (hst) return fail(hr->oom ? ACR_ERR_OOM : ACR_ERR_CUDA, "HODLR arithmetic: %s", hr->err.c_str());
            if (hres.bad_level >= 0)
                return fail(ACR_ERR_SINGULAR, "singular eliminated block: level %d, block %d (zero pivot in a HODLR leaf "
                            "or capacitance matrix)", hres.bad_level, hres.bad_block);
            th = hres.th;
            for (size_t q = 0; q < hres.check.size() && q < 32; ++q) h->st.h_check[q] = hres.check[q];
            float hm = 0.f;
            cudaEventElapsedTime(&hm, he0, he1);
            h_ms = hm;
            h->st.h_levels = th;
            h->st.h_ms = h_ms;
            h->st.h_flops = hr->flops;
            h->st.h_nodes = hr->nodes;
            h->st.h_sketch_redo = hr->sketch_redo;
            h->st.launches_factor += launch_count() - hl0;
            if (th > 0) {
                h->band0 = true;  // level 0 keeps A_i, C_i as diagonals
            } else {
                hres = hred::Result<T>();
                hr.reset();
                h->hdiag.release();
            }
        }
    }
    const bool b0 = h->band0;

    // ---- persistent arena -------------------------------------------------
    const size_t arena_bytes = plan_levels(n, b, sizeof(T), h->lev, b0, th);
    CK(h->arena.alloc(arena_bytes, h->stream));
    h->st.factor_bytes = arena_bytes;
    const int T_ = h->levels() - 1;
    const int t0d = th > 0 ? th : (b0 ? 1 : 0);  // first level reduced with dense products

    // ---- temporaries: D_odd, A_even, C_even per level (ping-pong) ---------
    auto temp_blocks = [&](int t) {
        const Level& L = h->lev[t];
        return (t < th || (b0 && t == 0)) ? (size_t)0 : (size_t)L.nk + 2 * (size_t)L.ne;
    };
    size_t tmax[2] = {0, 0};
    for (int t = 0; t <= T_; ++t) tmax[t & 1] = std::max(tmax[t & 1], temp_blocks(t));
    DevBuf tmp[2];
    CK(tmp[0].alloc(tmax[0] * blk, s));
    CK(tmp[1].alloc(tmax[1] * blk, s));
    auto t_dodd = [&](int t) { return tmp[t & 1].as<T>(); };
    auto t_aev = [&](int t) { return tmp[t & 1].as<T>() + (size_t)h->lev[t].nk * bb; };
    auto t_cev = [&](int t) { return t_aev(t) + (size_t)h->lev[t].ne * bb; };

    // ---- info / pivots / bad flag ------------------------------------------
    std::vector<int> info_off(T_ + 1);
    int ninfo = 0, maxne = 0;
    for (int t = 0; t <= T_; ++t) { info_off[t] = ninfo; ninfo += h->lev[t].ne; maxne = std::max(maxne, h->lev[t].ne); }
    DevBuf dinfo, dpiv;
    CK(dinfo.alloc((ninfo + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(dinfo.p, 0, (ninfo + 1) * sizeof(int), s));
    CK(dpiv.alloc((size_t)maxne * b * sizeof(int), s));
    int* d_bad = dinfo.as<int>() + ninfo;

    // ---- problem tables (built on the host, one upload) --------------------
    std::vector<GemmProb<T>> probs;
    std::vector<size_t> g1_off(T_ + 1), g1_cnt(T_ + 1), g2_off(T_ + 1), g2_cnt(T_ + 1);
    for (int t = t0d; t < T_; ++t) {
        const Level& L = h->lev[t];
        const Level& Ln = h->lev[t + 1];
        T* dinv = h->P<T>(L.off_dinv);
        T* xa = h->P<T>(L.off_xa);
        T* xc = h->P<T>(L.off_xc);
        T* ak = h->P<T>(L.off_ak);
        T* ck = h->P<T>(L.off_ck);
        g1_off[t] = probs.size();
        for (int e = 0; e < L.ne; ++e) {
            const int j = 2 * e;
            if (j > 0) probs.push_back({xa + e * bb, nullptr, {dinv + e * bb, nullptr}, {t_aev(t) + e * bb, nullptr}, T(1), T(0)});
            if (j + 1 < L.m) probs.push_back({xc + e * bb, nullptr, {dinv + e * bb, nullptr}, {t_cev(t) + e * bb, nullptr}, T(1), T(0)});
        }
        g1_cnt[t] = probs.size() - g1_off[t];
        g2_off[t] = probs.size();
        T* ndinv = h->P<T>(Ln.off_dinv);
        T* nak = h->P<T>(Ln.off_ak);
        T* nck = h->P<T>(Ln.off_ck);
        for (int k = 0; k < L.nk; ++k) {
            const int i = 2 * k + 1;
            const bool kev = (k % 2) == 0;
            const int ks = k / 2;
            T* Di = t_dodd(t) + k * bb;
            T* Ai = ak + k * bb;
            T* Ci = ck + k * bb;
            GemmProb<T> pd{kev ? ndinv + ks * bb : t_dodd(t + 1) + ks * bb, Di, {Ai, nullptr}, {xc + k * bb, nullptr}, T(-1), T(1)};
            if (i + 1 < L.m) { pd.a[1] = Ci; pd.bm[1] = xa + (k + 1) * bb; }
            probs.push_back(pd);
            if (i >= 3)
                probs.push_back({kev ? t_aev(t + 1) + ks * bb : nak + ks * bb, nullptr, {Ai, nullptr}, {xa + k * bb, nullptr}, T(-1), T(0)});
            if (i + 2 < L.m)
                probs.push_back({kev ? t_cev(t + 1) + ks * bb : nck + ks * bb, nullptr, {Ci, nullptr}, {xc + (k + 1) * bb, nullptr}, T(-1), T(0)});
        }
        g2_cnt[t] = probs.size() - g2_off[t];
    }
    DevBuf dprobs;
    CK(dprobs.alloc(std::max<size_t>(1, probs.size()) * sizeof(GemmProb<T>), s));
    if (!probs.empty())
        CK(cudaMemcpyAsync(dprobs.p, probs.data(), probs.size() * sizeof(GemmProb<T>), cudaMemcpyHostToDevice, s));
    const GemmProb<T>* dp = dprobs.as<GemmProb<T>>();

    // ---- tensor-core tables: one tensor map per level array, same problems ----
    bool tc = false;
    DevBuf dmaps, dtc, dterr;
    std::vector<size_t> tc1_off(T_ + 1), tc1_cnt(T_ + 1), tc2_off(T_ + 1), tc2_cnt(T_ + 1);
    if constexpr (sizeof(T) == 4) {
        if (h->prec == ACR_FP32TC_IR && tc_supported(b)) {
            tc = true;
            const size_t mb = tc_map_bytes();
            std::vector<unsigned char> maps;
            auto add_map = [&](const T* base, int count, int role) -> int {
                const size_t at = maps.size();
                maps.resize(at + mb);
                if (tc_encode_map(maps.data() + at, reinterpret_cast<const float*>(base), b, count, role) != 0)
                    return -1;
                return (int)(at / mb);
            };
            std::vector<TcProb> tp;
            for (int t = t0d; t < T_; ++t) {
                const Level& L = h->lev[t];
                const Level& Ln = h->lev[t + 1];
                const int mDinv = add_map(h->P<T>(L.off_dinv), L.ne, 0), mAev = add_map(t_aev(t), L.ne, 1),
                          mCev = add_map(t_cev(t), L.ne, 1), mAk = add_map(h->P<T>(L.off_ak), L.nk, 0),
                          mCk = add_map(h->P<T>(L.off_ck), L.nk, 0), mXa = add_map(h->P<T>(L.off_xa), L.ne, 1),
                          mXc = add_map(h->P<T>(L.off_xc), L.ne, 1);
                if (std::min({mDinv, mAev, mCev, mAk, mCk, mXa, mXc}) < 0)
                    return fail(ACR_ERR_CUDA, "tensor map encoding failed (level %d)", t);
                auto mk1 = [&](T* out, const T* cin, float al, float be, int am, int az, int bm, int bz) {
                    TcProb q;
                    memset(&q, 0, sizeof(q));
                    q.out = reinterpret_cast<float*>(out);
                    q.cin = reinterpret_cast<const float*>(cin);
                    q.alpha = al; q.beta = be; q.nterm = 1;
                    q.amap[0] = am; q.az[0] = az; q.bmap[0] = bm; q.bz[0] = bz;
                    return q;
                };
                tc1_off[t] = tp.size();
                for (int e = 0; e < L.ne; ++e) {
                    const int j = 2 * e;
                    if (j > 0) tp.push_back(mk1(h->P<T>(L.off_xa) + e * bb, nullptr, 1.f, 0.f, mDinv, e, mAev, e));
                    if (j + 1 < L.m) tp.push_back(mk1(h->P<T>(L.off_xc) + e * bb, nullptr, 1.f, 0.f, mDinv, e, mCev, e));
                }
                tc1_cnt[t] = tp.size() - tc1_off[t];
                tc2_off[t] = tp.size();
                for (int k = 0; k < L.nk; ++k) {
                    const int i = 2 * k + 1;
                    const bool kev = (k % 2) == 0;
                    const int ks = k / 2;
                    TcProb pd = mk1(kev ? h->P<T>(Ln.off_dinv) + ks * bb : t_dodd(t + 1) + ks * bb,
                                    t_dodd(t) + k * bb, -1.f, 1.f, mAk, k, mXc, k);
                    if (i + 1 < L.m) { pd.nterm = 2; pd.amap[1] = mCk; pd.az[1] = k; pd.bmap[1] = mXa; pd.bz[1] = k + 1; }
                    tp.push_back(pd);
                    if (i >= 3)
                        tp.push_back(mk1(kev ? t_aev(t + 1) + ks * bb : h->P<T>(Ln.off_ak) + ks * bb, nullptr, -1.f, 0.f,
                                         mAk, k, mXa, k));
                    if (i + 2 < L.m)
                        tp.push_back(mk1(kev ? t_cev(t + 1) + ks * bb : h->P<T>(Ln.off_ck) + ks * bb, nullptr, -1.f, 0.f,
                                         mCk, k, mXc, k + 1));
                }
                tc2_cnt[t] = tp.size() - tc2_off[t];
            }
            CK(dmaps.alloc(std::max<size_t>(maps.size(), 128), s));
            if (!maps.empty()) CK(cudaMemcpyAsync(dmaps.p, maps.data(), maps.size(), cudaMemcpyHostToDevice, s));
            CK(dtc.alloc(std::max<size_t>(1, tp.size()) * sizeof(TcProb), s));
            if (!tp.empty()) CK(cudaMemcpyAsync(dtc.p, tp.data(), tp.size() * sizeof(TcProb), cudaMemcpyHostToDevice, s));
            CK(dterr.alloc(sizeof(int), s));
            CK(cudaMemsetAsync(dterr.p, 0, sizeof(int), s));
            // the host tables must outlive the asynchronous uploads
            CK(cudaStreamSynchronize(s));
        }
    }

    Events evown;
    cudaEvent_t e0, e1;
    CK(evown.make(&e0));
    CK(evown.make(&e1));
    CK(cudaEventRecord(e0, s));

    // ---- level 0 staging (or the blocks of level th, from HODLR form) ----------
    if (th > 0 && th <= T_) {
        const Level& L = h->lev[th];
        // even blocks j -> slot j/2 of the eliminated arrays, odd i -> slot i/2
        // of the kept ones
        std::vector<int> dev_, dod, aev, cev, ak, ck;
        for (int j = 0; j < L.m; ++j) {
            if (j & 1) {
                dod.push_back(j);
                ak.push_back(2 * j);
                ck.push_back(2 * j + 1);
            } else {
                dev_.push_back(j);
                aev.push_back(2 * j);
                cev.push_back(2 * j + 1);
            }
        }
        hr->rs.add(h->arena.p, arena_bytes);
        hr->rs.add(tmp[th & 1].p, tmax[th & 1] * blk);
        int est = hr->expand(*hres.Dn, {{dev_, h->P<T>(L.off_dinv)}, {dod, t_dodd(th)}});
        if (!est && L.m > 1)
            est = hr->expand(*hres.ACn, {{aev, t_aev(th)}, {cev, t_cev(th)}, {ak, h->P<T>(L.off_ak)},
                                         {ck, h->P<T>(L.off_ck)}});
        if (est) return fail(ACR_ERR_CUDA, "HODLR arithmetic: %s", hr->err.c_str());
        hres.Dn.reset();
        hres.ACn.reset();
        hr->drop_tmp();
    } else if (th == 0) {
        const Level& L = h->lev[0];
        if (b0) {
            const double* oa = h->op.as<double>() + 3 * (size_t)n * b;  // a with a_0 = 0
            const double* oc = oa + (size_t)n * b;                       // c with c_{n-1} = 0
            CK(stage_diagonals<T>(oa, oc, n, b, h->P<T>(L.off_xa), h->P<T>(L.off_xc), h->P<T>(L.off_ak),
                                  h->P<T>(L.off_ck), d_bad, dD, s));
        } else {
            CK(stage_level0<T>(banded ? 1 : 0, n, b, dA, dD, dC, h->P<T>(L.off_dinv), t_dodd(0), t_aev(0),
                               h->P<T>(L.off_ak), t_cev(0), h->P<T>(L.off_ck), d_bad, s));
        }
    }
    const int use_tc = (h->prec == ACR_FP32TC_IR) ? 1 : 0;
    // ---- the reduction ---------------------------------------------------------
    // per-class device time: one event pair around every inversion / product launch
    std::vector<cudaEvent_t> evs;
    std::vector<int> evcls;  // 0: inversion, 1: products
    auto mark = [&](int cls) -> cudaError_t {
        cudaEvent_t e;
        cudaError_t err = evown.make(&e);
        if (err != cudaSuccess) return err;
        evs.push_back(e);
        evcls.push_back(cls);
        return cudaEventRecord(e, s);
    };
    const long long l0 = launch_count();
    long long inv_l = 0, gemm_l = 0;
    for (int t = th; t <= T_; ++t) {
        const Level& L = h->lev[t];
        long long c0 = launch_count();
        CK(mark(0));
        if (b0 && t == 0)
            CK(tridiag_inverse<T>(dD, n, b, h->P<T>(L.off_dinv), dinfo.as<int>() + info_off[t], s));
        else if (tc && gj_tc_supported(b)) {
            if constexpr (sizeof(T) == 4)
                CK(gj_inverse_tc(h->P<T>(L.off_dinv), b, L.ne, dinfo.as<int>() + info_off[t], dpiv.as<int>(),
                                 dterr.as<int>(), s));
        } else
            CK(gj_inverse<T>(h->P<T>(L.off_dinv), b, L.ne, dinfo.as<int>() + info_off[t], dpiv.as<int>(), s));
        CK(mark(0));
        inv_l += launch_count() - c0;
        if (t == T_) break;
        if (b0 && t == 0) {
            // elementwise Schur complement of the structured level 0
            const Level& Ln = h->lev[1];
            const double* oa = h->op.as<double>() + 3 * (size_t)n * b;
            const double* oc = oa + (size_t)n * b;
            CK(mark(2));
            CK(schur_level0<T>(dD, oa, oc, n, b, h->P<T>(L.off_dinv), h->P<T>(Ln.off_dinv), t_dodd(1), t_aev(1),
                               h->P<T>(Ln.off_ak), t_cev(1), h->P<T>(Ln.off_ck), s));
            CK(mark(2));
            continue;
        }
        c0 = launch_count();
        CK(mark(1));
        if (tc) {
            const TcProb* tq = dtc.as<TcProb>();
            CK(gemm_tc(tq + tc1_off[t], (int)tc1_cnt[t], dmaps.p, b, dterr.as<int>(), s));
            CK(gemm_tc(tq + tc2_off[t], (int)tc2_cnt[t], dmaps.p, b, dterr.as<int>(), s));
        } else {
            CK(gemm_batched<T>(dp + g1_off[t], (int)g1_cnt[t], b, use_tc, s));
            CK(gemm_batched<T>(dp + g2_off[t], (int)g2_cnt[t], b, use_tc, s));
        }
        CK(mark(1));
        gemm_l += launch_count() - c0;
    }
    CK(cudaEventRecord(e1, s));
    std::vector<int> info(ninfo + 1);
    CK(cudaMemcpyAsync(info.data(), dinfo.p, (ninfo + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (tc) {
        int terr = 0;
        CK(cudaMemcpy(&terr, dterr.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (terr) return fail(ACR_ERR_TIMEOUT, "tensor-core product kernel gave up on a bounded pipeline wait");
    }
    if (info[ninfo]) return fail(ACR_ERR_INVALID_ARG, "input holds a NaN or Inf");
    for (int t = 0; t <= T_; ++t)
        for (int e = 0; e < h->lev[t].ne; ++e)
            if (info[info_off[t] + e])
                return fail(ACR_ERR_SINGULAR, "singular eliminated block: level %d, block %d (pivot %d)", t, 2 * e,
                            info[info_off[t] + e] - 1);
    double cls_ms[3] = {0.0, 0.0, 0.0};
    for (size_t i = 0; i + 1 < evs.size(); i += 2) {
        float d = 0.f;
        cudaEventElapsedTime(&d, evs[i], evs[i + 1]);
        cls_ms[evcls[i]] += d;
    }
    h->st.factor_ms = ms + h_ms;
    // structured level 0: O(b^2) per block (tridiagonal inverse: ~3 b^2;
    // elementwise Schur complement: ~8 b^2 per kept block); levels below th:
    // the HODLR arithmetic's own products (h_flops)
    const size_t t0 = th > 0 ? (size_t)th : (b0 ? 1 : 0);
    double l0_inv = 0.0, l0_schur = 0.0;
    if (b0 && th == 0) {
        l0_inv = 3.0 * (double)b * b * h->lev[0].ne;
        l0_schur = 8.0 * (double)b * b * h->lev[0].nk;
    }
    double inv_fl = l0_inv;
    for (size_t t = t0; t < h->lev.size(); ++t) inv_fl += 2.0 * (double)b * b * b * h->lev[t].ne;
    h->st.factor_flops = factor_flops(h->lev, b, t0) + l0_inv + l0_schur + h->st.h_flops;
    h->st.inv_ms = cls_ms[0];
    h->st.inv_flops = inv_fl;
    h->st.gemm_ms = cls_ms[1];
    h->st.gemm_flops = h->st.factor_flops - inv_fl - l0_schur - h->st.h_flops;
    h->st.inv_launches = inv_l;
    h->st.gemm_launches = gemm_l;
    h->st.launches_factor += launch_count() - l0 + (th == 0 ? 1 : 0);  // + the staging kernel
    if (h->tol > 0) {
        const long long c0 = launch_count();
        cudaEvent_t ce0, ce1;
        CK(evown.make(&ce0));
        CK(evown.make(&ce1));
        CK(cudaEventRecord(ce0, s));
        const int st = compress_factor<T>(h, th > 0 ? &hres : nullptr);
        if (st != ACR_OK) return st;
        CK(cudaEventRecord(ce1, s));
        CK(cudaEventSynchronize(ce1));
        float cms = 0.f;
        cudaEventElapsedTime(&cms, ce0, ce1);
        h->st.factor_ms += cms;
        h->st.compress_ms = cms;
        h->st.launches_factor += launch_count() - c0;
    }
    return ACR_OK;
}

// ---------------------------------------------------------------------------
// Solve sweeps on a device panel F0 (N x nrhs, ld N, element T), in place.
// ---------------------------------------------------------------------------
template <class T>
struct SweepPlan {
    DevBuf ws;       // level vectors F_t (t >= 1) and G_t
    DevBuf dprobs;
    DevBuf hprobs;   // the same problems on compressed blocks
    DevBuf htasks;   // their node tasks
    DevBuf htbuf;    // node products V^T x
    std::vector<size_t> task_start;  // first task of every problem (+ total)
    DevBuf halist;                   // indices of the low-rank tasks
    std::vector<size_t> a_start;     // first low-rank task (in halist) of every problem
    DevBuf hterms;                   // compressed terms with low-rank nodes: (problem << 1) | term
    std::vector<size_t> t_start;     // first entry (in hterms) of every problem
    int rkmax = 0;                   // largest rank of a low-rank node
    std::vector<int> prk;            // largest low-rank node rank of every problem
    std::vector<int> pwmax;          // widest row tile of every problem
    bool hodlr = false;
    std::vector<size_t> fw_g_off, fw_g_cnt, fw_f_off, fw_f_cnt, bk_off, bk_cnt;
    int nrhs = 0;
    double bytes = 0.0;             // algorithmic bytes of one pass
    std::vector<cudaEvent_t> evs;   // start/end of every pass
    long long launches = 0;
    cudaGraphExec_t gexec = nullptr;  // the captured pass
    cudaStream_t gstream = nullptr;   // its stream
    long long glaunches = 0;          // kernels in it
    int applications = 0;
    bool no_graph = false;
    ~SweepPlan() {
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        if (gexec) {
            cudaStreamSynchronize(gstream);  // no replay may still be running
            cudaGraphExecDestroy(gexec);
        }
    }
    double elapsed_ms() const {
        double t = 0.0;
        for (size_t i = 0; i + 1 < evs.size(); i += 2) {
            float d = 0.f;
            cudaEventElapsedTime(&d, evs[i], evs[i + 1]);
            t += d;
        }
        return t;
    }
    int passes() const { return (int)(evs.size() / 2); }
};

template <class T>
int build_sweep(acr_ctx* h, T* F0, int nrhs, SweepPlan<T>& sp) {
    const int b = h->b, T_ = h->levels() - 1;
    const size_t bb = h->bb();
    cudaStream_t s = h->stream;
    std::vector<size_t> foff(T_ + 1), goff(T_ + 1);
    size_t tot = 0;
    for (int t = 0; t <= T_; ++t) {
        const Level& L = h->lev[t];
        foff[t] = tot;
        if (t > 0) tot += (size_t)L.m * b * nrhs;
        goff[t] = tot;
        tot += (size_t)L.ne * b * nrhs;
    }
    CK(sp.ws.alloc(tot * sizeof(T), s));
    T* base = sp.ws.template as<T>();
    auto Fp = [&](int t) { return t == 0 ? F0 : base + foff[t]; };
    auto Gp = [&](int t) { return base + goff[t]; };
    std::vector<SweepProb<T>> pr;
    // compressed blocks: the same problems on HODLR blocks (ids) instead of
    // dense block pointers
    std::vector<HSweepProb<T>> hp;
    const bool H = h->compressed;
    auto toh = [](const SweepProb<T>& p) {
        HSweepProb<T> q;
        memset(&q, 0, sizeof(q));
        q.out = p.out; q.cin = p.cin; q.ldo = p.ldo; q.ldc = p.ldc; q.ldx = p.ldx; q.alpha = p.alpha;
        q.x[0] = p.x[0]; q.x[1] = p.x[1];
        q.blk[0] = q.blk[1] = -1;
        return q;
    };
    const T* hd = H && h->band0 ? h->hdiag.template as<T>() : nullptr;
    sp.fw_g_off.assign(T_ + 1, 0); sp.fw_g_cnt.assign(T_ + 1, 0);
    sp.fw_f_off.assign(T_ + 1, 0); sp.fw_f_cnt.assign(T_ + 1, 0);
    sp.bk_off.assign(T_ + 1, 0); sp.bk_cnt.assign(T_ + 1, 0);
    auto mk = [](T* out, long long ldo, const T* cin, long long ldc, long long ldx, T alpha) {
        SweepProb<T> p;
        memset(&p, 0, sizeof(p));
        p.out = out; p.ldo = ldo; p.cin = cin; p.ldc = ldc; p.ldx = ldx; p.alpha = alpha;
        return p;
    };
    for (int t = 0; t <= T_; ++t) {
        const Level& L = h->lev[t];
        const long long ldF = (long long)L.m * b, ldG = (long long)L.ne * b;
        const T* dinv = h->P<T>(L.off_dinv);
        sp.fw_g_off[t] = pr.size();
        for (int e = 0; e < L.ne; ++e) {
            SweepProb<T> p = mk(Gp(t) + (size_t)e * b, ldG, nullptr, 0, ldF, T(1));
            p.m[0] = dinv + e * bb;
            p.x[0] = Fp(t) + (size_t)(2 * e) * b;
            pr.push_back(p);
            if (H) {
                HSweepProb<T> q = toh(p);
                q.blk[0] = h->bid[t][0][e];
                hp.push_back(q);
            }
        }
        sp.fw_g_cnt[t] = pr.size() - sp.fw_g_off[t];
        sp.fw_f_off[t] = pr.size();
        if (t < T_) {
            const T* ak = h->P<T>(L.off_ak);
            const T* ck = h->P<T>(L.off_ck);
            const long long ldN = (long long)L.nk * b;
            for (int k = 0; k < L.nk; ++k) {
                const int i = 2 * k + 1;
                SweepProb<T> p = mk(Fp(t + 1) + (size_t)k * b, ldN, Fp(t) + (size_t)i * b, ldF, ldG, T(-1));
                const size_t os = (h->band0 && t == 0) ? (size_t)b : bb;  // diagonal storage at level 0
                if (h->band0 && t == 0) p.diag_mask = 3;
                p.m[0] = ak + k * os;
                p.x[0] = Gp(t) + (size_t)k * b;
                if (i + 1 < L.m) { p.m[1] = ck + k * os; p.x[1] = Gp(t) + (size_t)(k + 1) * b; }
                pr.push_back(p);
                if (H) {
                    HSweepProb<T> q = toh(p);
                    if (h->band0 && t == 0) {
                        q.dg[0] = hd + h->hd_off[2] + (size_t)k * b;
                        if (i + 1 < L.m) q.dg[1] = hd + h->hd_off[3] + (size_t)k * b;
                    } else {
                        q.blk[0] = h->bid[t][3][k];
                        if (i + 1 < L.m) q.blk[1] = h->bid[t][4][k];
                    }
                    hp.push_back(q);
                }
            }
        }
        sp.fw_f_cnt[t] = pr.size() - sp.fw_f_off[t];
    }
    // back-substitution
    for (int t = T_; t >= 0; --t) {
        const Level& L = h->lev[t];
        const long long ldF = (long long)L.m * b, ldG = (long long)L.ne * b;
        sp.bk_off[t] = pr.size();
        if (t == T_) {
            pr.push_back(mk(Fp(t), ldF, Gp(t), ldG, 0, T(0)));
            if (H) hp.push_back(toh(pr.back()));
        } else {
            const T* xa = h->P<T>(L.off_xa);
            const T* xc = h->P<T>(L.off_xc);
            const long long ldU = (long long)L.nk * b;
            T* Un = Fp(t + 1);
            for (int i = 0; i < L.m; ++i) {
                if (i & 1) {
                    pr.push_back(mk(Fp(t) + (size_t)i * b, ldF, Un + (size_t)((i - 1) / 2) * b, ldU, 0, T(0)));
                    if (H) hp.push_back(toh(pr.back()));
                } else {
                    const int e = i / 2;
                    SweepProb<T> p = mk(Fp(t) + (size_t)i * b, ldF, Gp(t) + (size_t)e * b, ldG, ldU, T(-1));
                    if (h->band0 && t == 0) {
                        // u_j = g_j - D_j^-1 (a_j .* u_{j-1} + c_j .* u_{j+1})
                        int nt = 0;
                        if (i > 0) { p.x[nt] = Un + (size_t)((i - 2) / 2) * b; p.sx[nt] = xa + (size_t)e * b; ++nt; }
                        if (i + 1 < L.m) { p.x[nt] = Un + (size_t)(i / 2) * b; p.sx[nt] = xc + (size_t)e * b; ++nt; }
                        if (nt) p.m[0] = h->P<T>(L.off_dinv) + e * bb;
                    } else {
                        if (i > 0) { p.m[0] = xa + e * bb; p.x[0] = Un + (size_t)((i - 2) / 2) * b; }
                        if (i + 1 < L.m) { p.m[1] = xc + e * bb; p.x[1] = Un + (size_t)(i / 2) * b; }
                    }
                    pr.push_back(p);
                    if (H) {
                        HSweepProb<T> q = toh(p);
                        if (h->band0 && t == 0) {
                            int nt = 0;
                            if (i > 0) q.sx[nt++] = hd + h->hd_off[0] + (size_t)e * b;
                            if (i + 1 < L.m) q.sx[nt++] = hd + h->hd_off[1] + (size_t)e * b;
                            if (nt) q.blk[0] = h->bid[0][0][e];
                        } else {
                            if (i > 0) q.blk[0] = h->bid[t][1][e];
                            if (i + 1 < L.m) q.blk[1] = h->bid[t][2][e];
                        }
                        hp.push_back(q);
                    }
                }
            }
        }
        sp.bk_cnt[t] = pr.size() - sp.bk_off[t];
    }
    CK(sp.dprobs.alloc(pr.size() * sizeof(SweepProb<T>), s));
    CK(cudaMemcpyAsync(sp.dprobs.p, pr.data(), pr.size() * sizeof(SweepProb<T>), cudaMemcpyHostToDevice, s));
    sp.nrhs = nrhs;
    sp.hodlr = H;
    if (H) {
        // node tasks of every compressed term (pass A of the apply), in problem order
        std::vector<HTask> tasks;
        long long tcount = 0;
        sp.task_start.assign(hp.size() + 1, 0);
        for (size_t pi = 0; pi < hp.size(); ++pi) {
            sp.task_start[pi] = tasks.size();
            HSweepProb<T>& q = hp[pi];
            for (int t = 0; t < 2; ++t) {
                q.tbase[t] = -1;
                q.node_base[t] = 0;
                q.leaf_off[t] = 0;
                if (q.dg[t] || q.blk[t] < 0 || !q.x[t]) continue;
                q.tbase[t] = (int)tasks.size();
                const HBlk& hbk = h->hblks_host[q.blk[t]];
                q.node_base[t] = hbk.node_base;
                q.leaf_off[t] = hbk.leaf_off;
                for (int nu = 0; nu < h->npb; ++nu) {
                    int l = 1;
                    while (((1 << (l + 1)) - 2) <= nu) ++l;
                    const HNode& hn = h->hnodes_host[(size_t)hbk.node_base + nu];
                    HTask tk;
                    tk.node = hbk.node_base + nu;
                    tk.prob = (int)pi;
                    tk.term = t;
                    tk.level = l;
                    tk.ni = nu - ((1 << l) - 2);
                    tk.pad = 0;
                    tk.toff = hn.rank > 0 ? tcount : -1;
                    if (hn.rank > 0) tcount += (long long)hn.rank * nrhs;
                    tasks.push_back(tk);
                }
            }
        }
        sp.task_start[hp.size()] = tasks.size();
        // pass A runs only the low-rank tasks: their indices, and per problem
        // the first position in that list
        std::vector<int> alist;
        sp.a_start.assign(hp.size() + 1, 0);
        for (size_t pi = 0; pi < hp.size(); ++pi) {
            sp.a_start[pi] = alist.size();
            for (size_t ti = sp.task_start[pi]; ti < sp.task_start[pi + 1]; ++ti)
                if (tasks[ti].toff >= 0) alist.push_back((int)ti);
        }
        sp.a_start[hp.size()] = alist.size();
        // pass A per compressed term: the terms that own a low-rank node
        std::vector<int> terms;
        sp.t_start.assign(hp.size() + 1, 0);
        for (size_t pi = 0; pi < hp.size(); ++pi) {
            sp.t_start[pi] = terms.size();
            for (int t = 0; t < 2; ++t) {
                const int tb = hp[pi].tbase[t];
                if (tb < 0) continue;
                bool any = false;
                for (int nu = 0; nu < h->npb; ++nu) any |= tasks[(size_t)tb + nu].toff >= 0;
                if (any) terms.push_back(((int)pi << 1) | t);
            }
        }
        sp.t_start[hp.size()] = terms.size();
        sp.rkmax = 0;
        for (const HNode& hn : h->hnodes_host) sp.rkmax = std::max(sp.rkmax, hn.rank);
        // widest row tile of every problem: leaf + per tree level the widest
        // node (rank, or the node size when dense)
        std::vector<int> bw(h->hblks_host.size(), 0);
        for (size_t g = 0; g < bw.size(); ++g) {
            int w = h->leaf;
            for (int l = 1; l <= h->hL; ++l) {
                const int sz = b >> l;
                int m = 0;
                for (int ni = 0; ni < (1 << l); ++ni) {
                    const HNode& hn = h->hnodes_host[(size_t)h->hblks_host[g].node_base + (1 << l) - 2 + ni];
                    m = std::max(m, hn.rank < 0 ? sz : hn.rank);
                }
                w += m;
            }
            bw[g] = w;
        }
        sp.pwmax.assign(hp.size(), 0);
        for (size_t pi = 0; pi < hp.size(); ++pi)
            for (int t = 0; t < 2; ++t)
                if (hp[pi].blk[t] >= 0 && !hp[pi].dg[t]) sp.pwmax[pi] = std::max(sp.pwmax[pi], bw[hp[pi].blk[t]]);
        // largest low-rank node of every problem: pass A sizes its partial
        // sums by the launch's largest rank, not the plan's
        std::vector<int> brk(h->hblks_host.size(), 0);
        for (size_t g = 0; g < brk.size(); ++g)
            for (int nu = 0; nu < h->npb; ++nu)
                brk[g] = std::max(brk[g], h->hnodes_host[(size_t)h->hblks_host[g].node_base + nu].rank);
        sp.prk.assign(hp.size(), 0);
        for (size_t pi = 0; pi < hp.size(); ++pi)
            for (int t = 0; t < 2; ++t)
                if (hp[pi].blk[t] >= 0 && !hp[pi].dg[t]) sp.prk[pi] = std::max(sp.prk[pi], brk[hp[pi].blk[t]]);
        CK(sp.hterms.alloc(std::max<size_t>(1, terms.size()) * sizeof(int), s));
        if (!terms.empty())
            CK(cudaMemcpyAsync(sp.hterms.p, terms.data(), terms.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(sp.halist.alloc(std::max<size_t>(1, alist.size()) * sizeof(int), s));
        if (!alist.empty())
            CK(cudaMemcpyAsync(sp.halist.p, alist.data(), alist.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(sp.htasks.alloc(std::max<size_t>(1, tasks.size()) * sizeof(HTask), s));
        if (!tasks.empty())
            CK(cudaMemcpyAsync(sp.htasks.p, tasks.data(), tasks.size() * sizeof(HTask), cudaMemcpyHostToDevice, s));
        CK(sp.htbuf.alloc(std::max<long long>(1, tcount) * sizeof(T), s));
        CK(sp.hprobs.alloc(hp.size() * sizeof(HSweepProb<T>), s));
        CK(cudaMemcpyAsync(sp.hprobs.p, hp.data(), hp.size() * sizeof(HSweepProb<T>), cudaMemcpyHostToDevice, s));
        const double pbh = (double)b * nrhs * sizeof(T);
        sp.bytes = 0.0;
        for (const HSweepProb<T>& q : hp) {
            for (int t = 0; t < 2; ++t) {
                if (q.dg[t]) sp.bytes += (double)b * sizeof(T) + pbh;
                else if (q.blk[t] >= 0) sp.bytes += h->hblk_bytes[q.blk[t]] + pbh;
            }
            if (q.sx[0]) sp.bytes += (q.sx[1] ? 2.0 : 1.0) * b * sizeof(T) + (q.x[1] ? pbh : 0.0);
            if (q.cin) sp.bytes += pbh;
            sp.bytes += pbh;
        }
        CK(cudaStreamSynchronize(s));  // host tables go out of scope
        return ACR_OK;
    }
    // algorithmic traffic: every block read once, every panel operand read
    // once and every output panel written once
    const double pb = (double)b * nrhs * sizeof(T);
    sp.bytes = 0.0;
    for (const SweepProb<T>& p : pr) {
        for (int t = 0; t < 3; ++t)
            if (p.m[t]) sp.bytes += ((p.diag_mask >> t) & 1 ? (double)b * sizeof(T) : (double)bb * sizeof(T)) + pb;
        if (p.sx[0]) {  // combined mode: second panel and the two scaling vectors
            if (p.x[1]) sp.bytes += pb + (double)b * sizeof(T);
            sp.bytes += (double)b * sizeof(T);
        }
        if (p.cin) sp.bytes += pb;
        sp.bytes += pb;
    }
    return ACR_OK;
}

template <class T>
int issue_sweep(acr_ctx* h, SweepPlan<T>& sp) {
    const int b = h->b, T_ = h->levels() - 1, nrhs = sp.nrhs;
    cudaStream_t s = h->stream;
    const SweepProb<T>* dp = sp.dprobs.template as<SweepProb<T>>();
    if (sp.hodlr) {
        const HSweepProb<T>* hq = sp.hprobs.template as<HSweepProb<T>>();
        const HBlk* hb = h->hblks.as<HBlk>();
        const HNode* hn = h->hnodes.as<HNode>();
        const T* pool = h->hpool.as<T>();
        const HTask* tk = sp.htasks.template as<HTask>();
        T* tb = sp.htbuf.template as<T>();
        const int* al = sp.halist.template as<int>();
        const int* tl = sp.hterms.template as<int>();
        auto seg = [&](size_t off, size_t cnt) -> cudaError_t {
            const size_t a0 = sp.a_start[off], a1 = sp.a_start[off + cnt];
            const size_t t0 = sp.t_start[off], t1 = sp.t_start[off + cnt];
            int wmax = 0, rk = 0;
            for (size_t pi = off; pi < off + cnt; ++pi) {
                wmax = std::max(wmax, sp.pwmax[pi]);
                rk = std::max(rk, sp.prk[pi]);
            }
            return hsweep<T>(hq, (int)off, (int)cnt, tk, al, (int)a0, (int)(a1 - a0), tl + t0, (int)(t1 - t0),
                             rk, wmax, tb, hb, hn, pool, b, h->leaf, h->hL, nrhs, s);
        };
        for (int t = 0; t <= T_; ++t) {
            CK(seg(sp.fw_g_off[t], sp.fw_g_cnt[t]));
            if (sp.fw_f_cnt[t]) CK(seg(sp.fw_f_off[t], sp.fw_f_cnt[t]));
        }
        for (int t = T_; t >= 0; --t) CK(seg(sp.bk_off[t], sp.bk_cnt[t]));
    } else {
        for (int t = 0; t <= T_; ++t) {
            CK(sweep_batched<T>(dp + sp.fw_g_off[t], (int)sp.fw_g_cnt[t], b, nrhs, s));
            if (sp.fw_f_cnt[t]) CK(sweep_batched<T>(dp + sp.fw_f_off[t], (int)sp.fw_f_cnt[t], b, nrhs, s));
        }
        for (int t = T_; t >= 0; --t) CK(sweep_batched<T>(dp + sp.bk_off[t], (int)sp.bk_cnt[t], b, nrhs, s));
    }
    return ACR_OK;
}

// One application of the sweeps.  The launch sequence of a plan never changes
// (fixed buffers), so it is captured into a CUDA graph at the second
// application and replayed afterwards -- except on the NULL stream or a stream
// the caller is capturing, where the launches are issued directly.
template <class T>
int run_sweep(acr_ctx* h, SweepPlan<T>& sp) {
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    sp.evs.push_back(e0);
    CK(cudaEventCreate(&e1));
    sp.evs.push_back(e1);
    // capture from the second application on: a plan used once is never
    // captured, and every kernel's shared-memory limit has been raised by then
    // (raising it is not a stream operation)
    ++sp.applications;
    if (!sp.gexec && !sp.no_graph && sp.applications >= 2) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool legacy = s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread;
        if (legacy || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
            cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            sp.no_graph = true;  // the NULL stream cannot be captured: launch directly
        } else {
            sp.gstream = s;
            const long long c0 = launch_count();
            const int st = issue_sweep<T>(h, sp);
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(s, &g);  // always ends the capture
            // the captured launches ran nothing yet: count them per replay
            sp.glaunches = launch_count() - c0;
            count_launches((int)-sp.glaunches);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            // a capture or instantiation the driver refuses is not an error of
            // the solve: launch directly from now on
            cudaError_t ei = ee;
            if (ee == cudaSuccess) ei = cudaGraphInstantiate(&sp.gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                cudaGetLastError();
                sp.gexec = nullptr;
                sp.no_graph = true;
            }
        }
    }
    CK(cudaEventRecord(e0, s));
    if (sp.gexec) {
        CK(cudaGraphLaunch(sp.gexec, s));
        count_launches((int)sp.glaunches);
        sp.launches += sp.glaunches;
    } else {
        const long long c0 = launch_count();
        const int st = issue_sweep<T>(h, sp);
        sp.launches += launch_count() - c0;
        if (st) return st;
    }
    CK(cudaEventRecord(e1, s));
    return ACR_OK;
}

// r = f - M x with the FP64 operator copy.
struct ResidPlan {
    DevBuf dprobs;
    int nprob = 0;
};

// f == NULL builds the plain product r = M x.
int build_resid_dense(acr_ctx* h, const double* x, const double* f, double* r, int nrhs, ResidPlan& rp) {
    const int n = h->n, b = h->b;
    const size_t bb = h->bb();
    const double* oA = h->op.as<double>();
    const double* oD = oA + (size_t)n * bb;
    const double* oC = oD + (size_t)n * bb;
    const long long N = (long long)n * b;
    std::vector<SweepProb<double>> pr;
    for (int i = 0; i < n; ++i) {
        SweepProb<double> p;
        memset(&p, 0, sizeof(p));
        p.out = r + (size_t)i * b; p.ldo = N;
        p.cin = f ? f + (size_t)i * b : nullptr; p.ldc = N;
        p.ldx = N; p.alpha = f ? -1.0 : 1.0;
        p.m[0] = oD + i * bb; p.x[0] = x + (size_t)i * b;
        if (i > 0) { p.m[1] = oA + i * bb; p.x[1] = x + (size_t)(i - 1) * b; }
        if (i + 1 < n) { p.m[2] = oC + i * bb; p.x[2] = x + (size_t)(i + 1) * b; }
        pr.push_back(p);
    }
    CK(rp.dprobs.alloc(pr.size() * sizeof(SweepProb<double>), h->stream));
    CK(cudaMemcpyAsync(rp.dprobs.p, pr.data(), pr.size() * sizeof(SweepProb<double>), cudaMemcpyHostToDevice, h->stream));
    rp.nprob = (int)pr.size();
    return ACR_OK;
}

int residual(acr_ctx* h, const double* x, const double* f, double* r, int nrhs, ResidPlan* rp) {
    const int n = h->n, b = h->b;
    if (h->in_kind == ACR_BANDED) {
        const size_t N = (size_t)n * b;
        const double* o = h->op.as<double>();
        CK(resid_banded(n, b, o, o + N, o + 2 * N, o + 3 * N, o + 4 * N, x, f, r, nrhs, h->stream));
    } else {
        CK(sweep_batched<double>(rp->dprobs.as<SweepProb<double>>(), rp->nprob, b, nrhs, h->stream));
    }
    return ACR_OK;
}

// ---------------------------------------------------------------------------
// Refinement.  The preconditioner z = M^-1 v is one pass of the solve sweeps
// in the factor's precision Tf; the residual and every Krylov quantity are
// FP64 with the original operator.
// ---------------------------------------------------------------------------
template <class Tf>
struct Precond {
    acr_ctx* h = nullptr;
    SweepPlan<Tf> sp;
    DevBuf buf;
    long long NQ = 0;
    int init(acr_ctx* hh, int nrhs) {
        h = hh;
        NQ = (long long)h->n * h->b * nrhs;
        CK(buf.alloc(NQ * sizeof(Tf), h->stream));
        return build_sweep<Tf>(h, buf.as<Tf>(), nrhs, sp);
    }
    int apply(const double* v, double* z) {
        cudaStream_t s = h->stream;
        if constexpr (sizeof(Tf) == 4) {
            CK(convert_d2f(v, buf.as<float>(), NQ, s));
            int st = run_sweep<float>(h, sp);
            if (st) return st;
            CK(convert_f2d(buf.as<float>(), z, NQ, s));
        } else {
            CK(cudaMemcpyAsync(buf.p, v, NQ * 8, cudaMemcpyDeviceToDevice, s));
            int st = run_sweep<double>(h, sp);
            if (st) return st;
            CK(cudaMemcpyAsync(z, buf.p, NQ * 8, cudaMemcpyDeviceToDevice, s));
        }
        return ACR_OK;
    }
};

// FP64 operator products on fixed buffers: res: r = f - M x;  mv: w = M z.
struct Oper {
    acr_ctx* h = nullptr;
    int nrhs = 0;
    const double *x = nullptr, *f = nullptr;
    double *r = nullptr, *z = nullptr, *w = nullptr;
    ResidPlan prs, pmv;
    int init(acr_ctx* hh, const double* x_, const double* f_, double* r_, double* z_, double* w_, int nq) {
        h = hh; x = x_; f = f_; r = r_; z = z_; w = w_; nrhs = nq;
        if (h->in_kind != ACR_BANDED) {
            int st = build_resid_dense(h, x, f, r, nrhs, prs);
            if (st) return st;
            if (z) return build_resid_dense(h, z, nullptr, w, nrhs, pmv);
        }
        return ACR_OK;
    }
    int res() { return residual(h, x, f, r, nrhs, &prs); }
    int mv(const double* zin) {  // w = M zin (zin must be z for dense operators)
        if (h->in_kind == ACR_BANDED) return residual(h, zin, nullptr, w, nrhs, nullptr);
        if (zin != z) CK(cudaMemcpyAsync(z, zin, (size_t)h->n * h->b * nrhs * 8, cudaMemcpyDeviceToDevice, h->stream));
        return residual(h, z, nullptr, w, nrhs, &pmv);
    }
};

template <class Tf>
int refine(acr_ctx* h, const double* f, double* x, int nrhs, bool x0_given, std::vector<double>& rel,
           int& iters) {
    const long long N = (long long)h->n * h->b, NQ = N * nrhs;
    cudaStream_t s = h->stream;
    const double tol = h->opts.ir_tol;
    const int maxit = std::max(1, h->opts.ir_max_iter);
    const int method = h->opts.refine;
    Precond<Tf> P;
    int st = P.init(h, nrhs);
    if (st) return st;
    DevBuf r, zb, wb, ws, sq, coef;
    CK(r.alloc(NQ * 8, s));
    CK(zb.alloc(NQ * 8, s));
    CK(wb.alloc(NQ * 8, s));
    CK(ws.alloc((size_t)64 * nrhs * 1024 * 8, s));
    CK(sq.alloc((size_t)64 * nrhs * 8, s));
    CK(coef.alloc((size_t)64 * nrhs * 8, s));
    Oper op;
    if ((st = op.init(h, x, f, r.as<double>(), zb.as<double>(), wb.as<double>(), nrhs))) return st;
    std::vector<double> fn2(nrhs), hs(64 * nrhs);
    CK(col_sumsq(f, N, nrhs, ws.as<double>(), sq.as<double>(), s));
    CK(cudaMemcpyAsync(fn2.data(), sq.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
    iters = 0;
    if (!x0_given) {
        if ((st = P.apply(f, x))) return st;
        iters = 1;
    }
    // A column whose residual has reached tol is frozen: later corrections
    // leave it untouched, so every column follows the iteration it would
    // follow alone whatever other columns share the call (the kernels'
    // per-column arithmetic does not depend on nrhs).
    std::vector<char> frozen(nrhs, 0);
    auto check = [&](bool& conv) -> int {
        int e = op.res();
        if (e) return e;
        CK(col_sumsq(r.as<double>(), N, nrhs, ws.as<double>(), sq.as<double>(), s));
        CK(cudaMemcpyAsync(hs.data(), sq.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        conv = true;
        for (int q = 0; q < nrhs; ++q) {
            rel[q] = fn2[q] > 0 ? std::sqrt(hs[q] / fn2[q]) : std::sqrt(hs[q]);
            if (rel[q] <= tol) frozen[q] = 1;
            if (!frozen[q]) conv = false;
        }
        return ACR_OK;
    };
    bool conv = false;
    if ((st = check(conv))) return st;
    if (conv || method == ACR_REFINE_NONE) return conv ? ACR_OK : fail(ACR_ERR_NOT_CONVERGED, "residual %g above ir_tol %g and refinement is off", *std::max_element(rel.begin(), rel.end()), tol);
    if (method == ACR_REFINE_IR) {
        std::vector<double> mask(nrhs);
        while (iters < maxit && !conv) {
            if ((st = P.apply(r.as<double>(), zb.as<double>()))) return st;
            ++iters;
            for (int q = 0; q < nrhs; ++q) mask[q] = frozen[q] ? 0.0 : 1.0;
            CK(cudaMemcpyAsync(coef.p, mask.data(), nrhs * 8, cudaMemcpyHostToDevice, s));
            CK(multi_axpy(x, zb.as<double>(), 1, coef.as<double>(), N, nrhs, s));
            if ((st = check(conv))) return st;
        }
    } else {
        // restarted FGMRES(m), right preconditioned, one Krylov space per column
        const int m = std::min(ACR_FGMRES_RESTART, maxit);
        DevBuf V, Z, hacc, sq2, hsb, needb;
        CK(V.alloc((size_t)(m + 1) * NQ * 8, s));
        CK(Z.alloc((size_t)m * NQ * 8, s));
        CK(hacc.alloc((size_t)(m + 1) * nrhs * 8, s));
        CK(sq2.alloc((size_t)64 * nrhs * 8, s));
        CK(hsb.alloc((size_t)nrhs * 8, s));
        CK(needb.alloc((size_t)nrhs * sizeof(int), s));
        double* Vp = V.as<double>();
        double* Zp = Z.as<double>();
        std::vector<double> H((size_t)nrhs * (m + 1) * m), g((size_t)nrhs * (m + 1)), cs((size_t)nrhs * m),
            sn((size_t)nrhs * m), sc(nrhs), hh((size_t)(m + 1) * nrhs), y((size_t)m * nrhs);
        auto Hq = [&](int q, int i, int j) -> double& { return H[((size_t)q * (m + 1) + i) * m + j]; };
        while (iters < maxit && !conv) {
            std::fill(H.begin(), H.end(), 0.0);
            std::fill(g.begin(), g.end(), 0.0);
            // a frozen column restarts from a zero vector: its Krylov space
            // stays {0}, its y is 0 and x keeps its value
            std::vector<int> jdq(nrhs, 0);
            for (int q = 0; q < nrhs; ++q) {
                const double beta = frozen[q] ? 0.0 : std::sqrt(hs[q]);
                g[(size_t)q * (m + 1)] = beta;
                sc[q] = beta > 0 ? 1.0 / beta : 0.0;
            }
            CK(cudaMemcpyAsync(coef.p, sc.data(), nrhs * 8, cudaMemcpyHostToDevice, s));
            CK(col_scale(Vp, r.as<double>(), coef.as<double>(), N, nrhs, s));
            int jd = 0;
            for (int j = 0; j < m && iters < maxit; ++j) {
                double* Vj = Vp + (size_t)j * NQ;
                double* Zj = Zp + (size_t)j * NQ;
                if ((st = P.apply(Vj, Zj))) return st;
                ++iters;
                if ((st = op.mv(Zj))) return st;
                double* w = wb.as<double>();
                // classical Gram-Schmidt: h1 = V^T w with |w|^2 in one read of
                // V, w -= V h1 with |w'|^2 in a second.  A column repeats the
                // pass (h2 = V^T w', w' -= V h2, decided on the device) only
                // where the first cancelled the norm below 1e-2 |w|: a pass
                // leaves w' off orthogonal by about u |w| / |w'|, so above
                // that ratio the basis stays orthogonal to ~1e-12, well
                // within the refinement targets.  Column j of H (h1 [+ h2])
                // comes back with the final norm.
                const int nv = j + 1;
                double* sqp = sq.as<double>();
                double* sq2p = sq2.as<double>();
                CK(multi_dot_self(Vp, nv, w, N, nrhs, ws.as<double>(), sqp, s));
                CK(gs_coef(sqp, coef.as<double>(), hacc.as<double>(), nv * nrhs, true, s));
                CK(gs_update_norm(w, Vp, nv, coef.as<double>(), N, nrhs, nullptr, ws.as<double>(),
                                  sq2p + (size_t)63 * nrhs, s));
                if (N <= 4LL * 1024 * 1024) {
                    CK(gs_reorth(w, Vp, nv, sqp + (size_t)nv * nrhs, sq2p + (size_t)63 * nrhs, 1e-4, sq2p,
                                 coef.as<double>(), hacc.as<double>(), needb.as<int>(), hsb.as<double>(), N, nrhs,
                                 ws.as<double>(), s));
                } else {  // unconditional second pass
                    CK(multi_dot(Vp, nv, w, N, nrhs, ws.as<double>(), sq2p, s));
                    CK(gs_coef(sq2p, coef.as<double>(), hacc.as<double>(), nv * nrhs, false, s));
                    CK(gs_update_norm(w, Vp, nv, coef.as<double>(), N, nrhs, nullptr, ws.as<double>(), hsb.as<double>(),
                                      s));
                }
                CK(cudaMemcpyAsync(hh.data(), hacc.p, (size_t)(j + 1) * nrhs * 8, cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(hs.data(), hsb.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i)
                    for (int q = 0; q < nrhs; ++q) Hq(q, i, j) = hh[(size_t)i * nrhs + q];
                bool all = true;
                for (int q = 0; q < nrhs; ++q) {
                    const double hn = std::sqrt(hs[q]);
                    Hq(q, j + 1, j) = hn;
                    sc[q] = hn > 0 ? 1.0 / hn : 0.0;
                    // Givens rotations on column j of this column's Hessenberg
                    for (int i = 0; i < j; ++i) {
                        const double c = cs[(size_t)q * m + i], sv = sn[(size_t)q * m + i];
                        const double a = Hq(q, i, j), bq = Hq(q, i + 1, j);
                        Hq(q, i, j) = c * a + sv * bq;
                        Hq(q, i + 1, j) = -sv * a + c * bq;
                    }
                    const double a = Hq(q, j, j), bq = Hq(q, j + 1, j);
                    const double rr = std::hypot(a, bq);
                    const double c = rr > 0 ? a / rr : 1.0, sv = rr > 0 ? bq / rr : 0.0;
                    cs[(size_t)q * m + j] = c;
                    sn[(size_t)q * m + j] = sv;
                    Hq(q, j, j) = rr;
                    Hq(q, j + 1, j) = 0.0;
                    double* gq = &g[(size_t)q * (m + 1)];
                    gq[j + 1] = -sv * gq[j];
                    gq[j] = c * gq[j];
                    const double est = fn2[q] > 0 ? std::fabs(gq[j + 1]) / std::sqrt(fn2[q]) : std::fabs(gq[j + 1]);
                    // a column stops its cycle at its first step below the
                    // target; later steps do not enter its update
                    if (jdq[q] == 0 && (frozen[q] || est <= 0.5 * tol)) jdq[q] = j + 1;
                    if (jdq[q] == 0) all = false;
                }
                CK(cudaMemcpyAsync(coef.p, sc.data(), nrhs * 8, cudaMemcpyHostToDevice, s));
                CK(col_scale(Vp + (size_t)(j + 1) * NQ, w, coef.as<double>(), N, nrhs, s));
                jd = j + 1;
                if (all) break;
            }
            // y = R^-1 g per column, x += Z y
            for (int q = 0; q < nrhs; ++q) {
                const double* gq = &g[(size_t)q * (m + 1)];
                const int jq = jdq[q] > 0 ? jdq[q] : jd;
                for (int i = jd - 1; i >= jq; --i) y[(size_t)i * nrhs + q] = 0.0;
                for (int i = jq - 1; i >= 0; --i) {
                    double t = gq[i];
                    for (int k = i + 1; k < jq; ++k) t -= Hq(q, i, k) * y[(size_t)k * nrhs + q];
                    const double d = Hq(q, i, i);
                    y[(size_t)i * nrhs + q] = std::fabs(d) > 0 ? t / d : 0.0;
                }
            }
            CK(cudaMemcpyAsync(coef.p, y.data(), (size_t)jd * nrhs * 8, cudaMemcpyHostToDevice, s));
            CK(multi_axpy(x, Zp, jd, coef.as<double>(), N, nrhs, s));
            if ((st = check(conv))) return st;
        }
    }
    {
        CK(cudaStreamSynchronize(s));
        std::lock_guard<std::mutex> lk(h->mu);
        h->st.sweep_ms += P.sp.elapsed_ms();
        h->st.sweep_bytes += P.sp.bytes * P.sp.passes();
        h->st.sweep_launches += P.sp.launches;
        h->st.sweep_passes += P.sp.passes();
    }
    if (!conv)
        return fail(ACR_ERR_NOT_CONVERGED, "refinement took %d preconditioner solves without ||r||/||b|| <= %g (worst %g)",
                    iters, tol, *std::max_element(rel.begin(), rel.end()));
    return ACR_OK;
}

int solve_impl(acr_ctx* h, double* B, int nrhs, double* resid_out, int* iters_out) {
    const int n = h->n, b = h->b;
    const long long N = (long long)n * b;
    cudaStream_t s = h->stream;
    const size_t bytes = (size_t)N * nrhs * 8;
    const bool dev = ptr_kind(B, h->dev) == PTR_DEVICE;
    DevBuf dB;
    double* f = B;
    Events evown;
    cudaEvent_t e0, e1;
    CK(evown.make(&e0));
    CK(evown.make(&e1));
    if (!dev) {
        CK(dB.alloc(bytes, s));
        CK(cudaMemcpyAsync(dB.p, B, bytes, cudaMemcpyHostToDevice, s));
        f = dB.as<double>();
    }
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->st.sweep_ms = 0.0;
        h->st.sweep_bytes = 0.0;
        h->st.sweep_launches = 0;
        h->st.sweep_passes = 0;
    }
    const long long lc0 = launch_count();
    CK(cudaEventRecord(e0, s));
    int iters = 0, status = ACR_OK;
    std::vector<double> rel(nrhs, 0.0);
    {
        DevBuf x, f0;
        CK(x.alloc(bytes, s));
        if (h->prec == ACR_FP64) {
            // direct FP64 sweep; refinement only if the residual misses ir_tol
            SweepPlan<double> sp;
            int st = build_sweep<double>(h, x.as<double>(), nrhs, sp);
            if (st) return st;
            CK(cudaMemcpyAsync(x.p, f, bytes, cudaMemcpyDeviceToDevice, s));
            if ((st = run_sweep<double>(h, sp))) return st;
            CK(cudaStreamSynchronize(s));
            {
                std::lock_guard<std::mutex> lk(h->mu);
                h->st.sweep_ms += sp.elapsed_ms();
                h->st.sweep_bytes += sp.bytes;
                h->st.sweep_launches += sp.launches;
                h->st.sweep_passes += 1;
            }
            status = refine<double>(h, f, x.as<double>(), nrhs, true, rel, iters);
        } else {
            status = refine<float>(h, f, x.as<double>(), nrhs, false, rel, iters);
        }
        if (status != ACR_OK && status != ACR_ERR_NOT_CONVERGED) return status;
        CK(cudaMemcpyAsync(f, x.p, bytes, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaEventRecord(e1, s));
    if (!dev) CK(cudaMemcpyAsync(B, dB.p, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->st.solve_ms = ms;
        h->st.launches_solve = launch_count() - lc0;
        h->st.ir_iters = iters;
        double mx = 0.0;
        for (double v : rel) mx = std::max(mx, v);
        h->st.ir_resid_max = mx;
    }
    if (resid_out) memcpy(resid_out, rel.data(), sizeof(double) * nrhs);
    if (iters_out) *iters_out = iters;
    return status;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void acr_default_opts(acr_opts* o) {
    if (o) default_opts(o);
}

const char* acr_last_error(void) { return g_err.c_str(); }

int acr_factor_bytes(int nblk, int blksz, double tol, const acr_opts* o, size_t* bytes) {
    (void)tol;
    if (nblk < 1 || blksz < 1 || !bytes) return fail(ACR_ERR_INVALID_ARG, "bad arguments");
    acr_opts op;
    if (o) op = *o; else default_opts(&op);
    const size_t es = op.precision == ACR_FP64 ? 8 : 4;
    std::vector<Level> lev;
    size_t arena = plan_levels(nblk, blksz, es, lev);
    const size_t N = (size_t)nblk * blksz;
    const size_t opb = op.input_kind == ACR_BANDED ? 5 * N * 8 : 3 * (size_t)nblk * blksz * blksz * 8;
    *bytes = arena + opb;
    return ACR_OK;
}

int acr_solve_bytes(int nblk, int blksz, int nrhs, const acr_opts* o, size_t* bytes) {
    if (nblk < 1 || blksz < 1 || nrhs < 0 || !bytes) return fail(ACR_ERR_INVALID_ARG, "bad arguments");
    acr_opts op;
    if (o) op = *o; else default_opts(&op);
    const size_t es = op.precision == ACR_FP64 ? 8 : 4;
    const size_t NQ = (size_t)nblk * blksz * (size_t)nrhs;
    const int maxit = op.ir_max_iter > 0 ? op.ir_max_iter : 20;
    const size_t m = op.refine == ACR_REFINE_FGMRES ? (size_t)std::min(ACR_FGMRES_RESTART, maxit) : 0;
    // FP64 vectors: staged B, x, r, z, w and the FGMRES bases V (m + 1) and Z (m);
    // factor-precision vectors: the preconditioner's input, its level vectors
    // (about 2), the node products of the compressed apply (bounded by 2) and
    // the direct sweep's of FP64 mode (2); Gram-Schmidt partials; tables
    *bytes = NQ * (8 * (2 * m + 6) + 7 * es) + 2 * (size_t)64 * 1024 * 8 * nrhs + ((size_t)64 << 20);
    return ACR_OK;
}

}  // extern "C"

namespace {
// Freed stream-ordered memory stays in the device's default pool (up to
// 64 GiB, or the process's own higher setting), so that repeated
// factorizations and the per-call temporaries reuse mapped memory instead of
// mapping it again on every call.  A property of this process's pool only.
void keep_pool_memory(int dev) {
    static std::mutex mu;
    static std::set<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(dev)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t cur = 0, want = 64ull << 30;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < want)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
    }
    cudaGetLastError();
    done.insert(dev);
}
}  // namespace

extern "C" {

int acr_factor_ex(int nblk, int blksz, const double* A, const double* D, const double* C, double tol,
                  const acr_opts* o, acr_handle* out) {
    if (!out) return fail(ACR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nblk < 1 || blksz < 1) return fail(ACR_ERR_INVALID_ARG, "nblk and blksz must be >= 1 (got %d, %d)", nblk, blksz);
    if (!D || (nblk > 1 && (!A || !C))) return fail(ACR_ERR_INVALID_ARG, "NULL block array");
    if ((size_t)nblk * blksz > (size_t)1 << 31) return fail(ACR_ERR_INVALID_ARG, "system too large");
    acr_opts op;
    if (o) op = *o; else default_opts(&op);
    if (op.precision < ACR_FP64 || op.precision > ACR_FP32_IR) return fail(ACR_ERR_INVALID_ARG, "unknown precision %d", op.precision);
    if (op.input_kind != ACR_DENSE && op.input_kind != ACR_BANDED) return fail(ACR_ERR_INVALID_ARG, "unknown input_kind %d", op.input_kind);
    if (op.m_stop > 1) return fail(ACR_ERR_INVALID_ARG, "m_stop > 1 is not supported (reduction runs to one block)");
    if (op.h_levels < -1) return fail(ACR_ERR_INVALID_ARG, "h_levels must be >= -1 (got %d)", op.h_levels);
    if (op.ir_max_iter <= 0) op.ir_max_iter = 20;
    if (!(op.ir_tol > 0)) op.ir_tol = 1e-8;
    {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaGetLastError();
        const double* arr[3] = {A, D, C};
        const char* nm[3] = {"A", "D", "C"};
        for (int q = 0; q < 3; ++q)
            if ((q == 1 || nblk > 1) && ptr_kind(arr[q], cur) == PTR_OTHER_DEVICE)
                return fail(ACR_ERR_INVALID_ARG, "%s is device memory of another GPU than the current device %d", nm[q], cur);
    }
    acr_ctx* h = new (std::nothrow) acr_ctx();
    if (!h) return fail(ACR_ERR_OOM, "host allocation failed");
    h->n = nblk; h->b = blksz; h->prec = op.precision; h->in_kind = op.input_kind; h->tol = tol; h->opts = op;
    cudaGetDevice(&h->dev);
    keep_pool_memory(h->dev);
    if (op.stream) {
        h->stream = static_cast<cudaStream_t>(op.stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(ACR_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    h->es = op.precision == ACR_FP64 ? 8 : 4;
    // ranks below the factor's own rounding level only encode noise
    // truncation floor: a few units of the factor's rounding (FP32: 9.5e-7;
    // 32 eps was measured to cost four more FGMRES solves on the indefinite
    // 1M Helmholtz problem than 8 eps, for 15% less storage)
    h->tol_eff = tol > 0 ? std::max(tol, (h->es == 8 ? 32 * 2.220446049250313e-16 : 8 * 1.1920929e-7)) : 0.0;
    h->st.nblk = nblk; h->st.blksz = blksz; h->st.precision = op.precision; h->st.compressed = 0;
    int st = (h->es == 8) ? run_factor<double>(h, A, D, C) : run_factor<float>(h, A, D, C);
    if (st != ACR_OK) {
        std::string msg = g_err;
        cudaStreamSynchronize(h->stream);
        delete h;
        g_err = msg;
        return st;
    }
    h->st.levels = h->levels();
    *out = h;
    return ACR_OK;
}

int acr_factor(int nblk, int blksz, const double* A, const double* D, const double* C, double tol, acr_handle* out) {
    return acr_factor_ex(nblk, blksz, A, D, C, tol, nullptr, out);
}

int acr_solve_ex(acr_handle h, double* B, int nrhs, double* resid_out, int* iters_out) {
    if (!h) return fail(ACR_ERR_INVALID_ARG, "NULL handle");
    if (nrhs < 0 || (nrhs > 0 && !B)) return fail(ACR_ERR_INVALID_ARG, "bad right-hand side");
    if (iters_out) *iters_out = 0;
    if (nrhs == 0) return ACR_OK;
    if (ptr_kind(B, h->dev) == PTR_OTHER_DEVICE)
        return fail(ACR_ERR_INVALID_ARG, "B is device memory of another GPU than the handle's device %d", h->dev);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->dev) cudaSetDevice(h->dev);
    int st = solve_impl(h, B, nrhs, resid_out, iters_out);
    if (prev != h->dev) cudaSetDevice(prev);
    return st;
}

int acr_solve(acr_handle h, double* B, int nrhs) { return acr_solve_ex(h, B, nrhs, nullptr, nullptr); }

void acr_free(acr_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    delete h;
}

int acr_stats(acr_handle h, acr_stats_t* s) {
    if (!h || !s) return fail(ACR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(h->mu);
    *s = h->st;
    return ACR_OK;
}

}  // extern "C"

namespace {
template <class T>
int lowrank_truncate_impl(int count, int s, int R, const double* dU, const double* dV, double tol, int sketch,
                          double* dUo, double* dVo, int* dranks, std::vector<int>& hr, cudaStream_t st) {
    using namespace acr;
    const size_t nel = (size_t)count * s * R;
    DevBuf bU, bV, bVo, bUo, bW, bR2, bP;
    const T *U, *V;
    T *Vo, *Uo;
    if (sizeof(T) == 8) {
        U = reinterpret_cast<const T*>(dU);
        V = reinterpret_cast<const T*>(dV);
        Vo = reinterpret_cast<T*>(dVo);
        Uo = reinterpret_cast<T*>(dUo);
    } else {
        CK(bU.alloc(nel * sizeof(T), st));
        CK(bV.alloc(nel * sizeof(T), st));
        CK(bVo.alloc(nel * sizeof(T), st));
        CK(bUo.alloc(nel * sizeof(T), st));
        CK(convert_d2f(dU, bU.as<float>(), (long long)nel, st));
        CK(convert_d2f(dV, bV.as<float>(), (long long)nel, st));
        U = reinterpret_cast<const T*>(bU.p);
        V = reinterpret_cast<const T*>(bV.p);
        Vo = reinterpret_cast<T*>(bVo.p);
        Uo = reinterpret_cast<T*>(bUo.p);
    }
    RPT<T> P;
    memset(&P, 0, sizeof(P));
    P.U.base = U;
    P.U.gs = (long long)s * R;
    P.U.ld = s;
    P.V = P.U;
    P.V.base = V;
    P.Vout = P.U;
    P.Vout.base = Vo;
    P.s = s;
    P.R = R;
    P.wout = R;
    P.ni = 1;
    P.ng = count;
    const int kcap = std::min(s, R);
    if (hrecomp_smem_bytes(s, R, sizeof(T)) > 227 * 1024)
        return fail(ACR_ERR_INVALID_ARG, "s = %d, R = %d: the panels exceed the truncation kernel's shared memory", s, R);
    int ks = sketch;
    if (ks > 0 && (ks >= std::min(s, R) || hrecomp_sketch_smem_bytes(s, R, ks, sizeof(T)) > 227 * 1024)) ks = 0;
    CK(hrecomp_t<T>(P, dranks, tol, kcap, ks, st));
    CK(cudaMemcpyAsync(hr.data(), dranks, count * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<RProb<T>> redo;
    std::vector<int> at;
    for (int i = 0; i < count; ++i)
        if (hr[i] < 0) {
            RProb<T> q;
            q.U = U + (size_t)i * s * R;
            q.V = V + (size_t)i * s * R;
            q.Vout = Vo + (size_t)i * s * R;
            q.ldu = q.ldv = q.ldvo = s;
            q.s = s;
            q.R = R;
            q.wout = R;
            redo.push_back(q);
            at.push_back(i);
        }
    if (!redo.empty()) {
        CK(bP.alloc(redo.size() * sizeof(RProb<T>), st));
        CK(bR2.alloc(redo.size() * sizeof(int), st));
        CK(cudaMemcpyAsync(bP.p, redo.data(), redo.size() * sizeof(RProb<T>), cudaMemcpyHostToDevice, st));
        CK(hrecomp<T>(bP.as<RProb<T>>(), (int)redo.size(), s, R, bR2.as<int>(), tol, kcap, st));
        std::vector<int> r2(redo.size());
        CK(cudaMemcpyAsync(r2.data(), bR2.p, r2.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (size_t j = 0; j < at.size(); ++j) hr[at[j]] = -2 - r2[j];  // -2 - rank: resolved by the exact pass
        std::vector<int> fixed(hr);
        for (int& v : fixed) v = v <= -2 ? -2 - v : v;
        CK(cudaMemcpyAsync(dranks, fixed.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    CK(bW.alloc((size_t)count * R * R * sizeof(T), st));
    CK(lowrank_apply<T>(U, V, Vo, bW.as<T>(), Uo, count, s, R, st));
    if (sizeof(T) == 4) {
        CK(convert_f2d(bVo.as<float>(), dVo, (long long)nel, st));
        CK(convert_f2d(bUo.as<float>(), dUo, (long long)nel, st));
    }
    CK(cudaStreamSynchronize(st));
    return ACR_OK;
}
}  // namespace

extern "C" int acr_lowrank_truncate(int count, int s, int R, const double* U, const double* V, double tol,
                                    int precision, int sketch, double* Uout, double* Vout, int* ranks,
                                    int* exact_redo) {
    if (count < 0 || s < 1 || R < 1) return fail(ACR_ERR_INVALID_ARG, "count >= 0, s >= 1 and R >= 1 required");
    if (count == 0) {
        if (exact_redo) *exact_redo = 0;
        return ACR_OK;
    }
    if (!U || !V || !Uout || !Vout || !ranks) return fail(ACR_ERR_INVALID_ARG, "NULL argument");
    if (!(tol >= 0.0) || tol >= 1.0) return fail(ACR_ERR_INVALID_ARG, "tol must lie in [0, 1) (got %g)", tol);
    if (precision != ACR_FP64 && precision != ACR_FP32TC_IR && precision != ACR_FP32_IR)
        return fail(ACR_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (sketch < 0) return fail(ACR_ERR_INVALID_ARG, "sketch must be >= 0 (got %d)", sketch);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACR_ERR_CUDA, "no usable CUDA device");
    }
    const void* ptrs[5] = {U, V, Uout, Vout, ranks};
    PtrKind pk[5];
    for (int i = 0; i < 5; ++i) {
        pk[i] = ptr_kind(ptrs[i], dev);
        if (pk[i] == PTR_OTHER_DEVICE) return fail(ACR_ERR_INVALID_ARG, "argument %d is memory of another GPU", i + 1);
    }
    const size_t nel = (size_t)count * s * R;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACR_ERR_CUDA, "stream creation failed");
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } sg{st};
    int rc = ACR_OK;
    std::vector<int> hr(count);
    {
        DevBuf b[5];
        double* d[4];
        int* dr = ranks;
        for (int i = 0; i < 4; ++i) {
            d[i] = const_cast<double*>(static_cast<const double*>(ptrs[i]));
            if (pk[i] != PTR_DEVICE) {
                if (b[i].alloc(nel * 8, st) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ACR_ERR_OOM, "device allocation failed");
                }
                if (i < 2 && cudaMemcpyAsync(b[i].p, ptrs[i], nel * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ACR_ERR_CUDA, "copy failed");
                }
                d[i] = b[i].as<double>();
            }
        }
        if (pk[4] != PTR_DEVICE) {
            if (b[4].alloc((size_t)count * sizeof(int), st) != cudaSuccess) {
                cudaGetLastError();
                return fail(ACR_ERR_OOM, "device allocation failed");
            }
            dr = b[4].as<int>();
        }
        rc = precision == ACR_FP64
                 ? lowrank_truncate_impl<double>(count, s, R, d[0], d[1], tol, sketch, d[2], d[3], dr, hr, st)
                 : lowrank_truncate_impl<float>(count, s, R, d[0], d[1], tol, sketch, d[2], d[3], dr, hr, st);
        if (rc == ACR_OK) {
            bool ok = true;
            if (pk[2] != PTR_DEVICE) ok &= cudaMemcpyAsync(Uout, d[2], nel * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
            if (pk[3] != PTR_DEVICE) ok &= cudaMemcpyAsync(Vout, d[3], nel * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
            if (pk[4] != PTR_DEVICE)
                ok &= cudaMemcpyAsync(ranks, dr, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
            ok &= cudaStreamSynchronize(st) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                rc = fail(ACR_ERR_CUDA, "copy back failed");
            }
        }
    }
    if (exact_redo) {
        int c = 0;
        for (int v : hr) c += v <= -2;
        *exact_redo = c;
    }
    return rc;
}
