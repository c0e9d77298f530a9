// hred.cuh -- host driver of the reduction levels carried out in HODLR
// arithmetic (included by acr_api.cu only).
//
// Section 3 reduces every level with the blocks held as H-matrices: the
// eliminated diagonal blocks are inverted in H-arithmetic, and the products
// and sums of the Schur complement (Eq. "fund") are H-products and H-sums
// truncated to the tolerance.  Here each block is HODLR in the "stacked"
// format of k_harith.cu (dense leaves; per tree level l two b x K_l panels
// U_l, V_l whose row ranges are the nodes), and a batch of blocks (all the
// blocks one step of one level needs) is one HSet.  Every step is a short
// sequence of batched launches: products of row ranges of the panels
// (k_vgemm), truncations (k_hrecomp), copies (k_hcopy).
//
// Inverse of a HODLR block M (bottom-up Woodbury).  With G the inverse of the
// block diagonal of M at tree level l (known from the previous step; level L:
// the leaf inverses, pivoted Gauss-Jordan in FP64), each parent p at level
// l - 1 with children a, c and off-diagonal nodes U_a V_a^T, U_c V_c^T:
//     P = G U_l,  Q = G^T V_l,  T_nu = V_l[nu]^T P[nu],
//     K_p = [[I, T_c], [T_a, I]],   Kinv_p = K_p^-1  (FP64, pivoted),
//     new nodes of the inverse:  U'_a = -P_a Kinv11,  U'_c = -P_c Kinv22,  V' = Q,
//     update of the children:    G_a += Yn_a Q_a^T,  G_c += Yn_c Q_c^T,
//                                Yn_a = -P_a Kinv12,  Yn_c = -P_c Kinv21.
// The updates are kept as pending terms (applied inside the later products
// with G); at the end every node of level l collects [U'_l | Yn_{l-1} .. Yn_1]
// x [Q_l | Q_{l-1} .. Q_1]^T and is truncated once, and the leaves absorb
// sum_l Yn_l Q_l^T.
//
// Product C = A B of two HODLR blocks (same tree).  With BD_l(X) the block
// diagonal of X at tree level l, node nu of level l of C (rows R, columns R'
// of the sibling) is
//     [BD_l(A) U^B_l | U^A_l | (U^A_m W_m)_{m < l}] x [V^B_l | BD_l(B)^T V^A_l | (V^B_m)_{m < l}]^T
// restricted to (R, R'), where W_m (per node of level m) = V^A_m[sib]^T U^B_m[sib]
// collects the products that pass through the ancestors' off-diagonal
// blocks.  Leaves: A_leaf B_leaf + sum_m (U^A_m W_m)[leaf] V^B_m[leaf]^T.
// A sum of products (the Schur complement D - A1 B1 - A2 B2) concatenates the
// factors of all terms and truncates each node once.
#pragma once

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "acr_internal.h"

namespace acr {
namespace hred {

constexpr int HMAXL_TREE = HMAXL - 2;  // deepest HODLR tree

// ---------------------------------------------------------------- buffers
// Device ranges every descriptor must stay inside: each operand a descriptor
// names is checked on the host before upload, so an indexing mistake in this
// driver becomes an error return instead of an out-of-bounds access.  A
// buffer leaves the set when it is released.
struct Ranges {
    std::vector<std::pair<uintptr_t, uintptr_t>> r;
    void add(const void* p, size_t bytes) {
        if (!p || !bytes) return;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
        auto it = std::lower_bound(r.begin(), r.end(), std::make_pair(lo, (uintptr_t)0));
        r.insert(it, {lo, lo + bytes});
    }
    void remove(const void* p) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
        auto it = std::lower_bound(r.begin(), r.end(), std::make_pair(lo, (uintptr_t)0));
        if (it != r.end() && it->first == lo) r.erase(it);
    }
    // Live device buffers never overlap, so the only candidate is the last
    // range starting at or below p.
    bool has(const void* p, size_t bytes) const {
        if (!bytes) return true;
        if (!p) return false;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(p), hi = lo + bytes;
        auto it = std::upper_bound(r.begin(), r.end(), std::make_pair(lo, UINTPTR_MAX));
        if (it == r.begin()) return false;
        --it;
        return it->first <= lo && hi <= it->second;
    }
};

struct HBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    size_t bytes = 0;
    Ranges* rs = nullptr;
    HBuf() = default;
    HBuf(const HBuf&) = delete;
    HBuf& operator=(const HBuf&) = delete;
    ~HBuf() { release(); }
    void release() {
        if (p) {
            if (rs) rs->remove(p);
            cudaFreeAsync(p, s);
        }
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n, cudaStream_t st, Ranges* r = nullptr) {
        release();
        s = st;
        bytes = std::max<size_t>(n, 16);
        const cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        rs = r;
        if (rs) rs->add(p, bytes);
        return e;
    }
};

// A sequence of launches whose descriptors are uploaded in one copy.
struct Plan {
    std::vector<unsigned char> h;
    std::vector<std::function<cudaError_t(const unsigned char*)>> steps;
    size_t put(const void* src, size_t n) {
        const size_t off = (h.size() + 15) & ~(size_t)15;
        h.resize(off + n);
        if (n) memcpy(h.data() + off, src, n);
        return off;
    }
    cudaError_t run(cudaStream_t s, HBuf& dev) {
        if (!h.empty()) {
            cudaError_t e = dev.alloc(h.size(), s);
            if (e != cudaSuccess) return e;
            e = cudaMemcpyAsync(dev.p, h.data(), h.size(), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
        }
        for (auto& f : steps) {
            const cudaError_t e = f(static_cast<const unsigned char*>(dev.p));
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

// ---------------------------------------------------------------- block sets
template <class T>
struct HSet {
    int nb = 0, b = 0, L = 0, leaf = 0;
    int K[HMAXL + 1] = {0};
    HBuf buf;
    T* leaves = nullptr;
    T* U[HMAXL + 1] = {nullptr};
    T* V[HMAXL + 1] = {nullptr};
    std::vector<int> rank;  // per block, per node: (2^l - 2) + i
    int npb() const { return (1 << (L + 1)) - 2; }
    T* lf(int g, int lam) const { return leaves + ((size_t)g * (b / leaf) + lam) * leaf * leaf; }
    T* Up(int g, int l) const { return U[l] + (size_t)g * b * K[l]; }
    T* Vp(int g, int l) const { return V[l] + (size_t)g * b * K[l]; }
    int rk(int g, int l, int i) const { return rank[(size_t)g * npb() + (1 << l) - 2 + i]; }
    size_t words() const {
        size_t w = (size_t)nb * b * leaf;
        for (int l = 1; l <= L; ++l) w += 2 * (size_t)nb * b * K[l];
        return w;
    }
    cudaError_t alloc(int nb_, int b_, int L_, const int* K_, cudaStream_t s, Ranges& rs) {
        nb = nb_; b = b_; L = L_; leaf = b >> L;
        for (int l = 1; l <= L; ++l) K[l] = K_[l];
        const size_t w = words();
        cudaError_t e = buf.alloc(w * sizeof(T), s, &rs);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(buf.p, 0, w * sizeof(T), s);
        if (e != cudaSuccess) return e;
        T* p = static_cast<T*>(buf.p);
        leaves = p;
        p += (size_t)nb * b * leaf;
        for (int l = 1; l <= L; ++l) {
            U[l] = K[l] ? p : nullptr;
            p += (size_t)nb * b * K[l];
            V[l] = K[l] ? p : nullptr;
            p += (size_t)nb * b * K[l];
        }
        rank.assign((size_t)nb * npb(), 0);
        return cudaSuccess;
    }
    int maxrank(int l) const {
        int m = 0;
        for (int g = 0; g < nb; ++g)
            for (int i = 0; i < (1 << l); ++i) m = std::max(m, rk(g, l, i));
        return m;
    }
};

// ---------------------------------------------------------------- the driver
template <class T>
struct Red {
    cudaStream_t s = nullptr;
    int b = 0, L = 0, leaf = 0;
    double tol = 0.0;
    int kcap = 0;  // largest rank a node may keep
    Ranges rs;
    std::string err;
    std::vector<std::unique_ptr<HBuf>> tmp;  // temporaries of the current step
    double flops = 0.0;  // algorithmic flops of the products issued (2 M N K per term)
    bool oom = false;    // a device allocation was refused
    bool sketch = true;  // randomized first truncation pass where a rank hint is given
    long long nodes = 0;        // node truncations
    long long sketch_redo = 0;  // nodes the sketch left to the exact pass
    // host time blocked on the device (uploads that wait for the stream,
    // synchronisations); the rest of the driver's wall time is host work
    double wait_ms = 0.0;
    struct WaitClock {
        double& acc;
        std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
        explicit WaitClock(double& a) : acc(a) {}
        ~WaitClock() {
            acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    };

    int fail(const char* m) {
        if (err.empty()) err = m;
        return -1;
    }
    template <class X>
    X* get(size_t n) {
        tmp.emplace_back(new HBuf());
        if (tmp.back()->alloc(std::max<size_t>(n, 1) * sizeof(X), s, &rs) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return nullptr;
        }
        return static_cast<X*>(tmp.back()->p);
    }
    void drop_tmp() { tmp.clear(); }

    // ---- operand addressing ------------------------------------------------------
    // A host-side operand: address base + map(g) gs + ((i >> sh) ^ x) is with
    // the block map given as an index into the plan's maps (-1: identity).
    struct Op {
        const T* base = nullptr;
        long long gs = 0, is = 0;
        int sh = 0, x = 0, ld = 1;
        int map = -1;
    };
    static Op op(const T* base, long long gs, long long is, int ld, int map = -1, int sh = 0, int x = 0) {
        Op o;
        o.base = base; o.gs = gs; o.is = is; o.ld = ld; o.map = map; o.sh = sh; o.x = x;
        return o;
    }
    // Plan with block maps: uploaded with the launches' other data
    struct TPlan {
        Plan pl;
        std::vector<std::vector<int>> maps;
        std::vector<size_t> moff;
        int map(const std::vector<int>& m) {
            maps.push_back(m);
            moff.push_back(pl.put(m.data(), std::max<size_t>(1, m.size()) * sizeof(int)));
            return (int)maps.size() - 1;
        }
    };
    HAddr<T> resolve(const Op& o, const TPlan& tp, const unsigned char* d) const {
        HAddr<T> a;
        a.base = o.base; a.gs = o.gs; a.is = o.is; a.ishift = o.sh; a.ixor = o.x; a.ld = o.ld; a.pad = 0;
        a.gmap = (o.map >= 0) ? reinterpret_cast<const int*>(d + tp.moff[o.map]) : nullptr;
        return a;
    }
    // Host check that every (g, i) address of an operand, with its rows x cols
    // extent, lies in one registered device buffer.
    const char* where = "";  // the batch being built (for error messages)
    bool chk(const TPlan& tp, const Op& o, int ng, int ni, long long rows, long long cols) {
        if (!o.base || rows <= 0 || cols <= 0 || ng <= 0 || ni <= 0) return true;
        long long gmin = 0, gmax = ng - 1;
        if (o.map >= 0) {
            const std::vector<int>& m = tp.maps[o.map];
            gmin = LLONG_MAX; gmax = -1;
            for (int g = 0; g < ng && g < (int)m.size(); ++g)
                if (m[g] >= 0) { gmin = std::min<long long>(gmin, m[g]); gmax = std::max<long long>(gmax, m[g]); }
            if ((int)m.size() < ng) return fail("internal: block map shorter than its batch"), false;
            if (gmax < 0) return true;
        }
        long long fmin = LLONG_MAX, fmax = -1;
        for (int i = 0; i < ni; ++i) {
            const long long f = (long long)((i >> o.sh) ^ o.x);
            fmin = std::min(fmin, f);
            fmax = std::max(fmax, f);
        }
        const T* lo = o.base + gmin * o.gs + fmin * o.is;
        const T* hi = o.base + gmax * o.gs + fmax * o.is + (rows - 1) + (cols - 1) * o.ld + 1;
        if (!rs.has(lo, (size_t)(hi - lo) * sizeof(T))) {
            char m[512];
            uintptr_t rlo = 0, rhi = 0;
            const uintptr_t a = reinterpret_cast<uintptr_t>(lo);
            for (const auto& q : rs.r)
                if (q.first <= a) { rlo = q.first; rhi = q.second; }
            snprintf(m, sizeof(m),
                     "internal: a batch of the HODLR arithmetic points outside its buffers (%s: ng %d ni %d rows %lld "
                     "cols %lld gs %lld is %lld ld %d map %d sh %d x %d; bytes [%#zx, %#zx) vs buffer [%#zx, %#zx))",
                     where, ng, ni, rows, cols, o.gs, o.is, o.ld, o.map, o.sh, o.x, (size_t)a,
                     (size_t)reinterpret_cast<uintptr_t>(hi), (size_t)rlo, (size_t)rhi);
            fail(m);
            return false;
        }
        return true;
    }

    // ---- one product batch -------------------------------------------------------
    struct GB {
        int M = 0, N = 0, ni = 1, ng = 1;
        Op C, Cin;
        T beta = T(0);
        struct Tm {
            Op A, B;
            int K = 0;
            bool ta = false, tb = false;
            T alpha = T(1);
        };
        std::vector<Tm> t;
    };
    static GB gb(int ng, int ni, int M, int N, const Op& C) {
        GB g;
        g.ng = ng; g.ni = ni; g.M = M; g.N = N; g.C = C;
        return g;
    }
    static void tm(GB& g, const Op& A, bool ta, const Op& B, bool tb, int K, T alpha = T(1)) {
        if (K <= 0) return;
        typename GB::Tm x;
        x.A = A; x.B = B; x.K = K; x.ta = ta; x.tb = tb; x.alpha = alpha;
        g.t.push_back(x);
    }
    // Adds the batch (split into launches of at most VT_MAXT terms, the later
    // ones accumulating into C).
    void add(TPlan& tp, GB g) {
        if (g.M <= 0 || g.N <= 0 || g.ng <= 0 || g.ni <= 0) return;
        chk(tp, g.C, g.ng, g.ni, g.M, g.N);
        if (g.Cin.base) chk(tp, g.Cin, g.ng, g.ni, g.M, g.N);
        for (const auto& x : g.t) {
            chk(tp, x.A, g.ng, g.ni, x.ta ? x.K : g.M, x.ta ? g.M : x.K);
            chk(tp, x.B, g.ng, g.ni, x.tb ? g.N : x.K, x.tb ? x.K : g.N);
            flops += 2.0 * g.M * g.N * x.K * g.ng * g.ni;
        }
        size_t t0 = 0;
        bool first = true;
        do {
            const size_t t1 = std::min(g.t.size(), t0 + VT_MAXT);
            VPT<T> P;
            memset(&P, 0, sizeof(P));
            P.M = g.M; P.N = g.N; P.ni = g.ni; P.ng = g.ng; P.nt = (int)(t1 - t0);
            Op cin = first ? g.Cin : g.C;
            const T beta = first ? g.beta : T(1);
            P.beta = beta;
            const Op C = g.C;
            std::vector<typename GB::Tm> ts(g.t.begin() + t0, g.t.begin() + t1);
            const TPlan* tpp = &tp;
            cudaStream_t st = s;
            tp.pl.steps.push_back([=](const unsigned char* d) {
                VPT<T> Q = P;
                Q.C = resolve(C, *tpp, d);
                Q.Cin = resolve(cin, *tpp, d);
                for (size_t k = 0; k < ts.size(); ++k) {
                    Q.t[k].A = resolve(ts[k].A, *tpp, d);
                    Q.t[k].B = resolve(ts[k].B, *tpp, d);
                    Q.t[k].K = ts[k].K;
                    Q.t[k].flags = (ts[k].ta ? 1 : 0) | (ts[k].tb ? 2 : 0);
                    Q.t[k].alpha = ts[k].alpha;
                }
                return vgemm_t<T>(Q, st);
            });
            t0 = t1;
            first = false;
        } while (t0 < g.t.size());
    }
    // ---- one copy batch ----------------------------------------------------------
    void copy(TPlan& tp, int ng, int ni, const Op& src, const Op& dst, int rows, int cols, T alpha, T beta = T(0),
              const Op* dv = nullptr, const Op* dc = nullptr) {
        if (rows <= 0 || cols <= 0 || ng <= 0 || ni <= 0) return;
        if ((long long)rows * cols >= (1LL << 31)) {
            fail("internal: copy too large");
            return;
        }
        chk(tp, src, ng, ni, rows, cols);
        chk(tp, dst, ng, ni, rows, cols);
        if (dv) chk(tp, *dv, ng, ni, rows, 1);
        if (dc) chk(tp, *dc, ng, ni, cols, 1);
        CPT<T> P;
        memset(&P, 0, sizeof(P));
        P.rows = rows; P.cols = cols; P.ni = ni; P.ng = ng; P.alpha = alpha; P.beta = beta;
        const Op S = src, Dd = dst, V = dv ? *dv : Op(), Cc = dc ? *dc : Op();
        const TPlan* tpp = &tp;
        cudaStream_t st = s;
        tp.pl.steps.push_back([=](const unsigned char* d) {
            CPT<T> Q = P;
            Q.src = resolve(S, *tpp, d);
            Q.dst = resolve(Dd, *tpp, d);
            Q.dv = resolve(V, *tpp, d);
            Q.dc = resolve(Cc, *tpp, d);
            return hcopy_t<T>(Q, st);
        });
    }
    void fn(TPlan& tp, std::function<cudaError_t(const unsigned char*)> f) { tp.pl.steps.push_back(f); }
    int run(TPlan& tp) {
        if (!err.empty()) return -1;
        WaitClock wc(wait_ms);
        tmp.emplace_back(new HBuf());
        const cudaError_t e = tp.pl.run(s, *tmp.back());  // descriptors: not a range operands may use
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(cudaGetErrorString(e));
        }
        return 0;
    }

    // ------------------------------------------------------------ truncation
    // Accumulated factors of one tree level, stacked per block: U (nb x b x R)
    // and V (nb x b x R); node i of block g is U rows [i s, (i+1) s) and V rows
    // of the sibling i^1.
    struct Acc {
        T* U = nullptr;
        T* V = nullptr;
        int R = 0;
    };
    // Truncates every node of every tree level (k_hrecomp), reads the ranks,
    // allocates `out` with the largest kept rank per tree level as capacity,
    // and writes U' = U (V^T V'), V' and the leaves (leaves_src: nb x b x leaf).
    // khint[l]: the rank expected at tree level l (the operands' ranks); with
    // it, a level whose accumulated width is well above that rank is first
    // truncated through a randomized sketch of width hint + 10 (rounded up
    // to 8), and only the nodes the sketch does not resolve get the exact
    // pass.  Returns -2 (nothing done) when a level's panels exceed the
    // truncation kernel's shared memory.
    int sync_wait(const char* msg) {
        cudaError_t se;
        {
            WaitClock wc(wait_ms);
            se = cudaStreamSynchronize(s);
        }
        if (se != cudaSuccess) {
            cudaGetLastError();
            return fail(msg);
        }
        return 0;
    }
    int read_ranks(const std::vector<int*>& rkd, int nb, std::vector<std::vector<int>>& hr) {
        for (int l = 1; l <= L; ++l) {
            if (!rkd[l]) continue;
            hr[l].resize((size_t)nb << l);
            if (cudaMemcpyAsync(hr[l].data(), rkd[l], hr[l].size() * sizeof(int), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                return fail("rank readback failed");
        }
        return sync_wait("HODLR truncation failed on the device");
    }
    int truncate(const std::vector<Acc>& acc, int nb, const T* leaves_src, HSet<T>& out,
                 const int* khint = nullptr) {
        std::vector<T*> vt(L + 1, nullptr);
        std::vector<int*> rkd(L + 1, nullptr);
        std::vector<int> ksl(L + 1, 0);
        for (int l = 1; l <= L; ++l) {
            const int R = acc[l].R, s_ = b >> l;
            if (R && hrecomp_smem_bytes(s_, R, sizeof(T)) > 227 * 1024) return -2;
            if (R && khint && sketch) {
                const int ks = std::max(16, (khint[l] + 10 + 7) / 8 * 8);
                if (ks + 8 <= std::min(s_, R) && hrecomp_sketch_smem_bytes(s_, R, ks, sizeof(T)) <= 227 * 1024)
                    ksl[l] = ks;
            }
        }
        where = "truncate phase 1";
        TPlan p1;
        for (int l = 1; l <= L; ++l) {
            const int R = acc[l].R, s_ = b >> l;
            if (R == 0) continue;
            nodes += (long long)nb << l;
            vt[l] = get<T>((size_t)nb * b * R);
            rkd[l] = get<int>((size_t)nb << l);
            if (!vt[l] || !rkd[l]) return fail("device allocation failed (HODLR truncation)");
            const long long bs = (long long)b * R;
            const Op U = op(acc[l].U, bs, s_, b), V = op(acc[l].V, bs, s_, b, -1, 0, 1),
                     Vo = op(vt[l], bs, s_, b, -1, 0, 1);
            chk(p1, U, nb, 1 << l, s_, R);
            chk(p1, V, nb, 1 << l, s_, R);
            chk(p1, Vo, nb, 1 << l, s_, R);
            int* rr = rkd[l];
            const double tl = tol;
            const int kc = kcap, ks = ksl[l];
            cudaStream_t st = s;
            const TPlan* tpp = &p1;
            fn(p1, [=](const unsigned char* d) {
                RPT<T> Q;
                memset(&Q, 0, sizeof(Q));
                Q.U = resolve(U, *tpp, d);
                Q.V = resolve(V, *tpp, d);
                Q.Vout = resolve(Vo, *tpp, d);
                Q.s = s_; Q.R = R; Q.wout = R; Q.ni = 1 << l; Q.ng = nb;
                return hrecomp_t<T>(Q, rr, tl, kc, ks, st);
            });
        }
        if (run(p1)) return -1;
        std::vector<std::vector<int>> hr(L + 1);
        if (read_ranks(rkd, nb, hr)) return -1;
        // the nodes the sketch left open: the exact pass, as one list
        std::vector<RProb<T>> redo;
        std::vector<std::pair<int, size_t>> where_;
        int smax = 0, Rmax = 0;
        for (int l = 1; l <= L; ++l) {
            if (!ksl[l]) continue;
            const int R = acc[l].R, s_ = b >> l;
            for (size_t e = 0; e < hr[l].size(); ++e) {
                if (hr[l][e] >= 0) continue;
                const size_t g = e >> l;
                const int i = (int)(e & ((1u << l) - 1));
                const size_t base = g * b * R;
                RProb<T> q;
                q.U = acc[l].U + base + (size_t)i * s_;
                q.V = acc[l].V + base + (size_t)(i ^ 1) * s_;
                q.Vout = vt[l] + base + (size_t)(i ^ 1) * s_;
                q.ldu = q.ldv = q.ldvo = b;
                q.s = s_; q.R = R; q.wout = R;
                redo.push_back(q);
                where_.push_back({l, e});
                smax = std::max(smax, s_);
                Rmax = std::max(Rmax, R);
            }
        }
        if (!redo.empty()) {
            where = "truncate exact pass";
            sketch_redo += (long long)redo.size();
            int* rk2 = get<int>(redo.size());
            if (!rk2) return fail("device allocation failed (HODLR truncation)");
            TPlan pr;
            const size_t off = pr.pl.put(redo.data(), redo.size() * sizeof(RProb<T>));
            const int n = (int)redo.size();
            const double tl = tol;
            const int kc = kcap;
            cudaStream_t st = s;
            fn(pr, [=](const unsigned char* d) {
                return hrecomp<T>(reinterpret_cast<const RProb<T>*>(d + off), n, smax, Rmax, rk2, tl, kc, st);
            });
            if (run(pr)) return -1;
            std::vector<int> r2(redo.size());
            if (cudaMemcpyAsync(r2.data(), rk2, r2.size() * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return fail("rank readback failed");
            if (sync_wait("HODLR truncation failed on the device")) return -1;
            for (size_t j = 0; j < redo.size(); ++j) hr[where_[j].first][where_[j].second] = r2[j];
        }
        int Kn[HMAXL + 1] = {0};
        for (int l = 1; l <= L; ++l)
            for (int v : hr[l]) Kn[l] = std::max(Kn[l], v);
        if (out.alloc(nb, b, L, Kn, s, rs) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return fail("device allocation failed (HODLR block set)");
        }
        for (int l = 1; l <= L; ++l)
            if (!hr[l].empty())
                for (int g = 0; g < nb; ++g)
                    for (int i = 0; i < (1 << l); ++i)
                        out.rank[(size_t)g * out.npb() + (1 << l) - 2 + i] = hr[l][((size_t)g << l) + i];
        where = "truncate phase 2";
        TPlan p2;
        for (int l = 1; l <= L; ++l) {
            const int R = acc[l].R, Kl = Kn[l], s_ = b >> l;
            if (R == 0 || Kl == 0) continue;
            T* T1 = get<T>(((size_t)nb << l) * R * Kl);
            if (!T1) return fail("device allocation failed (HODLR truncation)");
            const long long bs = (long long)b * R;
            GB g1 = gb(nb, 1 << l, R, Kl, op(T1, (long long)(1 << l) * R * Kl, (long long)R * Kl, R));
            tm(g1, op(acc[l].V, bs, s_, b, -1, 0, 1), true, op(vt[l], bs, s_, b, -1, 0, 1), false, s_);
            add(p2, g1);
            GB g2 = gb(nb, 1 << l, s_, Kl, op(out.U[l], (long long)b * Kl, s_, b));
            tm(g2, op(acc[l].U, bs, s_, b), false, op(T1, (long long)(1 << l) * R * Kl, (long long)R * Kl, R), false, R);
            add(p2, g2);
            copy(p2, nb, 1, op(vt[l], bs, 0, b), op(out.V[l], (long long)b * Kl, 0, b), b, Kl, T(1));
        }
        const long long bl = (long long)b * leaf;
        copy(p2, nb, 1, op(leaves_src, bl, 0, (int)bl), op(out.leaves, bl, 0, (int)bl), (int)bl, 1, T(1));
        return run(p2);
    }

    // ------------------------------------------------------------ inverse
    // out (sel.size() blocks) = inverse of the blocks sel[] of D.  bad: index
    // (into sel) of the first block with a zero or non-finite pivot in a leaf
    // or a capacitance matrix, -1 if none.  tri: the blocks' FP64 tridiagonal
    // form (level 0 of a 5-point operator with strictly diagonally dominant
    // rows), whose leaves are inverted in O(leaf^2) each; NULL: the leaves are
    // inverted by pivoted Gauss-Jordan in FP64.
    int hinv(const HSet<T>& D, const std::vector<int>& sel, HSet<T>& out, int& bad, const double* tri = nullptr) {
        bad = -1;
        const int nI = (int)sel.size(), nl = 1 << L;
        const long long bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        if (nI == 0) return 0;
        int K[HMAXL + 1] = {0};
        for (int l = 1; l <= L; ++l) K[l] = D.K[l];
        T* Gl = get<T>((size_t)nI * bl);
        double* Ld = sizeof(T) == 8 ? reinterpret_cast<double*>(Gl) : get<double>((size_t)nI * bl);
        size_t ninfo = (size_t)nI * nl, npiv = (size_t)nI * nl * leaf;
        for (int l = 1; l <= L; ++l)
            if (K[l]) {
                ninfo += (size_t)nI << (l - 1);
                npiv = std::max(npiv, ((size_t)nI << (l - 1)) * 2 * K[l]);
            }
        int* info = get<int>(ninfo);
        int* piv = get<int>(npiv);
        if (!Gl || !Ld || !info || !piv) return fail("device allocation failed (HODLR inverse)");
        std::vector<T*> P(L + 1, nullptr), Q(L + 1, nullptr), Un(L + 1, nullptr), Yn(L + 1, nullptr),
            Tc(L + 1, nullptr), Kt(L + 1, nullptr);
        std::vector<double*> Kd(L + 1, nullptr);
        std::vector<int*> infoK(L + 1, nullptr);
        size_t io = (size_t)nI * nl;
        for (int l = 1; l <= L; ++l) {
            if (!K[l]) continue;
            const size_t pb = (size_t)nI * b * K[l], np = (size_t)nI << (l - 1);
            P[l] = get<T>(pb); Q[l] = get<T>(pb); Un[l] = get<T>(pb); Yn[l] = get<T>(pb);
            Tc[l] = get<T>(((size_t)nI << l) * K[l] * K[l]);
            Kd[l] = get<double>(np * 4 * K[l] * K[l]);
            Kt[l] = sizeof(T) == 8 ? reinterpret_cast<T*>(Kd[l]) : get<T>(np * 4 * K[l] * K[l]);
            infoK[l] = info + io;
            io += np;
            if (!P[l] || !Q[l] || !Un[l] || !Yn[l] || !Tc[l] || !Kd[l] || !Kt[l])
                return fail("device allocation failed (HODLR inverse)");
        }
        TPlan tp;
        const int ms = tp.map(sel);
        auto dU = [&](int l, long long is, int x = 0, int sh = 0) { return op(D.U[l], (long long)b * K[l], is, b, ms, sh, x); };
        auto dV = [&](int l, long long is, int x = 0, int sh = 0) { return op(D.V[l], (long long)b * K[l], is, b, ms, sh, x); };
        auto pan = [&](T* base, int Kk, long long is, int x = 0) { return op(base, (long long)b * Kk, is, b, -1, 0, x); };
        where = "hinv leaves";
        // ---- leaf inverses (FP64) ----
        if (tri) {
            cudaStream_t st = s;
            const int lf = leaf, bb_ = b;
            const TPlan* tpp = &tp;
            fn(tp, [=](const unsigned char* d) -> cudaError_t {
                cudaError_t e = cudaMemsetAsync(info, 0, (size_t)nI * nl * sizeof(int), st);
                if (e != cudaSuccess) return e;
                return tri_leaf_inverse<T>(tri, reinterpret_cast<const int*>(d + tpp->moff[ms]), nI, bb_, lf, Gl, st);
            });
        } else {
            copy(tp, nI, 1, op(D.leaves, bl, 0, (int)bl, ms), op(Gl, bl, 0, (int)bl), (int)bl, 1, T(1));
            cudaStream_t st = s;
            const int lf = leaf;
            fn(tp, [=](const unsigned char*) -> cudaError_t {
                cudaError_t e;
                if (sizeof(T) == 4) {
                    e = convert_f2d(reinterpret_cast<const float*>(Gl), Ld, (long long)nI * bl, st);
                    if (e != cudaSuccess) return e;
                }
                e = gj_inverse_small<double>(Ld, lf, nI * nl, info, piv, st);
                if (e != cudaSuccess) return e;
                if (sizeof(T) == 4) e = convert_d2f(Ld, reinterpret_cast<float*>(Gl), (long long)nI * bl, st);
                return e;
            });
        }
        const Op Gleaf = op(Gl, bl, l2, leaf);
        for (int l = L; l >= 1; --l) {
            const int Kl = K[l], s_ = b >> l;
            if (!Kl) continue;
            // products of the current inverse with U_l and V_l: node products
            // of the levels below (stage 1), then per leaf row block (stage 2)
            std::vector<T*> tP(L + 1, nullptr), dQ(L + 1, nullptr);
            for (int m = l + 1; m <= L; ++m)
                if (K[m]) {
                    tP[m] = get<T>(((size_t)nI << m) * K[m] * Kl);
                    dQ[m] = get<T>(((size_t)nI << m) * K[m] * Kl);
                    if (!tP[m] || !dQ[m]) return fail("device allocation failed (HODLR inverse)");
                }
            where = "hinv stage 1";
            for (int m = l + 1; m <= L; ++m) {
                if (!K[m]) continue;
                const int Km = K[m], sm = b >> m;
                const long long tg = (long long)(1 << m) * Km * Kl, ti = (long long)Km * Kl;
                GB gt = gb(nI, 1 << m, Km, Kl, op(tP[m], tg, ti, Km));
                tm(gt, pan(Q[m], Km, sm), true, dU(l, sm), false, sm);
                add(tp, gt);
                GB gd = gb(nI, 1 << m, Km, Kl, op(dQ[m], tg, ti, Km));
                tm(gd, pan(Un[m], Km, sm, 1), true, dV(l, sm, 1), false, sm);
                tm(gd, pan(Yn[m], Km, sm), true, dV(l, sm), false, sm);
                add(tp, gd);
            }
            where = "hinv stage 2";
            GB gp = gb(nI, nl, leaf, Kl, pan(P[l], Kl, leaf));
            tm(gp, Gleaf, false, dU(l, leaf), false, leaf);
            GB gq = gb(nI, nl, leaf, Kl, pan(Q[l], Kl, leaf));
            tm(gq, Gleaf, true, dV(l, leaf), false, leaf);
            for (int m = l + 1; m <= L; ++m) {
                if (!K[m]) continue;
                const int Km = K[m];
                const long long tg = (long long)(1 << m) * Km * Kl, ti = (long long)Km * Kl;
                tm(gp, pan(Un[m], Km, leaf), false, op(tP[m], tg, ti, Km, -1, L - m, 1), false, Km);
                tm(gp, pan(Yn[m], Km, leaf), false, op(tP[m], tg, ti, Km, -1, L - m, 0), false, Km);
                tm(gq, pan(Q[m], Km, leaf), false, op(dQ[m], tg, ti, Km, -1, L - m, 0), false, Km);
            }
            add(tp, gp);
            add(tp, gq);
            where = "hinv cores";
            GB gc = gb(nI, 1 << l, Kl, Kl, op(Tc[l], (long long)(1 << l) * Kl * Kl, (long long)Kl * Kl, Kl));
            tm(gc, dV(l, s_), true, pan(P[l], Kl, s_), false, s_);
            add(tp, gc);
            {
                const size_t np = (size_t)nI << (l - 1);
                T* tc = Tc[l];
                double* kd = Kd[l];
                T* kt = Kt[l];
                int* ik = infoK[l];
                cudaStream_t st = s;
                fn(tp, [=](const unsigned char*) -> cudaError_t {
                    cudaError_t e = hkmat<T>(tc, kd, (int)np, Kl, st);
                    if (e != cudaSuccess) return e;
                    e = gj_inverse_small<double>(kd, 2 * Kl, (int)np, ik, piv, st);
                    if (e != cudaSuccess) return e;
                    if (sizeof(T) == 4)
                        e = convert_d2f(kd, reinterpret_cast<float*>(kt), (long long)np * 4 * Kl * Kl, st);
                    return e;
                });
            }
            where = "hinv new nodes";
            // per parent p: node a = 2p (rows 2p s), node c = 2p + 1 (rows 2p s + s)
            const int K2 = 2 * Kl, npar = 1 << (l - 1);
            const long long kg = (long long)npar * 4 * Kl * Kl, ki = 4LL * Kl * Kl, bg = (long long)b * Kl;
            const long long offs[4][2] = {{0, 0}, {s_, Kl + (long long)Kl * K2}, {0, (long long)Kl * K2}, {s_, Kl}};
            T* dsts[4] = {Un[l], Un[l], Yn[l], Yn[l]};
            for (int q = 0; q < 4; ++q) {
                GB g4 = gb(nI, npar, s_, Kl, op(dsts[q] + offs[q][0], bg, 2LL * s_, b));
                tm(g4, op(P[l] + offs[q][0], bg, 2LL * s_, b), false, op(Kt[l] + offs[q][1], kg, ki, K2), false, Kl,
                   T(-1));
                add(tp, g4);
            }
        }
        where = "hinv assembly";
        // leaves absorb the pending updates; nodes gather [U'_l | Yn_{l-1} ..]
        {
            GB gf = gb(nI, nl, leaf, leaf, Gleaf);
            gf.Cin = Gleaf;
            gf.beta = T(1);
            for (int l = 1; l <= L; ++l)
                if (K[l]) tm(gf, pan(Yn[l], K[l], leaf), false, pan(Q[l], K[l], leaf), true, K[l]);
            add(tp, gf);
        }
        std::vector<Acc> acc(L + 1);
        for (int l = 1; l <= L; ++l) {
            int R = 0;
            for (int m = 1; m <= l; ++m) R += K[m];
            acc[l].R = R;
            if (!R) continue;
            acc[l].U = get<T>((size_t)nI * b * R);
            acc[l].V = get<T>((size_t)nI * b * R);
            if (!acc[l].U || !acc[l].V) return fail("device allocation failed (HODLR inverse)");
            int c0 = 0;
            for (int m = l; m >= 1; --m) {
                if (!K[m]) continue;
                const long long ab = (long long)b * R;
                copy(tp, nI, 1, pan(m == l ? Un[m] : Yn[m], K[m], 0), op(acc[l].U + (size_t)c0 * b, ab, 0, b), b, K[m],
                     T(1));
                copy(tp, nI, 1, pan(Q[m], K[m], 0), op(acc[l].V + (size_t)c0 * b, ab, 0, b), b, K[m], T(1));
                c0 += K[m];
            }
        }
        if (run(tp)) return -1;
        if (const int tr = truncate(acc, nI, Gl, out, D.K)) return tr;
        std::vector<int> hi(ninfo);
        if (cudaMemcpy(hi.data(), info, ninfo * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail("pivot readback failed");
        for (int g = 0; g < nI && bad < 0; ++g)
            for (int lam = 0; lam < nl; ++lam)
                if (hi[(size_t)g * nl + lam]) { bad = g; break; }
        io = (size_t)nI * nl;
        for (int l = 1; l <= L && bad < 0; ++l) {
            if (!K[l]) continue;
            const int np = 1 << (l - 1);
            for (int g = 0; g < nI && bad < 0; ++g)
                for (int p = 0; p < np; ++p)
                    if (hi[io + (size_t)g * np + p]) { bad = g; break; }
            io += (size_t)nI * np;
        }
        return 0;
    }

    // ------------------------------------------------------------ sums of products
    struct Term {
        int kind = 0;  // 0: alpha A B (both HODLR);  1: alpha diag(dl) A diag(dr)
        T alpha = T(1);
        const HSet<T>* A = nullptr;
        const HSet<T>* B = nullptr;
        std::vector<int> ia, ib;           // per output block; -1: the term is absent there
        const T* dl = nullptr;             // kind 1: dl = dl + dlmap[g] * b, dr likewise
        const T* dr = nullptr;
        std::vector<int> dlmap, drmap;
    };
    // out (nO blocks) = alpha0 D[id[g]] + sum of the terms, every node of the
    // result truncated once (D == NULL: no D term; id[g] < 0: none for g).
    int hsum(int nO, T alpha0, const HSet<T>* D, const std::vector<int>& id, const std::vector<Term>& terms,
             HSet<T>& out) {
        const int nl = 1 << L;
        const long long bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        std::vector<std::vector<int>> col(terms.size(), std::vector<int>(L + 1, 0));
        std::vector<Acc> acc(L + 1);
        for (int l = 1; l <= L; ++l) {
            int R = D ? D->K[l] : 0;
            for (size_t t = 0; t < terms.size(); ++t) {
                col[t][l] = R;
                const Term& x = terms[t];
                if (x.kind == 1) R += x.A->K[l];
                else {
                    R += x.B->K[l] + x.A->K[l];
                    for (int m = 1; m < l; ++m) R += x.B->K[m];
                }
            }
            acc[l].R = R;
            if (R) {
                if (hrecomp_smem_bytes(b >> l, R, sizeof(T)) > 227 * 1024) return -2;
                acc[l].U = get<T>((size_t)nO * b * R);
                acc[l].V = get<T>((size_t)nO * b * R);
                if (!acc[l].U || !acc[l].V) return fail("device allocation failed (HODLR sum)");
            }
        }
        T* Lo = get<T>((size_t)nO * bl);
        if (!Lo) return fail("device allocation failed (HODLR sum)");
        TPlan tp;
        {
            std::vector<std::pair<void*, size_t>> z;
            z.push_back({Lo, (size_t)nO * bl * sizeof(T)});
            for (int l = 1; l <= L; ++l)
                if (acc[l].R) {
                    z.push_back({acc[l].U, (size_t)nO * b * acc[l].R * sizeof(T)});
                    z.push_back({acc[l].V, (size_t)nO * b * acc[l].R * sizeof(T)});
                }
            cudaStream_t st = s;
            fn(tp, [=](const unsigned char*) -> cudaError_t {
                for (auto& q : z) {
                    const cudaError_t e = cudaMemsetAsync(q.first, 0, q.second, st);
                    if (e != cudaSuccess) return e;
                }
                return cudaSuccess;
            });
        }
        auto accU = [&](int l, int c, long long is = 0) { return op(acc[l].U + (size_t)c * b, (long long)b * acc[l].R, is, b); };
        auto accV = [&](int l, int c, long long is = 0) { return op(acc[l].V + (size_t)c * b, (long long)b * acc[l].R, is, b); };
        const Op Lleaf = op(Lo, bl, l2, leaf);
        where = "hsum D";
        if (D) {
            const int md = tp.map(id);
            copy(tp, nO, 1, op(D->leaves, bl, 0, (int)bl, md), op(Lo, bl, 0, (int)bl), (int)bl, 1, alpha0);
            for (int l = 1; l <= L; ++l) {
                const int Kd = D->K[l];
                if (!Kd) continue;
                copy(tp, nO, 1, op(D->U[l], (long long)b * Kd, 0, b, md), accU(l, 0), b, Kd, alpha0);
                copy(tp, nO, 1, op(D->V[l], (long long)b * Kd, 0, b, md), accV(l, 0), b, Kd, T(1));
            }
        }
        for (size_t t = 0; t < terms.size(); ++t) {
            const Term& x = terms[t];
            const HSet<T>& A = *x.A;
            if (x.kind == 1) {
                const int ma = tp.map(x.ia);
                auto aU = [&](int l, long long is) { return op(A.U[l], (long long)b * A.K[l], is, b, ma); };
                auto aV = [&](int l, long long is) { return op(A.V[l], (long long)b * A.K[l], is, b, ma); };
                const Op aleaf = op(A.leaves, bl, l2, leaf, ma);
                where = "hsum scaled term";
                const int mdl = tp.map(x.dlmap), mdr = tp.map(x.drmap);
                const Op dlf = op(x.dl, b, leaf, 1, mdl), drf = op(x.dr, b, leaf, 1, mdr);
                copy(tp, nO, nl, aleaf, Lleaf, leaf, leaf, x.alpha, T(1), &dlf, &drf);
                const Op dlb = op(x.dl, b, 0, 1, mdl), drb = op(x.dr, b, 0, 1, mdr);
                for (int l = 1; l <= L; ++l) {
                    const int Ka = A.K[l];
                    if (!Ka) continue;
                    copy(tp, nO, 1, aU(l, 0), accU(l, col[t][l]), b, Ka, x.alpha, T(0), &dlb);
                    copy(tp, nO, 1, aV(l, 0), accV(l, col[t][l]), b, Ka, T(1), T(0), &drb);
                }
                continue;
            }
            const HSet<T>& B = *x.B;
            where = "hsum product term";
            // a term absent for a block is absent on both operands
            std::vector<int> ian(x.ia), ibn(x.ib);
            for (size_t g = 0; g < ian.size() && g < ibn.size(); ++g)
                if (ian[g] < 0 || ibn[g] < 0) ian[g] = ibn[g] = -1;
            const int ma2 = tp.map(ian), mb = tp.map(ibn);
            auto aU = [&](int l, long long is, int x_ = 0, int sh = 0) { return op(A.U[l], (long long)b * A.K[l], is, b, ma2, sh, x_); };
            auto aV = [&](int l, long long is, int x_ = 0, int sh = 0) { return op(A.V[l], (long long)b * A.K[l], is, b, ma2, sh, x_); };
            const Op aleaf = op(A.leaves, bl, l2, leaf, ma2);
            auto bU = [&](int l, long long is, int x_ = 0, int sh = 0) { return op(B.U[l], (long long)b * B.K[l], is, b, mb, sh, x_); };
            auto bV = [&](int l, long long is, int x_ = 0, int sh = 0) { return op(B.V[l], (long long)b * B.K[l], is, b, mb, sh, x_); };
            const Op bleaf = op(B.leaves, bl, l2, leaf, mb);
            // cores W_l (per node) and UW_l = U^A_l W_l (per diagonal block)
            std::vector<T*> Wc(L + 1, nullptr), UW(L + 1, nullptr);
            for (int l = 1; l <= L; ++l)
                if (A.K[l] && B.K[l]) {
                    Wc[l] = get<T>(((size_t)nO << l) * A.K[l] * B.K[l]);
                    UW[l] = get<T>((size_t)nO * b * B.K[l]);
                    if (!Wc[l] || !UW[l]) return fail("device allocation failed (HODLR sum)");
                }
            for (int l = 1; l <= L; ++l) {
                const int KA = A.K[l], KB = B.K[l], s_ = b >> l;
                const int cP = col[t][l], cA = cP + KB;
                // stage 1: node products of A's levels below l on U^B_l, and
                // of B's levels below l on V^A_l
                std::vector<T*> tP(L + 1, nullptr), uQ(L + 1, nullptr);
                for (int m = l + 1; m <= L; ++m) {
                    const int sm = b >> m, KAm = A.K[m], KBm = B.K[m];
                    if (KAm && KB) {
                        tP[m] = get<T>(((size_t)nO << m) * KAm * KB);
                        if (!tP[m]) return fail("device allocation failed (HODLR sum)");
                        GB g1 = gb(nO, 1 << m, KAm, KB, op(tP[m], (long long)(1 << m) * KAm * KB, (long long)KAm * KB, KAm));
                        tm(g1, aV(m, sm, 1), true, bU(l, sm, 1), false, sm);
                        add(tp, g1);
                    }
                    if (KBm && KA) {
                        uQ[m] = get<T>(((size_t)nO << m) * KBm * KA);
                        if (!uQ[m]) return fail("device allocation failed (HODLR sum)");
                        GB g1 = gb(nO, 1 << m, KBm, KA, op(uQ[m], (long long)(1 << m) * KBm * KA, (long long)KBm * KA, KBm));
                        tm(g1, bU(m, sm), true, aV(l, sm), false, sm);
                        add(tp, g1);
                    }
                }
                // stage 2: P = BD_l(A) U^B_l (into U_acc, scaled), Q = BD_l(B)^T V^A_l (into V_acc)
                if (KB) {
                    GB g2 = gb(nO, nl, leaf, KB, accU(l, cP, leaf));
                    tm(g2, aleaf, false, bU(l, leaf), false, leaf, x.alpha);
                    for (int m = l + 1; m <= L; ++m)
                        if (tP[m])
                            tm(g2, aU(m, leaf), false,
                               op(tP[m], (long long)(1 << m) * A.K[m] * KB, (long long)A.K[m] * KB, A.K[m], -1, L - m, 0),
                               false, A.K[m], x.alpha);
                    add(tp, g2);
                    copy(tp, nO, 1, bV(l, 0), accV(l, cP), b, KB, T(1));
                }
                if (KA) {
                    GB g2 = gb(nO, nl, leaf, KA, accV(l, cA, leaf));
                    tm(g2, bleaf, true, aV(l, leaf), false, leaf);
                    for (int m = l + 1; m <= L; ++m)
                        if (uQ[m])
                            tm(g2, bV(m, leaf), false,
                               op(uQ[m], (long long)(1 << m) * B.K[m] * KA, (long long)B.K[m] * KA, B.K[m], -1, L - m, 1),
                               false, B.K[m]);
                    add(tp, g2);
                    copy(tp, nO, 1, aU(l, 0), accU(l, cA), b, KA, x.alpha);
                }
                if (Wc[l]) {
                    const Op w = op(Wc[l], (long long)(1 << l) * KA * KB, (long long)KA * KB, KA);
                    GB g3 = gb(nO, 1 << l, KA, KB, w);
                    tm(g3, aV(l, s_, 1), true, bU(l, s_, 1), false, s_);
                    add(tp, g3);
                    GB g4 = gb(nO, 1 << l, s_, KB, op(UW[l], (long long)b * KB, s_, b));
                    tm(g4, aU(l, s_), false, w, false, KA);
                    add(tp, g4);
                }
            }
            // far pieces of the nodes: alpha UW_m, V^B_m (m < l)
            for (int l = 2; l <= L; ++l) {
                int c = col[t][l] + B.K[l] + A.K[l];
                for (int m = 1; m < l; ++m) {
                    const int KB = B.K[m];
                    if (!KB) continue;
                    if (UW[m]) copy(tp, nO, 1, op(UW[m], (long long)b * KB, 0, b), accU(l, c), b, KB, x.alpha);
                    copy(tp, nO, 1, bV(m, 0), accV(l, c), b, KB, T(1));
                    c += KB;
                }
            }
            // leaves: alpha (A_leaf B_leaf + sum_m UW_m V^B_m^T)
            GB g5 = gb(nO, nl, leaf, leaf, Lleaf);
            g5.Cin = Lleaf;
            g5.beta = T(1);
            tm(g5, aleaf, false, bleaf, false, leaf, x.alpha);
            for (int m = 1; m <= L; ++m)
                if (UW[m]) tm(g5, op(UW[m], (long long)b * B.K[m], leaf, b), false, bV(m, leaf), true, B.K[m], x.alpha);
            add(tp, g5);
        }
        if (run(tp)) return -1;
        int hint[HMAXL + 1] = {0};
        for (int l = 1; l <= L; ++l) {
            if (D) hint[l] = D->K[l];
            for (const Term& x : terms) {
                hint[l] = std::max(hint[l], x.A->K[l]);
                if (x.kind != 1) hint[l] = std::max(hint[l], x.B->K[l]);
            }
        }
        return truncate(acc, nO, Lo, out, hint);
    }

    // out (nO blocks) = alpha diag(dl) A[ia] diag(dr): ranks unchanged, no
    // truncation (absent blocks, ia < 0, are zero).
    int hscale(int nO, const HSet<T>& A, const std::vector<int>& ia, T alpha, const T* dl, const std::vector<int>& dlmap,
               const T* dr, const std::vector<int>& drmap, HSet<T>& out) {
        if (out.alloc(nO, b, L, A.K, s, rs) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return fail("device allocation failed (HODLR scale)");
        }
        const int nl = 1 << L;
        const long long bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        TPlan tp;
        where = "hscale";
        const int ma = tp.map(ia), mdl = tp.map(dlmap), mdr = tp.map(drmap);
        const Op dlf = op(dl, b, leaf, 1, mdl), drf = op(dr, b, leaf, 1, mdr);
        copy(tp, nO, nl, op(A.leaves, bl, l2, leaf, ma), op(out.leaves, bl, l2, leaf), leaf, leaf, alpha, T(0), &dlf, &drf);
        const Op dlb = op(dl, b, 0, 1, mdl), drb = op(dr, b, 0, 1, mdr);
        for (int l = 1; l <= L; ++l) {
            if (!A.K[l]) continue;
            const long long bk = (long long)b * A.K[l];
            copy(tp, nO, 1, op(A.U[l], bk, 0, b, ma), op(out.U[l], bk, 0, b), b, A.K[l], alpha, T(0), &dlb);
            copy(tp, nO, 1, op(A.V[l], bk, 0, b, ma), op(out.V[l], bk, 0, b), b, A.K[l], T(1), T(0), &drb);
        }
        for (int g = 0; g < nO; ++g)
            if (ia[g] >= 0)
                for (int l = 1; l <= L; ++l)
                    for (int i = 0; i < (1 << l); ++i)
                        out.rank[(size_t)g * out.npb() + (1 << l) - 2 + i] = A.rk(ia[g], l, i);
        return run(tp);
    }

    // As hscale, into the blocks g with ia[g] >= 0 of an existing set whose
    // capacities equal A's (the other blocks are left as they are).
    int hscale_into(int nO, const HSet<T>& A, const std::vector<int>& ia, T alpha, const T* dl,
                    const std::vector<int>& dlmap, const T* dr, const std::vector<int>& drmap, HSet<T>& out) {
        const int nl = 1 << L;
        const long long bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        TPlan tp;
        where = "hscale_into";
        const int ma = tp.map(ia), mdl = tp.map(dlmap), mdr = tp.map(drmap), mo = tp.map(ia_to_self(ia));
        const Op dlf = op(dl, b, leaf, 1, mdl), drf = op(dr, b, leaf, 1, mdr);
        copy(tp, nO, nl, op(A.leaves, bl, l2, leaf, ma), op(out.leaves, bl, l2, leaf, mo), leaf, leaf, alpha, T(0), &dlf,
             &drf);
        const Op dlb = op(dl, b, 0, 1, mdl), drb = op(dr, b, 0, 1, mdr);
        for (int l = 1; l <= L; ++l) {
            if (!A.K[l]) continue;
            const long long bk = (long long)b * A.K[l];
            copy(tp, nO, 1, op(A.U[l], bk, 0, b, ma), op(out.U[l], bk, 0, b, mo), b, A.K[l], alpha, T(0), &dlb);
            copy(tp, nO, 1, op(A.V[l], bk, 0, b, ma), op(out.V[l], bk, 0, b, mo), b, A.K[l], T(1), T(0), &drb);
        }
        for (int g = 0; g < nO; ++g)
            if (ia[g] >= 0)
                for (int l = 1; l <= L; ++l)
                    for (int i = 0; i < (1 << l); ++i)
                        out.rank[(size_t)g * out.npb() + (1 << l) - 2 + i] = A.rk(ia[g], l, i);
        return run(tp);
    }
    static std::vector<int> ia_to_self(const std::vector<int>& ia) {
        std::vector<int> m(ia.size());
        for (size_t g = 0; g < ia.size(); ++g) m[g] = ia[g] >= 0 ? (int)g : -1;
        return m;
    }

    // Y_q = H[idx[q]] X_q for b x nv panels X_q = X + q b nv, Y_q likewise
    // (leading dimension b): per leaf row block, the leaf and every tree
    // level's node product U (V^T x).
    int happly(const HSet<T>& H, const std::vector<int>& idx, const T* X, int nv, T* Y) {
        const int nq = (int)idx.size(), nl = 1 << L;
        std::vector<T*> tv(L + 1, nullptr);
        TPlan tp;
        where = "happly";
        const int mh = tp.map(idx);
        const long long xg = (long long)b * nv, bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        for (int m = 1; m <= L; ++m) {
            if (!H.K[m]) continue;
            const int sm = b >> m, Km = H.K[m];
            tv[m] = get<T>(((size_t)nq << m) * Km * nv);
            if (!tv[m]) return fail("device allocation failed (HODLR apply)");
            GB g1 = gb(nq, 1 << m, Km, nv, op(tv[m], (long long)(1 << m) * Km * nv, (long long)Km * nv, Km));
            tm(g1, op(H.V[m], (long long)b * Km, sm, b, mh, 0, 1), true, op(X, xg, sm, b, -1, 0, 1), false, sm);
            add(tp, g1);
        }
        GB g2 = gb(nq, nl, leaf, nv, op(Y, xg, leaf, b));
        tm(g2, op(H.leaves, bl, l2, leaf, mh), false, op(X, xg, leaf, b), false, leaf);
        for (int m = 1; m <= L; ++m)
            if (tv[m])
                tm(g2, op(H.U[m], (long long)b * H.K[m], leaf, b, mh), false,
                   op(tv[m], (long long)(1 << m) * H.K[m] * nv, (long long)H.K[m] * nv, H.K[m], -1, L - m, 0), false,
                   H.K[m]);
        add(tp, g2);
        return run(tp);
    }

    // A posteriori accuracy of inverses: max over the blocks q of
    // ||D[sel[q]] (Dinv[q] x) - x|| / ||x|| for seeded random x (nv columns).
    int inverse_check(const HSet<T>& D, const std::vector<int>& sel, const HSet<T>& Dinv, double& worst) {
        const int nq = (int)sel.size(), nv = 2;
        const size_t n = (size_t)nq * b * nv;
        std::vector<T> hx(n);
        uint64_t z = 0x9e3779b97f4a7c15ull;
        for (size_t i = 0; i < n; ++i) {  // SplitMix64 uniforms in [-1, 1)
            z += 0x9e3779b97f4a7c15ull;
            uint64_t w = z;
            w = (w ^ (w >> 30)) * 0xbf58476d1ce4e5b9ull;
            w = (w ^ (w >> 27)) * 0x94d049bb133111ebull;
            w ^= w >> 31;
            hx[i] = (T)((double)(w >> 11) * (2.0 / 9007199254740992.0) - 1.0);
        }
        T* X = get<T>(n);
        T* Y = get<T>(n);
        T* Z = get<T>(n);
        if (!X || !Y || !Z) return fail("device allocation failed (inverse check)");
        if (cudaMemcpyAsync(X, hx.data(), n * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail("inverse check upload failed");
        std::vector<int> id(nq);
        for (int q = 0; q < nq; ++q) id[q] = q;
        if (happly(Dinv, id, X, nv, Y) || happly(D, sel, Y, nv, Z)) return -1;
        std::vector<T> hz(n);
        WaitClock wc(wait_ms);
        if (cudaMemcpyAsync(hz.data(), Z, n * sizeof(T), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return fail("inverse check failed on the device");
        }
        worst = 0.0;
        for (int q = 0; q < nq; ++q) {
            double num = 0.0, den = 0.0;
            for (size_t i = (size_t)q * b * nv; i < (size_t)(q + 1) * b * nv; ++i) {
                const double d = (double)hz[i] - (double)hx[i];
                num += d * d;
                den += (double)hx[i] * (double)hx[i];
            }
            const double e = den > 0 ? std::sqrt(num / den) : 0.0;
            worst = std::max(worst, std::isfinite(e) ? e : 1e300);
        }
        return 0;
    }

    // Dense b x b copies (column-major, ld b) of blocks of X: the blocks
    // idx[q] go to base + q bb (idx[q] < 0: a zero block), for each of the
    // given (idx, base) groups.
    int expand(const HSet<T>& X, const std::vector<std::pair<std::vector<int>, T*>>& groups) {
        TPlan tp;
        where = "expand";
        const int nl = 1 << L;
        const long long bb = (long long)b * b, bl = (long long)b * leaf, l2 = (long long)leaf * leaf;
        for (const auto& gr : groups) {
            const int nq = (int)gr.first.size();
            if (!nq) continue;
            T* Dd = gr.second;
            const int mx = tp.map(gr.first);
            // leaves on the diagonal; the off-diagonal nodes: even node 2p at
            // (rows 2p s, columns (2p+1) s), odd node 2p+1 at ((2p+1) s, 2p s)
            copy(tp, nq, nl, op(X.leaves, bl, l2, leaf, mx), op(Dd, bb, (long long)leaf * (1 + b), b), leaf, leaf, T(1));
            for (int l = 1; l <= L; ++l) {
                const int s_ = b >> l, np = 1 << (l - 1);
                const long long bk = (long long)b * X.K[l], step = 2LL * s_ * (1 + (long long)b);
                for (int odd = 0; odd < 2; ++odd) {
                    GB g = gb(nq, np, s_, s_, op(Dd + (odd ? s_ : (long long)s_ * b), bb, step, b));
                    if (X.K[l])
                        tm(g, op(X.U[l] + (odd ? s_ : 0), bk, 2LL * s_, b, mx), false,
                           op(X.V[l] + (odd ? 0 : s_), bk, 2LL * s_, b, mx), true, X.K[l]);
                    add(tp, g);
                }
            }
        }
        return run(tp);
    }
};

// ---------------------------------------------------------------- the levels
template <class T>
struct Result {
    int th = 0;                                  // levels reduced in HODLR arithmetic
    std::vector<double> check;                   // per level: the inverse check ||D Dinv x - x|| / ||x||
    std::vector<std::unique_ptr<HSet<T>>> dinv;  // per level: the ceil(m/2) inverses
    std::vector<std::unique_ptr<HSet<T>>> x;     // per level (null at 0): XA_e at 2e, XC_e at 2e+1
    std::vector<std::unique_ptr<HSet<T>>> ac;    // per level (null at 0): A_i at 2i, C_i at 2i+1
    std::unique_ptr<HSet<T>> Dn, ACn;            // the blocks of level th when it is reduced densely
    int bad_level = -1, bad_block = -1;          // singular eliminated block (level, block)
};

// Reduces levels 0, 1, ... of a 5-point operator in HODLR arithmetic while
// the ranks stay at most `hrank`, fewer than `hmax` levels are done (hmax <=
// 0: no limit) and every level's inverses pass the a posteriori check
// ||D_j (D_j^-1 x) - x|| / ||x|| <= chk_max on random x: a level whose
// inverses miss it (a near-singular indefinite block amplifies the
// truncation) and the levels after it are reduced densely.  Dband: FP64 [sub, diag, super] per block on the
// device; a, c: the diagonals of A_i, C_i (n*b each, a_0 = c_{n-1} = 0) in T.
// Returns 0, or -1 with R.err set; a singular eliminated block is reported
// through res.bad_level / bad_block.
template <class T>
int reduce(Red<T>& R, int n, const double* Dband, const T* a, const T* c, int hmax, int hrank, double chk_max,
           Result<T>& res, bool dominant = false) {
    const int b = R.b, L = R.L;
    auto D = std::make_unique<HSet<T>>();
    {
        int K1[HMAXL + 1];
        for (int l = 0; l <= HMAXL; ++l) K1[l] = 1;
        if (D->alloc(n, b, L, K1, R.s, R.rs) != cudaSuccess) {
            cudaGetLastError();
            R.oom = true;
            return R.fail("device allocation failed (level 0 blocks)");
        }
        HBandOut<T> o;
        for (int l = 0; l <= HMAXL; ++l) { o.U[l] = D->U[l]; o.V[l] = D->V[l]; }
        if (hband<T>(Dband, n, b, L, D->leaves, o, R.s) != cudaSuccess) return R.fail("level 0 staging failed");
        std::fill(D->rank.begin(), D->rank.end(), 1);
    }
    std::unique_ptr<HSet<T>> AC;  // null at level 0 (diagonal A_i, C_i)
    int m = n, t = 0;
    while (true) {
        const int ne = (m + 1) / 2, nk = m / 2;
        std::vector<int> sel(ne);
        for (int e = 0; e < ne; ++e) sel[e] = 2 * e;
        auto Dinv = std::make_unique<HSet<T>>();
        int bad = -1;
        int st = R.hinv(*D, sel, *Dinv, bad, (t == 0 && dominant) ? Dband : nullptr);
        if (st == -2) break;  // ranks beyond the truncation kernel's capacity: dense from here
        if (st) return -1;
        if (bad >= 0) {
            res.bad_level = t;
            res.bad_block = 2 * bad;
            return 0;
        }
        {
            double worst = 0.0;
            if (R.inverse_check(*D, sel, *Dinv, worst)) return -1;
            res.check.push_back(worst);
            if (!(worst <= chk_max)) break;  // dense from this level on
        }
        if (m == 1) {
            res.dinv.push_back(std::move(Dinv));
            res.x.emplace_back();
            res.ac.push_back(std::move(AC));
            res.th = t + 1;
            R.drop_tmp();
            return 0;
        }
        auto X = std::make_unique<HSet<T>>();
        auto Dn = std::make_unique<HSet<T>>();
        auto ACn = std::make_unique<HSet<T>>();
        std::vector<int> id(nk);
        for (int k = 0; k < nk; ++k) id[k] = 2 * k + 1;
        if (t == 0) {
            // products with the diagonal A_i, C_i are row and column scalings
            // (a, c: the diagonals of all blocks; dl, dr pick block dlmap[g] / drmap[g])
            typename Red<T>::Term t1, t2;
            t1.kind = t2.kind = 1;
            t1.alpha = t2.alpha = T(-1);
            t1.A = t2.A = Dinv.get();
            t1.dl = a; t1.dr = c;  // a_i Dinv_{(i-1)/2} c_{i-1}
            t2.dl = c; t2.dr = a;  // c_i Dinv_{(i+1)/2} a_{i+1}
            t1.ia.resize(nk); t2.ia.resize(nk);
            t1.dlmap.resize(nk); t1.drmap.resize(nk); t2.dlmap.resize(nk); t2.drmap.resize(nk);
            for (int k = 0; k < nk; ++k) {
                const int i = 2 * k + 1;
                t1.ia[k] = (i - 1) / 2;
                t1.dlmap[k] = i;
                t1.drmap[k] = i - 1;
                t2.ia[k] = i + 1 < m ? (i + 1) / 2 : -1;
                t2.dlmap[k] = i;
                t2.drmap[k] = i + 1 < m ? i + 1 : -1;
            }
            st = R.hsum(nk, T(1), D.get(), id, {t1, t2}, *Dn);
            if (st == -2) break;
            if (st) return -1;
            // A'_k = -a_i Dinv_{(i-1)/2} a_{i-1} (i >= 3) at 2k, C'_k = -c_i Dinv_{(i+1)/2} c_{i+1} (i + 2 < m) at 2k+1;
            // the diagonals of the kept blocks' A and C are the even and odd
            // halves of one interleaved list: a block index into a for A', into
            // c for C' (c shifted by n blocks in a combined a|c array is not
            // needed: two scalings, one per parity)
            std::vector<int> iaA(2 * nk, -1), iaC(2 * nk, -1), lA(2 * nk, -1), rA(2 * nk, -1), lC(2 * nk, -1),
                rC(2 * nk, -1);
            for (int k = 0; k < nk; ++k) {
                const int i = 2 * k + 1;
                if (i >= 3) { iaA[2 * k] = (i - 1) / 2; lA[2 * k] = i; rA[2 * k] = i - 1; }
                if (i + 2 < m) { iaC[2 * k + 1] = (i + 1) / 2; lC[2 * k + 1] = i; rC[2 * k + 1] = i + 1; }
            }
            if (R.hscale(2 * nk, *Dinv, iaA, T(-1), a, lA, a, rA, *ACn)) return -1;
            if (R.hscale_into(2 * nk, *Dinv, iaC, T(-1), c, lC, c, rC, *ACn)) return -1;
        } else {
            typename Red<T>::Term tx;
            tx.A = Dinv.get();
            tx.B = AC.get();
            tx.ia.assign(2 * ne, -1);
            tx.ib.assign(2 * ne, -1);
            for (int e = 0; e < ne; ++e) {
                const int j = 2 * e;
                if (j > 0) { tx.ia[2 * e] = e; tx.ib[2 * e] = 2 * j; }              // XA_e = Dinv_e A_j
                if (j + 1 < m) { tx.ia[2 * e + 1] = e; tx.ib[2 * e + 1] = 2 * j + 1; }  // XC_e = Dinv_e C_j
            }
            st = R.hsum(2 * ne, T(0), nullptr, {}, {tx}, *X);
            if (st == -2) break;
            if (st) return -1;
            typename Red<T>::Term t1, t2;
            t1.alpha = t2.alpha = T(-1);
            t1.A = t2.A = AC.get();
            t1.B = t2.B = X.get();
            t1.ia.resize(nk); t1.ib.resize(nk); t2.ia.resize(nk); t2.ib.resize(nk);
            for (int k = 0; k < nk; ++k) {
                const int i = 2 * k + 1;
                t1.ia[k] = 2 * i;      // A_i XC_{(i-1)/2} = AC[2i] X[i]
                t1.ib[k] = i;
                t2.ia[k] = i + 1 < m ? 2 * i + 1 : -1;  // C_i XA_{(i+1)/2} = AC[2i+1] X[i+1]
                t2.ib[k] = i + 1 < m ? i + 1 : -1;
            }
            st = R.hsum(nk, T(1), D.get(), id, {t1, t2}, *Dn);
            if (st == -2) break;
            if (st) return -1;
            typename Red<T>::Term ta;
            ta.alpha = T(-1);
            ta.A = AC.get();
            ta.B = X.get();
            ta.ia.assign(2 * nk, -1);
            ta.ib.assign(2 * nk, -1);
            for (int k = 0; k < nk; ++k) {
                const int i = 2 * k + 1;
                if (i >= 3) { ta.ia[2 * k] = 2 * i; ta.ib[2 * k] = i - 1; }                    // -A_i XA_{(i-1)/2}
                if (i + 2 < m) { ta.ia[2 * k + 1] = 2 * i + 1; ta.ib[2 * k + 1] = i + 2; }   // -C_i XC_{(i+1)/2}
            }
            st = R.hsum(2 * nk, T(0), nullptr, {}, {ta}, *ACn);
            if (st == -2) break;
            if (st) return -1;
        }
        res.dinv.push_back(std::move(Dinv));
        res.x.push_back(t == 0 ? nullptr : std::move(X));
        res.ac.push_back(std::move(AC));
        D = std::move(Dn);
        AC = std::move(ACn);
        m = nk;
        ++t;
        R.drop_tmp();
        int mr = 0;
        for (int l = 1; l <= L; ++l) mr = std::max({mr, D->maxrank(l), AC->maxrank(l)});
        if ((hmax > 0 && t >= hmax) || mr > hrank) break;
        // automatic choice in FP32: the next level is not tried when the
        // checks' growth, extrapolated geometrically (c_t^2 / c_{t-1}, with
        // c_{t-1} taken at least 1e-3 of the limit), passes the limit.  In
        // FP32 the check grows by orders of magnitude per level once the
        // reduced blocks turn ill-conditioned (Helmholtz 1024^2: 1.5e-7,
        // 3e-7, 6.5e-3, then 12 against a limit of 9.5e-3), and such a level
        // would fail its check only after its whole H-inverse had been built.
        // FP64 checks move up and down by orders of magnitude between levels
        // (and every level done in HODLR arithmetic there is more accurate
        // than a dense level compressed afterwards), so FP64 tries them all.
        if (sizeof(T) == 4 && hmax <= 0 && res.check.size() >= 2) {
            const double c1 = res.check[res.check.size() - 1];
            const double c0 = std::max(res.check[res.check.size() - 2], 1e-3 * chk_max);
            if (c1 * (c1 / c0) > chk_max) break;
        }
    }
    R.drop_tmp();
    res.th = t;
    res.Dn = std::move(D);
    res.ACn = std::move(AC);
    return 0;
}

}  // namespace hred
}  // namespace acr
