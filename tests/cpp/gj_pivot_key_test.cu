// Host-only check of the FP32 pivot key of the register Gauss-Jordan panel
// (no CUDA call is made): the panel picks its pivot by reducing
// gj_pivot_key(|x|) -- a maximum over the rows of each warp, the lowest row
// among the warp's maxima, then the same over the warps -- and this must pick
// the row that a float comparison picks (largest |x| among the rows >= k,
// lowest row on ties), for every value a column can hold: signed zeros
// (|x| taken as x < 0 ? -x : x leaves -0 negative), denormals, infinities,
// ties, and rows with no candidate.  Built and run by tests/test_gj_host.py;
// prints "OK" and exits 0 when every check holds.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "acr_internal.h"

using acr::gj_pivot_key;
using acr::gj_pivot_mag;

static int fails = 0;
#define CHECK(c)                                                      \
    do {                                                              \
        if (!(c)) {                                                   \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);          \
            ++fails;                                                  \
        }                                                             \
    } while (0)

static float mag(float x) { return x < 0.f ? -x : x; }

// the float-comparison arg-max over rows [k, n)
static int ref_pivot(const float* x, int n, int k, float* best) {
    float val = -1.f;
    int idx = 0x7fffffff;
    for (int r = k; r < n; ++r) {
        const float a = mag(x[r]);
        if (a > val || (a == val && r < idx)) { val = a; idx = r; }
    }
    *best = val;
    return idx;
}

// the panel's order: NT threads of RPT rows (row t + i * NT), a lane's own
// best by float comparison, then key maxima / lowest-row minima per warp of
// 32 lanes and over the warps
static int key_pivot(const float* x, int n, int k, int NT, int RPT, float* best) {
    const int NW = NT / 32;
    unsigned wk[32];
    unsigned wi[32];
    for (int w = 0; w < NW; ++w) {
        unsigned kmax = 0, imin = 0xffffffffu;
        unsigned keys[32], idxs[32];
        for (int l = 0; l < 32; ++l) {
            const int t = w * 32 + l;
            float val = -1.f;
            int idx = 0x7fffffff;
            for (int i = 0; i < RPT; ++i) {
                const int r = t + i * NT;
                if (r >= k && r < n) {
                    const float a = mag(x[r]);
                    if (a > val) { val = a; idx = r; }
                }
            }
            keys[l] = gj_pivot_key(val, idx != 0x7fffffff);
            idxs[l] = (unsigned)idx;
            if (keys[l] > kmax) kmax = keys[l];
        }
        for (int l = 0; l < 32; ++l)
            if (keys[l] == kmax && idxs[l] < imin) imin = idxs[l];
        wk[w] = kmax;
        wi[w] = imin;
    }
    unsigned bk = 0, bi = 0xffffffffu;
    for (int w = 0; w < NW; ++w)
        if (wk[w] > bk) bk = wk[w];
    for (int w = 0; w < NW; ++w)
        if (wk[w] == bk && wi[w] < bi) bi = wi[w];
    *best = bk ? gj_pivot_mag(bk) : -1.f;
    return (int)bi;
}

static uint64_t st = 0x9e3779b97f4a7c15ull;
static uint32_t rnd() {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return (uint32_t)(st >> 32);
}

int main() {
    // keys order as magnitudes; -0 and +0 tie; the inverse recovers |x|
    CHECK(gj_pivot_key(0.f, false) == 0u);
    CHECK(gj_pivot_key(-0.f, true) == gj_pivot_key(0.f, true));
    CHECK(gj_pivot_key(-0.f, true) < gj_pivot_key(1e-45f, true));
    CHECK(gj_pivot_key(1e-45f, true) < gj_pivot_key(1.17549435e-38f, true));
    CHECK(gj_pivot_key(1.f, true) < gj_pivot_key(INFINITY, true));
    CHECK(gj_pivot_key(3e38f, true) < gj_pivot_key(INFINITY, true));
    const float probe[] = {0.f, 1e-45f, 3e-39f, 1.17549435e-38f, 0.5f, 1.f, 2.5f, 3e38f, INFINITY};
    for (float a : probe) {
        const float b = gj_pivot_mag(gj_pivot_key(a, true));
        CHECK(std::memcmp(&a, &b, sizeof(a)) == 0);
    }
    CHECK(gj_pivot_mag(gj_pivot_key(-0.f, true)) == 0.f);

    // a column of signed zeros below one tiny positive: the positive wins
    {
        float x[64];
        for (int r = 0; r < 64; ++r) x[r] = (r & 1) ? -0.f : 0.f;
        x[40] = 1e-30f;
        float bv, kv;
        CHECK(ref_pivot(x, 64, 3, &bv) == 40);
        CHECK(key_pivot(x, 64, 3, 32, 2, &kv) == 40 && kv == 1e-30f);
        x[40] = -0.f;  // all zeros: the lowest candidate row, magnitude 0
        CHECK(key_pivot(x, 64, 3, 32, 2, &kv) == 3 && kv == 0.f);
        CHECK(ref_pivot(x, 64, 3, &bv) == 3 && bv == 0.f);
    }

    // random columns over two panel shapes (512 x 1 and 512 x 2 rows)
    const float pool[] = {0.f, -0.f, 1e-45f, -1e-45f, 3e-39f, -3e-39f, 1.f, -1.f, 2.5f, -2.5f,
                          3e38f, -3e38f, INFINITY, -INFINITY};
    const int npool = sizeof(pool) / sizeof(pool[0]);
    static float x[1024];
    int cases = 0;
    for (int it = 0; it < 4000; ++it) {
        const int RPT = (it & 1) ? 2 : 1, NT = 512, n = (it % 7 == 0) ? NT * RPT - (int)(rnd() % 200) : NT * RPT;
        const int mode = (int)(rnd() % 3);
        for (int r = 0; r < n; ++r) {
            if (mode == 0) {
                x[r] = pool[rnd() % npool];
            } else if (mode == 1) {  // few distinct values: many ties
                x[r] = pool[rnd() % 4] * (float)(1 + (int)(rnd() % 2));
            } else {
                const float u = ((float)(rnd() >> 8) / 16777216.f) - 0.5f;
                x[r] = (rnd() % 5 == 0) ? ((rnd() & 1) ? -0.f : 0.f) : u * 1e-20f;
            }
        }
        const int k = (int)(rnd() % (uint32_t)n);
        float bv, kv;
        const int pr = ref_pivot(x, n, k, &bv);
        const int pk = key_pivot(x, n, k, NT, RPT, &kv);
        CHECK(pr == pk);
        CHECK(bv == kv);  // equal magnitudes (-0 == +0)
        ++cases;
        if (fails > 10) break;
    }
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("OK %d cases\n", cases);
    return 0;
}
