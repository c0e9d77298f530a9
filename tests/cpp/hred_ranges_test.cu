// Host-only checks of the HODLR driver's range checker (no CUDA call is made):
// every batched launch of the HODLR arithmetic names its operands by an
// address template (base + block * gs + ((node >> sh) ^ x) * is, leading
// dimension ld, optional block map), and the driver refuses a launch whose
// template could reach outside the live buffers.  Built and run by
// tests/test_hred_host.py; prints "OK" and exits 0 when every check holds.
#include <cstdio>
#include <cstdlib>

#include "hred.cuh"

using namespace acr::hred;

static int fails = 0;
#define CHECK(c)                                                      \
    do {                                                              \
        if (!(c)) {                                                   \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);          \
            ++fails;                                                  \
        }                                                             \
    } while (0)

int main() {
    // ---- Ranges: sorted, non-overlapping live buffers
    Ranges rs;
    char* a = reinterpret_cast<char*>(0x100000);
    char* b = reinterpret_cast<char*>(0x200000);
    rs.add(b, 4096);
    rs.add(a, 1024);
    CHECK(rs.has(a, 1024));
    CHECK(rs.has(a + 1000, 24));
    CHECK(!rs.has(a + 1000, 25));        // one byte past the end
    CHECK(!rs.has(a - 1, 2));            // starts before the buffer
    CHECK(rs.has(b + 4095, 1));
    CHECK(!rs.has(a + 1024, 1));         // the gap between buffers
    CHECK(rs.has(a, 0));                 // empty ranges are always inside
    CHECK(!rs.has(nullptr, 4));
    rs.remove(a);
    CHECK(!rs.has(a, 1));
    CHECK(rs.has(b, 4096));

    // ---- the template checker of a batch (float operands)
    Red<float> R;
    float* base = reinterpret_cast<float*>(0x1000000);
    const int nb = 4, bsz = 64, K = 8;  // 4 blocks of a 64 x K panel, stride 64 * K
    R.rs.add(base, (size_t)nb * bsz * K * sizeof(float));
    Red<float>::TPlan tp;
    // every block, node i of 2 at tree level 1: rows [32 i, 32 i + 32), all K columns
    auto o = Red<float>::op(base, (long long)bsz * K, 32, bsz);
    CHECK(R.chk(tp, o, nb, 2, 32, K));
    CHECK(R.err.empty());
    // one column too many reaches into the next block, and past the last one
    CHECK(!R.chk(tp, o, nb, 2, 32, K + 1));
    CHECK(!R.err.empty());
    R.err.clear();
    // the sibling form (i ^ 1) covers the same rows
    auto os = Red<float>::op(base, (long long)bsz * K, 32, bsz, -1, 0, 1);
    CHECK(R.chk(tp, os, nb, 2, 32, K));
    // a shift that maps 4 nodes onto 2 row ranges stays inside; without it it does not
    auto oh = Red<float>::op(base, (long long)bsz * K, 32, bsz, -1, 1, 0);
    CHECK(R.chk(tp, oh, nb, 4, 32, K));
    auto on = Red<float>::op(base, (long long)bsz * K, 32, bsz);
    CHECK(!R.chk(tp, on, nb, 4, 32, K));
    R.err.clear();
    // block maps: absent blocks (-1) are not checked, the used ones are
    const int m1 = tp.map({3, -1, 0, 2});
    auto om = Red<float>::op(base, (long long)bsz * K, 32, bsz, m1);
    CHECK(R.chk(tp, om, 4, 2, 32, K));
    const int m2 = tp.map({4, -1, -1, -1});  // block 4 does not exist
    auto om2 = Red<float>::op(base, (long long)bsz * K, 32, bsz, m2);
    CHECK(!R.chk(tp, om2, 4, 2, 32, K));
    R.err.clear();
    const int m3 = tp.map({-1, -1, -1, -1});  // nothing used: nothing to check
    CHECK(R.chk(tp, Red<float>::op(base + (1 << 20), 1, 1, 1, m3), 4, 2, 32, K));
    // a map shorter than its batch is an internal error
    const int m4 = tp.map({0});
    CHECK(!R.chk(tp, Red<float>::op(base, (long long)bsz * K, 32, bsz, m4), 4, 2, 32, K));

    if (fails) return 1;
    std::printf("OK\n");
    return 0;
}
