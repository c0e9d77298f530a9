// k_tc.cu -- batched block products on the 5th-generation tensor cores.
//
// The Schur complement products of Eq. "fund" (D_j^-1 A_j, D_j^-1 C_j and
// D_i - A_i XC_{i-1} - C_i XA_{i+1}, ...) are dense b x b contractions.  This
// kernel runs them with tcgen05.mma (kind::tf32, FP32 accumulation in TMEM)
// at FP32 accuracy by the error-corrected TF32 product (Ootomo and Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing
// the FP32 theoretical peak performance", IJHPCA 2022): the three-term
// split  x ~= hi + lo,  hi = x rounded to
// the nearest TF32 value,  lo = (x - hi) rounded to the nearest TF32 value:
//     A B  ~=  Ahi Bhi + Ahi Blo + Alo Bhi       (the Alo Blo term is ~2^-22;
// launches that feed cancelling updates, the inversion's, add it as a fourth).
//
// One CTA computes one 128 x 128 tile of one problem:
//   warp 0      TMA producer: A tile (128 rows x 32 k, the operand's natural
//               column-major layout) and B tile (32 k x 128 cols, loaded with
//               the 128-byte swizzle = the K-major operand layout);
//   warp 1      allocates 128 TMEM columns and issues the MMAs (one thread);
//   warps 2..9  split each stage into hi/lo operand tiles (A transposed into
//               the K-major swizzled layout), then run the epilogue
//               (tcgen05.ld, alpha/beta, coalesced column-major stores).
// A 3-stage ring of raw copies feeds a 2-stage ring of split operands, with
// mbarrier handshakes; every wait is bounded and a timeout sets *err instead
// of hanging.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <cstring>

#include "acr_internal.h"

namespace acr {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE_BYTES = BM * BK * 4;  // 16 KB, every operand tile
// Two rings: RAW stages receive the TMA copies (A_raw, B_raw); CONV stages
// hold the split operands (A_hi, A_lo, B_hi, B_lo) the MMAs read.  A raw
// stage is released as soon as it is converted, so the copies of later
// k-steps overlap the conversion and the MMAs of earlier ones.
constexpr int RAW = 3, CONV = 2;
constexpr int RAW_BYTES = 2 * TILE_BYTES, CONV_BYTES = 4 * TILE_BYTES;
constexpr int SMEM_BYTES = RAW * RAW_BYTES + CONV * CONV_BYTES + 1024 /*align*/ + 256 /*barriers*/;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
constexpr int NTHREADS = 320;  // producer, MMA issuer, 8 converter / epilogue warps
constexpr long long WAIT_LIMIT = 1LL << 22;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase with parity `ph`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t ph, long long limit) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(ph)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), start address in 16-byte units.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading-dimension offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride between 8-row groups
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Round to the nearest TF32 value (ties away from zero): add half a TF32 ulp
// to the magnitude bits, then clear the 13 low mantissa bits.  Both parts of
// the split are rounded this way, so the MMA sees exactly representable
// operands and the split error (<= 2^-23 |x|) has no bias that could grow
// along the 1024-long contractions.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}
__device__ __forceinline__ float tf32_hi(float x) { return tf32_rn(x); }

// byte offset of element (row, k) in a 128-row x 32-k K-major SW128 tile
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
    return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + ((k & 3) << 2));
}

}  // namespace tc

using namespace tc;

// Problem z: out[:, cols] = alpha * sum_t A_t[:, ka0 : ka0 + kdim] B_t[0 : kdim, cols] + beta * cin,
// rows 0..b-1 (ld b).  Output column tile tn covers columns ((tn < nskip) ? tn : tn + nshift) * BN,
// so a launch can leave out a band of column tiles (nskip = INT_MAX: no band).
__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm_tc(const TcProb* __restrict__ probs, const CUtensorMap* __restrict__ maps, int b, int tiles_m,
          int* __restrict__ err, int kdim, int ka0, int nskip, int nshift, int lolo, long long wlimit,
          int withhold) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* raw = base;                           // [RAW][A_raw | B_raw]
    unsigned char* cvt = base + RAW * RAW_BYTES;         // [CONV][A_hi | A_lo | B_hi | B_lo]
    uint64_t* bars = reinterpret_cast<uint64_t*>(cvt + CONV * CONV_BYTES);
    uint64_t* full = bars;                  // [RAW]  TMA bytes landed
    uint64_t* raw_free = bars + RAW;        // [RAW]  converters done with the raw stage
    uint64_t* conv_full = bars + 2 * RAW;   // [CONV] split operands ready
    uint64_t* conv_free = conv_full + CONV; // [CONV] MMAs done with them
    uint64_t* accb = conv_free + CONV;      // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
    __shared__ int s_fail;

    // a CTA that gave up on a wait raises *err; later CTAs do no work at all
    if (*reinterpret_cast<volatile int*>(err) != 0) return;
    const TcProb P = probs[blockIdx.y];
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int m0 = tm * BM, n0 = (tn < nskip ? tn : tn + nshift) * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kt = kdim / BK;
    const int niter = P.nterm * kt;

    if (threadIdx.x == 0) {
        for (int i = 0; i < RAW; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&raw_free[i], 8);
        }
        for (int i = 0; i < CONV; ++i) {
            mbar_init(&conv_full[i], 8);
            mbar_init(&conv_free[i], 1);
        }
        mbar_init(accb, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem_d = *tmem_slot;

    if (warp == 0) {
        // withhold != 0 (failure-path tests only): no copies are issued, so
        // every consumer wait runs out and the CTA takes its timeout path
        if (lane == 0 && !withhold) {
            for (int it = 0; it < niter; ++it) {
                const int r = it % RAW;
                if (it >= RAW && !mbar_wait(&raw_free[r], (uint32_t)(((it / RAW) & 1) ^ 1), wlimit)) { s_fail = 1; break; }
                unsigned char* st = raw + r * RAW_BYTES;
                const int term = it / kt, kq = (it % kt) * BK;
                mbar_expect_tx(&full[r], 2 * TILE_BYTES);
                tma_load_3d(st, &maps[P.amap[term]], &full[r], m0, ka0 + kq, P.az[term]);
                tma_load_3d(st + TILE_BYTES, &maps[P.bmap[term]], &full[r], kq, n0, P.bz[term]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int it = 0; it < niter; ++it) {
                const int c = it % CONV;
                if (!mbar_wait(&conv_full[c], (uint32_t)((it / CONV) & 1), wlimit)) { s_fail = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char* cv = cvt + c * CONV_BYTES;
                const uint32_t a_hi = smem_u32(cv);
                const uint32_t a_lo = smem_u32(cv + TILE_BYTES);
                const uint32_t b_hi = smem_u32(cv + 2 * TILE_BYTES);
                const uint32_t b_lo = smem_u32(cv + 3 * TILE_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint32_t off = kk * 32;  // 8 tf32 along K = 32 bytes inside the swizzle row
                    const uint32_t acc0 = (it > 0 || kk > 0) ? 1u : 0u;
                    mma_tf32(tmem_d, sdesc_sw128(a_hi + off), sdesc_sw128(b_hi + off), acc0);
                    mma_tf32(tmem_d, sdesc_sw128(a_hi + off), sdesc_sw128(b_lo + off), 1u);
                    mma_tf32(tmem_d, sdesc_sw128(a_lo + off), sdesc_sw128(b_hi + off), 1u);
                    if (lolo) mma_tf32(tmem_d, sdesc_sw128(a_lo + off), sdesc_sw128(b_lo + off), 1u);
                }
                mma_commit(&conv_free[c]);
            }
            mma_commit(accb);
        }
    } else {
        // ---- converters (warps 2..9, 256 threads: two per scheduler) --------
        const int t = threadIdx.x - 64;
        const int am = t & (BM - 1), ah = t >> 7;  // A: row am, k chunks [4 ah, 4 ah + 4)
        for (int it = 0; it < niter; ++it) {
            const int r = it % RAW, c = it % CONV;
            if (!mbar_wait(&full[r], (uint32_t)((it / RAW) & 1), wlimit)) { s_fail = 1; break; }
            if (it >= CONV && !mbar_wait(&conv_free[c], (uint32_t)(((it / CONV) & 1) ^ 1), wlimit)) { s_fail = 1; break; }
            const unsigned char* st = raw + r * RAW_BYTES;
            unsigned char* cv = cvt + c * CONV_BYTES;
            const float* araw = reinterpret_cast<const float*>(st);   // [k][m], 32 x 128
            const float4* braw = reinterpret_cast<const float4*>(st + TILE_BYTES);
            unsigned char* ahi = cv;
            unsigned char* alo = cv + TILE_BYTES;
            float4* bhi = reinterpret_cast<float4*>(cv + 2 * TILE_BYTES);
            float4* blo = reinterpret_cast<float4*>(cv + 3 * TILE_BYTES);
            // A: row am, 4 chunks of 4 k -> K-major swizzled hi / lo
#pragma unroll
            for (int qq = 0; qq < BK / 8; ++qq) {
                const int q = ah * (BK / 8) + qq;
                float4 h, l;
                float x;
                x = araw[(4 * q + 0) * BM + am]; h.x = tf32_hi(x); l.x = tf32_rn(x - h.x);
                x = araw[(4 * q + 1) * BM + am]; h.y = tf32_hi(x); l.y = tf32_rn(x - h.y);
                x = araw[(4 * q + 2) * BM + am]; h.z = tf32_hi(x); l.z = tf32_rn(x - h.z);
                x = araw[(4 * q + 3) * BM + am]; h.w = tf32_hi(x); l.w = tf32_rn(x - h.w);
                const uint32_t o = sw128_off(am, 4 * q);
                *reinterpret_cast<float4*>(ahi + o) = h;
                *reinterpret_cast<float4*>(alo + o) = l;
            }
            // B: already in the K-major swizzled layout; split element-wise
#pragma unroll
            for (int j = 0; j < TILE_BYTES / 16 / 256; ++j) {
                const int i = t + j * 256;
                const float4 v = braw[i];
                float4 h, l;
                h.x = tf32_hi(v.x); l.x = tf32_rn(v.x - h.x);
                h.y = tf32_hi(v.y); l.y = tf32_rn(v.y - h.y);
                h.z = tf32_hi(v.z); l.z = tf32_rn(v.z - h.z);
                h.w = tf32_hi(v.w); l.w = tf32_rn(v.w - h.w);
                bhi[i] = h;
                blo[i] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&raw_free[r]);
                mbar_arrive(&conv_full[c]);
            }
        }
        // ---- epilogue ---------------------------------------------------------
        const bool ok = mbar_wait(accb, 0, wlimit);
        if (!ok) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        const int row = m0 + q * 32 + lane;
        const int half = (warp - 2) >> 2;  // two warps per quarter: columns [64 half, 64 half + 64)
#pragma unroll 1
        for (int cj = half * (BN / 64); cj < (half + 1) * (BN / 64); ++cj) {
            uint32_t r[32];
            const uint32_t taddr = tmem_d + ((uint32_t)(q * 32) << 16) + (uint32_t)(cj * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (ok && row < b) {
                // all 32 loads first: out may alias cin, so a load placed after
                // a store could not be moved ahead of it, and the chunk would
                // pay one memory round trip per column
                const size_t o0 = (size_t)row + (size_t)(n0 + cj * 32) * b;
                float cv[32];
                if (P.cin) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) cv[c] = P.cin[o0 + (size_t)c * b];
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) cv[c] = 0.f;
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) P.out[o0 + (size_t)c * b] = P.alpha * __uint_as_float(r[c]) + P.beta * cv[c];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(BN));
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and launch.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    // looked up once; every thread sees the final value (solves and factors
    // may run concurrently from several host threads)
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool tc_supported(int b) { return b >= 128 && b % 128 == 0 && encode_fn() != nullptr; }

// role 0: left operand (column-major rows are the MMA's M): box 128 rows x 32 k, no swizzle.
// role 1: right operand (K contiguous): box 32 k x 128 cols, 128-byte swizzle.
// `count` matrices of d0 (contiguous) x d1 FP32 elements, one after another.
int tc_encode_map_dims(void* map_out, const float* base, int d0, int d1, int count, int role) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)(count > 0 ? count : 1)};
    cuuint64_t strides[2] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * d1 * 4};
    cuuint32_t box[3] = {role == 0 ? (cuuint32_t)BM : (cuuint32_t)BK, role == 0 ? (cuuint32_t)BK : (cuuint32_t)BN, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<float*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    role == 0 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

int tc_encode_map(void* map_out, const float* base, int b, int count, int role) {
    return tc_encode_map_dims(map_out, base, b, b, count, role);
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t gemm_tc_ex(const TcProb* d_probs, int nprob, const void* d_maps, int b, int kdim, int ka0,
                       int tiles_n, int nskip, int nshift, int lolo, int* d_err, cudaStream_t s) {
    if (nprob <= 0 || tiles_n <= 0) return cudaSuccess;
    if (b % BM || kdim % BK || kdim <= 0 || ka0 % BK) return cudaErrorInvalidValue;
    ensure_smem((const void*)k_gemm_tc, SMEM_BYTES);
    const int tiles_m = b / BM;
    dim3 g(tiles_m * tiles_n, nprob);
    // ACR_TEST_TC_WITHHOLD=1 (failure-path tests): the producer issues no
    // copies and every wait gives up after a short limit, exercising the
    // bounded-wait path that ends in ACR_ERR_TIMEOUT with the context usable
    const char* wh = getenv("ACR_TEST_TC_WITHHOLD");
    const int withhold = (wh && wh[0] == '1') ? 1 : 0;
    const long long wlimit = withhold ? (1LL << 12) : WAIT_LIMIT;
    k_gemm_tc<<<g, NTHREADS, SMEM_BYTES, s>>>(d_probs, static_cast<const CUtensorMap*>(d_maps), b, tiles_m, d_err,
                                              kdim, ka0, nskip, nshift, lolo, wlimit, withhold);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gemm_tc(const TcProb* d_probs, int nprob, const void* d_maps, int b, int* d_err, cudaStream_t s) {
    return gemm_tc_ex(d_probs, nprob, d_maps, b, b, 0, b / BN, 1 << 30, 0, 0, d_err, s);
}

}  // namespace acr
