// noalloc.cu -- batched block inversion that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// batch of block inverses: code running inside another framework's memory
// pool that has already reserved nearly all of the GPU's memory, latency-
// critical paths that cannot absorb an allocation (or its failure, or the
// device synchronisation cudaFree can cause), and hosts that hand the library
// only the buffers it computes on.  acr_block_inverse_noalloc serves them: it
// runs the same batched Gauss-Jordan inversion as the factorization, but takes
// every temporary from one fixed scratch array compiled into this library.
//
// The scratch is a file-scope __device__ array of ACR_NOALLOC_SCRATCH_BYTES
// (16 MiB).  Every GPU on which the library's module is loaded holds it until
// the process exits.  In host code the array's name is only a host-side
// stand-in, so its device address is looked up with cudaGetSymbolAddress,
// with the device current, and cached per device together with the identity
// of the CUDA context it belongs to.  A device reset destroys that context
// (and the module with the array); the next call sees a different context and
// looks the address up again instead of using the stale one.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/acr.h"
#include "acr_internal.h"

namespace {

constexpr size_t kScratchBytes = ACR_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (driver entry points
// cuCtxGetCurrent and cuCtxGetId); 0 if there is none or it cannot be read.
unsigned long long current_context_id() {
    typedef int (*GetCurrent)(void**);
    typedef int (*GetId)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

int err(int code, const char* fmt, long long a = 0, long long b = 0, long long c = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b, c);
    return acr::set_last_error(code, buf);
}

// Device memory of GPU `dev` (or managed memory).  Memory of another GPU is
// refused: the kernels run on the current device and would fault reading it.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int acr_block_inverse_noalloc(int blksz, int count, double* mats, int* info, void* stream) {
    if (blksz < 1 || count < 0) return err(ACR_ERR_INVALID_ARG, "blksz must be >= 1 and count >= 0 (got %lld, %lld)", blksz, count);
    if (count == 0) return ACR_OK;
    if (!mats || !info) return err(ACR_ERR_INVALID_ARG, "mats and info must not be NULL");
    const size_t need = acr::gj_scratch_bytes<double>(blksz, count);
    if (need > kScratchBytes)
        return err(ACR_ERR_INVALID_ARG,
                   "batch needs %lld scratch bytes, above the fixed %lld-byte scratch (blksz %lld): split the batch",
                   (long long)need, (long long)kScratchBytes, blksz);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return err(ACR_ERR_INVALID_ARG, "no usable current CUDA device (%lld)", dev);
    }
    if (!on_device(mats, dev) || !on_device(info, dev))
        return err(ACR_ERR_INVALID_ARG, "mats and info must be device memory of the current device %lld", dev);
    void* scratch = nullptr;
    {
        // first call on this device (or in a new context after a device
        // reset): look up the array's device address with this device
        // current (not capturable: make this call before any capture)
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return err(ACR_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed (error %lld)", (long long)e);
            }
            g_scratch_addr[dev] = p;
            g_scratch_ctx[dev] = current_context_id();
        }
        scratch = g_scratch_addr[dev];
    }
    const cudaError_t e = acr::gj_inverse_scratch<double>(mats, blksz, count, info, scratch, kScratchBytes,
                                                          static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return err(ACR_ERR_CUDA, "launch failed (error %lld)", (long long)e);
    }
    return ACR_OK;
}
