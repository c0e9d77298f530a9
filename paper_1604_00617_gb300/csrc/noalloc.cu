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
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress and cached.
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

int err(int code, const char* fmt, long long a = 0, long long b = 0, long long c = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b, c);
    return acr::set_last_error(code, buf);
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int acr_block_inverse_noalloc(int blksz, int count, double* mats, int* info, void* stream) {
    if (blksz < 1 || count < 0) return err(ACR_ERR_INVALID_ARG, "blksz must be >= 1 and count >= 0 (got %lld, %lld)", blksz, count);
    if (count == 0) return ACR_OK;
    if (!mats || !info) return err(ACR_ERR_INVALID_ARG, "mats and info must not be NULL");
    if (!on_device(mats) || !on_device(info))
        return err(ACR_ERR_INVALID_ARG, "mats and info must be device memory");
    const size_t need = acr::gj_scratch_bytes<double>(blksz, count);
    if (need > kScratchBytes)
        return err(ACR_ERR_INVALID_ARG,
                   "batch needs %lld scratch bytes, above the fixed %lld-byte scratch (blksz %lld): split the batch",
                   (long long)need, (long long)kScratchBytes, blksz);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return err(ACR_ERR_CUDA, "no usable current device (%lld)", dev);
    }
    void* scratch = nullptr;
    {
        // first call on this device: look up the array's device address with
        // this device current (not capturable: make this call before capture)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return err(ACR_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed (error %lld)", (long long)e);
            }
            g_scratch_addr[dev] = p;
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
