// Device scratch for rascas_propagate_noalloc: a file-scope device array, so
// that the entry point needs no cudaMalloc.  Every GPU that loads the library
// holds these 8 MiB until the process exits.
#include <mutex>
#include <cuda_runtime.h>
#include "internal.h"

namespace rg {

namespace {
constexpr size_t kNoAllocBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {};
std::mutex g_lock;
}  // namespace

// Device address of the scratch array on `device` (which must be current).
// The host-side symbol is only a stand-in for the array, so the address is
// taken once per device with cudaGetSymbolAddress and cached.
cudaError_t noalloc_scratch(int device, void** ptr, size_t* bytes) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_lock);
    if (g_addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *ptr = g_addr[device];
    *bytes = kNoAllocBytes;
    return cudaSuccess;
}

}  // namespace rg
