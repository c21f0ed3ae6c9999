// Device scratch for rascas_propagate_noalloc: a file-scope device array, so
// that the entry point needs no cudaMalloc.  Every GPU that loads the library
// holds these 8 MiB until the process exits.
#include <cuda_runtime.h>
#include "internal.h"

namespace rg {

namespace {
constexpr size_t kNoAllocBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
}  // namespace

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in for the array, so the address is looked up with
// cudaGetSymbolAddress.  rascas_create calls this once per context, with the
// context's device current: the lookup loads the module that holds the array
// (under lazy module loading its 8 MiB are allocated then), and a context
// created after a device reset gets the address of the reloaded module.
cudaError_t noalloc_scratch(void** ptr, size_t* bytes) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *ptr = p;
    *bytes = kNoAllocBytes;
    return cudaSuccess;
}

}  // namespace rg
