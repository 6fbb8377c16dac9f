// noalloc.cu -- forward projection that allocates no device memory.
//
// Some callers must not allocate: a plugin inside a host framework that owns the whole
// device-memory budget and forbids raw allocations in its execution step, or a
// latency-critical loop that cannot afford the allocator's locks and possible
// synchronisation.  cnsf_forward_project allocates its scratch (zero-padded copies of
// the image) stream-ordered on every call; this entry point uses a fixed array in the
// library's own device memory instead.  That array is reserved on every GPU that loads
// the library and stays reserved until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "cnsf.h"
#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CNSF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[kMaxDevices];   // device address of the array, per device

// Once per device, with that device current: the array's name in host code is only a
// host-side stand-in, so its device address is looked up here and passed to the kernels.
static int noalloc_scratch_address(int dev, void **addr)
{
    if (dev < 0 || dev >= kMaxDevices) return CNSF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return record_cuda_error(e);
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return CNSF_OK;
}

}  // namespace cnsf

using namespace cnsf;

extern "C" CNSF_API int cnsf_forward_project_noalloc(const cnsf_geometry *geom, const void *image, void *sino,
                                                     int32_t batch, int32_t dtype, void *stream)
{
    try {
        if (!geom || batch < 0 || (dtype != CNSF_F32 && dtype != CNSF_F64)) return CNSF_ERR_INVALID;
        if (batch > 0 && (!image || !sino)) return CNSF_ERR_INVALID;
        if (batch > 65535) return CNSF_ERR_UNSUPPORTED;
        int dev = -1;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return record_cuda_error(e);
        if (dev != geom->device) return CNSF_ERR_INVALID;
        if (batch == 0) return CNSF_OK;
        if (forward_scratch_bytes(geom, batch, dtype) > (size_t)CNSF_NOALLOC_SCRATCH_BYTES)
            return CNSF_ERR_UNSUPPORTED;
        void *scratch = nullptr;
        int s = noalloc_scratch_address(dev, &scratch);
        if (s != CNSF_OK) return s;
        // The padding kernels write every element of the copies they use, zeros included,
        // so whatever an earlier call left in the array never reaches the result.
        return launch_forward_with_scratch(geom, image, sino, batch, dtype, scratch,
                                           (size_t)CNSF_NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}
