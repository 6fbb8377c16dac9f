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

#include "cnsf.h"
#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CNSF_NOALLOC_SCRATCH_BYTES];

// The array's name in host code is only a host-side stand-in, so its device address is
// looked up for the current device (a host-side query, repeated on every call so that a
// device reset that reloads the module cannot leave a stale address behind).
static int noalloc_scratch_address(void **addr)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return record_cuda_error(e);
    *addr = p;
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
        int s = noalloc_scratch_address(&scratch);
        if (s != CNSF_OK) return s;
        // The padding kernels write every element of the copies they use, zeros included,
        // so whatever an earlier call left in the array never reaches the result.
        return launch_forward_with_scratch(geom, image, sino, batch, dtype, scratch,
                                           (size_t)CNSF_NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}
