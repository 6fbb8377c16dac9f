// capi.cu -- extern "C" entry points of include/cnsf.h: argument checks, device checks and
// error translation around the kernel launchers.  No exception crosses this boundary.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <exception>

#include "cnsf.h"
#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

static thread_local char g_last_cuda[256] = "no CUDA error recorded";

int record_cuda_error(cudaError_t e)
{
    std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return CNSF_ERR_CUDA;
}

// The geometry's tables live on one device; calls must be made with that device current.
static int check_device(const cnsf_geometry *geo)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    return dev == geo->device ? CNSF_OK : CNSF_ERR_INVALID;
}

static int check_call(const cnsf_geometry *geo, const void *in, void *out, int32_t batch, int32_t dtype)
{
    if (!geo || batch < 0) return CNSF_ERR_INVALID;
    if (dtype != CNSF_F32 && dtype != CNSF_F64) return CNSF_ERR_INVALID;
    if (batch > 0 && (!in || !out)) return CNSF_ERR_INVALID;
    if (batch > 65535) return CNSF_ERR_UNSUPPORTED;   // grid z/y extent
    return check_device(geo);
}

}  // namespace cnsf

using namespace cnsf;

extern "C" {

int cnsf_geometry_create(const cnsf_geometry_desc *desc, cnsf_geometry **out)
{
    try {
        return build_geometry(desc, out);
    } catch (const std::bad_alloc &) {
        return CNSF_ERR_NOMEM;
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

void cnsf_geometry_destroy(cnsf_geometry *geom)
{
    try {
        destroy_geometry(geom);
    } catch (...) {
    }
}

int cnsf_geometry_shape(const cnsf_geometry *geom, int32_t *n_x, int32_t *n_y, int32_t *n_views, int32_t *n_det)
{
    if (!geom) return CNSF_ERR_INVALID;
    if (n_x) *n_x = geom->gc.nx;
    if (n_y) *n_y = geom->gc.ny;
    if (n_views) *n_views = geom->gc.nv;
    if (n_det) *n_det = geom->gc.nd;
    return CNSF_OK;
}

int cnsf_forward_project(const cnsf_geometry *geom, const void *image, void *sino, int32_t batch, int32_t dtype,
                         void *stream)
{
    try {
        int s = check_call(geom, image, sino, batch, dtype);
        if (s != CNSF_OK) return s;
        return launch_forward(geom, image, sino, batch, dtype, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_back_project(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch, int32_t dtype,
                      void *stream)
{
    try {
        int s = check_call(geom, sino, image, batch, dtype);
        if (s != CNSF_OK) return s;
        return launch_back(geom, sino, image, batch, dtype, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_forward_project_ref(const cnsf_geometry *geom, const void *image, void *sino, int32_t batch, int32_t dtype,
                             void *stream)
{
    try {
        int s = check_call(geom, image, sino, batch, dtype);
        if (s != CNSF_OK) return s;
        return launch_forward_ref(geom, image, sino, batch, dtype, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_back_project_ref(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch, int32_t dtype,
                          void *stream)
{
    try {
        int s = check_call(geom, sino, image, batch, dtype);
        if (s != CNSF_OK) return s;
        return launch_back_ref(geom, sino, image, batch, dtype, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_count_nonzeros(const cnsf_geometry *geom, uint64_t *count, void *stream)
{
    try {
        if (!geom || !count) return CNSF_ERR_INVALID;
        int s = check_device(geom);
        if (s != CNSF_OK) return s;
        return count_nonzeros(geom, count, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

size_t cnsf_solver_workspace_bytes(const cnsf_geometry *geom, int32_t dtype)
{
    if (!geom || (dtype != CNSF_F32 && dtype != CNSF_F64)) return 0;
    return solver_workspace_bytes(geom, dtype);
}

static int solver_call(const cnsf_geometry *geom, int algo, const void *sino, void *image, int32_t iters,
                       double relax, int32_t resume, int32_t dtype, void *ws, size_t ws_bytes, void *stream)
{
    try {
        int s = check_call(geom, sino, image, 1, dtype);
        if (s != CNSF_OK) return s;
        if (iters < 0 || !(relax > 0.0 && relax < 2.0)) return CNSF_ERR_INVALID;
        return run_solver(geom, algo, sino, image, iters, relax, resume, dtype, ws, ws_bytes, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_sirt(const cnsf_geometry *geom, const void *sino, void *image, int32_t iters, double relax, int32_t dtype,
              void *ws, size_t ws_bytes, void *stream)
{
    return solver_call(geom, 0, sino, image, iters, relax, 0, dtype, ws, ws_bytes, stream);
}

int cnsf_cgls(const cnsf_geometry *geom, const void *sino, void *image, int32_t iters, int32_t resume, int32_t dtype,
              void *ws, size_t ws_bytes, void *stream)
{
    return solver_call(geom, 1, sino, image, iters, 1.0, resume, dtype, ws, ws_bytes, stream);
}

const char *cnsf_status_string(int status)
{
    switch (status) {
        case CNSF_OK: return "ok";
        case CNSF_ERR_INVALID: return "invalid argument or geometry";
        case CNSF_ERR_CUDA: return "CUDA runtime error";
        case CNSF_ERR_NOMEM: return "out of memory";
        case CNSF_ERR_UNSUPPORTED: return "unsupported request";
        case CNSF_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

const char *cnsf_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
