// capi.cu -- extern "C" entry points of include/cnsf.h: argument checks, device checks and
// error translation around the kernel launchers.  No exception crosses this boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <vector>

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

// Per-device memory pools of the library's own for the projections' stream-ordered scratch.
// The default pool returns its free memory to the driver at every synchronisation, so a
// call made after one mapped its scratch afresh (about 0.3 ms for the 90 MB of a 16-image
// forward projection); these pools keep up to CNSF_SCRATCH_KEEP_BYTES mapped.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static cudaError_t scratch_pool(cudaMemPool_t *pool)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = CNSF_SCRATCH_KEEP_BYTES;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *pool = g_pool[dev];
    return cudaSuccess;
}

cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    // under capture the allocation becomes the graph's own (kept across its replays)
    if (cs != cudaStreamCaptureStatusNone) return cudaMallocAsync(ptr, bytes, st);
    cudaMemPool_t pool;
    if ((e = scratch_pool(&pool)) != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
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
        // lengths must be finite as well as positive (the geometry builder checks the rest)
        if (desc && (!std::isfinite(desc->pixel_mm) || !std::isfinite(desc->det_spacing_mm) ||
                     !std::isfinite(desc->det_width_mm) ||
                     (desc->detector != CNSF_DETECTOR_PARALLEL &&
                      (!std::isfinite(desc->d_po_mm) || !std::isfinite(desc->d_ps_mm)))))
            return CNSF_ERR_INVALID;
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

int cnsf_geometry_paths(const cnsf_geometry *geom, int32_t *symmetric, int32_t *exact_differences)
{
    if (!geom) return CNSF_ERR_INVALID;
    if (symmetric) *symmetric = geom->sym8 ? 8 : geom->sym ? 4 : 1;
    if (exact_differences) *exact_differences = geom->exact;
    return CNSF_OK;
}

int cnsf_geometry_device_bytes(const cnsf_geometry *geom, size_t *bytes)
{
    if (!geom || !bytes) return CNSF_ERR_INVALID;
    *bytes = geom->device_bytes;
    return CNSF_OK;
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

size_t cnsf_cgls_batched_workspace_bytes(const cnsf_geometry *geom, int32_t batch, int32_t dtype)
{
    if (!geom || batch < 0 || batch > 65535 || (dtype != CNSF_F32 && dtype != CNSF_F64)) return 0;
    return cgls_batched_workspace_bytes(geom, batch, dtype);
}

int cnsf_cgls_batched(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch, int32_t iters,
                      int32_t resume, int32_t dtype, void *ws, size_t ws_bytes, void *stream)
{
    try {
        int s = check_call(geom, sino, image, batch, dtype);
        if (s != CNSF_OK) return s;
        if (iters < 0) return CNSF_ERR_INVALID;
        return run_cgls_batched(geom, sino, image, batch, iters, resume, dtype, ws, ws_bytes, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

}  // extern "C"

namespace {

// Subsets must share everything but their views, live on the current device, and the rows
// must be a permutation of the total views.
int check_subsets(const cnsf_geometry *const *sub, int32_t nsub)
{
    if (!sub || nsub < 1) return CNSF_ERR_INVALID;
    for (int k = 0; k < nsub; ++k) {
        if (!sub[k]) return CNSF_ERR_INVALID;
        const GeomConsts &a = sub[0]->gc, &b = sub[k]->gc;
        if (a.nx != b.nx || a.ny != b.ny || a.nd != b.nd || a.h != b.h || a.cx != b.cx || a.cy != b.cy ||
            a.ds != b.ds || a.tau != b.tau || a.doff != b.doff || a.dpo != b.dpo || a.dps != b.dps ||
            a.par != b.par || a.arc != b.arc || sub[k]->device != sub[0]->device)
            return CNSF_ERR_INVALID;
    }
    return check_device(sub[0]);
}

}  // namespace

extern "C" {

size_t cnsf_asd_pocs_workspace_bytes(const cnsf_geometry *const *subsets, int32_t n_subsets, int32_t dtype)
{
    try {
        if (dtype != CNSF_F32 && dtype != CNSF_F64) return 0;
        if (!subsets || n_subsets < 1) return 0;
        for (int k = 0; k < n_subsets; ++k)
            if (!subsets[k]) return 0;
        return asd_workspace_bytes(subsets, n_subsets, dtype);
    } catch (...) {
        return 0;
    }
}

int cnsf_asd_pocs(const cnsf_geometry *const *subsets, int32_t n_subsets, const int32_t *rows, const void *sino,
                  void *image, const cnsf_asd_pocs_params *params, int32_t dtype, void *ws, size_t ws_bytes,
                  void *stream)
{
    try {
        int s = check_subsets(subsets, n_subsets);
        if (s != CNSF_OK) return s;
        if (!rows || !sino || !image || !params || (dtype != CNSF_F32 && dtype != CNSF_F64)) return CNSF_ERR_INVALID;
        const cnsf_asd_pocs_params &P = *params;
        if (P.iters < 0 || P.tv_steps < 0 || !(P.relax > 0.0 && P.relax < 2.0) ||
            !(P.relax_red > 0.0 && P.relax_red <= 1.0) || !(P.alpha >= 0.0) ||
            !(P.alpha_red > 0.0 && P.alpha_red <= 1.0) || !(P.r_max > 0.0) || !(P.tv_eps >= 0.0) ||
            !std::isfinite(P.data_tol) || (P.projector != CNSF_PROJECTOR_CNSF && P.projector != CNSF_PROJECTOR_REF))
            return CNSF_ERR_INVALID;
        long long total = 0;
        for (int k = 0; k < n_subsets; ++k) total += subsets[k]->gc.nv;
        std::vector<char> seen((size_t)total, 0);
        std::vector<int> rows_copy((size_t)total);   // pageable: the upload is staged before return
        for (long long t = 0; t < total; ++t) {
            if (rows[t] < 0 || rows[t] >= total || seen[(size_t)rows[t]]) return CNSF_ERR_INVALID;
            seen[(size_t)rows[t]] = 1;
            rows_copy[(size_t)t] = rows[t];
        }
        return run_asd_pocs(subsets, n_subsets, rows_copy.data(), sino, image, P, dtype, ws, ws_bytes,
                            (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        return CNSF_ERR_NOMEM;
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_plan_create(const cnsf_geometry *geom, int32_t op, const void *in, void *out, int32_t batch, int32_t dtype,
                     cnsf_plan **plan)
{
    try {
        if (!plan) return CNSF_ERR_INVALID;
        *plan = nullptr;
        if (op < CNSF_OP_FORWARD || op > CNSF_OP_BACK_REF) return CNSF_ERR_INVALID;
        int s = check_call(geom, in, out, batch, dtype);
        if (s != CNSF_OK) return s;
        return plan_create(geom, op, in, out, batch, dtype, plan);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_projection_scratch_bytes(const cnsf_geometry *geom, int32_t op, int32_t batch, int32_t dtype,
                                  size_t *bytes)
{
    try {
        if (!geom || !bytes || batch < 0) return CNSF_ERR_INVALID;
        if (dtype != CNSF_F32 && dtype != CNSF_F64) return CNSF_ERR_INVALID;
        switch (op) {
        case CNSF_OP_FORWARD: *bytes = forward_alloc_bytes(geom, batch, dtype); return CNSF_OK;
        case CNSF_OP_BACK: *bytes = back_alloc_bytes(geom, batch, dtype); return CNSF_OK;
        case CNSF_OP_FORWARD_REF:
        case CNSF_OP_BACK_REF: *bytes = 0; return CNSF_OK;
        default: return CNSF_ERR_INVALID;
        }
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_plan_launch(const cnsf_plan *plan, void *stream)
{
    try {
        if (!plan) return CNSF_ERR_INVALID;
        return plan_launch(plan, (cudaStream_t)stream);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

void cnsf_plan_destroy(cnsf_plan *plan)
{
    try {
        plan_destroy(plan);
    } catch (...) {
    }
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

int cnsf_scratch_pool_stats(size_t *reserved, size_t *used_high, int32_t reset_high)
{
    try {
        cudaMemPool_t pool;
        cudaError_t e = scratch_pool(&pool);
        uint64_t r = 0, h = 0;
        if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
        if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h);
        if (e == cudaSuccess && reset_high) {
            uint64_t zero = 0;   // the only value the attribute may be set to
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
        }
        if (e != cudaSuccess) return record_cuda_error(e);
        if (reserved) *reserved = (size_t)r;
        if (used_high) *used_high = (size_t)h;
        return CNSF_OK;
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

int cnsf_scratch_trim(void)
{
    try {
        cudaMemPool_t pool;
        cudaError_t e = scratch_pool(&pool);
        if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
        return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
    } catch (...) {
        return CNSF_ERR_INTERNAL;
    }
}

const char *cnsf_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
