// cnsf_runtime.h -- internal entry points between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cnsf.h"

namespace cnsf {

// Remember the CUDA error text for cnsf_last_cuda_error (per host thread); returns CNSF_ERR_CUDA.
int record_cuda_error(cudaError_t e = cudaGetLastError());

// Stream-ordered scratch for one call: from the library's per-device pool (which keeps up to
// CNSF_SCRATCH_KEEP_BYTES mapped across synchronisations), or the graph's own allocation
// while `st` is being captured.  Freed with cudaFreeAsync.
cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st);

int build_geometry(const cnsf_geometry_desc *d, cnsf_geometry **out);
void destroy_geometry(cnsf_geometry *geo);
// Precompute the back projector's per-(tile, view) coefficients when they fit 1 GiB (back.cu).
int build_tile_view_table(cnsf_geometry *geo);

// Kernel launchers (arguments already validated by the C ABI layer).
int launch_forward(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype,
                   cudaStream_t stream);
int launch_back(const cnsf_geometry *geo, const void *sino, void *img, int batch, int dtype,
                cudaStream_t stream);
int count_nonzeros(const cnsf_geometry *geo, uint64_t *count, cudaStream_t stream);

// Reference projector (reference.cu): bin-averaged exact chords, FP64 entries.
int launch_forward_ref(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype,
                       cudaStream_t stream);
int launch_back_ref(const cnsf_geometry *geo, const void *sino, void *img, int batch, int dtype,
                    cudaStream_t stream);

// Projection plans (plan.cu): op 0 forward, 1 back, 2 reference forward, 3 reference back.
int plan_create(const cnsf_geometry *geo, int op, const void *in, void *out, int batch, int dtype, cnsf_plan **res);
int plan_launch(const cnsf_plan *p, cudaStream_t stream);
void plan_destroy(cnsf_plan *p);

// Forward projection into caller-provided scratch (bytes from forward_scratch_bytes).
size_t forward_scratch_bytes(const cnsf_geometry *geo, int batch, int dtype);
int launch_forward_with_scratch(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype,
                                void *scratch, size_t scratch_bytes, cudaStream_t stream);

// Device bytes a projection call allocates stream-ordered, all held at once (forward.cu,
// back.cu, batch.cu).
size_t forward_alloc_bytes(const cnsf_geometry *geo, int batch, int dtype);
size_t back_alloc_bytes(const cnsf_geometry *geo, int batch, int dtype);
size_t forward_batch_alloc_bytes(const cnsf_geometry *geo);
size_t back_batch_alloc_bytes(const cnsf_geometry *geo);

// FP32 projections of a batch through the symmetric kernels (geo->sym8 or geo->sym;
// CNSF_ERR_UNSUPPORTED otherwise): each image as in a single-image call, so its result does
// not depend on the batch.
int launch_forward_sym(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t stream);
int launch_back_sym(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t stream);

// Images per launch group of the symmetric kernels: as many as keep the group's scratch
// within 256 MiB, at least one, at most the batch.
inline int sym_batch_group(size_t per_image_bytes, int batch)
{
    const size_t cap = (size_t)256 << 20;
    size_t g = per_image_bytes > 0 ? cap / per_image_bytes : (size_t)batch;
    if (g < 1) g = 1;
    if (g > (size_t)batch) g = (size_t)batch;
    return batch > 0 ? (int)g : 1;
}

// Batches of FP32 images (batch.cu): each entry evaluated once per chunk of <= 16 images.
int launch_forward_batch(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t stream);
int launch_back_batch(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t stream);

// Iterative drivers (solver.cu): algo 0 = SIRT, 1 = CGLS.
size_t solver_workspace_bytes(const cnsf_geometry *geo, int dtype);
// CGLS over a batch of problems with one geometry (solver.cu).
size_t cgls_batched_workspace_bytes(const cnsf_geometry *geo, int batch, int dtype);
int run_cgls_batched(const cnsf_geometry *geo, const void *sino, void *image, int batch, int iters, int resume,
                     int dtype, void *ws, size_t ws_bytes, cudaStream_t stream);
// ASD-POCS (solver.cu) over ordered subsets of views, one geometry per subset.
size_t asd_workspace_bytes(const cnsf_geometry *const *subsets, int n_subsets, int dtype);
int run_asd_pocs(const cnsf_geometry *const *subsets, int n_subsets, const int *rows, const void *sino, void *image,
                 const cnsf_asd_pocs_params &params, int dtype, void *ws, size_t ws_bytes, cudaStream_t stream);
int run_solver(const cnsf_geometry *geo, int algo, const void *sino, void *image, int iters, double relax,
               int resume, int dtype, void *ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace cnsf
