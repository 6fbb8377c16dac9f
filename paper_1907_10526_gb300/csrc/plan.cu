// plan.cu -- a projection call captured once into a CUDA graph and replayed.
//
// Iterative reconstruction calls the same projection on the same buffers many times.  A
// plan records one call (its launches, stream-ordered scratch allocations and frees) on a
// private stream as a CUDA graph; launching the plan then submits the whole call with one
// graph launch on the caller's stream, so the host's per-call work (argument checks,
// launch configuration, a dozen kernel launches) is paid once.
#include <cuda_runtime.h>

#include <new>

#include "cnsf.h"
#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

struct cnsf_plan {
    int device;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace cnsf {

int plan_create(const cnsf_geometry *geo, int op, const void *in, void *out, int batch, int dtype, cnsf_plan **res)
{
    typedef int (*Fn)(const cnsf_geometry *, const void *, void *, int, int, cudaStream_t);
    const Fn fns[4] = {launch_forward, launch_back, launch_forward_ref, launch_back_ref};
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return record_cuda_error(e);
    cnsf_plan *p = new (std::nothrow) cnsf_plan();
    if (!p) {
        cudaStreamDestroy(cap);
        return CNSF_ERR_NOMEM;
    }
    p->device = geo->device;
    int s = CNSF_OK;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = fns[op](geo, in, out, batch, dtype, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &p->graph);
        if (s == CNSF_OK && e2 != cudaSuccess) s = record_cuda_error(e2);
    } else {
        s = record_cuda_error(e);
    }
    if (s == CNSF_OK) {
        e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) s = record_cuda_error(e);
    }
    cudaStreamDestroy(cap);
    if (s != CNSF_OK) {
        plan_destroy(p);
        return s;
    }
    *res = p;
    return CNSF_OK;
}

int plan_launch(const cnsf_plan *p, cudaStream_t st)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (dev != p->device) return CNSF_ERR_INVALID;
    e = cudaGraphLaunch(p->exec, st);
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

void plan_destroy(cnsf_plan *p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
}

}  // namespace cnsf
