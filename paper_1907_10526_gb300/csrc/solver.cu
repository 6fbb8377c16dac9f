// solver.cu -- SIRT and CGLS drivers around the forward and back projectors.
//
// Neither algorithm is in the paper (its reconstructions use ASD-POCS); both are the
// textbook forms named in the header.  CGLS carries x, r and p in FP64 (the projections run
// in the requested precision).  Every iteration is launched asynchronously on the
// caller's stream: the step lengths are computed on the device from FP64 dot products
// and read by the update kernels, so the host never waits inside the loop.  Reductions
// are two-pass with a fixed block order, so a result does not depend on what else runs
// on the GPU.
#include <cuda_runtime.h>

#include <algorithm>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

constexpr int RED_BLOCKS = 1024;   // partial sums of a dot product
constexpr int RED_THREADS = 256;

// ---------------------------------------------------------------- workspace layout
// [ scalars | partials | x64 | p64 | r64 | pT | sT | qT | rT ]   (T = projector precision)
// CGLS keeps its state (x, p, r) in FP64 whatever the projector precision: recursive CG
// with FP32 vectors loses orthogonality within tens of iterations, while the FP32
// projections only add their own ~1e-7 error.  SIRT uses sT/qT/rT/pT as scratch.
struct SolverWs {
    double *scal;        // [0] gamma, [1] <q,q>, [2] gamma_new
    double *part;        // RED_BLOCKS partial sums
    double *x64, *p64;   // image-sized, FP64
    double *r64;         // sinogram-sized, FP64
    void *pT, *sT;       // image-sized, projector precision
    void *qT, *rT;       // sinogram-sized, projector precision
};

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

static size_t ws_layout(const cnsf_geometry *geo, int dtype, SolverWs *w, void *base)
{
    const GeomConsts &g = geo->gc;
    size_t el = dtype == CNSF_F64 ? sizeof(double) : sizeof(float);
    size_t ns = (size_t)g.nv * g.nd, ni = (size_t)g.nx * g.ny;
    size_t off = 0;
    size_t o_scal = off; off += align256(8 * sizeof(double));
    size_t o_part = off; off += align256(RED_BLOCKS * sizeof(double));
    size_t o_x = off; off += align256(ni * sizeof(double));
    size_t o_p = off; off += align256(ni * sizeof(double));
    size_t o_r = off; off += align256(ns * sizeof(double));
    size_t o_pT = off; off += align256(ni * el);
    size_t o_sT = off; off += align256(ni * el);
    size_t o_qT = off; off += align256(ns * el);
    size_t o_rT = off; off += align256(ns * el);
    if (w && base) {
        char *b = (char *)base;
        w->scal = (double *)(b + o_scal);
        w->part = (double *)(b + o_part);
        w->x64 = (double *)(b + o_x);
        w->p64 = (double *)(b + o_p);
        w->r64 = (double *)(b + o_r);
        w->pT = b + o_pT; w->sT = b + o_sT; w->qT = b + o_qT; w->rT = b + o_rT;
    }
    return off;
}

size_t solver_workspace_bytes(const cnsf_geometry *geo, int dtype) { return ws_layout(geo, dtype, nullptr, nullptr); }

// ---------------------------------------------------------------- vector kernels
template <typename T>
__global__ void fill_kernel(T *x, size_t n, T v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

// w = 1/w where w > 0, else 0 (SIRT row and column weights)
template <typename T>
__global__ void recip_kernel(T *w, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w[i] = w[i] > T(0) ? T(1) / w[i] : T(0);
}

// r = R (y - Ax), in place on Ax
template <typename T>
__global__ void sirt_residual_kernel(T *ax, const T *__restrict__ y, const T *__restrict__ R, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        ax[i] = R[i] * (y[i] - ax[i]);
}

// x += relax C g
template <typename T>
__global__ void sirt_update_kernel(T *x, const T *__restrict__ g, const T *__restrict__ C, T relax, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] += relax * C[i] * g[i];
}

// Deterministic <a, a> in FP64: fixed grid of RED_BLOCKS blocks, each summing a fixed
// strided subset, then one block summing the partials in order.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) sumsq_partial_kernel(const T *__restrict__ a, size_t n,
                                                                    double *__restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < n; i += (size_t)RED_BLOCKS * RED_THREADS) {
        double v = (double)a[i];
        s = fma(v, v, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(RED_THREADS) sum_final_kernel(const double *__restrict__ part, double *out)
{
    __shared__ double sh[RED_THREADS];
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <typename Ti, typename To>
__global__ void convert_kernel(To *dst, const Ti *__restrict__ src, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (To)src[i];
}

// r64 = y - Ax (FP64), rT = r64 in projector precision
template <typename T>
__global__ void cgls_init_r_kernel(double *r64, T *rT, const T *__restrict__ y, const T *__restrict__ ax, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double r = (double)y[i] - (double)ax[i];
        r64[i] = r;
        rT[i] = (T)r;
    }
}

// p64 = s, pT = s
template <typename T>
__global__ void cgls_init_p_kernel(double *p64, T *pT, const T *__restrict__ sT, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        p64[i] = (double)sT[i];
        pT[i] = sT[i];
    }
}

// CGLS step: alpha = gamma / <q,q> (0 when either vanishes); x += alpha p over the image
// and r -= alpha q over the sinogram (FP64 state), rT = r for the back projection; one launch.
template <typename T>
__global__ void cgls_xr_kernel(double *x, const double *__restrict__ p, size_t nimg, double *r, T *rT,
                               const T *__restrict__ q, size_t nsino, const double *__restrict__ scal)
{
    const double gam = scal[0], qq = scal[1];
    const double alpha = (gam > 0.0 && qq > 0.0) ? gam / qq : 0.0;
    const size_t n = nimg + nsino;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (i < nimg) {
            x[i] = fma(alpha, p[i], x[i]);
        } else {
            const size_t k = i - nimg;
            const double rv = fma(-alpha, (double)q[k], r[k]);
            r[k] = rv;
            rT[k] = (T)rv;
        }
    }
}

// p = s + beta p (FP64), beta = gamma_new / gamma (0 when gamma vanishes); pT = p
template <typename T>
__global__ void cgls_p_kernel(double *p, T *pT, const T *__restrict__ s, size_t n, const double *__restrict__ scal)
{
    const double gam = scal[0], gnew = scal[2];
    const double beta = gam > 0.0 ? gnew / gam : 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double pv = fma(beta, p[i], (double)s[i]);
        p[i] = pv;
        pT[i] = (T)pv;
    }
}

// gamma <- gamma_new (after every thread of cgls_p_kernel has read the old gamma)
__global__ void cgls_roll_kernel(double *scal) { scal[0] = scal[2]; }

static inline dim3 grid_for(size_t n) { return dim3((unsigned)std::min<size_t>((n + 255) / 256, 4096)); }

// Run `iters` identical iterations.  The launches of one iteration (projections with their
// stream-ordered scratch, reductions, updates: tens of small launches) are captured once
// into a CUDA graph on a private stream and the graph is launched `iters` times on the
// caller's stream, so the host submits one launch per iteration.  Short runs (fewer than
// `min_graph` iterations) launch directly.  `body(stream)` issues one iteration and returns
// a status; it must not depend on the iteration index (step-dependent choices are made by
// the kernels from device scalars).
template <typename Body>
static int run_iterations(int iters, cudaStream_t st, Body body, int min_graph = 3)
{
    if (iters < min_graph) {
        for (int k = 0; k < iters; ++k) {
            int s = body(st);
            if (s != CNSF_OK) return s;
        }
        return CNSF_OK;
    }
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return record_cuda_error(e);
    int s = CNSF_OK;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = body(cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (s == CNSF_OK && e2 != cudaSuccess) s = record_cuda_error(e2);
    } else {
        s = record_cuda_error(e);
    }
    if (s == CNSF_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) s = record_cuda_error(e);
    }
    for (int k = 0; s == CNSF_OK && k < iters; ++k) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) s = record_cuda_error(e);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);   // returns at once; the stream is released when its work is done
    return s;
}

template <typename T>
static void sumsq(const T *a, size_t n, SolverWs &w, double *dst, cudaStream_t st)
{
    sumsq_partial_kernel<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, n, w.part);
    sum_final_kernel<<<1, RED_THREADS, 0, st>>>(w.part, dst);
}

// ---------------------------------------------------------------- drivers
template <typename T>
static int sirt_impl(const cnsf_geometry *geo, const T *y, T *x, int iters, double relax, int dtype, SolverWs &w,
                     cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const size_t ns = (size_t)g.nv * g.nd, ni = (size_t)g.nx * g.ny;
    T *R = (T *)w.qT, *r = (T *)w.rT, *C = (T *)w.pT, *gr = (T *)w.sT;
    int s;
    // R = 1/(A 1), C = 1/(A^T 1)
    fill_kernel<T><<<grid_for(ni), 256, 0, st>>>(gr, ni, T(1));
    if ((s = launch_forward(geo, gr, R, 1, dtype, st)) != CNSF_OK) return s;
    recip_kernel<T><<<grid_for(ns), 256, 0, st>>>(R, ns);
    fill_kernel<T><<<grid_for(ns), 256, 0, st>>>(r, ns, T(1));
    if ((s = launch_back(geo, r, C, 1, dtype, st)) != CNSF_OK) return s;
    recip_kernel<T><<<grid_for(ni), 256, 0, st>>>(C, ni);
    s = run_iterations(iters, st, [&](cudaStream_t q) -> int {
        int t;
        if ((t = launch_forward(geo, x, r, 1, dtype, q)) != CNSF_OK) return t;
        sirt_residual_kernel<T><<<grid_for(ns), 256, 0, q>>>(r, y, R, ns);
        if ((t = launch_back(geo, r, gr, 1, dtype, q)) != CNSF_OK) return t;
        sirt_update_kernel<T><<<grid_for(ni), 256, 0, q>>>(x, gr, C, (T)relax, ni);
        return CNSF_OK;
    });
    if (s != CNSF_OK) return s;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

template <typename T>
static int cgls_impl(const cnsf_geometry *geo, const T *y, T *x, int iters, int resume, int dtype, SolverWs &w,
                     cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const size_t ns = (size_t)g.nv * g.nd, ni = (size_t)g.nx * g.ny;
    T *pT = (T *)w.pT, *sT = (T *)w.sT, *qT = (T *)w.qT, *rT = (T *)w.rT;
    int s;
    if (!resume) {
        // x = x0; r = y - A x0; s = A^T r; p = s; gamma = <s,s>
        convert_kernel<T, double><<<grid_for(ni), 256, 0, st>>>(w.x64, x, ni);
        if ((s = launch_forward(geo, x, qT, 1, dtype, st)) != CNSF_OK) return s;
        cgls_init_r_kernel<T><<<grid_for(ns), 256, 0, st>>>(w.r64, rT, y, qT, ns);
        if ((s = launch_back(geo, rT, sT, 1, dtype, st)) != CNSF_OK) return s;
        cgls_init_p_kernel<T><<<grid_for(ni), 256, 0, st>>>(w.p64, pT, sT, ni);
        sumsq<T>(sT, ni, w, w.scal + 0, st);
    }
    s = run_iterations(iters, st, [&](cudaStream_t q) -> int {
        int t;
        if ((t = launch_forward(geo, pT, qT, 1, dtype, q)) != CNSF_OK) return t;
        sumsq<T>(qT, ns, w, w.scal + 1, q);
        cgls_xr_kernel<T><<<grid_for(ni + ns), 256, 0, q>>>(w.x64, w.p64, ni, w.r64, rT, qT, ns, w.scal);
        if ((t = launch_back(geo, rT, sT, 1, dtype, q)) != CNSF_OK) return t;
        sumsq<T>(sT, ni, w, w.scal + 2, q);
        cgls_p_kernel<T><<<grid_for(ni), 256, 0, q>>>(w.p64, pT, sT, ni, w.scal);
        cgls_roll_kernel<<<1, 1, 0, q>>>(w.scal);
        return CNSF_OK;
    });
    if (s != CNSF_OK) return s;
    convert_kernel<double, T><<<grid_for(ni), 256, 0, st>>>(x, w.x64, ni);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// ================================================================ batched CGLS
// CGLS on a batch of independent problems with one geometry (the same A): each image keeps
// its own FP64 state and step lengths; the projections run once per iteration over the
// whole batch.  In FP32 they take the symmetric kernels when the geometry has the symmetry
// (each image projected as in a single-image call) and the batched kernels (batch.cu)
// otherwise, whatever the batch size; in both the arithmetic per image does not depend on
// the batch's size or other members, so every iterate is the same whichever requests it is
// batched with.

// workspace: [ scal (B x 8) | part (B x RED_BLOCKS) | x64 | p64 | r64 | pT | sT | qT | rT ], each B x
static size_t cglsb_layout(const cnsf_geometry *geo, int B, int dtype, SolverWs *w, void *base)
{
    const GeomConsts &g = geo->gc;
    size_t el = dtype == CNSF_F64 ? sizeof(double) : sizeof(float);
    size_t ns = (size_t)B * g.nv * g.nd, ni = (size_t)B * g.nx * g.ny;
    size_t off = 0;
    size_t o_scal = off; off += align256((size_t)B * 8 * sizeof(double));
    size_t o_part = off; off += align256((size_t)B * RED_BLOCKS * sizeof(double));
    size_t o_x = off; off += align256(ni * sizeof(double));
    size_t o_p = off; off += align256(ni * sizeof(double));
    size_t o_r = off; off += align256(ns * sizeof(double));
    size_t o_pT = off; off += align256(ni * el);
    size_t o_sT = off; off += align256(ni * el);
    size_t o_qT = off; off += align256(ns * el);
    size_t o_rT = off; off += align256(ns * el);
    if (w && base) {
        char *b = (char *)base;
        w->scal = (double *)(b + o_scal);
        w->part = (double *)(b + o_part);
        w->x64 = (double *)(b + o_x);
        w->p64 = (double *)(b + o_p);
        w->r64 = (double *)(b + o_r);
        w->pT = b + o_pT; w->sT = b + o_sT; w->qT = b + o_qT; w->rT = b + o_rT;
    }
    return off;
}

size_t cgls_batched_workspace_bytes(const cnsf_geometry *geo, int batch, int dtype)
{
    return cglsb_layout(geo, batch, dtype, nullptr, nullptr);
}

// per image b (blockIdx.y): partial sums of squares of its n values
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) sumsq_partial_batched_kernel(const T *__restrict__ a, size_t n,
                                                                            double *__restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    const T *ab = a + blockIdx.y * n;
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < n; i += (size_t)RED_BLOCKS * RED_THREADS) {
        double v = (double)ab[i];
        s = fma(v, v, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.y * RED_BLOCKS + blockIdx.x] = sh[0];
}

// scal[8 b + slot] = sum of image b's partials (one block per image)
__global__ void __launch_bounds__(RED_THREADS) sum_final_batched_kernel(const double *__restrict__ part, double *scal,
                                                                        int slot)
{
    __shared__ double sh[RED_THREADS];
    const double *pb = part + blockIdx.x * RED_BLOCKS;
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) s += pb[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[8 * blockIdx.x + slot] = sh[0];
}

// x_b += alpha_b p_b and r_b -= alpha_b q_b, alpha_b = gamma_b / <q_b, q_b>, for every image
template <typename T>
__global__ void cglsb_xr_kernel(double *x, const double *__restrict__ p, size_t nimg, double *r, T *rT,
                                const T *__restrict__ q, size_t nsino, int B, const double *__restrict__ scal)
{
    const size_t ni = (size_t)B * nimg, n = ni + (size_t)B * nsino;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i < ni ? i / nimg : (i - ni) / nsino;
        const double gam = scal[8 * b], qq = scal[8 * b + 1];
        const double alpha = (gam > 0.0 && qq > 0.0) ? gam / qq : 0.0;
        if (i < ni) {
            x[i] = fma(alpha, p[i], x[i]);
        } else {
            const size_t k = i - ni;
            const double rv = fma(-alpha, (double)q[k], r[k]);
            r[k] = rv;
            rT[k] = (T)rv;
        }
    }
}

// p_b = s_b + beta_b p_b, beta_b = gamma_new_b / gamma_b
template <typename T>
__global__ void cglsb_p_kernel(double *p, T *pT, const T *__restrict__ s, size_t nimg, int B,
                               const double *__restrict__ scal)
{
    const size_t n = (size_t)B * nimg;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / nimg;
        const double gam = scal[8 * b], gnew = scal[8 * b + 2];
        const double beta = gam > 0.0 ? gnew / gam : 0.0;
        const double pv = fma(beta, p[i], (double)s[i]);
        p[i] = pv;
        pT[i] = (T)pv;
    }
}

__global__ void cglsb_roll_kernel(double *scal, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) scal[8 * b] = scal[8 * b + 2];
}

template <typename T>
static void sumsq_batched(const T *a, size_t n, int B, double *part, double *scal, int slot, cudaStream_t st)
{
    sumsq_partial_batched_kernel<T><<<dim3(RED_BLOCKS, B), RED_THREADS, 0, st>>>(a, n, part);
    sum_final_batched_kernel<<<B, RED_THREADS, 0, st>>>(part, scal, slot);
}

template <typename T>
static int proj_fwd_b(const cnsf_geometry *geo, const T *x, T *y, int B, int dtype, cudaStream_t st)
{
    if (dtype == CNSF_F32 && (geo->sym8 || geo->sym)) return launch_forward_sym(geo, (const float *)x, (float *)y, B, st);
    if (dtype == CNSF_F32) return launch_forward_batch(geo, (const float *)x, (float *)y, B, st);
    return launch_forward(geo, x, y, B, dtype, st);
}

template <typename T>
static int proj_back_b(const cnsf_geometry *geo, const T *y, T *x, int B, int dtype, cudaStream_t st)
{
    if (dtype == CNSF_F32 && (geo->sym8 || geo->sym)) return launch_back_sym(geo, (const float *)y, (float *)x, B, st);
    if (dtype == CNSF_F32) return launch_back_batch(geo, (const float *)y, (float *)x, B, st);
    return launch_back(geo, y, x, B, dtype, st);
}

template <typename T>
static int cglsb_impl(const cnsf_geometry *geo, const T *y, T *x, int B, int iters, int resume, int dtype,
                      SolverWs &w, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const size_t ns = (size_t)g.nv * g.nd, ni = (size_t)g.nx * g.ny;
    T *pT = (T *)w.pT, *sT = (T *)w.sT, *qT = (T *)w.qT, *rT = (T *)w.rT;
    int s;
    if (!resume) {
        convert_kernel<T, double><<<grid_for(B * ni), 256, 0, st>>>(w.x64, x, B * ni);
        if ((s = proj_fwd_b<T>(geo, x, qT, B, dtype, st)) != CNSF_OK) return s;
        cgls_init_r_kernel<T><<<grid_for(B * ns), 256, 0, st>>>(w.r64, rT, y, qT, B * ns);
        if ((s = proj_back_b<T>(geo, rT, sT, B, dtype, st)) != CNSF_OK) return s;
        cgls_init_p_kernel<T><<<grid_for(B * ni), 256, 0, st>>>(w.p64, pT, sT, B * ni);
        sumsq_batched<T>(sT, ni, B, w.part, w.scal, 0, st);
    }
    s = run_iterations(iters, st, [&](cudaStream_t q) -> int {
        int t;
        if ((t = proj_fwd_b<T>(geo, pT, qT, B, dtype, q)) != CNSF_OK) return t;
        sumsq_batched<T>(qT, ns, B, w.part, w.scal, 1, q);
        cglsb_xr_kernel<T><<<grid_for(B * (ni + ns)), 256, 0, q>>>(w.x64, w.p64, ni, w.r64, rT, qT, ns, B, w.scal);
        if ((t = proj_back_b<T>(geo, rT, sT, B, dtype, q)) != CNSF_OK) return t;
        sumsq_batched<T>(sT, ni, B, w.part, w.scal, 2, q);
        cglsb_p_kernel<T><<<grid_for(B * ni), 256, 0, q>>>(w.p64, pT, sT, ni, B, w.scal);
        cglsb_roll_kernel<<<(B + 127) / 128, 128, 0, q>>>(w.scal, B);
        return CNSF_OK;
    });
    if (s != CNSF_OK) return s;
    convert_kernel<double, T><<<grid_for(B * ni), 256, 0, st>>>(x, w.x64, B * ni);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int run_cgls_batched(const cnsf_geometry *geo, const void *sino, void *image, int batch, int iters, int resume,
                     int dtype, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < cgls_batched_workspace_bytes(geo, batch, dtype) || ((uintptr_t)ws & 255u) != 0)
        return CNSF_ERR_INVALID;
    if (batch == 0) return CNSF_OK;
    SolverWs w;
    cglsb_layout(geo, batch, dtype, &w, ws);
    return dtype == CNSF_F64
               ? cglsb_impl<double>(geo, (const double *)sino, (double *)image, batch, iters, resume, dtype, w, st)
               : cglsb_impl<float>(geo, (const float *)sino, (float *)image, batch, iters, resume, dtype, w, st);
}

// ================================================================ ASD-POCS
// Adaptive steepest descent POCS (Sidky & Pan 2008), the reconstruction method of Sec. IV-E.
// One outer iteration: a data-consistency sweep over the ordered subsets of views
// (x += beta C_s A_s^T R_s (y_s - A_s x), then x = max(x, 0)), then tv_steps normalised
// steepest-descent steps on the smoothed TV, with the TV step length adapted from the sizes
// of the two moves.  All control scalars (beta, the TV step, the norms) live on the device, so
// the whole loop is launched without a host round trip.

// workspace: [ scal | part | rows | ysub | R | rbuf | C (S images) | gr | xprev | xdata | d ]
struct AsdWs {
    double *scal;   // [0] beta, [1] TV step, [2] dp^2, [3] dd^2, [4] |grad TV|^2, [5] dg^2
    double *part;
    int *rows;
    void *ysub, *R, *rbuf, *C, *gr, *xprev, *xdata, *d;
};

static size_t asd_layout(const cnsf_geometry *const *sub, int nsub, int dtype, AsdWs *w, void *base)
{
    const GeomConsts &g = sub[0]->gc;
    size_t el = dtype == CNSF_F64 ? sizeof(double) : sizeof(float);
    size_t rows = 0;
    for (int k = 0; k < nsub; ++k) rows += (size_t)sub[k]->gc.nv;
    const size_t ns = rows * g.nd, ni = (size_t)g.nx * g.ny;
    size_t off = 0;
    size_t o_scal = off; off += align256(8 * sizeof(double));
    size_t o_part = off; off += align256(RED_BLOCKS * sizeof(double));
    size_t o_rows = off; off += align256(rows * sizeof(int));
    size_t o_y = off; off += align256(ns * el);
    size_t o_R = off; off += align256(ns * el);
    size_t o_rb = off; off += align256(ns * el);
    size_t o_C = off; off += align256((size_t)nsub * ni * el);
    size_t o_gr = off; off += align256(ni * el);
    size_t o_xp = off; off += align256(ni * el);
    size_t o_xd = off; off += align256(ni * el);
    size_t o_d = off; off += align256(ni * el);
    if (w && base) {
        char *b = (char *)base;
        w->scal = (double *)(b + o_scal);
        w->part = (double *)(b + o_part);
        w->rows = (int *)(b + o_rows);
        w->ysub = b + o_y; w->R = b + o_R; w->rbuf = b + o_rb; w->C = b + o_C;
        w->gr = b + o_gr; w->xprev = b + o_xp; w->xdata = b + o_xd; w->d = b + o_d;
    }
    return off;
}

size_t asd_workspace_bytes(const cnsf_geometry *const *sub, int nsub, int dtype)
{
    return asd_layout(sub, nsub, dtype, nullptr, nullptr);
}

// ysub[t][:] = y[rows[t]][:]
template <typename T>
__global__ void gather_rows_kernel(const T *__restrict__ y, const int *__restrict__ rows, T *__restrict__ ysub,
                                   size_t nrows, int nd)
{
    const size_t n = nrows * nd;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t t = i / nd;
        ysub[i] = y[(size_t)rows[t] * nd + (i - t * nd)];
    }
}

// x += beta C g with beta = scal[0]; the last subset of a sweep also clips x to >= 0
template <typename T>
__global__ void asd_update_kernel(T *x, const T *__restrict__ g, const T *__restrict__ C, size_t n,
                                  const double *__restrict__ scal, int clip)
{
    const T beta = (T)scal[0];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const T v = x[i] + beta * C[i] * g[i];
        x[i] = clip ? (v > T(0) ? v : T(0)) : v;
    }
}

// sum of (a - b)^2, deterministic partials as sumsq_partial_kernel
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) diffsq_partial_kernel(const T *__restrict__ a, const T *__restrict__ b,
                                                                     size_t n, double *__restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < n; i += (size_t)RED_BLOCKS * RED_THREADS) {
        const double v = (double)a[i] - (double)b[i];
        s = fma(v, v, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Gradient of TV(x) = sum sqrt(eta^2 + Dx^2 + Dy^2), backward differences that vanish across
// the image border: a pixel enters its own term and, with a minus sign, those of its right
// and lower neighbours.
template <typename T>
__global__ void tv_grad_kernel(const T *__restrict__ x, T *__restrict__ d, int nx, int ny, T eta2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || r >= ny) return;
    const size_t c = (size_t)r * nx + i;
    const T v = x[c];
    const T dx = i > 0 ? v - x[c - 1] : T(0), dy = r > 0 ? v - x[c - nx] : T(0);
    T gsum = (dx + dy) / sqrt(eta2 + dx * dx + dy * dy);
    if (i + 1 < nx) {
        const T vr = x[c + 1];
        const T ex = vr - v, ey = r > 0 ? vr - x[c + 1 - nx] : T(0);
        gsum -= ex / sqrt(eta2 + ex * ex + ey * ey);
    }
    if (r + 1 < ny) {
        const T vd = x[c + nx];
        const T ex = i > 0 ? vd - x[c + nx - 1] : T(0), ey = vd - v;
        gsum -= ey / sqrt(eta2 + ex * ex + ey * ey);
    }
    d[c] = gsum;
}

// x -= step d / |d| (step = scal[1], |d|^2 = scal[4]); nothing when d = 0
template <typename T>
__global__ void tv_step_kernel(T *x, const T *__restrict__ d, size_t n, const double *__restrict__ scal)
{
    const double nd2 = scal[4];
    if (!(nd2 > 0.0)) return;
    const T f = (T)(scal[1] / sqrt(nd2));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] -= f * d[i];
}

// scal[6] counts the iterations done (so that one captured iteration serves them all)
__global__ void asd_start_kernel(double *scal, double relax)
{
    scal[0] = relax;
    scal[1] = 0.0;
    scal[6] = 0.0;
}

// first iteration: TV step = alpha dp
__global__ void asd_first_kernel(double *scal, double alpha)
{
    if (scal[6] == 0.0) scal[1] = alpha * sqrt(scal[2]);
}

// after the TV steps: shrink the TV step when the TV move outgrew the data move (while the
// data residual is above its tolerance), and relax the data step
__global__ void asd_adapt_kernel(double *scal, double r_max, double alpha_red, double data_tol, double relax_red)
{
    const double dp = sqrt(scal[2]), dd = sqrt(scal[3]), dg = sqrt(scal[5]);
    if (dg > r_max * dp && (data_tol <= 0.0 || dd > data_tol)) scal[1] *= alpha_red;
    scal[0] *= relax_red;
    scal[6] += 1.0;
}

template <typename T>
static void diffsq(const T *a, const T *b, size_t n, double *part, double *dst, cudaStream_t st)
{
    diffsq_partial_kernel<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, n, part);
    sum_final_kernel<<<1, RED_THREADS, 0, st>>>(part, dst);
}

typedef int (*ProjFn)(const cnsf_geometry *, const void *, void *, int, int, cudaStream_t);

template <typename T>
static int asd_impl(const cnsf_geometry *const *sub, int nsub, const int *rows_host, const T *y, T *x,
                    const cnsf_asd_pocs_params &P, int dtype, AsdWs &w, cudaStream_t st)
{
    const GeomConsts &g = sub[0]->gc;
    const ProjFn fwd = P.projector == CNSF_PROJECTOR_REF ? launch_forward_ref : launch_forward;
    const ProjFn bwd = P.projector == CNSF_PROJECTOR_REF ? launch_back_ref : launch_back;
    const size_t ni = (size_t)g.nx * g.ny;
    size_t nrows = 0;
    for (int k = 0; k < nsub; ++k) nrows += (size_t)sub[k]->gc.nv;
    const size_t ns = nrows * g.nd;
    T *ysub = (T *)w.ysub, *R = (T *)w.R, *rb = (T *)w.rbuf, *C = (T *)w.C, *gr = (T *)w.gr;
    T *xprev = (T *)w.xprev, *xdata = (T *)w.xdata, *d = (T *)w.d;
    cudaError_t e = cudaMemcpyAsync(w.rows, rows_host, nrows * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return record_cuda_error(e);
    gather_rows_kernel<T><<<grid_for(ns), 256, 0, st>>>(y, w.rows, ysub, nrows, g.nd);
    // per subset: R_s = 1/(A_s 1), C_s = 1/(A_s^T 1)
    int s;
    size_t off = 0;
    for (int k = 0; k < nsub; ++k) {
        const size_t nk = (size_t)sub[k]->gc.nv * g.nd;
        fill_kernel<T><<<grid_for(ni), 256, 0, st>>>(gr, ni, T(1));
        if ((s = fwd(sub[k], gr, R + off, 1, dtype, st)) != CNSF_OK) return s;
        recip_kernel<T><<<grid_for(nk), 256, 0, st>>>(R + off, nk);
        fill_kernel<T><<<grid_for(nk), 256, 0, st>>>(rb + off, nk, T(1));
        if ((s = bwd(sub[k], rb + off, C + k * ni, 1, dtype, st)) != CNSF_OK) return s;
        recip_kernel<T><<<grid_for(ni), 256, 0, st>>>(C + k * ni, ni);
        off += nk;
    }
    asd_start_kernel<<<1, 1, 0, st>>>(w.scal, P.relax);
    const dim3 tvb(16, 16), tvg((g.nx + 15) / 16, (g.ny + 15) / 16);
    const T eta2 = (T)(P.tv_eps * P.tv_eps);
    s = run_iterations(P.iters, st, [&](cudaStream_t q) -> int {
        int t;
        cudaError_t ce;
        if ((ce = cudaMemcpyAsync(xprev, x, ni * sizeof(T), cudaMemcpyDeviceToDevice, q)) != cudaSuccess)
            return record_cuda_error(ce);
        size_t o = 0;
        for (int k = 0; k < nsub; ++k) {   // data-consistency sweep over the ordered subsets
            const size_t nk = (size_t)sub[k]->gc.nv * g.nd;
            if ((t = fwd(sub[k], x, rb + o, 1, dtype, q)) != CNSF_OK) return t;
            sirt_residual_kernel<T><<<grid_for(nk), 256, 0, q>>>(rb + o, ysub + o, R + o, nk);
            if ((t = bwd(sub[k], rb + o, gr, 1, dtype, q)) != CNSF_OK) return t;
            asd_update_kernel<T><<<grid_for(ni), 256, 0, q>>>(x, gr, C + k * ni, ni, w.scal, k == nsub - 1);
            o += nk;
        }
        diffsq<T>(x, xprev, ni, w.part, w.scal + 2, q);
        if (P.data_tol > 0.0) {
            o = 0;
            for (int k = 0; k < nsub; ++k) {
                if ((t = fwd(sub[k], x, rb + o, 1, dtype, q)) != CNSF_OK) return t;
                o += (size_t)sub[k]->gc.nv * g.nd;
            }
            diffsq<T>(rb, ysub, ns, w.part, w.scal + 3, q);
        }
        asd_first_kernel<<<1, 1, 0, q>>>(w.scal, P.alpha);
        if ((ce = cudaMemcpyAsync(xdata, x, ni * sizeof(T), cudaMemcpyDeviceToDevice, q)) != cudaSuccess)
            return record_cuda_error(ce);
        for (int m = 0; m < P.tv_steps; ++m) {
            tv_grad_kernel<T><<<tvg, tvb, 0, q>>>(x, d, g.nx, g.ny, eta2);
            sumsq_partial_kernel<T><<<RED_BLOCKS, RED_THREADS, 0, q>>>(d, ni, w.part);
            sum_final_kernel<<<1, RED_THREADS, 0, q>>>(w.part, w.scal + 4);
            tv_step_kernel<T><<<grid_for(ni), 256, 0, q>>>(x, d, ni, w.scal);
        }
        diffsq<T>(x, xdata, ni, w.part, w.scal + 5, q);
        asd_adapt_kernel<<<1, 1, 0, q>>>(w.scal, P.r_max, P.alpha_red, P.data_tol, P.relax_red);
        return CNSF_OK;
    });
    if (s != CNSF_OK) return s;
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int run_asd_pocs(const cnsf_geometry *const *sub, int nsub, const int *rows, const void *sino, void *image,
                 const cnsf_asd_pocs_params &P, int dtype, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ws || ws_bytes < asd_workspace_bytes(sub, nsub, dtype) || ((uintptr_t)ws & 255u) != 0)
        return CNSF_ERR_INVALID;
    AsdWs w;
    asd_layout(sub, nsub, dtype, &w, ws);
    return dtype == CNSF_F64
               ? asd_impl<double>(sub, nsub, rows, (const double *)sino, (double *)image, P, dtype, w, st)
               : asd_impl<float>(sub, nsub, rows, (const float *)sino, (float *)image, P, dtype, w, st);
}

int run_solver(const cnsf_geometry *geo, int algo, const void *sino, void *image, int iters, double relax,
               int resume, int dtype, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (ws_bytes < solver_workspace_bytes(geo, dtype) || !ws) return CNSF_ERR_INVALID;
    if (((uintptr_t)ws & 255u) != 0) return CNSF_ERR_INVALID;
    SolverWs w;
    ws_layout(geo, dtype, &w, ws);
    if (algo == 0) {
        return dtype == CNSF_F64 ? sirt_impl<double>(geo, (const double *)sino, (double *)image, iters, relax, dtype, w, st)
                                 : sirt_impl<float>(geo, (const float *)sino, (float *)image, iters, relax, dtype, w, st);
    }
    return dtype == CNSF_F64 ? cgls_impl<double>(geo, (const double *)sino, (double *)image, iters, resume, dtype, w, st)
                             : cgls_impl<float>(geo, (const float *)sino, (float *)image, iters, resume, dtype, w, st);
}

}  // namespace cnsf
