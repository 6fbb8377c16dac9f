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
    for (int k = 0; k < iters; ++k) {
        if ((s = launch_forward(geo, x, r, 1, dtype, st)) != CNSF_OK) return s;
        sirt_residual_kernel<T><<<grid_for(ns), 256, 0, st>>>(r, y, R, ns);
        if ((s = launch_back(geo, r, gr, 1, dtype, st)) != CNSF_OK) return s;
        sirt_update_kernel<T><<<grid_for(ni), 256, 0, st>>>(x, gr, C, (T)relax, ni);
    }
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
    for (int k = 0; k < iters; ++k) {
        if ((s = launch_forward(geo, pT, qT, 1, dtype, st)) != CNSF_OK) return s;
        sumsq<T>(qT, ns, w, w.scal + 1, st);
        cgls_xr_kernel<T><<<grid_for(ni + ns), 256, 0, st>>>(w.x64, w.p64, ni, w.r64, rT, qT, ns, w.scal);
        if ((s = launch_back(geo, rT, sT, 1, dtype, st)) != CNSF_OK) return s;
        sumsq<T>(sT, ni, w, w.scal + 2, st);
        cgls_p_kernel<T><<<grid_for(ni), 256, 0, st>>>(w.p64, pT, sT, ni, w.scal);
        cgls_roll_kernel<<<1, 1, 0, st>>>(w.scal);
    }
    convert_kernel<double, T><<<grid_for(ni), 256, 0, st>>>(x, w.x64, ni);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
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
