/*
 * cnsf.h -- C ABI of the GB300 (sm_103a) CNSF fan-beam projector.
 *
 * The library computes the matrix-free forward projection y = A c and its
 * adjoint A^T y of Zhang & Entezari, "A Convolutional Forward and
 * Back-Projection Model for Fan-Beam Geometry" (arXiv 1907.10526).  Each entry
 * of A is the convolutional non-separable footprint of Eq. (18): the pixel
 * basis (first-order box spline, Sec. III.A) projected along the ray through
 * the centre of a detector cell (Eq. 16, Theorem 2) and convolved with the
 * effective detector blur tau' of Eq. (17), evaluated on the fly; no system
 * matrix is stored.
 *
 * Conventions (the paper's Sec. II.A leaves them open):
 *   view k:   theta_k = angles_rad[k] (or 2*pi*k/n_views), u = (cos, sin),
 *             source p = d_po * u, flat detector perpendicular to u at distance
 *             d_ps from the source, detector axis w = (-sin, cos);
 *   cell j:   centre s_j = (j - (n_det-1)/2) * det_spacing + det_offset_mm,
 *             width det_width_mm (tau); a cell value is the mean of the line
 *             integrals over the cell (Eq. 2 with a normalised box blur);
 *   pixel:    pixel (i, r) of an n_x x n_y image of side pixel_mm is centred at
 *             (center_x + (i - (n_x-1)/2) h, center_y + (r - (n_y-1)/2) h).
 *
 * Memory layouts (all buffers contiguous, owned by the caller):
 *   image     [batch][n_y][n_x]      (column index i fastest)
 *   sinogram  [batch][n_views][n_det] (cell index j fastest)
 *   element type float (CNSF_F32) or double (CNSF_F64).
 *
 * Device pointers, unless a function says otherwise, live on the device that
 * was current when the geometry was created; that device must be current
 * when any call is made.  Calls that take a stream are asynchronous on it
 * (a NULL stream is the legacy default stream) and overwrite their outputs.
 * No function throws; each returns a cnsf_status.  One geometry may be used
 * from several host threads and streams at once: it is immutable after
 * creation, and every call keeps its scratch memory private to that call.
 */
#ifndef CNSF_H
#define CNSF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CNSF_API __attribute__((visibility("default")))
#else
#define CNSF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CNSF_OK = 0,
    CNSF_ERR_INVALID = 1,     /* bad argument or geometry, nothing launched          */
    CNSF_ERR_CUDA = 2,        /* a CUDA runtime call failed (see cnsf_last_cuda_error) */
    CNSF_ERR_NOMEM = 3,       /* device or host allocation failed                    */
    CNSF_ERR_UNSUPPORTED = 4, /* valid request the library does not implement        */
    CNSF_ERR_INTERNAL = 5     /* a consistency check of the library failed           */
} cnsf_status;

typedef enum { CNSF_F32 = 0, CNSF_F64 = 1 } cnsf_dtype;

/* Acquisition kind.  FLAT: fan beam from a point source onto a flat detector line (Sec. II.A).
 * ARC: fan beam onto the arc of radius d_ps about the source (the equiangular fan of Sec. I);
 * the cell coordinate s is the arc length from the point p - d_ps u, so cell j's central ray
 * leaves the source at the angle s_j / d_ps from -u; det_spacing and det_width are arc
 * lengths; every cell must lie within 80 degrees of -u.
 * PARALLEL: parallel beam, the limit D_po -> infinity (Sec. III, Theorem 1): every ray of a
 * view runs along -u, the detector line passes through the rotation centre, the detector
 * coordinate of a point x is s = x . w, and the blur is tau at every depth, so the entries of
 * Eq. (18) are the exact bin averages; d_po_mm and d_ps_mm are ignored. */
typedef enum { CNSF_DETECTOR_FLAT = 0, CNSF_DETECTOR_ARC = 1, CNSF_DETECTOR_PARALLEL = 2 } cnsf_detector;

typedef struct cnsf_geometry cnsf_geometry; /* opaque, immutable after creation */

/* Fan-beam acquisition (Sec. II.A, Fig. 1). */
typedef struct {
    int32_t n_x, n_y;          /* image columns and rows (>= 1)                      */
    double pixel_mm;           /* h, side of the square pixel (> 0)                  */
    double center_x_mm;        /* image centre relative to the rotation centre       */
    double center_y_mm;
    int32_t n_views;           /* >= 1                                               */
    const double *angles_rad;  /* host array of n_views angles, copied; NULL selects
                                  theta_k = 2*pi*k/n_views                           */
    int32_t n_det;             /* detector cells (>= 1)                              */
    double det_spacing_mm;     /* Delta_s, pitch of the cell centres (> 0)           */
    double det_width_mm;       /* tau, cell width (> 0)                              */
    double det_offset_mm;      /* shift of the detector centre along w               */
    double d_po_mm;            /* source to rotation centre (D_po); fan beams only    */
    double d_ps_mm;            /* source to detector (D_ps > D_po); fan beams only    */
    int32_t detector;          /* cnsf_detector: FLAT, ARC or PARALLEL               */
    int32_t options;           /* cnsf_option bits (0: the library chooses)          */
} cnsf_geometry_desc;

/* Choices of evaluation that leave the operator unchanged (the paper has no counterpart;
 * they select among implementations of the same entries of Eq. 18).
 *   CNSF_OPT_NO_SYMMETRY: never use the quarter-turn symmetry below.  By default, when the
 *     image is square (n_x = n_y) and centred on the rotation axis (center_x = center_y = 0),
 *     and the views are closed under a quarter turn (n_views divisible by 4 and, for given
 *     angles, angles_rad[k + n_views/4] = angles_rad[k] + pi/2 to 1e-12 rad), the view
 *     v + k n_views/4 sees the image of view v turned by k quarter turns, a quarter turn maps
 *     the pixel lattice onto itself, and so every entry a(v + k n_views/4, j, n) equals
 *     a(v, j, n turned back by k quarter turns).  The FP32 projections then evaluate each
 *     distinct entry once and apply it to the four (view, pixel) pairs it belongs to (a
 *     batch image by image, each with the bits of its single-image call, in launch groups
 *     whose scratch stays within 256 MiB).  When moreover the detector is centred (det_offset = 0) and the views are
 *     closed under reflection (angles_rad[(n_views - k) mod n_views] = -angles_rad[k] to
 *     1e-12 rad, true of the default angles), mirroring the acquisition of view v in the x
 *     axis gives view -v with cell j at n_det - 1 - j and pixel row r at n_y - 1 - r, so each
 *     distinct entry of the views 0 .. n_views/8 serves eight entries of A (four at the two
 *     views that are their own mirror images); CNSF_OPT_NO_REFLECTION keeps to the quarter
 *     turns.  Results agree with the general kernels to FP32 rounding.
 *   CNSF_OPT_EXACT_DIFFERENCES / CNSF_OPT_PLAIN_DIFFERENCES: how the FP32 kernels form the
 *     window difference of Eq. (18), B H(s'+tau'/2) - B H(s'-tau'/2) (H the antiderivative of
 *     the footprint trapezoid).  PLAIN subtracts the two antiderivative values (relative error
 *     ~ 6e-8 B / tau' per entry); EXACT adds the trapezoid's pieces over the window, which
 *     are non-negative, with the cut points taken relative to s' (error ~ 1e-7 whatever
 *     tau'), at about twice the cost.  With neither bit the geometry takes EXACT when the
 *     smallest effective blur tau' of any entry falls below B/32 (PLAIN would lose more than
 *     five bits there) and PLAIN otherwise; cnsf_geometry_paths reports the choice.  FP64
 *     always uses the plain form (its error ~1e-16 B/tau'). */
typedef enum {
    CNSF_OPT_NO_SYMMETRY = 1,
    CNSF_OPT_EXACT_DIFFERENCES = 2,
    CNSF_OPT_PLAIN_DIFFERENCES = 4,
    CNSF_OPT_NO_REFLECTION = 8
} cnsf_option;

/* Build a geometry and its device tables on the current device (Sec. II.A and
 * Eq. 17: per-view rotations, per-cell effective-blur slopes, per-ray walk
 * tables).  Synchronous.  Rejects (CNSF_ERR_INVALID): non-positive sizes,
 * non-positive or non-finite lengths, offsets or view angles and, for the fan beams, d_ps <= d_po and images that reach within two
 * pixels of the source circle (the footprint model needs every pixel in front of the
 * source), and arcs that reach 80 degrees from -u; CNSF_ERR_UNSUPPORTED for an unknown
 * detector kind or n_views * n_det or n_x * n_y of 2^31 or more.
 * On success *out owns device memory until cnsf_geometry_destroy. */
CNSF_API int cnsf_geometry_create(const cnsf_geometry_desc *desc, cnsf_geometry **out);

/* Release a geometry (NULL is allowed).  The caller must first make sure that no
 * work launched with it is still pending. */
CNSF_API void cnsf_geometry_destroy(cnsf_geometry *geom);

/* The evaluation paths a geometry's FP32 projections take (the paper has no
 * counterpart): *symmetric = the number of entries of A each evaluated entry serves -- 1
 * (no symmetry used), 4 (quarter turns) or 8 (quarter turns and reflections);
 * *exact_differences = 1 when the window differences are formed piece by piece (see
 * cnsf_option).  Either pointer may be NULL. */
CNSF_API int cnsf_geometry_paths(const cnsf_geometry *geom, int32_t *symmetric, int32_t *exact_differences);

/* Device bytes the geometry's tables hold from creation to destruction (the paper has no
 * counterpart; for callers that budget device memory, such as a scheduler caching several
 * geometries).  *bytes is a host pointer.  CNSF_ERR_INVALID for a NULL argument. */
CNSF_API int cnsf_geometry_device_bytes(const cnsf_geometry *geom, size_t *bytes);

/* Scratch pool.  Projections called outside stream capture take their stream-ordered
 * scratch (cnsf_projection_scratch_bytes) from a device memory pool of the library's own,
 * one per device, created on first use.  After a synchronisation the pool keeps up to
 * CNSF_SCRATCH_KEEP_BYTES of freed scratch mapped for the next call (CUDA's default pool
 * returns it to the driver, and the next call maps it again); scratch allocated while a
 * stream is captured (plans, solvers) is the graph's own and never comes from the pool.
 * cnsf_scratch_pool_stats: for the current device's pool, *reserved = device bytes it holds
 * now (in use or kept) and *used_high = the most bytes in use at once since its creation or
 * the last reset (host pointers, either may be NULL); reset_high != 0 resets that mark
 * after reading it.  cnsf_scratch_trim: returns the current device's kept scratch to the
 * driver (memory of calls still in flight stays).  Both create the pool if needed;
 * CNSF_ERR_CUDA when a CUDA call fails.  (Not in the paper: device-memory management of
 * this library.) */
#define CNSF_SCRATCH_KEEP_BYTES (512ull << 20)
CNSF_API int cnsf_scratch_pool_stats(size_t *reserved, size_t *used_high, int32_t reset_high);
CNSF_API int cnsf_scratch_trim(void);

/* Sizes of a geometry: any output pointer may be NULL. */
CNSF_API int cnsf_geometry_shape(const cnsf_geometry *geom, int32_t *n_x, int32_t *n_y, int32_t *n_views,
                        int32_t *n_det);

/* Forward projection y = A c (Eq. 6 with the entries of Eq. 18), detector-driven
 * gather without atomics.  image: device [batch][n_y][n_x]; sino: device
 * [batch][n_views][n_det], overwritten.  batch >= 0 (0 launches nothing).
 * Allocates its scratch (zero-padded copies of the image, partial sinograms of line
 * parts) stream-ordered on `stream` and frees it the same way
 * (cnsf_projection_scratch_bytes gives its size).  FP32 batches on a symmetric geometry
 * give every image the bits of its single-image call; other FP32 batches evaluate each
 * entry once for a chunk of up to 16 images (results equal to single-image calls to FP32
 * rounding). */
CNSF_API int cnsf_forward_project(const cnsf_geometry *geom, const void *image, void *sino, int32_t batch,
                         int32_t dtype, void *stream);

/* Back projection c = A^T y, the exact adjoint of cnsf_forward_project (same
 * entries), pixel-driven gather without atomics.  sino: device
 * [batch][n_views][n_det]; image: device [batch][n_y][n_x], overwritten.  FP32
 * allocates scratch stream-ordered on `stream` (the sinogram as weighted cell-pair
 * records — on a symmetric geometry the base views' records with the values of the views
 * that share their entries, even-aligned pairs only on the eight-fold path, both
 * alignments on the quarter-turn path; the general path an odd-aligned copy, and an
 * even-aligned one when n_det is odd or the pointer is not 8-byte aligned; partial images of groups of views, summed in a fixed order;
 * interleaved copies for batch >= 2 off the symmetric path) and frees it the same way.
 * Batches as cnsf_forward_project.  FP64 uses no scratch. */
CNSF_API int cnsf_back_project(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch,
                      int32_t dtype, void *stream);

/* Reference projector (Sec. IV, "Ref"): the same operator shape with the exact entries
 * a_ref = (1/tau) int over the cell of the pixel's exact line integrals (Eq. 1-2),
 * integrated by Gauss-Legendre on the smooth pieces between the detector coordinates
 * of the pixel corners, in FP64 whatever dtype (about 1e-15 relative).  For the
 * parallel kind this equals cnsf_forward_project (Theorem 1); for the fan kinds it is
 * what the CNSF entries approximate.  Ray-driven, no atomics, no scratch; layouts and
 * errors as cnsf_forward_project.  Tens of times slower than the CNSF path: a
 * high-accuracy mode and the yardstick of the approximation error. */
CNSF_API int cnsf_forward_project_ref(const cnsf_geometry *geom, const void *image, void *sino, int32_t batch,
                                      int32_t dtype, void *stream);

/* Adjoint of cnsf_forward_project_ref (same entries, pixel-driven, no atomics, no
 * scratch); layouts and errors as cnsf_back_project. */
CNSF_API int cnsf_back_project_ref(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch,
                                   int32_t dtype, void *stream);

/* Number of non-zero entries of A: pairs (view, cell, pixel) whose pixel centre lies
 * strictly inside the support of the footprint, |s'| < (zeta_1 + zeta_2 + tau')/2
 * (Eq. 18), decided in FP32 along the forward kernel's enumeration.
 * Synchronous; *count is a host pointer. */
CNSF_API int cnsf_count_nonzeros(const cnsf_geometry *geom, uint64_t *count, void *stream);

/* Iterative reconstruction drivers.  Neither is in the paper (its experiments use
 * ASD-POCS); they are the textbook algorithms, built on the projector pair above:
 *   SIRT  x <- x + relax * C A^T (R (y - A x)),  R = 1/(A 1), C = 1/(A^T 1)
 *         (0 where a sum is 0);
 *   CGLS  conjugate gradients on A^T A x = A^T y (Hestenes-Stiefel form).
 * y: device sinogram [n_views][n_det]; x: device image [n_y][n_x], holding x0 on entry
 * and the result on exit (batch 1).  ws: device workspace of at least
 * cnsf_solver_workspace_bytes bytes, 256-byte aligned, owned by the caller and used by
 * one call at a time.  All iterations are launched asynchronously on `stream`; step
 * lengths are computed on the device (FP64 dot products with a fixed reduction order, so
 * results are the same whatever else runs on the GPU).  CGLS with resume != 0 continues
 * from the state a previous call on the same ws, geometry and sinogram left (x must be
 * that call's result); resume = 0 starts from x0. */
CNSF_API size_t cnsf_solver_workspace_bytes(const cnsf_geometry *geom, int32_t dtype);

CNSF_API int cnsf_sirt(const cnsf_geometry *geom, const void *sino, void *image, int32_t iters, double relax,
                       int32_t dtype, void *ws, size_t ws_bytes, void *stream);

CNSF_API int cnsf_cgls(const cnsf_geometry *geom, const void *sino, void *image, int32_t iters, int32_t resume,
                       int32_t dtype, void *ws, size_t ws_bytes, void *stream);

/* CGLS on `batch` independent problems that share the geometry (the same A): sino device
 * [batch][n_views][n_det], image device [batch][n_y][n_x] (x0 in, result out), each image
 * with its own FP64 state and step lengths, the projections run once per iteration over
 * the batch.  In FP32 the projections take the symmetric kernels when the geometry has the
 * symmetry (see cnsf_option) and the batched kernels otherwise, whatever the batch size;
 * in both the arithmetic for one image does not depend on the batch's size or other
 * members: an image's iterates are bitwise the same whichever problems it is batched with
 * (they may differ from cnsf_cgls's at the FP32 rounding level).  Workspace: device, 256-byte aligned, of
 * cnsf_cgls_batched_workspace_bytes; `resume` continues from the state it holds.
 * batch in [0, 65535]. */
CNSF_API size_t cnsf_cgls_batched_workspace_bytes(const cnsf_geometry *geom, int32_t batch, int32_t dtype);
CNSF_API int cnsf_cgls_batched(const cnsf_geometry *geom, const void *sino, void *image, int32_t batch,
                               int32_t iters, int32_t resume, int32_t dtype, void *ws, size_t ws_bytes,
                               void *stream);

/* ASD-POCS (adaptive steepest descent POCS with total variation, Sidky & Pan 2008), the
 * reconstruction method of Sec. IV-E, on the device.  One outer iteration:
 *   1. a data-consistency sweep over the ordered subsets of views, subset by subset
 *      x += beta C_s A_s^T R_s (y_s - A_s x), R_s = 1/(A_s 1), C_s = 1/(A_s^T 1) (0 where
 *      the sum is 0), then x = max(x, 0);
 *   2. dp = |x - x_before_1|; dd = |A x - y| when data_tol > 0;
 *   3. on the first iteration the TV step is alpha * dp;
 *   4. tv_steps steps x -= step * d/|d|, d = grad TV(x) (none when d = 0), with
 *      TV(x) = sum sqrt(tv_eps^2 + Dx^2 + Dy^2) over backward differences that vanish
 *      across the image border;
 *   5. dg = |x - x_after_1|; if dg > r_max dp and (data_tol <= 0 or dd > data_tol) the TV
 *      step is multiplied by alpha_red;
 *   6. beta *= relax_red.
 * Fields left at the values in brackets reproduce Sidky and Pan's choices. */
typedef enum { CNSF_PROJECTOR_CNSF = 0, CNSF_PROJECTOR_REF = 1 } cnsf_projector;

typedef struct {
    int32_t iters;         /* outer iterations (>= 0)                                  */
    int32_t tv_steps;      /* TV steps per iteration (>= 0) [20]                       */
    double relax;          /* beta, initial data-step relaxation, (0, 2) [1]           */
    double relax_red;      /* beta reduction per iteration, (0, 1] [0.995]             */
    double alpha;          /* first TV step relative to the first data move, >= 0 [0.2] */
    double alpha_red;      /* TV step reduction, (0, 1] [0.95]                         */
    double r_max;          /* TV/data move ratio that triggers a reduction, > 0 [0.95] */
    double data_tol;       /* residual tolerance; <= 0: the test is always met [0]     */
    double tv_eps;         /* TV smoothing, >= 0 [1e-4]                                */
    int32_t projector;     /* cnsf_projector: the CNSF entries or the reference ones    */
} cnsf_asd_pocs_params;

/* Device bytes of the workspace of cnsf_asd_pocs for these subsets (0 on bad input). */
CNSF_API size_t cnsf_asd_pocs_workspace_bytes(const cnsf_geometry *const *subsets, int32_t n_subsets,
                                              int32_t dtype);

/* Run ASD-POCS.  subsets: n_subsets geometries (host array of handles) that differ only
 * in their views, swept in this order (one subset: the simultaneous SIRT form of the
 * data step).  rows: host array of the subsets' views in order, the sinogram row of
 * each (a permutation of 0 .. total views - 1).  sino: device [total views][n_det] in
 * the original row order.  image: device [n_y][n_x], x0 in, the result out.  ws: device
 * workspace of cnsf_asd_pocs_workspace_bytes, 256-byte aligned, owned by the caller
 * (not touched by any other call while this one runs).  Asynchronous on `stream`
 * (the rows array is copied before return).  CNSF_ERR_INVALID for inconsistent
 * subsets, a bad permutation, parameters outside their ranges or a short workspace. */
CNSF_API int cnsf_asd_pocs(const cnsf_geometry *const *subsets, int32_t n_subsets, const int32_t *rows,
                           const void *sino, void *image, const cnsf_asd_pocs_params *params, int32_t dtype,
                           void *ws, size_t ws_bytes, void *stream);

/* Size of the static device array used by cnsf_forward_project_noalloc: 16 MiB. */
#define CNSF_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* Forward projection that allocates no memory (the paper has no counterpart: this
 * exists for callers that may not allocate device memory, such as a plugin inside a
 * framework that owns the device-memory budget, or a loop that must not wait on the
 * allocator).  Same arguments, layouts and result as cnsf_forward_project; its scratch
 * (the zero-padded copies of the image) lives in one file-scope device array of
 * CNSF_NOALLOC_SCRATCH_BYTES that every GPU loading the library reserves until the
 * process exits.  The request must fit:
 *     batch * (n_y*(n_x + 2*pad) + n_x*(n_y + 2*pad)) * sizeof(element) <= 16 MiB,
 * pad being the geometry's padding (8 for 1 mm cells and pixels), e.g. batch <= 7 at
 * 512^2 FP32, batch 1 up to ~1400^2 FP32; larger requests return CNSF_ERR_UNSUPPORTED
 * and launch nothing.  Every call looks up the array's device address for the current
 * device (a host-side query; the first one on a device may load the library's device
 * code, so make the first call before any stream capture).  Every call on a device shares
 * the one array: calls whose work overlaps on the GPU (different streams without ordering
 * between them) race and may corrupt each other's results.  The array keeps the last
 * call's contents; nothing in it needs clearing because each call rewrites every element
 * it reads.  Each ray's lines are walked in one part (no partial sinograms to allocate).
 * In FP32 on a geometry with the quarter-turn symmetry (see cnsf_option) whose image copy
 * with its four rotations, 2 * n_x * (n_x + 2*pad) * 16 bytes, fits the array (n_x up to
 * ~700), the images of the batch are projected one after the other by the quarter-turn
 * kernel in that copy, each with the bits of its single-image call; otherwise by the
 * general kernel, several times slower than cnsf_forward_project at large
 * n_views x n_det. */
CNSF_API int cnsf_forward_project_noalloc(const cnsf_geometry *geom, const void *image, void *sino,
                                          int32_t batch, int32_t dtype, void *stream);

/* Projection plans (the paper has no counterpart: a host-side convenience for iterative
 * use).  A plan captures one projection call -- op CNSF_OP_FORWARD, CNSF_OP_BACK,
 * CNSF_OP_FORWARD_REF or CNSF_OP_BACK_REF with the fixed device buffers `in` and `out`,
 * batch and dtype, as for the corresponding cnsf_*_project* call -- into a CUDA graph on
 * the current device; cnsf_plan_launch replays it on `stream` with one graph launch
 * (asynchronous, the same result as the direct call; the buffers' contents are read and
 * written at replay time, their addresses are fixed at creation).  The geometry and the
 * buffers must outlive the plan.  A plan is replayed by one stream at a time (its
 * scratch allocations belong to the graph).  Creation is synchronous with respect to the
 * host and launches nothing; errors as the corresponding call, CNSF_ERR_INVALID for an
 * unknown op or a launch from another device. */
typedef struct cnsf_plan cnsf_plan;
typedef enum { CNSF_OP_FORWARD = 0, CNSF_OP_BACK = 1, CNSF_OP_FORWARD_REF = 2, CNSF_OP_BACK_REF = 3 } cnsf_op;
CNSF_API int cnsf_plan_create(const cnsf_geometry *geom, int32_t op, const void *in, void *out, int32_t batch,
                              int32_t dtype, cnsf_plan **plan);
CNSF_API int cnsf_plan_launch(const cnsf_plan *plan, void *stream);

/* Device bytes that one projection call (op as for cnsf_plan_create) with this batch
 * and dtype allocates stream-ordered, all held at once -- an upper bound that callers
 * budgeting device memory add to their buffers.  Launches nothing, needs no current
 * device.  *bytes is a host pointer.  CNSF_ERR_INVALID for a NULL argument, a negative
 * batch, an unknown op or dtype. */
CNSF_API int cnsf_projection_scratch_bytes(const cnsf_geometry *geom, int32_t op, int32_t batch, int32_t dtype,
                                           size_t *bytes);
CNSF_API void cnsf_plan_destroy(cnsf_plan *plan);   /* NULL is allowed; no replay may be pending */

/* Status code to a static English string. */
CNSF_API const char *cnsf_status_string(int status);

/* Text of the last CUDA error seen by this host thread (static storage). */
CNSF_API const char *cnsf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CNSF_H */
