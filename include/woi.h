/*
 * woi.h -- C ABI of libwoi, a GB300 (sm_103a) implementation of the
 * Walk-on-Interfaces (WoI) Monte Carlo estimator of
 *
 *     Ding & Stinchcombe, "Walk-on-Interfaces: A Monte Carlo Estimator for an
 *     Elliptic Interface Problem with Nonhomogeneous Flux Jump Conditions and
 *     a Neumann Boundary Condition", arXiv 2508.16767.
 *
 * Problem (Sec. 1, Eq. interface_problem): div(sigma grad u) = 0 with sigma
 * piecewise constant on a tree of regions Omega_1 ⊃ Omega_i; sigma_1 d_n u = b_1
 * on the outer boundary dOmega_1; [u] = 0 and [sigma d_n u] = b_i across each
 * interface dOmega_i (jump = exterior minus interior).  The estimator returns
 * u(x) and grad u(x) (Sec. 4.3 Eq. woi_estimator and Sec. 4.5 Eq.
 * naive_woi_grad_estimator; Algorithm 3 / Eq. variance_reduced_woi_estimator
 * for the variance-reduced variant) with their Monte Carlo standard errors.
 * u is defined up to an additive constant (Sec. 1); the estimator returns the
 * single-layer representation of Sec. 3 without any shift.
 *
 * Conventions shared by every entry point:
 *   - Surfaces are numbered 0..n_surf-1; surface 0 is the outer boundary
 *     (the paper's dOmega_1).  parent[0] = -1, parent[i] = index of the
 *     region that directly contains region i.
 *   - Arrays are row-major, FP64 unless stated.  Pointers passed to an
 *     estimate call may be host or device memory (detected per pointer with
 *     cudaPointerGetAttributes); every other pointer is host memory.
 *   - The caller owns every array it passes.  The library deep-copies
 *     geometry and data at create/set time; nothing passed in is retained.
 *   - Every call returns a woi_status.  On any error the outputs are left
 *     untouched and woi_last_error() returns a message for the calling thread.
 *   - A geometry handle may be used by one host thread / one stream at a time.
 *   - With device output pointers an estimate call is asynchronous on the
 *     given stream; with host output pointers it returns after the results are
 *     copied back.
 */
#ifndef WOI_H
#define WOI_H

#include <stdint.h>

#if defined(__GNUC__)
#define WOI_API __attribute__((visibility("default")))
#else
#define WOI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define WOI_MAX_DIM 6
#define WOI_MAX_SURF 128
#define WOI_MAX_STAR_DEGREE 16
#define WOI_MAX_M 32

/* opaque geometry handle (geometry, conductivities, flux data, device copies) */
typedef struct woi_geometry woi_geometry;

typedef enum {
    WOI_OK = 0,
    WOI_E_INVALID_ARG = 1,   /* bad pointer, size, option or range */
    WOI_E_GEOMETRY = 2,      /* surfaces overlap, are not nested as `parent` says, or a point lies outside */
    WOI_E_COMPAT = 3,        /* flux data violate the zero-mean compatibility condition of Sec. 1 */
    WOI_E_UNSUPPORTED = 4,   /* a combination the library does not implement */
    WOI_E_NO_DEVICE = 5,     /* no usable CUDA device */
    WOI_E_CUDA = 6,          /* a CUDA runtime call failed (message has the CUDA error string) */
    WOI_E_OOM = 7,           /* device or host allocation failed */
    WOI_E_TIMEOUT = 8,       /* a bounded device wait gave up */
    WOI_E_STATE = 9          /* call order violated (e.g. estimate before set_sigma_and_data) */
} woi_status;

#define WOI_MAX_ELLIPSOIDS 8
#define WOI_MAX_MESHES 16
#define WOI_MAX_MESH_TRIANGLES (1 << 22)   /* per geometry, all meshes together */

/* surface kinds */
enum { WOI_SPHERE = 0,     /* circle (2D) or (d-1)-sphere: centre, radius */
       WOI_STAR = 1,       /* 2D star-shaped curve about `center`:
                              r(t) = radius (1 + sum_{k=1..K} a_k cos kt + b_k sin kt) */
       WOI_ELLIPSOID = 2,  /* d >= 3: (y - center)^T A (y - center) = 1, A = matrix symmetric
                              positive definite (Sec. 5, Example 2); at most WOI_MAX_ELLIPSOIDS
                              per geometry */
       WOI_MESH = 3 };     /* d = 3: closed triangle mesh (Sec. 5), every edge shared by exactly two
                              triangles with opposite orientations, triangles counter-clockwise
                              seen from outside (positive enclosed volume); `center` is the
                              reference point of the surface's local coordinates (any point near
                              it).  A line crossing one mesh more than 32 times is not supported:
                              the call reports WOI_E_GEOMETRY (asynchronous calls through
                              woi_check_status).
                              At most WOI_MAX_MESHES per geometry */

typedef struct {
    int type;                         /* WOI_SPHERE, WOI_STAR or WOI_ELLIPSOID */
    double center[WOI_MAX_DIM];       /* first `dim` entries used */
    double radius;                    /* sphere radius, or the star's base radius (unused for ellipsoids) */
    int star_degree;                  /* K (star only), 0..WOI_MAX_STAR_DEGREE */
    const double *star_a;             /* [K+1], index 0 ignored (star only) */
    const double *star_b;             /* [K+1], index 0 ignored (star only) */
    const double *matrix;             /* [dim][dim] row-major A (ellipsoid only) */
    int n_vertices;                   /* mesh only */
    const double *vertices;           /* [n_vertices][3] (mesh only) */
    int n_triangles;                  /* mesh only */
    const int *triangles;             /* [n_triangles][3] vertex indices (mesh only) */
} woi_surface_desc;

/* flux bases (the data b_i of Sec. 1 on each surface) */
enum {
    WOI_FLUX_ZERO = 0,          /* b = 0                                                      */
    WOI_FLUX_FOURIER = 1,       /* 2D: coef = [a0, a1, b1, ..., aK, bK] in the surface's local
                                   angle t (atan2 about its centre / the star parameter)      */
    WOI_FLUX_REAL_SH = 2,       /* 3D spheres: coef[l*l + l + m], l <= 4, orthonormal real
                                   spherical harmonics of the unit vector from the centre, no
                                   Condon-Shortley phase: sin(phi) cos(theta) = sqrt(4pi/3) Y_1^1 */
    WOI_FLUX_HARMONIC_POLY = 3, /* any d: coef = [s, T, (c, e_1..e_d) x T];
                                   b(y) = s n(y) . grad P(y), P = sum c prod y_k^{e_k} harmonic */
    WOI_FLUX_POINT_CHARGE = 4   /* d >= 3: coef = [s, x0_1..x0_d]; b(y) = s n(y) . grad |y - x0|^{2-d}
                                   (the point-charge potential of Sec. 5, Example 2); x0 must lie
                                   outside the region the surface bounds (compatibility) */
};

typedef struct {
    int basis;                        /* WOI_FLUX_* */
    int n_coef;                       /* number of doubles in coef */
    const double *coef;
} woi_flux_desc;

enum { WOI_PLAIN = 0,                 /* Algorithm 2 */
       WOI_VR = 1 };                  /* Algorithm 3: two chains from dOmega^+ / dOmega^-.  2D Fourier
                                         data: parts cut at the roots of beta; d >= 3 data linear in the
                                         unit vector on a sphere: hemispheres; any other data and
                                         surface: the start is drawn from 16 uniform trials on the
                                         surface, weighted by the fraction of trials of each sign (same
                                         mean, no areas needed) */
enum { WOI_MIXED = 0,                 /* FP32 walks, compensated FP32 per-lane sums, FP64 reductions */
       WOI_FP64_PLAIN = 1 };          /* FP64 everywhere, one kernel launch per evaluation point */

typedef struct {
    int M;                            /* truncation: steps i = 0..M (Sec. 3, w_i = 1 - delta_iM / 2) */
    int variant;                      /* WOI_PLAIN or WOI_VR */
    int precision;                    /* WOI_MIXED or WOI_FP64_PLAIN */
    int sched_group;                  /* walkers per interface schedule (Algorithm 1): 1 or 32 */
    void *cuda_stream;                /* cudaStream_t to launch on; NULL = the legacy default stream */
    int block_size;                   /* 0 = autotuned / default */
    int walks_per_lane;               /* walks each lane runs per work unit (a unit is one warp's, or for a
                                         batch one block's, share of a point's walks); 0 = default */
    int timing;                       /* 1: record CUDA events around the walk kernel(s) on the launch
                                         stream (read back with woi_last_kernel_ms) */
    int tile_points;                  /* 0: every point has its own walks (streams keyed by point).
                                         32: shared trajectories (Sec. 4.6): the points
                                         [32 t, 32 t + 32) of the call all use the walks of stream id t,
                                         each tallied against all 32 points; errors of points in a tile
                                         are correlated.  Mixed precision, woi_estimate / _range only. */
} woi_opts;

/* Fills `o` with the defaults: M = 4, WOI_PLAIN, WOI_MIXED, sched_group 1, NULL stream. */
WOI_API void woi_default_opts(woi_opts *o);

/*
 * Create a geometry (Sec. 1: tree-structured domain; Sec. 4.6: analytic
 * surfaces with closed-form sampling and intersection).  Validates: 2 <= dim
 * <= 6; 1 <= n_surf <= WOI_MAX_SURF; parent forms a tree rooted at surface 0;
 * stars only in 2D with r(t) > 0; every surface strictly inside its parent and
 * disjoint from its siblings (circles/spheres analytically, stars on a dense
 * sample).  Returns WOI_E_INVALID_ARG / WOI_E_GEOMETRY on failure.  *out is
 * owned by the caller and released with woi_destroy_geometry.
 */
WOI_API woi_status woi_create_geometry(int dim, int n_surf, const woi_surface_desc *surfaces, const int *parent,
                               woi_geometry **out);

/*
 * |dOmega_i| of surface i as the estimator uses it (Eq. naive_woi_p0): closed
 * form for circles / d-spheres, Gauss-Legendre arc length for the star, and for
 * an ellipsoid |S^{d-1}| prod(a_k) E_u |diag(1/a) u| (u uniform on the unit
 * sphere, a_k the semi-axes) by a one-dimensional quadrature.  Host only.
 */
WOI_API woi_status woi_surface_area(const woi_geometry *geometry, int i, double *area);

/*
 * Set conductivities and flux data.  sigma[n_surf] (sigma_i >= 0, sigma_0 > 0,
 * sigma_i + sigma_parent > 0); flux[n_surf] with flux[0] the Neumann datum
 * sigma_1 d_n u = b_1 and flux[i] the jump [sigma d_n u] = b_i.  Computes the
 * unit-coefficient system of Sec. 3 (alpha_1 = 2, alpha_i =
 * 2 (sigma_i - sigma_p) / (sigma_p + sigma_i), beta_1 = 2 b_1 / sigma_1,
 * beta_i = -2 b_i / (sigma_p + sigma_i)) and the schedule of Thm 4.2.
 * WOI_E_COMPAT if some surface has |int b_i dA| > 1e-10 ||b_i||_1 (the
 * compatibility condition of Sec. 1), WOI_E_UNSUPPORTED for a basis that does
 * not fit the surface (e.g. REAL_SH outside 3D spheres).
 */
WOI_API woi_status woi_set_sigma_and_data(woi_geometry *geometry, const double *sigma, const woi_flux_desc *flux);

/*
 * Estimate u and grad u at n_pts points (points [n_pts][dim], host or
 * device) with n_walks walks per point (a multiple of sched_group) and the
 * counter-based stream `seed`.  Outputs (host or device, each may be NULL):
 * u[n_pts], grad[n_pts][dim], se_u[n_pts], se_grad[n_pts][dim]: the sample
 * mean of N * (walk tally) (Algorithm 1) and its standard error computed from
 * the schedule-group means.  Points must lie inside the outer surface
 * (WOI_E_GEOMETRY otherwise).
 */
WOI_API woi_status woi_estimate(woi_geometry *geometry, const woi_opts *opts, const double *points, int64_t n_pts,
                        int64_t n_walks, uint64_t seed, double *u, double *grad, double *se_u, double *se_grad);

/*
 * The walks [walk_begin, walk_begin + n_walks) of every point (both multiples
 * of sched_group), returned as raw moments for resumption and sharding:
 * moments[n_pts][2][dim+1] = (sum over walks of f, sum over schedule groups of
 * (group mean of f)^2) for f = (u tally, grad tally).  Ranges that tile
 * [0, W) add up to the moments of one call over [0, W).
 */
WOI_API woi_status woi_estimate_range(woi_geometry *geometry, const woi_opts *opts, const double *points, int64_t n_pts,
                              int64_t walk_begin, int64_t n_walks, uint64_t seed, double *moments);

/*
 * Mean and standard error from raw moments (Algorithm 1: the estimate is the mean
 * of the walk tallies, its standard error the one of the schedule-group means).
 * moments[n_pts][2][dim+1] as woi_estimate_range returns them -- for f = (u tally,
 * grad tally), the sum of f over n_walks walks and the sum over the
 * G = n_walks / sched_group schedule groups of (group mean of f)^2 -- typically the
 * element-wise sum of the moments of disjoint walk ranges (shards, resumed runs)
 * that together cover n_walks walks of every point.  Writes u[n_pts] = sum / n_walks,
 * grad[n_pts][dim] likewise, and se_u[n_pts], se_grad[n_pts][dim] = sqrt(s^2 / G)
 * with s^2 the sample variance of the G group means (0 when G = 1); each output
 * may be NULL.  moments and outputs may be host or device memory (detected per
 * pointer); with only device pointers the call is asynchronous on cuda_stream (a
 * cudaStream_t, NULL = the legacy default stream) and allocates nothing, otherwise
 * it stages through temporary device memory and returns after the results are
 * copied back.  Errors: WOI_E_INVALID_ARG for dim outside [2, 6], n_pts < 0,
 * n_walks < 1, sched_group not 1 or 32, n_walks not a multiple of sched_group, or a
 * null moments array with n_pts > 0; WOI_E_NO_DEVICE without a CUDA device.
 */
WOI_API woi_status woi_finalize_moments(int dim, int64_t n_pts, int64_t n_walks, int sched_group,
                                        const double *moments, void *cuda_stream, double *u, double *grad,
                                        double *se_u, double *se_grad);

/*
 * Per-walk values for pathwise replay: for one point x[dim] (host) with
 * stream ids point_id and instance_id (the instance index of a batch, 0 otherwise), the walks walk_ids[n] (host) give f_u[n] and
 * f_grad[n][dim] (host), each the full walk tally N sum_i c_i Phi(x, y_i)
 * (resp. grad_x Phi), in the precision opts->precision selects.
 */
WOI_API woi_status woi_walk_values(woi_geometry *geometry, const woi_opts *opts, const double *x, uint32_t point_id,
                                   uint32_t instance_id, const uint64_t *walk_ids, int64_t n, uint64_t seed,
                                   double *f_u, double *f_grad);

/*
 * woi_walk_values plus the states of each walk: trace[n][chains][M+1][dim+2]
 * (host) holds, per step i, the point y_i (dim values), Q_i and T_i (Eqs.
 * naive_woi_Q / naive_woi_T); chains = 2 for the variance-reduced variant,
 * else 1.  A chain that ended keeps its last state.
 */
WOI_API woi_status woi_walk_trace(woi_geometry *geometry, const woi_opts *opts, const double *x, uint32_t point_id,
                                  uint32_t instance_id, const uint64_t *walk_ids, int64_t n, uint64_t seed,
                                  double *f_u, double *f_grad, double *trace);

/*
 * Batched heterogeneous estimate: n_inst geometries (each with data set),
 * instance k with n_pts[k] points at points[k] (host or device) and n_walks[k]
 * walks per point.  All instances of one group run in one persistent kernel:
 * a block serves one instance at a time and its warps take (point, walk-chunk)
 * units from that instance's device work-queue head; outputs per
 * instance as for woi_estimate (u[k], grad[k], se_u[k], se_grad[k], each may
 * be NULL).  Random streams use instance id k.  opts applies to all instances
 * except M, which comes from m_per_inst[k] when m_per_inst is not NULL.
 * Instances are grouped by (dimension, non-sphere surfaces): one persistent launch per
 * group, then one finalize; the sequence is captured as a CUDA graph and
 * replayed while the same batch (handles, sizes, pointers, seed, options) is
 * run again.  With WOI_FP64_PLAIN the instances run one after another, one
 * launch per point (the FP64 baseline).  The call returns when the results are
 * written; batch calls share one library scratch area and must not overlap.
 */
WOI_API woi_status woi_estimate_batch(int n_inst, woi_geometry *const *geometries, const woi_opts *opts, const int *m_per_inst,
                              const double *const *points, const int64_t *n_pts, const int64_t *n_walks,
                              uint64_t seed, double *const *u, double *const *grad, double *const *se_u,
                              double *const *se_grad);

/*
 * Outcome of the last asynchronous estimate on this geometry (an estimate or
 * range call with device points and device outputs, which returns before its
 * kernels finish).  Waits for that call's work on its stream and returns
 * WOI_E_GEOMETRY if a line or ray of one of its walks crossed a mesh surface
 * more than 32 times (the crossing lists are bounded: the extra crossings were
 * dropped and that call's estimates are invalid), WOI_OK otherwise or if there
 * is nothing to check.  The counter is reset by every call and read once.
 * Synchronous calls (host points or outputs), woi_walk_values / woi_walk_trace
 * and woi_estimate_batch report the same condition in their own status.
 */
WOI_API woi_status woi_check_status(woi_geometry *geometry);

/*
 * Duration in milliseconds of the walk kernel(s) of the last estimate on this
 * handle that ran with opts->timing = 1 (CUDA events on its launch stream;
 * waits for the stop event).  WOI_E_STATE if no timed estimate ran.
 */
WOI_API woi_status woi_last_kernel_ms(woi_geometry *geometry, float *ms);

/*
 * Allocation-free variant of woi_estimate (mixed precision only).  The paper
 * has no counterpart: this entry point exists for callers that must not
 * allocate device memory while they run -- e.g. code inside a region where a
 * host framework owns the whole device heap through its own pool, real-time or
 * embedded hosts that fix their memory budget at start-up, or plug-ins that
 * are only allowed to launch work on memory handed to them.
 *
 * Every byte of scratch it needs (the instance's geometry tables, the work
 * queue head and the per-work-unit partial sums) lives in one fixed array of
 * WOI_NOALLOC_SCRATCH_BYTES (16 MiB) compiled into the library; each GPU that
 * loads the library holds that array until the process exits.  The call makes
 * no cudaMalloc / cudaFree and uses no allocating library routine.
 *
 * points [n_pts][dim] and the outputs u[n_pts], grad[n_pts][dim], se_u[n_pts],
 * se_grad[n_pts][dim] must be device pointers (outputs may be NULL).  The
 * call is asynchronous on opts->cuda_stream.  Sizes whose scratch would exceed
 * the array are rejected with WOI_E_INVALID_ARG (about 16 MiB / (16 (dim+1))
 * work units of 32 x walks_per_lane walks each -- e.g. 4096 points x 1e5 walks
 * in 3D fits with 64 walks per lane).  The launch shape is chosen as for
 * woi_estimate (explicit options, else the woi_autotune table), except that the
 * default is 64 walks per lane (fewer, larger work units).
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  All calls share the one array and it
 * keeps the contents of the last call, so calls that may overlap on the GPU
 * (different streams, or different host threads) race with each other and
 * must be serialised by the caller.
 */
#define WOI_NOALLOC_SCRATCH_BYTES (16u << 20)
WOI_API woi_status woi_estimate_noalloc(woi_geometry *geometry, const woi_opts *opts, const double *points,
                                        int64_t n_pts, int64_t n_walks, uint64_t seed, double *u, double *grad,
                                        double *se_u, double *se_grad);

/*
 * Autotuner of the FP32 walk kernel's launch shape.  Times the persistent
 * kernel on a probe of the given workload (the first few waves of work units)
 * for block sizes {128, 256} x walks per lane {8, 16, 32, 64}, and keeps the
 * fastest pair for this (dimension, star surface, variant, schedule group, M)
 * in a process-wide table that later calls with block_size = walks_per_lane = 0
 * use.  If the environment variable WOI_TUNE_CACHE names a file, the table is
 * read from it at the first call and written back after each tuning.  points
 * as for woi_estimate; *block_size / *walks_per_lane receive the choice (may be
 * NULL).  Synchronous.
 */
WOI_API woi_status woi_autotune(woi_geometry *geometry, const woi_opts *opts, const double *points, int64_t n_pts,
                                int64_t n_walks, uint64_t seed, int *block_size, int *walks_per_lane);

/* Release a geometry and its device buffers. NULL is accepted. */
WOI_API void woi_destroy_geometry(woi_geometry *geometry);

/* Message of the last failed call on this host thread ("" if none). */
WOI_API const char *woi_last_error(void);

/* Library version string. */
WOI_API const char *woi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WOI_H */
