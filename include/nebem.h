/*
 * nebem.h -- C-ABI of libnebem, a single-GPU (GB300, sm_103a) implementation of the
 * data-parallel hot path of the nearly exact Boundary Element Method (neBEM):
 * closed-form potential and field influence of uniformly charged flat rectangular
 * and triangular elements plus their periodic images, evaluated over large target
 * sets, used to fill the collocation influence matrix, to evaluate potential and
 * field at points, and to add the direct sum over space-charge carriers.
 *
 * Paper references are to "neBEM: A GPU-accelerated Electrostatic Field Solver":
 * Sec. 2 (Eq. 1-5: Poisson equation, point-charge potential, superposition of the
 * potential and of the field), Sec. 2 (Eq. Matrix: K . rho = phi by collocation at
 * element centroids, rho = K^-1 phi), Sec. 2.1 (closed-form potential Phi' and field
 * E' of a uniformly charged rectangle / right triangle; weighting-field reuse of the
 * factors), Sec. 4.1 (LU-based solve, Alg. 1; RHVector with the known-charge term),
 * Sec. 4.2 (space-charge kernel, Alg. 2), Sec. 4.3 (dynamic update, Alg. 4),
 * Sec. 5 Case 2 (periodic "virtual copies" of a THGEM unit cell).
 *
 * Units are SI: metres, volts, C/m^2 for charge densities, C for point charges,
 * V/m for fields.  The Coulomb constant is 1/(4 pi eps0) with
 * eps0 = 8.8541878128e-12 F/m.
 *
 * Conventions common to every call:
 *   - Return value: NEBEM_OK (0) or a negative nebem_status.  A failed call leaves
 *     the context's previous valid state unchanged unless stated otherwise;
 *     nebem_last_error() gives a human-readable message for the calling thread.
 *   - Ownership: caller buffers are never retained.  Host inputs are copied before
 *     the call returns; host outputs are written before it returns.  Device variants
 *     (suffix _device) read and write caller device memory asynchronously on the
 *     given CUDA stream (NULL = the context's own stream); the caller keeps those
 *     buffers alive until the stream reaches the call.
 *   - A context is bound to one CUDA device and is not thread-safe: calls on one
 *     context must be serialised by the caller.  Different contexts are independent.
 *   - Precision argument: NEBEM_FP64 runs every pair through the FP64 closed forms;
 *     NEBEM_MIXED evaluates element-point pairs farther than ratio_near element radii
 *     with FP32 Gauss rules whose order grows as the pair gets closer (target-minus-
 *     source differences formed exactly from two-float coordinates, FP32 arithmetic,
 *     FP64 accumulation), keeps nearer pairs in the FP64 closed forms, factors in FP32
 *     and refines in FP64 against the FP64 matrix.
 */
#ifndef NEBEM_H
#define NEBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nebem_status {
    NEBEM_OK = 0,
    NEBEM_INVALID_ARG = -1,        /* NULL where not allowed, negative size, bad enum */
    NEBEM_BAD_STATE = -2,          /* call out of order (e.g. eval before solve) */
    NEBEM_OUT_OF_MEMORY = -3,      /* device or host allocation failed */
    NEBEM_CUDA = -4,               /* a CUDA runtime call failed */
    NEBEM_SINGULAR = -5,           /* exact zero pivot in the LU factorisation */
    NEBEM_NOT_CONVERGED = -6,      /* iterative refinement hit its iteration limit */
    NEBEM_TIMEOUT = -7,            /* a bounded device-side wait gave up */
    NEBEM_DEGENERATE_ELEMENT = -8, /* zero-area, non-planar, non-convex or non-right-angled element */
    NEBEM_NO_DEVICE = -9,          /* no usable CUDA device */
    NEBEM_TOO_LARGE = -10          /* size beyond a documented limit */
} nebem_status;

/* Every count a call takes (points, carriers, matrix entries, the order of a dense
 * matrix) is at most NEBEM_MAX_COUNT; a larger one returns NEBEM_TOO_LARGE before any
 * buffer is read or any size is computed from it. */
#define NEBEM_MAX_COUNT 2147483647LL

typedef enum nebem_precision { NEBEM_FP64 = 0, NEBEM_MIXED = 1 } nebem_precision;

typedef enum nebem_kind { NEBEM_RECT = 0, NEBEM_TRI = 1, NEBEM_QUAD = 2 } nebem_kind;
typedef enum nebem_bc { NEBEM_CONDUCTOR = 0, NEBEM_DIELECTRIC = 1 } nebem_bc;

/* One flat boundary element (Sec. 2: rectangular and triangular surface elements with
 * uniform charge density; collocation at the centroid).  128 bytes.
 *   kind      NEBEM_RECT: v[0..3] in order around the rectangle, right angles, planar
 *             (v2 = v1 + v3 - v0 within 1e-9 relative).  NEBEM_TRI: v[0..2]; v[3] ignored.
 *             NEBEM_QUAD: v[0..3] in order around a planar convex quadrilateral (v3 within
 *             1e-9 of the size from the plane of v0, v1, v2; every corner convex); its
 *             centroid is the area centroid.  Quadrilaterals are the flat pieces of graded
 *             polar meshes and the primitives of Adaptive Modelling (nebem_set_primitives);
 *             they use the same edge formula as the other kinds.
 *   bc        NEBEM_CONDUCTOR: potential prescribed, V = voltages[conductor].
 *             NEBEM_DIELECTRIC: interface between relative permittivities eps_a on the
 *             -n side and eps_b on the +n side (eps_a != eps_b); conductor ignored.
 *   normal n  right-hand rule on v0, v1, v2, i.e. along (v1 - v0) x (v2 - v0). */
typedef struct nebem_element {
    int32_t kind;
    int32_t bc;
    int32_t conductor;
    int32_t reserved; /* must be 0 */
    double eps_a;
    double eps_b;
    double v[4][3];
} nebem_element;

/* Context options.  Obtain defaults with nebem_default_options(). */
typedef struct nebem_options {
    int32_t device;          /* CUDA device ordinal (default 0) */
    int32_t ir_max_iter;     /* iterative refinement limit in mixed solves (default 30) */
    double ir_tol;           /* stop when ||d sigma||_inf / ||sigma||_inf <= ir_tol (1e-8) */
    double ratio_0;          /* mixed eval: pairs with distance >= ratio_0 element radii use
                                the 4-node FP32 Gauss rule (default 64) */
    double ratio_a;          /* >= ratio_a radii: 6-node triangle / 3x3 rectangle rule
                                (default 24) */
    double ratio_b;          /* >= ratio_b radii: 16-node FP32 rule (default 8) */
    double ratio_near;       /* >= ratio_near radii: 36-node FP32 rule; nearer pairs take
                                the FP64 closed form (default 3) */
    double softening;        /* default Plummer softening of carrier charges, m (1e-6) */
    double sc_near;          /* space charge: pairs closer than this (m) form the FP32
                                difference from exact two-float coordinates (default 1e-4) */
    int32_t lu_block;        /* LU panel width, 32 or 64 (default 64) */
    int32_t wait_polls;      /* poll limit of the software waits on the device (the FP32
                                panel's grid barrier, the triangular sweeps' block flags);
                                0 = 4,194,304 polls (about 0.1-0.3 s).  A wait that runs out
                                gives NEBEM_TIMEOUT (see nebem_solve); default 0 */
    double mixed_point_tol;  /* mixed eval: a point whose estimated error exceeds this fraction
                                of its |phi| or |E| is evaluated again in two-float arithmetic
                                (see nebem_eval_err); 0 keeps the single FP32 pass (default 1e-6) */
    double reserved[3];
} nebem_options;

/* Result report of nebem_solve. */
typedef struct nebem_solve_info {
    int32_t precision;       /* the precision that ran */
    int32_t iterations;      /* refinement iterations (0 for FP64) */
    double correction;       /* last ||d sigma||_inf / ||sigma||_inf (mixed) */
    double residual;         /* ||K sigma - b||_inf / ||sigma||_inf, FP64 (scale of K) */
    double ms_fill;          /* device time of the influence-matrix fill */
    double ms_factor;        /* device time of the LU factorisation */
    double ms_solve;         /* device time of triangular solves and refinement */
    double reserved[4];
} nebem_solve_info;

typedef struct nebem_ctx nebem_ctx;

/* Fill *opt with the defaults listed above (a library utility: no counterpart in the
 * paper).  Errors: NEBEM_INVALID_ARG (opt NULL). */
int nebem_default_options(nebem_options *opt);

/* Create a context on opt->device (opt may be NULL: defaults).  *out receives the
 * context; it owns all device memory it allocates and frees it in nebem_destroy.  The
 * context holds one problem of Sec. 2 (geometry, voltages, charge densities, matrix and
 * factors); it has no counterpart of its own in the paper.  The options are checked on
 * the host before the device is touched.
 * Errors: NEBEM_INVALID_ARG (out NULL or bad option), NEBEM_NO_DEVICE, NEBEM_CUDA. */
int nebem_create(nebem_ctx **out, const nebem_options *opt);

/* Destroy a context and free its device memory (waits for its stream first).  NULL is
 * accepted (no-op).  Always returns NEBEM_OK.  A library utility with no counterpart in
 * the paper. */
int nebem_destroy(nebem_ctx *ctx);

/* Message for the last failed call on this thread (thread-local storage, valid until
 * the thread's next failing call; never NULL, never fails).  A library utility. */
const char *nebem_last_error(void);

/* Name of a status code (static storage; never NULL, never fails; unknown codes get a
 * generic name).  A library utility. */
const char *nebem_status_string(int status);

/* Define the geometry (Sec. 2: discretised boundaries; Sec. 5 Case 2: periodic
 * virtual copies).  el[n] is copied; each element's local frame (origin v0, x along
 * v0->v1, y along the normal), centroid, edge data and far-field Gauss nodes are built
 * in FP64 on the host and uploaded.
 *   lattice  NULL: no images.  Otherwise two primitive translations a1 = lattice[0..2],
 *            a2 = lattice[3..5]; the images are t = k1*a1 + k2*a2 for k1, k2 in
 *            [img_lo, img_hi] (at most 11 per axis), image index
 *            (k1 - img_lo) * m + (k2 - img_lo), m = img_hi - img_lo + 1; every element's
 *            influence is summed over all images (the base cell is the image t = 0,
 *            which must be in range).
 * Invalidates the factors, charge densities and the known-charge set.
 * Errors: NEBEM_INVALID_ARG, NEBEM_DEGENERATE_ELEMENT (index in nebem_last_error),
 * NEBEM_TOO_LARGE (more than 11 images per axis), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_set_geometry(nebem_ctx *ctx, const nebem_element *el, int64_t n, const double *lattice,
                       int32_t img_lo, int32_t img_hi);

/* Conductor potentials (Sec. 2: Dirichlet boundary conditions; Sec. 2.1: K does not
 * depend on them, so the factors are kept).  voltages[n_conductors] is copied.  Every
 * conductor element's index must be < n_conductors.  Invalidates sigma only.
 * Errors: NEBEM_BAD_STATE (no geometry), NEBEM_INVALID_ARG (voltages NULL with
 * n_conductors > 0, n_conductors < 0, a conductor index out of range, a non-finite
 * voltage). */
int nebem_set_bc(nebem_ctx *ctx, const double *voltages, int32_t n_conductors);

/* Solve K sigma = b (Eq. Matrix; Alg. 1 with an LU solve instead of an explicit inverse).
 *   precision  NEBEM_FP64: FP64 fill (closed forms for every pair), FP64 blocked LU with
 *              partial pivoting, FP64 triangular solves.  NEBEM_MIXED: mixed fill (pairs
 *              at >= 6 element radii by Gauss rules in two-float arithmetic, truncation
 *              below ~3e-12 of the pair, nearer pairs by the FP64 closed forms; an FP64
 *              matrix from an earlier FP64 fill is reused instead), FP32 LU with tensor-core
 *              trailing updates, FP64 iterative refinement (residual with that K) until
 *              ir_tol.
 *   Conductor rows: K_ij = ke sum_k Phi'(c_i; j + t_k), b_i = V - phi_sc(c_i).
 *   Interface rows: K_ij = ke sum_k n_i . E'(c_i; j + t_k) (principal value on the own
 *   element) + delta_ij (eps_a + eps_b) / (2 eps0 (eps_b - eps_a)), b_i = -n_i . E_sc(c_i).
 * The matrix and factors are kept on the device and reused by later solves with new
 * voltages or a new known-charge set.  sigma_out[n] (host, may be NULL) receives the
 * charge densities; info (may be NULL) the report.
 * Errors: NEBEM_BAD_STATE (no geometry or no voltages), NEBEM_SINGULAR,
 * NEBEM_NOT_CONVERGED (sigma and info are still written), NEBEM_TIMEOUT (a bounded device
 * wait ran out -- see wait_polls: in the FP32 factorisation, nothing is written; in a
 * triangular sweep, sigma_out is written with NaN in the 64-row blocks whose wait ran out,
 * and the context holds no valid charge densities until the next solve; every kernel has
 * returned, so the context stays usable), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_solve(nebem_ctx *ctx, int32_t precision, double *sigma_out, nebem_solve_info *info);

/* Weighting fields (Sec. 2.1: the influence matrix does not depend on the voltages, so a
 * weighting field is one more solve with the retained factors and a unit-readout
 * right-hand side): for each readout[j] (j < k), the charge densities with unit potential
 * on the elements of conductor readout[j], 0 on every other conductor, 0 on interface rows
 * and no known charges.  The matrix and factors are made on first use as in nebem_solve and
 * kept; all k right-hand sides go through each triangular sweep together (8 per pass, the
 * factors read once per pass), each column with the arithmetic of a single solve, so
 * column j equals nebem_set_bc (unit voltages) + nebem_solve bit for bit when no known
 * charges are set.  NEBEM_MIXED: FP32 solves with FP64 iterative refinement, each column
 * stopping when its own correction meets ir_tol.  The context's charge densities and
 * voltages are not changed.
 *   readout    k conductor indices (host), each the index of at least one conductor
 *              element; repeats allowed.  1 <= k <= 64.
 *   sigma_out  host, n * k doubles, column-major (column j = readout[j]'s densities);
 *              may be NULL.  info (may be NULL): iterations and correction are the largest
 *              over the columns, residual the largest ||K x_j - b_j|| / ||x_j||.
 * Errors: NEBEM_INVALID_ARG (NULL, k, precision, a readout with no element),
 * NEBEM_BAD_STATE (no geometry), NEBEM_SINGULAR, NEBEM_NOT_CONVERGED (some column missed
 * ir_tol; sigma_out is still written), NEBEM_TIMEOUT (a sweep's bounded wait ran out, see
 * wait_polls: sigma_out is written with NaN in the blocks whose wait ran out; the context's
 * own densities are not affected), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_weighting_fields(nebem_ctx *ctx, const int32_t *readout, int32_t k, int32_t precision, double *sigma_out,
                           nebem_solve_info *info);

/* Replace the charge densities (sigma_j of Eq. Potential; n values, host, copied)
 * without solving, e.g. to evaluate a stored solution.  Errors: NEBEM_BAD_STATE (no
 * geometry), NEBEM_INVALID_ARG (NULL, or n not the element count), NEBEM_CUDA. */
int nebem_set_sigma(nebem_ctx *ctx, const double *sigma, int64_t n);

/* Copy the current charge densities (sigma of Eq. Matrix; n values) to host memory.
 * Errors: NEBEM_BAD_STATE (none), NEBEM_INVALID_ARG (NULL, or n not the element count),
 * NEBEM_CUDA. */
int nebem_get_sigma(nebem_ctx *ctx, double *sigma_out, int64_t n);

/* Fill the influence matrix (Eq. Matrix; LHMatrix of Sec. 4.1), as nebem_solve does in
 * this precision, and copy it to host memory in column-major order, K_out[i + j*n] =
 * K_ij.  K_out may be NULL (device copy only).  A current FP64 matrix also answers a
 * NEBEM_MIXED request.  Errors: NEBEM_INVALID_ARG (bad precision), NEBEM_BAD_STATE (no
 * geometry), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_fill(nebem_ctx *ctx, int32_t precision, double *K_out);

/* Gather entries of the current influence matrix (Eq. Matrix; filled on demand as
 * nebem_fill does): out[e] = K[rows[e], cols[e]] for e < count (host arrays; indices
 * 0 <= r, c < n).  For checks of matrices too large to copy whole.  Errors:
 * NEBEM_BAD_STATE (no geometry), NEBEM_INVALID_ARG (NULL or index out of range),
 * NEBEM_TOO_LARGE (count), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_matrix_entries(nebem_ctx *ctx, const int64_t *rows, const int64_t *cols, int64_t count, double *out);

/* Potential and field at points (Eq. Potential and Eq. Field with the element charge
 * densities; Sec. 4.1 PFAtPoint = element part + known-charge part): phi(x) =
 * ke sum_j sigma_j sum_k Phi'(x; j + t_k) [+ ke sum_c q_c / sqrt(r^2 + s^2) when a
 * known-charge set is present], E likewise.  pts[n][3] row-major (host);
 * phi[n] and/or E[n][3] (host) may be NULL.  n = 0 is allowed.  A point with a NaN or
 * infinite coordinate gets NaN phi and E (both precisions; the other points are not
 * affected).  precision NEBEM_FP64: closed forms for every pair.  NEBEM_MIXED: FP32 Gauss
 * rules for far pairs and FP64 closed forms for near ones, then a two-float re-evaluation of
 * every point whose estimated error exceeds mixed_point_tol of its |phi| or |E| (see
 * nebem_eval_err).  Errors: NEBEM_BAD_STATE (no charge densities), NEBEM_INVALID_ARG. */
int nebem_eval(nebem_ctx *ctx, const double *pts, int64_t n, double *phi, double *E, int32_t precision);

/* Device variant of nebem_eval (same equations: Eq. Potential, Eq. Field): d_pts, d_phi, d_E are device pointers
 * (d_phi or d_E may be NULL); runs asynchronously on `stream` (a cudaStream_t, NULL =
 * context stream).  Uses context-owned scratch, so calls on one context must not overlap
 * in time.  Errors: as nebem_eval, plus NEBEM_TOO_LARGE (n), NEBEM_OUT_OF_MEMORY
 * (scratch) and NEBEM_CUDA (a launch failed); faults inside the kernels surface at the
 * caller's next synchronisation. */
int nebem_eval_device(nebem_ctx *ctx, const double *d_pts, int64_t n, double *d_phi, double *d_E,
                      int32_t precision, void *stream);

/* Mixed-precision evaluation (Sec. 2, Eq. Potential / Eq. Field: the same sums as
 * nebem_eval with precision NEBEM_MIXED) with an error estimate for every result.  The FP32
 * pass keeps, per point, the scales of its rounding and truncation errors, from the
 * per-element terms b_j = |sigma_j| |sum_k Phi'_jk| (for E: |sigma_j| |sum_k E'_jk|_1) over
 * its FP32 (element, image) pairs: B = ke sum_j b_j and S = ke sqrt(sum_j b_j^2).  Its
 * estimated absolute error of x = phi (V) and x = |E| (V/m) is
 * 1e-7 |x| + 7e-8 B + 5e-7 S (constants: nebem_set_error_model), which covers every error
 * measured against the FP64 path by 1.7 times or more (a statistical estimate, not a
 * bound).  A point whose estimate exceeds mixed_point_tol times its
 * |phi| or |E| (context option, default 1e-6) is evaluated again in two-float arithmetic
 * (about 44 bits) for the quantity or quantities whose estimate exceeds it (the other keeps
 * its value and estimate): first with the same Gauss rules and FP64 near pairs (estimate
 * 1e-9 B),
 * and where that estimate still exceeds the tolerance, with rules truncated below ~3e-12 of
 * each pair and FP64 closed forms within 6 element radii (estimate 1e-11 B).
 * nebem_eval / nebem_eval_device with NEBEM_MIXED
 * apply the same refinement; these calls also return the estimates.
 *   pts / d_pts  n x 3 points (host memory, copied / device memory).
 *   phi, E       outputs as in nebem_eval (either may be NULL; a NULL output is not used
 *                to decide the refinement).
 *   err / d_err  n x 2 output: estimated absolute error of phi and of |E| per point; may be
 *                NULL (then nothing is written).
 *   n_refined    (host variant, may be NULL) number of points evaluated again (first level).
 *   stream       as in nebem_eval_device (asynchronous, device pointers).
 * Known charges (nebem_space_charge) are added after the refinement, in their own
 * precision; their sum is not part of the estimate.  Not available with Adaptive
 * Modelling (NEBEM_BAD_STATE).  Errors as nebem_eval. */
int nebem_eval_err(nebem_ctx *ctx, const double *pts, int64_t n, double *phi, double *E, double *err,
                   int64_t *n_refined);
int nebem_eval_device_err(nebem_ctx *ctx, const double *d_pts, int64_t n, double *d_phi, double *d_E, double *d_err,
                          void *stream);

/* Constants of the FP32 pass's error estimate (see nebem_eval_err) for the following
 * mixed evaluations of this context: the estimate of each point is
 * gamma_r |x| + gamma_b B + gamma_s S for x = phi and x = |E| alike, with B and S the
 * point's error scales (see nebem_eval_err).  A negative constant restores its default.
 * With (0, 1, 0) or (0, 0, 1) and mixed_point_tol = 0, nebem_eval_err returns the scales
 * B or S themselves.  A library utility with no counterpart in the paper.  Errors:
 * NEBEM_INVALID_ARG (NULL, a non-finite constant). */
int nebem_set_error_model(nebem_ctx *ctx, double gamma_r, double gamma_b, double gamma_s);

/* Set the context's wait_polls option (see nebem_options) for the following calls; 0
 * restores the default.  A library utility with no counterpart in the paper.  Errors:
 * NEBEM_INVALID_ARG (NULL, polls < 0). */
int nebem_set_wait_polls(nebem_ctx *ctx, int32_t polls);

/* Measured throughput of the pipes the evaluation kernels use, on the context's device (a
 * measurement utility with no counterpart in the paper; about 0.1 s): rates[0] scalar FP32
 * FMA, rates[1] packed FP32x2 FMA (each lane counted), rates[2] MUFU reciprocal square
 * root, rates[3] FP64 FMA, in operations per second (an FMA counts as one operation).
 * Best of three timed launches after a warm-up, CUDA events on the context stream.
 * Errors: NEBEM_INVALID_ARG (NULL), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_peak_rates(nebem_ctx *ctx, double *rates);

/* Stage report of the last mixed evaluation of this context that ran without Adaptive
 * Modelling (nebem_eval, nebem_eval_device, nebem_eval_err and friends; a library utility
 * with no counterpart in the paper).  Waits for that evaluation to finish.  Device times
 * (ms, CUDA events on the evaluation's stream) of the FP32 pass (binning, far tiers, FP64
 * near pairs), of the flag step plus the first two-float level, and of the second flag
 * step plus the second level; point counts of the evaluation and of both levels, and of
 * the first level's points that needed only phi or only E re-evaluated.
 * Errors: NEBEM_INVALID_ARG (NULL), NEBEM_BAD_STATE (no such evaluation yet), NEBEM_CUDA. */
typedef struct nebem_eval_stats_t {
    int64_t points;
    int64_t refined_level1;
    int64_t refined_level2;
    double ms_fp32;
    double ms_level1;
    double ms_level2;
    int64_t refined_level1_phi_only; /* of refined_level1: points whose E estimate was within
                                        the tolerance (phi re-evaluated, E kept) */
    int64_t refined_level1_E_only;   /* of refined_level1: E re-evaluated, phi kept */
    double reserved[2];
} nebem_eval_stats_t;
int nebem_eval_stats(nebem_ctx *ctx, nebem_eval_stats_t *out);

/* Set the known-charge set (Sec. 4.2 OptKnCh; Alg. 4 UpdateSpaceCharge): n point
 * carriers at pos[n][3] (m) with charges q[n] (C), Plummer softening `softening` (m,
 * > 0; <= 0 selects the context default).  Copied to the device.  n = 0 clears it.
 * Invalidates sigma (the right-hand side changes), keeps the factors.  Errors:
 * NEBEM_BAD_STATE (no geometry), NEBEM_INVALID_ARG (NULL buffers with n > 0, n < 0, a
 * non-finite position or charge, index in nebem_last_error), NEBEM_TOO_LARGE (n),
 * NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_space_charge(nebem_ctx *ctx, const double *pos, const double *q, int64_t n, double softening);

/* Point -> line charge reduction (Sec. 4.2, Alg. 3) of the current point-charge set, which
 * then stands for the known charges (the LineCh branch of Alg. 4) until the next
 * nebem_space_charge call.
 *   voxel[3]  voxel edges (dx, dy, dz) in m, each > 0.
 * The grid is anchored at the minimum corner (xmin, ymin, zmin) of the cloud: a point
 * falls in voxel (i, j, k) = floor((x - xmin) / dx), ... (IEEE FP64), with flat index
 * (k * ny + j) * nx + i and ny, nx = floor((max - min) / d) + 1.  Every occupied voxel
 * gives one line charge along +z through the voxel centre (xmin + (i + 1/2) dx,
 * ymin + (j + 1/2) dy), from zmin + k dz to zmin + (k + 1) dz, with density
 * lambda = (sum of the voxel's charges, in point order) / dz in C/m.  Lines are listed in
 * increasing voxel index; the reduction is deterministic.  The line charges carry the
 * point charges' softening: phi = ke lambda int dt / sqrt(r(t)^2 + s^2).
 * While lines are in use, the right-hand side, nebem_eval's known-charge part,
 * nebem_space_charge_eval (exclude_self must be 0) and nebem_step use them, and
 * nebem_step repeats the reduction after every move.  The point charges are kept.
 *   n_lines  (may be NULL) receives the number of lines.
 * Invalidates sigma, keeps the factors.
 * Errors: NEBEM_BAD_STATE (no point charges), NEBEM_TOO_LARGE (more than 2^26 points, or
 * voxels * points >= 4e18), NEBEM_INVALID_ARG (an edge <= 0, or dx, dy so small against dz
 * that the near-line search, (3 dz/dx + 3)(3 dz/dy + 3) 5 voxels per target, exceeds 2e5). */
int nebem_space_charge_lines(nebem_ctx *ctx, const double *voxel, int64_t *n_lines);

/* Copy the current line charges (Sec. 4.2, Alg. 3) to the host: start[L][3], stop[L][3] (m), lambda[L] (C/m),
 * each may be NULL.  *n_lines (may be NULL) receives L.  capacity = 0 only queries L;
 * 0 < capacity < L returns NEBEM_TOO_LARGE and writes nothing.
 * Errors: NEBEM_BAD_STATE when the known charges are point charges. */
int nebem_get_lines(nebem_ctx *ctx, double *start, double *stop, double *lambda, int64_t capacity,
                    int64_t *n_lines);

/* Adaptive Modelling (Sec. 3.3; the PrimAfter parameter of the timing table in Sec. 5.3.1):
 * evaluate distant periodic copies with whole primitives carrying the average charge
 * density of their elements instead of the elements themselves.
 *   prims[n_prim]   flat polygons (kind NEBEM_RECT, NEBEM_TRI or NEBEM_QUAD; bc, conductor
 *                   and eps are ignored, reserved must be 0) that the elements tile.
 *   prim_of[n]      primitive of every element of the geometry, or -1 for an element that
 *                   belongs to none (it stands for itself in every copy).  The elements of
 *                   a primitive must lie in its plane (1e-9 of its radius) and their areas
 *                   must add up to its area (1e-9 relative).
 *   prim_after      copy k = (k1, k2) is distant when max(|k1|, |k2|) > prim_after;
 *                   prim_after < 0 switches Adaptive Modelling off.
 * Primitive p carries sigma_p = sum_{j in p} sigma_j A_j / A_p (its total charge over its
 * area), recomputed on the device whenever sigma changes.  Applies to every evaluation at
 * points (nebem_eval, nebem_eval_device, FastVolume nodes, the carriers of nebem_step);
 * not to the matrix fill nor to the server (nebem_server_*), which evaluate all copies
 * element by element.  Copied at the call; set_geometry clears it.
 * Errors: NEBEM_BAD_STATE (no geometry), NEBEM_INVALID_ARG (bad ids, tiling, planes),
 * NEBEM_DEGENERATE_ELEMENT (a degenerate primitive). */
int nebem_set_primitives(nebem_ctx *ctx, const nebem_element *prims, int32_t n_prim, const int32_t *prim_of,
                         int32_t prim_after);

/* Direct space-charge sum at points (Alg. 2, all pairs, softened):
 * phi_t = ke sum_{c != self(t)} q_c / sqrt(r^2 + s^2), E_t = ke sum q_c (x_t - x_c) /
 * (r^2 + s^2)^{3/2}.  exclude_self != 0 means target t is carrier t (n must equal the
 * carrier count) and is excluded.  With line charges in use (nebem_space_charge_lines) the
 * sum runs over the lines instead, exclude_self must be 0, and mixed precision evaluates
 * lines farther than 3 half-lengths with FP32 Gauss-Legendre nodes along the line (2 to
 * 6 by distance), nearer ones in FP64.  Host buffers as in nebem_eval.  Errors:
 * NEBEM_BAD_STATE (no known-charge set), NEBEM_INVALID_ARG (bad precision, NULL points,
 * exclude_self with n != carrier count or with lines), NEBEM_TOO_LARGE (n),
 * NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_space_charge_eval(nebem_ctx *ctx, const double *pts, int64_t n, double *phi, double *E,
                            int32_t precision, int32_t exclude_self);

/* Run `steps` dynamic space-charge updates (Alg. 4 with SpChTh = 0; carriers drift
 * instead of being tracked): per step (1) right-hand side with the known charges at the
 * collocation points, (2) sigma from the retained factors (mixed: FP32 solve + FP64
 * refinement), (3) E at every carrier from all elements (with images) and all other
 * carriers, (4) x_c += sign(q_c) * mu * E_c * dt.  With line charges in use, every step
 * starts with the reduction of Alg. 3 on the current positions, and (1) and (3) sum over
 * the lines (a carrier's own charge is part of its voxel's line).  Requires a solved geometry
 * (factors) and a known-charge set; positions stay on the device between steps.
 * pos_out[n][3] (host, may be NULL) receives the final positions.
 * Errors: NEBEM_BAD_STATE, NEBEM_NOT_CONVERGED, NEBEM_CUDA, NEBEM_TOO_LARGE (a step's voxel
 * grid too large; the positions are still advanced). */
int nebem_step(nebem_ctx *ctx, int32_t steps, double mu, double dt, int32_t precision, double *pos_out);

/* Dense LU factorisation of a caller's matrix on the device (Sec. 4.1, Alg. 1, with the
 * factors kept instead of forming the inverse): right-looking blocked LU with partial
 * pivoting (largest |a|, lowest row index on ties), FP64, in place.
 *   d_A    device, n x n column-major (lda = n); overwritten by L (unit lower, below the
 *          diagonal) and U.
 *   d_piv  device int32[n]; row k was swapped with row d_piv[k] at step k.
 * Runs on `stream` (NULL = the context stream) and synchronises it before returning.
 * Allocates its work buffer (about (lu_block + 1) * n doubles) on the context's device
 * for the duration of the call.  An exact zero pivot (the whole remaining column is zero)
 * does not stop the factorisation: that column is left unscaled, the remaining columns
 * are factored, and the call returns NEBEM_SINGULAR naming the first such column in
 * nebem_last_error.  d_A and d_piv then hold complete factors, P A = L U, with an exact
 * zero on U's diagonal there (which nebem_lu_solve_device cannot use).  Other errors:
 * NEBEM_INVALID_ARG, NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_lu_factor_device(nebem_ctx *ctx, double *d_A, int64_t n, int32_t *d_piv, void *stream);

/* FP32 variant (Sec. 4.1, Alg. 1; the factorisation inside mixed solves): d_A is float, n x n column-major.
 * The rank-64 trailing updates run on the tensor cores (tcgen05, TF32 with a hi/lo split
 * of both operands, FP32 accumulation; with n % 4 == 0 and d_A 16-byte aligned the
 * operands move by bulk copies and the products are added to the matrix by TMA
 * reduce-add).  Each 64-column panel is factored in one cooperative launch (all CTAs
 * resident, one bounded grid barrier per column) when the device supports it; pivots are
 * those of partial pivoting with the lowest row on ties.  Swaps and the unit-lower block
 * inverse run in FP32 on the CUDA cores.  Errors as nebem_lu_factor_device, plus
 * NEBEM_TIMEOUT if a bounded wait (tensor-core update or panel barrier) gave up. */
int nebem_lu_factor_device_f32(nebem_ctx *ctx, float *d_A, int64_t n, int32_t *d_piv, void *stream);

/* Solve A x = b in place with factors from nebem_lu_factor_device (Sec. 4.1, Alg. 1:
 * the solve with retained factors, P then L then U): d_b (device, n) is overwritten by
 * x.  Asynchronous on `stream` (NULL = the context stream); its work space is
 * stream-ordered.  Each triangular sweep is one launch over 64-row blocks that wait
 * (bounded) for the blocks before them; a wait that gives up writes NaN for its block
 * instead of hanging.  Errors: NEBEM_INVALID_ARG (NULL or n <= 0), NEBEM_TOO_LARGE (n),
 * NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_lu_solve_device(nebem_ctx *ctx, const double *d_LU, int64_t n, const int32_t *d_piv, double *d_b,
                          void *stream);

/* The same factorisation as nebem_lu_factor_device for callers that cannot allocate
 * device memory while they run: codes that reserve the device's memory up front for
 * their own pool (where a cudaMalloc would fail or fragment it), or loops that must not
 * allocate after start-up (cudaMalloc / cudaFree can synchronise the device).  There is
 * no counterpart in the paper; this is a property of the library, not of the method.
 *   d_A, d_piv  as in nebem_lu_factor_device (device memory owned by the caller).
 *   n           1 <= n <= 4096; larger n returns NEBEM_TOO_LARGE before any GPU work.
 *   stream      cudaStream_t the work runs on (NULL = the legacy default stream); the
 *               call synchronises it before returning.
 * Needs no context: it runs on the calling thread's current device.  Its work space is a
 * fixed static device array of the library (about 2.1 MB, held on every GPU that loads
 * the library until the process exits); every call looks up that array's device address
 * in the context current on the calling thread (no cached address, so a cudaDeviceReset
 * or a caller-made non-primary context is followed correctly; the first call in a context
 * loads the library's device code there).  All calls on a device share the array, so calls whose
 * GPU work overlaps in time race on it: serialise them.  No memory is allocated by the
 * call (it issues only kernel launches, a memset and one small device-to-host copy).
 * Errors: NEBEM_INVALID_ARG, NEBEM_TOO_LARGE, NEBEM_SINGULAR, NEBEM_CUDA. */
int nebem_lu_factor_device_noalloc(double *d_A, int64_t n, int32_t *d_piv, void *stream);

/* FastVolume map (Sec. 3.3; CreateFastVolPF of Sec. 4.1): evaluate potential and field
 * once at the nodes of a rectilinear grid -- node coordinates per axis, strictly
 * increasing, at least 2 per axis, so nodes can be packed where the field varies fast --
 * with the evaluation kernels of nebem_eval (elements with images, plus known charges),
 * and keep the node values on the device.  One map per context; a new build replaces it.
 * The map belongs to the current charge densities: after any change of them (solve,
 * set_sigma, set_geometry, space_charge, step) lookups fail with NEBEM_BAD_STATE until it
 * is rebuilt.  Axis arrays are host memory, copied.  At most 1e8 nodes.  A node placed
 * exactly on an element's edge or vertex takes the field there, which diverges
 * logarithmically (non-finite values that reach the cells around that node): keep nodes
 * off element boundaries, e.g. by offsetting regular grids by a small fraction.
 * Weighting-field maps, one per readout, come from nebem_weighting_fastvol_build.  Errors: NEBEM_BAD_STATE (no charge densities),
 * NEBEM_INVALID_ARG, NEBEM_TOO_LARGE, NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_fastvol_build(nebem_ctx *ctx, const double *x_nodes, int32_t nx, const double *y_nodes, int32_t ny,
                        const double *z_nodes, int32_t nz, int32_t precision);

/* Trilinear interpolation of the map at points (Sec. 3.3, the FastVolume lookup; host
 * buffers as in nebem_eval): the eight nodes of the cell that holds the point, weights
 * from its fractional position; points outside the grid box take the value at the
 * nearest point of the box; a point with a NaN or infinite coordinate gets NaN.
 * Errors: NEBEM_BAD_STATE (no map, or the charge densities changed since it was built),
 * NEBEM_INVALID_ARG, NEBEM_TOO_LARGE (n), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_fastvol_eval(nebem_ctx *ctx, const double *pts, int64_t n, double *phi, double *E);

/* Device variant of nebem_fastvol_eval (Sec. 3.3; asynchronous on `stream`, NULL = context
 * stream; device pointers, d_phi or d_E may be NULL).  Errors as nebem_fastvol_eval. */
int nebem_fastvol_eval_device(nebem_ctx *ctx, const double *d_pts, int64_t n, double *d_phi, double *d_E,
                              void *stream);

/* Weighting-field FastVolume maps (Sec. 2.1 weighting fields, Sec. 3.3 FastVolume): one
 * map per readout, each a handle of its own (independent of the context and of one
 * another; the context's own map and charge densities are not changed).  The k weighting
 * fields are solved as in nebem_weighting_fields, then the potential and field of each are
 * evaluated at the grid nodes (axes as in nebem_fastvol_build; elements with images only,
 * no known charges) in `precision` (NEBEM_MIXED: the refined mixed evaluation).
 * maps_out[k] receives the handles (each freed with nebem_fvmap_destroy); on an error none
 * is returned.  info (may be NULL) as in nebem_weighting_fields.  Errors: those of
 * nebem_weighting_fields and nebem_fastvol_build, NEBEM_BAD_STATE (Adaptive Modelling on),
 * NEBEM_OUT_OF_MEMORY. */
typedef struct nebem_fvmap nebem_fvmap;
int nebem_weighting_fastvol_build(nebem_ctx *ctx, const int32_t *readout, int32_t k, const double *x_nodes,
                                  int32_t nx, const double *y_nodes, int32_t ny, const double *z_nodes, int32_t nz,
                                  int32_t precision, nebem_fvmap **maps_out, nebem_solve_info *info);

/* Trilinear lookup of one map (as nebem_fastvol_eval; host buffers, phi or E may be NULL;
 * the map's own stream, synchronised before return).  Errors: NEBEM_INVALID_ARG,
 * NEBEM_TOO_LARGE (n), NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_fvmap_eval(nebem_fvmap *map, const double *pts, int64_t n, double *phi, double *E);

/* Device variant (asynchronous on `stream`, NULL = the map's own stream; device pointers,
 * d_phi or d_E may be NULL).  Errors as nebem_fvmap_eval. */
int nebem_fvmap_eval_device(nebem_fvmap *map, const double *d_pts, int64_t n, double *d_phi, double *d_E,
                            void *stream);

/* Free a map (NULL is allowed).  Always NEBEM_OK. */
int nebem_fvmap_destroy(nebem_fvmap *map);

/* Image translations of the current geometry in index order (the virtual copies of
 * Sec. 5 Case 2; count * 3 doubles, host).  *count receives the number of images; t_out
 * may be NULL to query it.  Errors: NEBEM_INVALID_ARG (count NULL), NEBEM_BAD_STATE (no
 * geometry). */
int nebem_image_table(nebem_ctx *ctx, double *t_out, int64_t *count);

/* Distance tier that the mixed evaluation assigns to every (point, element, image) pair,
 * for checks: codes[(p * n_el + j) * n_images + k] = 0 (FP32 4-node rule), 1 (6/9-node),
 * 2 (16-node), 3 (36-node) or 4 (FP64 closed form), decided in FP32 from two-float
 * coordinates against (ratio * element radius)^2 (the options' ratio_0, ratio_a, ratio_b,
 * ratio_near).  pts[n][3] and codes are host arrays; at most 2e8 pairs.  A check of the
 * mixed evaluation with no counterpart in the paper.  Errors: NEBEM_INVALID_ARG,
 * NEBEM_BAD_STATE (no geometry), NEBEM_TOO_LARGE, NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_pair_tiers(nebem_ctx *ctx, const double *pts, int64_t n, uint8_t *codes);

/* Influence of single elements (Sec. 2.1: the closed forms Phi' and E' of a uniformly
 * charged flat element; no charge density, no images) at points, for kernel checks: for
 * element e and point p, phi_out[e*n_pts + p] = Phi'(p) (m) and
 * E_out[(e*n_pts + p)*3 + c] = E'_c(p) (dimensionless), in FP64 closed form.
 * Host buffers; needs no geometry (a context provides the device).  At most 1e8 pairs.
 * Errors: NEBEM_INVALID_ARG (NULL or a size <= 0), NEBEM_DEGENERATE_ELEMENT (index in
 * nebem_last_error), NEBEM_TOO_LARGE, NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_element_influence(nebem_ctx *ctx, const nebem_element *el, int64_t n_el, const double *pts,
                            int64_t n_pts, double *phi_out, double *E_out);

/* ------------------------------------------------------------------ serving
 * Continuous batching over several resident solved contexts (a field-query server).
 * Requests are admitted as device memory frees up, split into point chunks that a
 * persistent batched evaluation kernel pulls from a device work queue; requests that
 * arrive while others run join the running kernel.  Results are bit-identical to
 * the same request evaluated alone.  The serving layer has no counterpart in the paper:
 * each request is the evaluation of Eq. Potential and Eq. Field at its points (the
 * element part of Sec. 4.1 PFAtPoint, with images). */
typedef struct nebem_server nebem_server;

typedef struct nebem_server_options {
    int64_t arena_points;   /* device staging capacity in points (default 4,194,304) */
    int32_t chunk_points;   /* points per work item (128, the only value accepted) */
    int32_t max_requests;   /* in-flight request slots (default 256) */
    int32_t workers;        /* persistent CTAs (0 = 2 per SM) */
    int32_t idle_us;        /* a persistent kernel with no work exits after this (default 2000) */
    double reserved[4];
} nebem_server_options;

/* Fill *opt with the defaults listed above.  Errors: NEBEM_INVALID_ARG (opt NULL). */
int nebem_server_default_options(nebem_server_options *opt);

/* Create a server over n_ctx solved contexts (all on one device; they must stay alive
 * until nebem_server_destroy).  Geometry index g in submit refers to ctxs[g].  The server
 * evaluates the elements' field (with images) from the context's current charge
 * densities; a context with known charges (nebem_space_charge) or with Adaptive
 * Modelling on (nebem_set_primitives) is refused with NEBEM_BAD_STATE, here and at
 * submit, as is a context whose densities have been invalidated.  Errors: NEBEM_INVALID_ARG
 * (NULL or empty context list, bad options, contexts on different devices),
 * NEBEM_BAD_STATE, NEBEM_OUT_OF_MEMORY, NEBEM_CUDA. */
int nebem_server_create(nebem_server **out, nebem_ctx *const *ctxs, int32_t n_ctx,
                        const nebem_server_options *opt);

/* Submit a request: n points pts[n][3] (host) for geometry `geometry`; results go to the
 * caller's host buffers phi[n] / E[n][3] (either may be NULL), which must stay valid
 * until the request completes.  Returns immediately with *req_id.  Admission waits in
 * the server's host queue while the arena is full.
 * Errors: NEBEM_INVALID_ARG, NEBEM_TOO_LARGE (n > arena_points), NEBEM_BAD_STATE. */
int nebem_server_submit(nebem_server *srv, int32_t geometry, const double *pts, int64_t n, double *phi,
                        double *E, int32_t precision, int64_t *req_id);

/* Drive the server (admission, launches, completions) and report whether req_id is
 * done (*done = 1; its outputs are written) or not (*done = 0).  Errors:
 * NEBEM_INVALID_ARG (NULL or unknown req_id), NEBEM_CUDA. */
int nebem_server_poll(nebem_server *srv, int64_t req_id, int32_t *done);

/* Drive the server until req_id completes or timeout_ms passes.  Errors:
 * NEBEM_TIMEOUT (the request keeps running), NEBEM_INVALID_ARG (NULL or unknown req_id),
 * NEBEM_CUDA. */
int nebem_server_wait(nebem_server *srv, int64_t req_id, int64_t timeout_ms);

/* Per-request timing (host clock, seconds since server creation): submit, admission,
 * completion (each output may be NULL).  Errors: NEBEM_BAD_STATE (not complete),
 * NEBEM_INVALID_ARG (NULL server or unknown req_id). */
int nebem_server_request_times(nebem_server *srv, int64_t req_id, double *t_submit, double *t_admit,
                               double *t_done);

/* Finish the admitted work and free the server (contexts are not destroyed); requests
 * still waiting for admission are dropped, their outputs left unwritten.  NULL is
 * accepted.  Always returns NEBEM_OK. */
int nebem_server_destroy(nebem_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* NEBEM_H */
