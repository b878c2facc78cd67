/*
 * bem.h -- C ABI of the GB300 (sm_103a) library for the electric potential
 * phi and field E of charged constant-density BEM triangles and rectangles
 * by Gaussian cubature (Glueck & Hilk, arXiv:1606.03743).
 *
 * The method (Sec. 4, Eq. 4.1): every element is replaced by the point
 * charges q_i = w_i sigma A of one of the paper's cubature rules (App. A for
 * triangles, App. B for rectangles), chosen by the distance ratio
 * DR = |P - Q_cen| / L (Sec. 2); below the near-field limit (DR < 4.5 for
 * triangles, 6 for rectangles by default, Sec. 4; see bem_default_limits)
 * the element is integrated analytically.  phi and E at a
 * field point are the sums over all elements (Sec. 5), times 1/(4 pi eps0).
 *
 * Conventions for every entry point:
 *  - Return value: BEM_OK (0) or a negative BEM_ERR_* code; the message of
 *    the last failure on the calling thread is bem_last_error().  No C++
 *    exception crosses this boundary.  On failure the outputs are not
 *    written (except where a call says otherwise).
 *  - Pointers: arrays may live in host memory or in device memory of the
 *    current CUDA device; the library tells them apart with
 *    cudaPointerGetAttributes and stages host arrays through its own device
 *    buffers.  The caller owns every array it passes; the mesh owns all
 *    device memory it allocates.
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default
 *    stream).  Device work is issued on that stream; a call returns after
 *    its results are complete (it synchronises the stream), because the
 *    status it returns depends on device-side checks.
 *  - Threads: one mesh must not be used from two threads at once.
 *  - Layouts are row-major, double precision, C order.
 */
#ifndef BEM_H
#define BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BEM_OK 0
#define BEM_ERR_INVALID -1  /* bad argument, NaN, degenerate or non-rectangular element */
#define BEM_ERR_OOM -2      /* device allocation failed or the memory budget is exceeded */
#define BEM_ERR_CAPACITY -3 /* a work list outgrew its fixed capacity (no-growth calls) */
#define BEM_ERR_CUDA -4     /* a CUDA runtime call or kernel launch failed */
#define BEM_ERR_TIMEOUT -5  /* a bounded wait ran out (serving loop) */
#define BEM_ERR_NOT_FOUND -6 /* unknown serving ticket */
#define BEM_ERR_NOT_CONVERGED -7 /* bem_solve stopped at its iteration limit above the tolerance */

/* element types */
#define BEM_TRIANGLE 0
#define BEM_RECTANGLE 1

/* arithmetic of the far-field cubature */
#define BEM_FP64 0  /* double precision throughout (the paper's arithmetic, Sec. 6) */
#define BEM_MIXED 1 /* FP32 point-charge sums with split-float (hi/lo) point-
                       centroid differences, running sums as FP32 hi + lo pairs;
                       near field and final sums in FP64 */

/* bem_options.flags: precomputed node records (mixed meshes only).  The
 * paper compares Gaussian points precomputed for all elements with points
 * computed on the fly (Sec. 6, Table 4).  With this flag bem_create stores,
 * for every element, the node records of all five rules of its type (3600
 * bytes per element, outside the scratch budget), and the far-field kernel
 * streams them into its node buffers with asynchronous copies, one element
 * ahead, instead of computing them per (warp, element).  Results agree with
 * the on-the-fly path to FP32 rounding (the charge scales the element sums
 * instead of each node's weight).  Linear and quadratic densities and the
 * field gradient use the on-the-fly expansion whatever the flag. */
#define BEM_FLAG_NODE_TABLE 1

typedef struct bem_mesh bem_mesh;

/* Options of bem_create (all fields: 0 / NULL = default). */
typedef struct {
    int32_t precision;        /* BEM_FP64 (default) or BEM_MIXED */
    int32_t flags;            /* 0 or BEM_FLAG_NODE_TABLE */
    const double* limits;     /* NULL or 10 host doubles: for triangles then
                                 rectangles, the 5 ascending DR limits
                                 [near, 33-pt, 19|17-pt, 12-pt, 7-pt] of the
                                 rule bands (Sec. 4): DR < limits[0] is
                                 integrated analytically, limits[0] <= DR <
                                 limits[1] uses the 33-point rule, ... and
                                 DR >= limits[4] the 4-point rule.  Default
                                 (bem_default_limits): triangles {4.5, 12,
                                 30, 120, 2250}, rectangles {6, 18, 45, 160,
                                 2800}. */
    double eps0;              /* vacuum permittivity; <= 0: 8.8541878128e-12 F/m */
    size_t device_mem_budget; /* upper bound in bytes on the scratch memory the
                                 mesh may hold (work lists, sort buffers);
                                 0 = 4 GiB */
} bem_options;

/*
 * bem_create -- upload and preprocess a mesh of constant-density elements.
 *   types  [n]      BEM_TRIANGLE or BEM_RECTANGLE
 *   verts  [n][4][3] corners: a triangle uses A, B, C (row 3 ignored); a
 *                   rectangle gives P0, P1, P2, P3 around the boundary, side
 *                   a = |P1 - P0| along u_x, side b = |P3 - P0| along u_y
 *                   (Eq. 3.2); P2 must equal P1 + P3 - P0 and the sides must
 *                   be orthogonal to 1e-9 relative.
 *   sigma  [n]      charge density of each element (Eq. 2.1)
 *   n      number of elements, >= 1 and < 2^31
 * Per element it computes the centroid Q_cen, the average side length L
 * (Sec. 2: (a+b+c)/3 for a triangle, (a+b)/2 for a rectangle), the area A
 * and the frame from which the cubature nodes of Eq. 3.2 / Eq. 3.3 are
 * expanded on the fly.  BEM_ERR_INVALID names the first bad element.
 * The mesh copies everything it needs; the caller's arrays may be freed
 * after the call.  *out receives the mesh (NULL on failure).
 */
int bem_create(const int32_t* types, const double* verts, const double* sigma, int64_t n,
               const bem_options* opt, void* stream, bem_mesh** out);

/* Release the mesh and every device buffer it owns.  NULL is a no-op. */
void bem_destroy(bem_mesh* mesh);

/*
 * bem_default_limits -- the default DR band limits of bem_options.limits
 * (10 host doubles, triangles then rectangles, in that field's layout).
 * Sec. 4 prints limits for the triangle potential at a 2e-15 relative error
 * (analytic below DR 3, then 33, 19, 12, 7, 4 points from DR 3, 8, 20, 80,
 * 1500) and notes that the field needs slightly higher ones, which then
 * serve potential and field together; it prints none for rectangles.  The
 * defaults repeat the paper's experiment (random unit-cube elements, the
 * 16 x 16 Gauss-Legendre reference, mean relative errors) for phi and E
 * together and take, per rule, the smallest DR from which both stay at or
 * below 2e-15, rounded up -- the near limit included: the 33-point rule
 * reaches 2e-15 for the triangle potential at DR 3, as printed, and for the
 * field at DR 4.1 (triangles) and 5.3 (rectangles).  Host only.
 */
int bem_default_limits(double* out /* 10 */);

/* Number of elements of the mesh (0 for NULL). */
int64_t bem_num_elements(const bem_mesh* mesh);

/*
 * bem_set_sigma -- replace the charge densities (n = bem_num_elements
 * doubles), e.g. between the iterations of a charge-density solve.
 */
int bem_set_sigma(bem_mesh* mesh, const double* sigma, void* stream);

/*
 * bem_set_sigma_linear -- charge densities that vary linearly over each
 * element.  The paper treats constant densities and notes that the
 * cubature applies as well to densities that vary over the element
 * (Sec. 7): each node then carries q_i = w_i area sigma(Q_i).  For element j
 * with frame coordinates (alpha, beta) of Q - Q_cen = alpha e0 + beta e1
 * (see bem_rule: triangle alpha = lambda_A - lambda_C, beta = lambda_B -
 * lambda_C; rectangle the natural coordinates x, y of Eq. 3.2)
 *   sigma_j(Q) = coef[3j] + coef[3j+1] alpha + coef[3j+2] beta
 * (a triangle with vertex values sA, sB, sC: coef = (m, sA - m, sB - m),
 * m = (sA + sB + sC) / 3).  bem_eval, bem_eval_noalloc and the server then
 * use these densities: the far field with sigma at every node (the rule
 * bands stay those of constant densities, which costs one polynomial degree
 * of margin: ~1e-11 relative at the band edges instead of ~1e-15), the near
 * field by the analytic integral of the linear density.  bem_set_sigma
 * returns the mesh to constant densities.  bem_assemble and bem_matvec keep
 * their constant unit / x densities; bem_eval_grad uses the linear ones.
 *   coef [n_el][3], host or device
 */
int bem_set_sigma_linear(bem_mesh* mesh, const double* coef, void* stream);

/*
 * bem_linear_coef_from_corners -- the coefficients of bem_set_sigma_linear
 * from density values at the corners of each element (Sec. 7's densities
 * that vary over the element, given where meshes usually carry them).  The
 * frame coordinates are those of Eq. 3.2 / Eq. 3.3 (see bem_rule):
 *   triangle (sA, sB, sC): the linear interpolant, coef = (m, sA - m, sB - m)
 *     with m = (sA + sB + sC) / 3;
 *   rectangle (s0, s1, s2, s3) at P0..P3 = natural coordinates (-1,-1),
 *     (1,-1), (1,1), (-1,1): the least-squares plane, ((s0+s1+s2+s3)/4,
 *     (s1+s2-s0-s3)/4, (s2+s3-s0-s1)/4), exact when s0 + s2 = s1 + s3.
 *   types  [n]     host
 *   values [n][4]  host; a triangle's fourth value is ignored
 *   coef   [n][3]  host, out
 * Host only; no device needed.  BEM_ERR_INVALID for an unknown type.
 */
int bem_linear_coef_from_corners(const int32_t* types, const double* values, int64_t n, double* coef);

/*
 * bem_set_sigma_quadratic -- charge densities that vary quadratically over
 * each element (the varying densities of Sec. 7, one order above
 * bem_set_sigma_linear), in the same frame coordinates:
 *   sigma_j(Q) = c0 + c1 alpha + c2 beta + c3 alpha^2 + c4 alpha beta + c5 beta^2,
 *   (c0 .. c5) = coef[6j .. 6j+5]
 * The far field takes sigma at every node (the constant-density rule bands
 * now lose two polynomial degrees of margin: up to ~1e-8 relative in E at the
 * edge of the 4-point rule's band), the near field the analytic integral of the
 * quadratic density.  bem_set_sigma or bem_set_sigma_linear replaces it;
 * bem_assemble and bem_matvec keep their constant densities, bem_eval_grad
 * uses the quadratic ones.
 *   coef [n_el][6], host or device
 */
int bem_set_sigma_quadratic(bem_mesh* mesh, const double* coef, void* stream);

/*
 * bem_eval -- phi and E at n field points (Eq. 2.1 approximated by Eq. 4.1
 * with the rule bands of Sec. 4 and the analytic near field).
 *   points [n][3]  field points
 *   phi    [n]     potential (V), or NULL to skip it
 *   E      [n][3]  field (V/m), or NULL to skip it
 * n = 0 is a no-op.  Each result depends only on its own field point and
 * the mesh: it is the same whatever other points share the call.  On a
 * field point that lies on an element (to 1e-12 of its mean side length)
 * the normal field is taken as the mean of both sides (zero contribution).
 */
int bem_eval(bem_mesh* mesh, const double* points, int64_t n, double* phi, double* E, void* stream);

/*
 * bem_eval_grad -- the field gradient dE_i / dx_j at n field points.  The
 * paper notes that point charges give higher derivatives of the field
 * directly (Sec. 7, for field maps by Hermite interpolation): each node
 * charge q_i adds q_i (delta_ij / r^3 - 3 r_i r_j / r^5), with the same rule
 * bands as bem_eval; below the near limit the analytic gradient of the
 * uniformly charged polygon is used (the derivative of the near-field
 * formula: edge line fields and the gradient of the solid angle).  The far
 * sums take the mesh's precision: FP64, or on a mixed mesh FP32 node terms
 * (the point-centroid difference split as in bem_eval) with per-element
 * sums b, c, c alpha, c beta, c alpha^2, c alpha beta, c beta^2 (b = q_i / r^3,
 * c = q_i / r^5) from which the element's tensor is formed, summed as FP32
 * hi + lo pairs (~1e-6 relative, as the mixed field); near pairs are FP64.
 * Linear and quadratic densities (bem_set_sigma_linear / _quadratic): the
 * node charges carry sigma(Q_i); near pairs move the in-plane derivative
 * onto the density (divergence theorem in the plane: the field of
 * d sigma / d tau minus edge integrals of sigma (P - Q) / R^3, in closed
 * form), the normal column from symmetry and zero trace.
 *   points [n][3]
 *   G      [n][6]  (dEx/dx, dEy/dy, dEz/dz, dEx/dy, dEx/dz, dEy/dz) in V/m^2;
 *                  the tensor is symmetric and, off the elements, traceless
 * Host or device arrays; allocates its partial sums per call.  A point on an
 * element edge gets that edge's (singular) contribution left out.
 */
int bem_eval_grad(bem_mesh* mesh, const double* points, int64_t n, double* G, void* stream);

/*
 * bem_assemble -- BEM collocation matrix (the linear system for the charge
 * densities that the paper's BEM context solves, Sec. 1 and Sec. 5):
 *   A[i][j] = potential at colloc[i] of element j with sigma_j = 1,
 * by the same rule bands, the analytic branch for near and self terms, and
 * 1/(4 pi eps0).
 *   colloc [m][3]       collocation points
 *   A      [m][n_el]    output, row-major (m * n_el doubles, n_el =
 *                       bem_num_elements)
 */
int bem_assemble(bem_mesh* mesh, const double* colloc, int64_t m, double* A, void* stream);

/*
 * bem_matvec -- matrix-free product y = A x of the collocation matrix at the
 * element centroids (the shell-matrix product of the paper's iterative BEM
 * solver context, Sec. 5): y[i] = potential at the centroid of element i of
 * all elements carrying charge density x[j].
 *   x [n_el], y [n_el]
 */
int bem_matvec(bem_mesh* mesh, const double* x, double* y, void* stream);

/*
 * bem_solve -- charge densities for prescribed potentials: solves
 *   sum_j A[i][j] sigma[j] = rhs[i]   (i, j = 0 .. n_el - 1)
 * with A the collocation matrix at the element centroids (bem_matvec): the
 * linear system for the charge densities of the BEM electrode problem,
 * solved before phi and E are evaluated from them (Sec. 1 names direct and
 * iterative solvers; the field code of Sec. 5 keeps its matrices unstored
 * and iterates).  This is restarted GMRES with a Jacobi (diagonal) right
 * preconditioner, every product a bem_matvec and every vector operation a
 * kernel of this library, so the matrix is never stored.  Each product has
 * the mesh's precision: an FP64 mesh reaches relative residuals near 1e-14,
 * a mixed mesh near 1e-7.
 *   rhs   [n_el]  potentials at the centroids (V), host or device
 *   sigma [n_el]  out: charge densities (C/m^2); in: the initial guess when
 *                 opt->flags has BEM_SOLVE_X0 (else the solve starts from 0)
 *   opt           may be NULL: restart 50, max_iter 1000 products, tol 1e-12
 *                 (FP64 mesh) or 1e-6 (mixed mesh)
 *   info  [3]     may be NULL: products used, final relative residual
 *                 |rhs - A sigma| / |rhs| (recomputed, not the GMRES estimate),
 *                 1 if converged else 0
 * With BEM_SOLVE_REFINE on an FP64 mesh the solve refines iteratively: FP64
 * residuals b - A sigma, corrections from GMRES on mixed-precision products
 * (to 1e-6), sigma += correction, until the FP64 residual meets tol -- the
 * same answer for a fraction of the FP64 products (this GPU's FP64 rate is
 * about 1/74 of its FP32 rate); info[0] then counts both kinds of product.
 * Returns BEM_ERR_NOT_CONVERGED (sigma holds the last iterate) if the
 * residual is above tol after max_iter products.  The mesh's own sigma is
 * not changed (bem_set_sigma sets it).  Deterministic: the same inputs give
 * the same bits.
 */
#define BEM_SOLVE_X0 1
#define BEM_SOLVE_REFINE 2
typedef struct {
    int32_t restart;  /* Krylov dimension per cycle (0: 50, at most 200) */
    int32_t max_iter; /* matrix-vector products in total (0: 1000) */
    double tol;       /* relative residual to reach (0: the default above) */
    int32_t flags;    /* BEM_SOLVE_X0 | BEM_SOLVE_REFINE */
} bem_solve_options;
int bem_solve(bem_mesh* mesh, const double* rhs, double* sigma, const bem_solve_options* opt, double* info,
              void* stream);

/* Element centroids Q_cen (Sec. 2), n_el x 3, written to a host or device array. */
int bem_centroids(bem_mesh* mesh, double* out, void* stream);

/*
 * bem_rule -- the expanded nodes of one cubature rule as the library stores
 * them (App. A, App. B): for rule index r = 0..4 (N = 4, 7, 12, 19|17, 33),
 * writes N rows (alpha, beta, w) to out (host, 33 * 3 doubles) and returns
 * N.  A node sits at Q = Q_cen + alpha e0 + beta e1 with e0 = A - Q_cen,
 * e1 = B - Q_cen for a triangle (alpha = lambda_A - lambda_C, beta =
 * lambda_B - lambda_C, Eq. 3.3) and e0 = (a/2) u_x, e1 = (b/2) u_y for a
 * rectangle (alpha = x, beta = y, Eq. 3.2).  Host only; no device needed.
 */
int bem_rule(int32_t type, int32_t r, double* out);

/* Statistics of the last bem_eval / bem_assemble / bem_matvec on this mesh:
 * out[0..5] pair counts per distance-ratio band for triangles (analytic,
 * 33, 19, 12, 7, 4 points), out[6..11] the same for rectangles (analytic,
 * 33, 17, 12, 7, 4 points), out[12] the number of near (analytic) pairs,
 * out[13] (warp, element) pairs where one band served all 32 x PT points
 * of the warp, out[14] those that fell back to per-point bands, out[15]
 * node evaluations executed by the far-field kernel (masked ones
 * included; compare with the pairs x nodes of out[0..11]).
 * out[0..11] and out[13..15] are filled only by calls made with statistics
 * enabled (bem_set_stats); out[12] always. */
int bem_last_stats(const bem_mesh* mesh, int64_t* out /* 16 */);

/* Enable (1) or disable (0) the per-band pair counts of the next calls; the
 * counting variant of the far-field kernel is slower, so it is off by default. */
int bem_set_stats(bem_mesh* mesh, int32_t enable);

/* Enable (1) or disable (0) per-phase timing with CUDA events recorded on the
 * call's stream.  bem_last_times then gives, in milliseconds, for the last
 * bem_eval / bem_matvec: out[0] spatial sort of the points, out[1] far-field
 * cubature kernel, out[2] near-pair scan + analytic near-field kernel,
 * out[3] finalisation (sum, scale, scatter). */
int bem_set_timing(bem_mesh* mesh, int32_t enable);
int bem_last_times(const bem_mesh* mesh, double* out /* 4 */);

/* Total number of CUDA kernels this library has launched in this process
 * (all meshes, all devices). */
int64_t bem_kernel_launches(void);

/*
 * bem_peak_rate -- measured throughput of one arithmetic pipe of the current
 * device, the denominator of the far-field kernel's roofline fraction.  The
 * paper has no counterpart (it reports times, not pipe rates); the cubature
 * sum of Eq. 4.1 is bound by FP32 fused multiply-adds plus one reciprocal
 * square root per node (mixed path) or by FP64 arithmetic (FP64 path).
 *   kind  BEM_PEAK_FFMA (scalar FP32 FMA), BEM_PEAK_FFMA2 (packed f32x2 FMA),
 *         BEM_PEAK_RSQRT (MUFU reciprocal square root), BEM_PEAK_DFMA (FP64 FMA)
 *   out   [3] host: out[0] lane operations per second (an FMA counts as one
 *         operation, a packed FFMA2 as two), out[1] duration of the best of
 *         three timed launches in ms (CUDA events), out[2] the SM clock in
 *         MHz during the run (clock64 over the global timer on one block)
 * Every SM runs 2048 threads, each with eight independent chains of the
 * instruction; a launch lasts about 50 ms.  Allocates a few bytes of device
 * memory and a stream for the call.  BEM_ERR_INVALID for an unknown kind.
 */
#define BEM_PEAK_FFMA 0
#define BEM_PEAK_FFMA2 1
#define BEM_PEAK_RSQRT 2
#define BEM_PEAK_DFMA 3
int bem_peak_rate(int32_t kind, double* out /* 3 */);

/*
 * bem_eval_noalloc -- bem_eval that allocates no device memory.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * let the library call cudaMalloc -- an application that hands all device
 * memory to its own pool up front, or a latency-critical loop (a particle
 * tracker asking for fields at every step) that must never wait on the
 * allocator.  bem_eval grows the mesh's scratch buffers on demand; this call
 * instead takes all of its scratch from one fixed array of
 * BEM_NOALLOC_BYTES bytes in device memory, which every GPU that loads the
 * library holds until the process exits.  It runs the same kernels, so its
 * results equal bem_eval's.
 *   points [n][3], phi [n] (or NULL), E [n][3] (or NULL): device arrays of
 *   the mesh's device; host arrays are rejected (BEM_ERR_INVALID).
 *   n <= BEM_NOALLOC_MAX_POINTS, else BEM_ERR_INVALID.
 * If the points have more than BEM_NOALLOC_MAX_NEAR near-field (analytic)
 * pairs the call returns BEM_ERR_CAPACITY and phi / E hold incomplete
 * values: split the points, or use bem_eval.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls on a device share the one array, which keeps the previous
 * call's contents (the call clears what must start at zero): calls that
 * overlap on the GPU -- from two host threads or on two streams -- race.
 * The call returns after its results are complete (it synchronises the
 * stream).
 */
#define BEM_NOALLOC_MAX_POINTS 16384
#define BEM_NOALLOC_MAX_NEAR 262144
#define BEM_NOALLOC_BYTES (40u << 20)
int bem_eval_noalloc(bem_mesh* mesh, const double* points, int64_t n, double* phi, double* E, void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of field-point queries on a device-resident
 * mesh (a particle tracker's stream of uneven requests).  A server thread
 * forms ticks of at most max_points_per_tick points: first every waiting
 * small request (at most 1/8 of a tick) whole, in arrival order, then the
 * other requests in arrival order, splitting one that does not fit the
 * space left (its next piece goes into this tick, the rest into later
 * ticks).  A tick's points are copied in, one CUDA graph of the whole
 * evaluation (captured at creation; the persistent far-field kernel walks
 * (point tile x element chunk) work items) is replayed, and the results are
 * copied back.  Two ticks can be in flight, so requests that arrive while
 * one tick runs are admitted into the next and overlap it; at most one of
 * them holds pieces of large requests, so a small request waits behind at
 * most one tick of large work.  Each result equals bem_eval's for the same
 * points bit for bit, whatever other requests shared its ticks and however
 * it was split.  While a server exists it owns the mesh: make no other call
 * on that mesh until bem_server_destroy.
 * ------------------------------------------------------------------------ */
typedef struct bem_server bem_server;

typedef struct {
    int64_t max_points_per_tick;     /* points one tick can take (0: 131072); a
                                        larger request is split across ticks.
                                        Smaller ticks finish sooner (lower
                                        latency for small requests), larger
                                        ones fill the GPU better */
    int64_t max_near_pairs_per_tick; /* near-field pairs one tick can take (0: 2^21);
                                        a tick that has more evaluates its
                                        requests one by one with bem_eval */
    size_t device_mem_budget;        /* bound on the server's device memory
                                        (0: 2 GiB), and never more than 3/4 of
                                        the device memory free at creation;
                                        max_points_per_tick is halved until two
                                        ticks' buffers fit.  All of it is
                                        allocated at creation: ticks allocate
                                        nothing */
    int32_t flags;                   /* reserved, must be 0 */
} bem_server_options;

/* Create a server on mesh (opt may be NULL).  Builds both ticks' device
 * buffers and CUDA graphs and starts the server thread. */
int bem_server_create(bem_mesh* mesh, const bem_server_options* opt, bem_server** out);

/* Finish every queued request, stop the thread, release everything. */
void bem_server_destroy(bem_server* server);

/* Queue n field points (host array [n][3], copied) for evaluation; *ticket
 * names the request.  Thread-safe.  BEM_ERR_INVALID for n < 1 or a
 * non-finite coordinate; BEM_ERR_OOM if the host copy cannot be made. */
int bem_submit(bem_server* server, const double* points, int64_t n, uint64_t* ticket);

/* Non-blocking: *done = 1 and the results copied to phi [n] / E [n][3]
 * (host arrays, either may be NULL) once the request has finished; the
 * ticket is then spent.  *done = 0 otherwise.  BEM_ERR_NOT_FOUND for an
 * unknown or spent ticket. */
int bem_poll(bem_server* server, uint64_t ticket, double* phi, double* E, int32_t* done);

/* Blocking with a bound: wait at most timeout_s seconds for the request,
 * then copy its results as bem_poll.  BEM_ERR_TIMEOUT if it is still
 * unfinished (the ticket stays valid). */
int bem_wait(bem_server* server, uint64_t ticket, double timeout_s, double* phi, double* E);

/* Drop a request: a queued one is removed, a running one's results are
 * discarded when its tick ends. */
int bem_cancel(bem_server* server, uint64_t ticket);

/* Stop (1) or resume (0) forming new ticks; queued requests wait meanwhile. */
int bem_server_pause(bem_server* server, int32_t paused);

/* Service statistics since creation or the last reset (reset = 1 clears them
 * after reading): out[0] requests completed, out[1] p50 and out[2] p99
 * latency (ms, submission to results on the host), out[3] mean latency
 * (ms), out[4] ticks, out[5] points evaluated, out[6] ticks that fell back
 * to per-request evaluation, out[7] points per tick (capacity), out[8]
 * device bytes held, out[9] graph launches. */
int bem_server_stats(bem_server* server, int32_t reset, double* out /* 10 */);

/* Latency of every request completed since creation or the last stats reset,
 * in completion order: ms[i] (submission to results on the host) and
 * points[i] (its size), for i < min(cap, *count); *count receives the number
 * of completed requests.  Host arrays of cap entries (cap = 0: count only). */
int bem_server_latencies(bem_server* server, int64_t cap, double* ms, int64_t* points, int64_t* count);

/* Message of the last failure on the calling thread ("" if none). */
const char* bem_last_error(void);

/* Library version string. */
const char* bem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H */
