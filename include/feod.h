/*
 * feod.h -- C ABI of the GB300 (sm_103a) matrix-free finite element operator library.
 *
 * The library applies the finite element operator decomposition A = P^T G^T B^T D B G P
 * (Fig. 1 and Eq. 1) of the steady p-Laplacian  -div(kappa(|grad u|) grad u) = f,
 * kappa = kappa_rho(rho_e) (eps^2 + |grad u|^2)^((p-2)/2), and its exact Jacobian
 * J(u) = P^T G^T B^T J_D(u_q) B G P (Eq. 2), where the pointwise operator D is differentiated
 * at each quadrature point with forward-mode dual numbers.  On top of these it runs a
 * matrix-free Newton-CG solve and the adjoint design gradient (the adjoint loads of the
 * design-sensitivity discussion that follows Eq. 3).
 *
 * Discretisation: structured lattice of n[0] x n[1] (x n[2]) elements (dim = 2 or 3) with
 * caller-given (jittered) vertices and a multilinear geometry map per element; continuous
 * Lagrange basis of order k = 1..6 on Gauss-Lobatto-Legendre nodes; (k+1)^dim Gauss-Legendre
 * points per element.  DOFs form the lattice (k n[0] + 1) x (k n[1] + 1) (x (k n[2] + 1)),
 * numbered lexicographically with x fastest; elements are numbered ex + n[0] (ey + n[1] ez).
 * Essential (Dirichlet) DOFs are the DOFs on the boundary of the lattice's box, except on faces
 * marked natural (subdomain interfaces).  On one GPU the subdomain restriction P is the identity
 * plus this Dirichlet elimination:
 *   - R(u) = A(u) - F with R_i = 0 on essential DOFs (u carries the boundary values);
 *   - J(u) v treats essential entries of v as zero and returns y_i = v_i on essential DOFs,
 *     so J is symmetric positive (semi)definite.
 *
 * Conventions for every call:
 *   - Vector arguments are DEVICE pointers owned by the caller, of length N_L (number of DOFs)
 *     unless stated otherwise; the library never frees or retains them beyond the call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are stream-ordered and
 *     asynchronous unless stated otherwise; the caller keeps inputs alive until the stream work
 *     completes.
 *   - Every call returns an fe_status and never aborts or traps; the message of the last non-OK
 *     status of a context is returned by fe_last_error().
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef FEOD_H
#define FEOD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ctx fe_ctx;

typedef enum {
    FE_OK = 0,
    FE_ERR_ARG = 1,            /* invalid argument (null pointer, size, range)               */
    FE_ERR_MESH = 2,           /* det J <= 0 at some quadrature point (inverted element)      */
    FE_ERR_CUDA = 3,           /* a CUDA runtime call failed, or a kernel's bounded wait
                                  timed out (see fe_selftest_wait_timeout)                    */
    FE_ERR_OOM = 4,            /* device or host allocation failed                           */
    FE_ERR_UNSUPPORTED = 5,    /* order / quadrature / size outside what is built            */
    FE_ERR_NAN = 6,            /* a NaN or Inf appeared in a norm                            */
    FE_ERR_NOT_CONVERGED = 7,  /* Newton or CG reached its iteration limit                   */
    FE_ERR_BREAKDOWN = 8,      /* CG found p^T J p <= 0 or the line search failed             */
    FE_ERR_STATE = 9           /* call out of order (e.g. cached Jacobian requested before
                                  fe_linearize)                                               */
} fe_status;

/* Structured lattice mesh of n[0] x n[1] (x n[2]) elements.  `vertices` is a HOST array
 * [(n[0]+1)(n[1]+1)(n[2]+1)][dim] (the last factor absent in 2D), lexicographic with x fastest; it
 * is copied during fe_setup.  natural_faces: the faces of the lattice's box whose DOFs are NOT
 * essential -- the boundary between this subdomain and its neighbours when the problem is split
 * by the subdomain restriction P (Fig. 1), where the neighbours' partial sums complete the
 * operator; bits 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+ (0 = every boundary DOF essential, the
 * single-domain problem). */
typedef struct {
    int dim;                   /* 2 or 3                                                      */
    int n[3];                  /* elements per direction x, y, z, each >= 1 (n[2] unused in 2D) */
    const double *vertices;
    int natural_faces;         /* mask of non-essential box faces (see above)                 */
} fe_mesh;

/* The pointwise law and the load.  kappa_rho(rho) = kappa_eps + rho^kappa_q multiplies the flux
 * when `rho` is given (one HOST value per element, copied), else kappa_rho = 1. */
typedef struct {
    double p;                  /* exponent; p >= 2, or p > 1 with eps > 0                     */
    double eps;                /* regularisation of |grad u|^2 (0 = the plain p-Laplacian)     */
    int f_kind;                /* 0: f = f_const; 1: manufactured source of u* = exp(x+y/2+z/3) */
    double f_const;
    const double *rho;         /* host, one value per element [N_e] or NULL                  */
    double kappa_eps;
    double kappa_q;
} fe_problem;

/* Launch-shape options (fe_setup picks them from the built-in tuning table). */
typedef struct {
    int tile;                  /* elements per tile edge: one CTA owns tile^dim elements;
                                  0 = tuned default                                           */
    int per_element;           /* 1: apply the cached Jacobian, and evaluate the residual and
                                  the tangent, with the per-element kernels (element-by-element
                                  sum factorisation, staged in-tile G^T) instead of the
                                  tile-level ones (3D); for comparison only                    */
} fe_setup_opts;

/* fe_setup: build a context for the mesh, order k (1..6) and quadrature q1d (0 or k+1 Gauss
 * points per direction).  Copies the mesh and design field to the device, builds the element
 * restriction G as explicit index arrays (tile slot codes and the transposed halo index that
 * makes G^T deterministic without atomics), and evaluates the geometric factors at every
 * quadrature point (w det J J^{-1}J^{-T}, 1/(w det J), w det J f).  Fig. 1 / the decomposition
 * paragraph: P, G and B are linear and topological and set up once, outside differentiation.
 * Synchronises the current device.  Errors: FE_ERR_ARG, FE_ERR_MESH (det J <= 0),
 * FE_ERR_UNSUPPORTED (order, q1d, or more than 2^30-1 DOFs), FE_ERR_OOM, FE_ERR_CUDA.
 * On success *out owns all device memory it allocated; release with fe_destroy. */
fe_status fe_setup(const fe_mesh *mesh, int order, int q1d, const fe_problem *prob, fe_ctx **out);
fe_status fe_setup_ex(const fe_mesh *mesh, int order, int q1d, const fe_problem *prob,
                      const fe_setup_opts *opts, fe_ctx **out);

/* Sizes of the decomposition's vectors (Fig. 1): N_L, the DOFs of the L-vector (on one GPU the
 * T-vector too), the free (non-essential) DOFs among them, and the elements N_e (the E-vector has
 * N_e (k+1)^dim entries, the Q-vector N_e (k+1)^dim points). */
fe_status fe_num_dofs(const fe_ctx *ctx, int64_t *n_l, int64_t *n_free);
fe_status fe_num_elements(const fe_ctx *ctx, int64_t *n_e);

/* fe_residual: r = R(u) = P^T G^T B^T D(B G P u) - F (Eq. 1 minus the load), FP64, essential
 * entries zero.  u, r: device double[N_L]; may not alias. */
fe_status fe_residual(fe_ctx *ctx, const double *u, double *r, void *stream);

/* fe_linearize: evaluate J_D at every quadrature point of u (Eq. 2) with 3 (2 in 2D) dual
 * directions and store it inside the context (partial assembly: FP64 and its FP32 rounding,
 * d(d+1)/2 symmetric entries per point), plus the Jacobi diagonal of J.  u: device double[N_L]. */
fe_status fe_linearize(fe_ctx *ctx, const double *u, void *stream);

/* Device-side failures: every wait inside a kernel is bounded.  One that times out (a tile's
 * tangent copy that does not land) abandons that kernel's work and sets the context's error word;
 * the next synchronous call on the context (fe_jacobian_action_host, fe_cg_solve, newton_solve,
 * fe_check_error) returns FE_ERR_CUDA and clears the word.  Results computed by the failed kernel
 * and by everything queued after it on the context are invalid until that check: callers of the
 * asynchronous calls (fe_residual, fe_jacobian_action, ...) read the word with fe_check_error. */

/* fe_check_error: synchronise `stream`, then return FE_ERR_CUDA (and clear the word) if a kernel
 * of this context has reported a timed-out wait since the last check, else FE_OK. */
fe_status fe_check_error(fe_ctx *ctx, void *stream);

/* fe_selftest_wait_timeout: diagnostic of that path.  Runs one CTA whose bounded wait on an
 * mbarrier phase that nothing completes (no arrival, no copy) gives up after about a second and
 * sets the error word; returns FE_ERR_CUDA exactly as a real timeout would, with the word cleared
 * and the context usable afterwards.  Synchronous on `stream`. */
fe_status fe_selftest_wait_timeout(fe_ctx *ctx, void *stream);

/* fe_jacobian_action: y = J(u) v (Eq. 2).
 *   u == NULL : uses the quadrature-point Jacobian cached by the last fe_linearize (partial
 *               assembly); FE_ERR_STATE if there is none.
 *   u != NULL : stateless: recomputes J_D(u_q) . (B G P v) with one dual direction seeded by the
 *               gradient of v, nothing cached.
 *   precision : 64 -> v, y are double[N_L] and all arithmetic is FP64;
 *               48 -> v, y are double[N_L]; double-float arithmetic: every value is the
 *                     unevaluated sum of two FP32 words (a 48-bit significand, FP32's exponent
 *                     range), computed on the FP32 pipes, from the FP64 tangent split into such
 *                     pairs (split on the first call after each linearisation, into storage
 *                     allocated on first use).  Each operation errs by a small multiple of 2^-48
 *                     relative to its operands, as one FP64 operation does by 2^-53.  Entries of
 *                     v, y and the tangent outside about [1e-30, 1e38] in magnitude lose
 *                     precision to FP32's range.  Cached linearisation only: with u != NULL it
 *                     returns FE_ERR_UNSUPPORTED;
 *               32 -> v, y are float[N_L], FP32 arithmetic and accumulation (the FP32 rounding of
 *                     the FP64 tangent when cached);
 *               -32 -> v, y are double[N_L] but the action is computed exactly as for 32 (the
 *                     inner operator of the mixed-precision Newton-CG).
 * v and y may not alias. */
fe_status fe_jacobian_action(fe_ctx *ctx, const double *u, const void *v, void *y, int precision,
                             void *stream);

/* Same as fe_jacobian_action with u == NULL but v_host/y_host are HOST buffers (pinned memory
 * recommended): copies v to the device, applies J, copies y back; synchronises `stream` before
 * returning.  For 3D problems whose tile kernel has several tile layers along z, the action runs
 * in z-chunks (32 for precision 64 and 8 otherwise, at most one per tile layer): each chunk's
 * DOF planes are copied in on a copy stream while earlier chunks compute, and the planes that are
 * complete are copied back on another while later chunks compute (the same kernels and sums as
 * the one-piece action: the same bits).  The call uses internal streams of its own, the chunks'
 * fix-ups on one of the device's highest priority. */
fe_status fe_jacobian_action_host(fe_ctx *ctx, const void *v_host, void *y_host, int precision,
                                  void *stream);

/* fe_jacobian_action_noalloc: the same y = J v as fe_jacobian_action with u == NULL (cached
 * linearisation, precision 64 / 32 / -32 with the same meaning; not 48, whose tangent storage
 * is allocated on first use), for callers that cannot call cudaMalloc while they run: an
 * application whose device memory is all handed out by its own pool allocator (a cudaMalloc would
 * fail, or take memory the pool counts on), or a host loop with a latency budget that cannot absorb
 * the device-wide synchronisation an allocation may cause.  The paper has no counterpart; it is a
 * deployment variant of the Jacobian action.
 *
 * Scratch: the cross-tile partial sums that fe_jacobian_action keeps in the context's halo buffer
 * go instead to one file-scope device array of FE_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU
 * that loads the library holds until the process exits.  A problem needs one word (8 bytes for
 * precision 64, else 4) per cross-tile partial sum -- about 127 per tile for 3D order 3 with the
 * default 2^3-element tile, so up to about 64^3 elements in FP32 and 50^3 in FP64; larger
 * problems return FE_ERR_UNSUPPORTED with a message and launch nothing.  Every scratch entry that
 * is read is written earlier in the same call, so nothing needs clearing between calls.
 *
 * The first call on a device resolves the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other contexts on the same device) race
 * and produce wrong results -- serialise them.  The call itself allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  v, y: device arrays as for fe_jacobian_action;
 * FE_ERR_STATE without a cached linearisation, FE_ERR_ARG if the current device is not the
 * context's or its index is beyond the 64 devices the address table covers. */
#define FE_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
fe_status fe_jacobian_action_noalloc(fe_ctx *ctx, const void *v, void *y, int precision, void *stream);

/* fe_jacobian_diagonal: diag(J) of the cached linearisation (1 on essential DOFs), FP64. */
fe_status fe_jacobian_diagonal(fe_ctx *ctx, double *diag, void *stream);

/* fe_load_vector: F_i = int f phi_i with essential entries zero, FP64. */
fe_status fe_load_vector(fe_ctx *ctx, double *F, void *stream);

/* fe_node_coords: physical coordinates of every DOF, device double[N_L][dim]. */
fe_status fe_node_coords(fe_ctx *ctx, double *xyz, void *stream);

/* fe_set_design: replace the per-element design field rho (device double[N_e], copied on the
 * stream).  Invalidates the cached linearisation. */
fe_status fe_set_design(fe_ctx *ctx, const double *rho, void *stream);

/* fe_adjoint_vjp (Section 2, the design-sensitivity paragraph after Eq. 3: derivatives of a
 * PDE-constrained objective by the adjoint method, with AD applied locally at the quadrature
 * points): per-element design gradient of the residual contracted with lambda,
 *   grad_rho[e] = lambda^T dR/drho_e = kappa_rho'(rho_e) int_e kappa(|grad u|) grad u . grad lambda,
 * obtained by seeding a dual number on rho at each quadrature point (AD local to the quadrature
 * point; no scatter, element-local reduction).  For the compliance c = F^T u with R(u; rho) = 0,
 * dc/drho = -grad_rho evaluated at the adjoint solution J lambda = F.  Needs a design field.
 * u, lambda: device double[N_L]; grad_rho: device double[N_e] (element order ex fastest). */
fe_status fe_adjoint_vjp(fe_ctx *ctx, const double *u, const double *lambda, double *grad_rho,
                         void *stream);

/* fe_compliance: the design problem's objective c = F^T u (F the load vector, zero on essential
 * DOFs), written to the DEVICE double *c; summed in a fixed order.  The compliance of Section 2's
 * design example (Fig. 2).  u: device double[N_L]. */
fe_status fe_compliance(fe_ctx *ctx, const double *u, double *c, void *stream);

/* fe_compliance_gradient: grad_rho = scale * dc/drho at the solution u of R(u; rho) = 0, by the
 * adjoint method of the paragraph after Eq. 3: linearise at u (fe_linearize), solve J(u) lambda = F
 * (J symmetric) by Jacobi-preconditioned CG to ||r|| <= rtol ||F|| in `precision` (as
 * fe_cg_solve's), then grad_rho = -scale lambda^T dR/drho (fe_adjoint_vjp's kernel).  Needs a
 * design field; replaces the cached linearisation by the one at u.  u: device double[N_L];
 * grad_rho: device double[N_e]; iters (may be NULL): the CG iterations.  Synchronous.  Errors as
 * fe_cg_solve's. */
fe_status fe_compliance_gradient(fe_ctx *ctx, const double *u, double scale, double rtol, int max_iter,
                                 int precision, double *grad_rho, int *iters, void *stream);

/* fe_element_matrices: dense element tangent matrices K_e = dr_e/du_e = B^T J_D(u_q) B (Eq. 3) of
 * the elements [e0, e0 + count) (lexicographic element order, x fastest) at the state u, each
 * [nl][nl] row-major in the local DOF order a + D1 (b + D1 c) (D1 = order + 1), no Dirichlet
 * convention.  The comparison of where the AD sits (Table 1's columns), not a solver path:
 *   method 0 (HND): the law's tangent written out by hand at each quadrature point;
 *   method 1 (RES): forward AD at the quadrature point (the law on dim dual directions);
 *   method 2 (ELM): forward AD at the element level (the element residual on dual numbers over
 *                   the element DOFs, 8 directions per pass, B and B^T inside the AD).
 * HND and RES form K_e = sum_q G_q^T T_q G_q with dense reference-gradient tables.  3D, order 1..3
 * (FE_ERR_UNSUPPORTED otherwise).  u: device double[N_L]; K: device double[count * nl * nl]. */
fe_status fe_element_matrices(fe_ctx *ctx, const double *u, int method, int64_t e0, int64_t count,
                              double *K, void *stream);

/* Newton-CG options.  Defaults (fe_newton_default_opts): rtol 1e-8, max_newton 50, max_cg 20000,
 * cg_rtol 1e-4, inner_precision 64, line_search 1, armijo 1e-4, max_halvings 20,
 * cg_batch 16, use_graph 2, forcing 0, eta_max 0.1. */
typedef struct {
    double rtol;               /* stop when ||R(u_k)||_2 <= rtol ||R(u_0)||_2                    */
    int max_newton;
    int max_cg;                /* per Newton step                                              */
    double cg_rtol;            /* inner CG stops when ||r_cg|| <= cg_rtol ||R(u_k)||           */
    int inner_precision;       /* CG precision, as fe_jacobian_action's: 64 FP64; 48 double-
                                  float J v in an FP64 CG; -32 FP32 J v in an FP64 CG; 32
                                  FP32 J v and FP32 CG vectors                                */
    int line_search;           /* 1: backtracking on ||R||_2                                   */
    double armijo;             /* accept alpha when ||R(u+alpha d)|| <= (1-armijo alpha)||R(u)|| */
    int max_halvings;
    int cg_batch;              /* CG iterations enqueued between host convergence checks
                                  (use_graph 0, 1) or per pass of the device loop (2)          */
    int use_graph;             /* 0: plain launches; 1: each CG batch replayed as a captured
                                  CUDA graph, host check after each; 2: the whole CG solve as
                                  one graph launch, a conditional WHILE node repeating the batch
                                  while the device-side CG flag says running                   */
    int forcing;               /* inner CG tolerance: 0 the fixed cg_rtol; 1 Eisenstat-Walker
                                  choice 2 (newton_solve); the batched Newton uses cg_rtol     */
    double eta_max;            /* forcing 1: the largest inner tolerance, in (0, 1)            */
} fe_newton_opts;

#define FE_NEWTON_HIST 64

typedef struct {
    int newton_iters;
    int cg_iters_total;
    int line_search_halvings;
    int status;                /* fe_status of the solve                                       */
    double r0, r_final;        /* ||R(u_0)||_2, ||R(u_final)||_2                                */
    double t_total_ms;         /* wall time of the solve (host clock, device synchronised)     */
    double t_cg_ms;            /* part of it spent in CG                                       */
    int64_t kernel_launches;   /* kernels this solve launched (graph replays included)         */
    double r_hist[FE_NEWTON_HIST];  /* ||R|| after each Newton step                            */
    int cg_hist[FE_NEWTON_HIST];    /* CG iterations of each Newton step                       */
} fe_newton_report;

fe_status fe_newton_default_opts(fe_newton_opts *opts);

/* newton_solve (Section 2, closing remarks: the matrix-free nonlinear solver that the residual of
 * Eq. 1 and the Jacobian action of Eq. 2 serve; the paper leaves its algorithm to later work, so
 * the one below -- inexact Newton with CG and a backtracking line search -- is this library's
 * reading): solve R(u) = 0 from u_inout (device double[N_L], carrying the boundary values),
 * overwritten with the solution.  Each step: R and J_D at u (fused, FP64 dual numbers), Jacobi-
 * preconditioned CG on J d = -R with the partially assembled J, then a backtracking line search
 * on ||R|| (R, its norm, u and the line search always FP64).  inner_precision 64: the CG runs in
 * FP64.  48: FP64 CG vectors and scalars with the double-float operator (the FP64 tangent split
 * into FP32 word pairs before each CG), for -R scaled by a power of two near its RMS (exact).  -32: the FP32 operator (FP32 arithmetic on the FP32 rounding of the stored tangent) is
 * applied to FP64 CG vectors; dot products, norms and updates FP64.  32: the CG runs on FP32
 * vectors with the FP32 operator, for -R scaled by a power of two near its RMS (exact), with its
 * inner products accumulated in compensated FP32 (Ogita-Rump-Oishi Dot2) and summed in FP64; its
 * scalars are FP64.  Inner tolerance: cg_rtol at every step (forcing 0), or (forcing 1) the
 * forcing term of Eisenstat and Walker's choice 2 (SIAM J. Sci. Comput. 17, 1996): eta_0 =
 * eta_max, eta_k = 0.9 (||R_k|| / ||R_k-1||)^2, raised to 0.9 eta_k-1^2 when that exceeds 0.1,
 * raised to 0.5 rtol ||R_0|| / ||R_k|| (no more accuracy than the Newton stop needs), then kept
 * in [1e-6, eta_max].  All reductions run in a fixed order, so results are bitwise reproducible on
 * a given GPU model.  Runs on an internal stream after synchronising `stream`; synchronous
 * (returns after the solve).  report may be NULL. */
fe_status newton_solve(fe_ctx *ctx, double *u_inout, const fe_newton_opts *opts,
                       fe_newton_report *report, void *stream);

/* fe_cg_solve: solve J x = b with the cached linearisation (e.g. the adjoint J lambda = F; J is
 * symmetric), x starting from 0, Jacobi-preconditioned CG to ||r|| <= rtol ||b||.  precision 64,
 * 48, -32 or 32 as newton_solve's inner_precision (with 32 the attainable relative residual is about
 * 1e-6, so a smaller rtol ends in FE_ERR_NOT_CONVERGED at max_iter).  b, x: device double[N_L].
 * Synchronous.  iters may be NULL. */
fe_status fe_cg_solve(fe_ctx *ctx, const double *b, double *x, double rtol, int max_iter,
                      int precision, int *iters, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Vector operations on device vectors of a context's length N_L, FP64, stream-ordered: the CG's
 * building blocks, exposed for solvers that run outside the library -- in particular the
 * subdomain-split solve, where the subdomain restriction P (Fig. 1) puts one exchange of
 * interface values after each local operator application and a sum over ranks after each local
 * inner product.  Calls on one context must not overlap on the GPU (fe_dot's reduction scratch
 * belongs to the context).
 * --------------------------------------------------------------------------------------------- */
/* fe_dot: *out (a DEVICE double) = sum_{begin <= i < end} a_i b_i, summed in a fixed order (the
 * same range gives the same bits on the same GPU model).  FE_ERR_ARG for a range outside [0, N_L]. */
fe_status fe_dot(fe_ctx *ctx, const double *a, const double *b, int64_t begin, int64_t end, double *out,
                 void *stream);
/* fe_axpby: y = alpha x + beta y (with beta == 0, y is only written). */
fe_status fe_axpby(fe_ctx *ctx, double alpha, const double *x, double beta, double *y, void *stream);
/* fe_pointwise_mul: z_i = d_i r_i (z may alias r; the Jacobi scaling of a residual). */
fe_status fe_pointwise_mul(fe_ctx *ctx, const double *d, const double *r, double *z, void *stream);
/* fe_reciprocal: y_i = 1 / x_i (y may alias x). */
fe_status fe_reciprocal(fe_ctx *ctx, const double *x, double *y, void *stream);
/* Faces of the DOF lattice: face 2a + s is the plane where coordinate a (0 x, 1 y, 2 z) is 0
 * (s = 0) or its last value (s = 1).  fe_face_size: number of DOFs of the face.  fe_face_add:
 * y_g += buf_i for the face's i-th DOF g (DOFs in lexicographic order of the two other axes, lower
 * axis fastest), on non-essential DOFs only (essential ones keep their value) -- P^T across an
 * interface: the neighbour's partial sums of the shared DOFs added to this subdomain's.  For
 * face 4 (z = 0) and 5 (z = last) of a 3D lattice the face's DOFs are the contiguous first and
 * last (k n[0] + 1)(k n[1] + 1) entries of a vector, so buf can be a neighbour's slice as is. */
fe_status fe_face_size(const fe_ctx *ctx, int face, int64_t *size);
fe_status fe_face_add(fe_ctx *ctx, int face, double *y, const double *buf, void *stream);

/* Profiling: when enabled, every kernel launch is bracketed by CUDA events on its stream.
 * fe_prof_read synchronises, then returns for kernel name index i (0 <= i < *count) its name,
 * number of launches and total milliseconds since the last reset. fe_launch_count returns the
 * number of kernels launched by the context since the last reset (graph replays included). */
fe_status fe_prof_enable(fe_ctx *ctx, int enable);
fe_status fe_prof_reset(fe_ctx *ctx);
fe_status fe_prof_read(fe_ctx *ctx, int i, const char **name, int64_t *launches, double *ms,
                       int *count);
fe_status fe_launch_count(const fe_ctx *ctx, int64_t *launches);

/* Device bytes held by the context. */
fe_status fe_memory_bytes(const fe_ctx *ctx, int64_t *bytes);

/* fe_measure_fp64_peak: the FP64 fused multiply-add rate of the current device, measured (the
 * paper has no counterpart: it is the denominator of the FP64-pipe roofline that the FP64
 * operators are reported against).  A kernel of independent FMA chains fills every SM; it runs
 * twice untimed, then `reps` times, each timed with CUDA events on `stream`.  *tflops_best and
 * *tflops_median (may be NULL) receive 2 x FMAs / second / 1e12 of the fastest and the median
 * launch.  Allocates and frees one small result array; synchronous.  FE_ERR_ARG for reps < 1. */
fe_status fe_measure_fp64_peak(int reps, double *tflops_best, double *tflops_median, void *stream);

void fe_destroy(fe_ctx *ctx);
const char *fe_last_error(const fe_ctx *ctx);
const char *fe_status_string(fe_status s);

/* ---------------------------------------------------------------------------------------------
 * Batched instances.  Many independent 3D problems of uneven size and order 1..4 (Eq. 1-2 each,
 * on its own mesh and law) share the launches of the FP32 Jacobian action: either one persistent
 * launch whose CTAs stride over a work list of (instance, tile) items and apply each item's
 * (order, tile edge) variant, or (work policy 3) one launch per variant with one CTA per item of
 * that variant; a batched fix-up completes the cross-tile sums.  The batch owns one context per
 * instance.  Batch vectors are the instances' vectors concatenated, instance i at element
 * offset fe_batch_info(..., i, &offset, ...) (offsets are multiples of 64; the gaps are unused
 * and ignored).
 *
 * Autotuning (fe_batch_create): per order present, the tile edge (the largest the kernels are
 * compiled for, or the next smaller) is timed on the order's largest instance, then the
 * persistent grid (CTAs per SM) and the work policy (0: instance by instance, 1: interleaved,
 * 2: largest instance first, each in the persistent launch; 3: one launch per variant) on the
 * whole batch; results are cached in the JSON file opts->tune_cache (read first, then
 * rewritten), keyed by the GPU name and the batch's (order, n, tile) signature.
 * --------------------------------------------------------------------------------------------- */
typedef struct fe_batch fe_batch;

typedef struct {
    const fe_mesh *mesh;       /* 3D lattice mesh of the instance (host, copied)                */
    int order;                 /* 1..4                                                         */
    const fe_problem *prob;    /* law and load of the instance (host, copied)                  */
} fe_batch_item;

typedef struct {
    const char *tune_cache;    /* autotuner cache file (JSON) or NULL                          */
    int tune;                  /* 1: time what the cache does not hold; 0: defaults            */
    int retune;                /* 1: ignore cached entries (and rewrite them)                  */
    int policy;                /* work policy: -1 tuned (or interleaved), 0 by instance,
                                  1 interleaved, 2 largest first (persistent launch), 3 one
                                  launch per variant                                          */
    int tile[4];               /* per order 1..4: 0 tuned (or the largest), else this edge     */
} fe_batch_opts;

/* fe_batch_create: set up `count` instances (FE_ERR_UNSUPPORTED for order > 4 or a tile edge that
 * is not compiled), tune, and return the batch.  opts may be NULL (no tuning, largest tiles,
 * interleaved work).  On failure *out is NULL and fe_batch_last_error(NULL) says why. */
fe_status fe_batch_create(const fe_batch_item *items, int count, const fe_batch_opts *opts,
                          fe_batch **out);
/* Instance i's offset in the batch vectors, its DOF count and its tile edge (any may be NULL). */
fe_status fe_batch_info(const fe_batch *b, int i, int64_t *offset, int64_t *n_dofs, int *tile);
/* Batch vector length, persistent grid, threads per CTA, work policy, kernels launched so far. */
fe_status fe_batch_shape(const fe_batch *b, int64_t *total, int *grid, int *threads, int *policy,
                         int64_t *launches);
/* FP32 tangent of every instance at u (device double batch vector), Eq. 2. */
fe_status fe_batch_linearize(fe_batch *b, const double *u, void *stream);
/* y = J v for all instances in one persistent launch (policy 3: one launch per variant present)
 * plus one fix-up launch; v, y: device float batch vectors (not aliased).  FE_ERR_STATE before fe_batch_linearize. */
fe_status fe_batch_jacobian_action(fe_batch *b, const float *v, float *y, void *stream);
/* Newton on every instance in lock step from u (device double batch vector, overwritten): per
 * step the FP64 residuals and FP32 tangents per instance, one Jacobi-preconditioned FP32 CG for
 * all instances (segmented reductions, per-instance flags; with opts->use_graph 1 CG batches
 * replayed as one captured graph with a host check after each, with 2 the whole CG as one graph
 * launch whose conditional WHILE node repeats while any instance runs), per-instance FP64 line
 * search.  opts->inner_precision is ignored
 * (FP32 CG, as newton_solve's 32).  reports: `count` per-instance reports or NULL; total: the
 * whole solve (max Newton steps, summed CG iterations, batch norms) or NULL.  Returns the first
 * failing instance's status, or FE_OK. */
fe_status fe_batch_newton_solve(fe_batch *b, double *u, const fe_newton_opts *opts,
                                fe_newton_report *reports, fe_newton_report *total, void *stream);
void fe_batch_destroy(fe_batch *b);
const char *fe_batch_last_error(const fe_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* FEOD_H */
