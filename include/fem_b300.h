/*
 * fem_b300.h -- C ABI of the B300 (sm_103a) energy-based FEM hot path.
 *
 * Method (arXiv 2602.12365, Sec. 2): the total potential of Eq. 2,
 *     Psi_h(u) = sum_e sum_q psi(grad u_h^e(xi_q)) w_q det J^e(xi_q),
 * is evaluated element by element (Algorithm 1: gather, field gradient,
 * density, integrate, accumulate); the residual is its gradient and the
 * tangent acts matrix-free as the directional derivative of the residual
 * (Eq. 1 and Eq. 3).  The density is the compressible Neo-Hookean law
 *     psi(F) = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2,
 * F = I + grad u, I1 = tr F^T F (+1 in 2D plane strain), J = det F.
 * Dirichlet data follow the condensation of Sec. 6.1: prescribed components
 * keep their values in u and are masked out of r and K.
 *
 * Conventions for every call below
 *   - Vectors u, v, r, y, a are DEVICE pointers to flat [n_nodes * dim]
 *     arrays, node-major and interleaved (node i, component k at i*dim+k),
 *     of the dtype passed (FEM_F64: double, FEM_F32: float).  The caller owns
 *     them; the library never frees or retains them after the call returns.
 *   - Calls are asynchronous and ordered on the CUDA stream passed as `stream`
 *     (a cudaStream_t, NULL = legacy default stream).  They allocate nothing
 *     and never synchronise; each uses workspace owned by the mesh handle, so
 *     calls on ONE handle must be ordered on one stream (two streams in
 *     flight on the same handle race on that workspace).
 *   - Kernels never trap.  Device-side conditions (some J <= 0, a non-finite
 *     value) are OR-ed into the handle's status word; fem_sync_status()
 *     synchronises the stream and returns and clears it.
 *   - Every call returns a fem_status; FEM_OK means the work was enqueued.
 *     fem_last_error() gives a message for the last failing call of the
 *     calling thread.  No C++ exception crosses this boundary.
 */
#ifndef FEM_B300_H
#define FEM_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FEM_OK = 0,
    FEM_ERR_ARG = 1,           /* bad argument (null, size, enum)                */
    FEM_ERR_CUDA = 2,          /* a CUDA runtime call failed                     */
    FEM_ERR_INVERTED = 3,      /* some J <= 0: energy +inf, derivatives invalid   */
    FEM_ERR_NONFINITE = 4,     /* NaN/Inf met in an input or a result            */
    FEM_ERR_NOT_CONVERGED = 5, /* Newton or CG iteration cap reached             */
    FEM_ERR_NEG_CURVATURE = 6, /* p^T K p <= 0 in CG                             */
    FEM_ERR_TIMEOUT = 7,       /* a bounded device wait gave up                   */
    FEM_ERR_BADMESH = 8,       /* mesh does not fit the tiling limits            */
    FEM_ERR_NOT_SPD = 9,       /* a nodal diagonal block is not positive definite */
    FEM_ERR_LINESEARCH = 10    /* backtracking found no acceptable step          */
} fem_status;

typedef enum { FEM_TRI3 = 0, FEM_TET4 = 1, FEM_HEX8 = 2 } fem_elem_type;

/* Arithmetic of a call: FEM_F64 everywhere, or FEM_F32 element kernels
 * (reductions and energy sums stay FP64 in both). */
typedef enum { FEM_F64 = 0, FEM_F32 = 1 } fem_dtype;

/* Mesh precision: FEM_PREC_FP64 keeps FP64 geometry only; FEM_PREC_MIXED keeps
 * FP32 geometry for the FEM_F32 kernels and FP64 geometry for FEM_F64 ones. */
typedef enum { FEM_PREC_FP64 = 0, FEM_PREC_MIXED = 1 } fem_precision;

/* Flags of fem_residual, fem_hvp, fem_sparse_assemble and the atomic
 * variants; any other bit is rejected with FEM_ERR_ARG */
#define FEM_MASK_OUT 1u /* zero prescribed components of the result          */
#define FEM_MASK_IN 2u  /* zero prescribed components of v before use (HVP)  */
#define FEM_MASK_BOTH (FEM_MASK_IN | FEM_MASK_OUT)

/* Status-word bits (fem_sync_status) */
#define FEM_FLAG_INVERTED 1  /* some J <= 0 was met                   */
#define FEM_FLAG_NONFINITE 2 /* some non-finite value was met          */
#define FEM_FLAG_TIMEOUT 4   /* a bounded device wait gave up          */

typedef struct fem_mesh fem_mesh; /* opaque; owns all device-side mesh data */

/*
 * Mesh description (all HOST pointers, read during fem_mesh_create only).
 *   coords    [n_nodes * dim] double, reference positions X.
 *   conn      [n_elems * n_en] int32, node ids; positive orientation.  n_en is
 *             3 (P1 triangle, 1 point, w = 1/2), 4 (P1 tetrahedron, 1 point,
 *             w = 1/6) or 8 (Q1 hexahedron, 2x2x2 Gauss, VTK vertex order).
 *   mu, lambda [n_elems] double per-element Lame moduli, or NULL to use the
 *             scalars mu0, lambda0 for every element.
 *   dirichlet [n_nodes * dim] uint8, 1 = prescribed component; NULL = none.
 *   tile_elems  elements per tile (0 = default: 1024 for P1, 512 for Q1).
 */
typedef struct {
    int32_t elem_type; /* fem_elem_type */
    int32_t precision; /* fem_precision */
    int64_t n_nodes;
    int64_t n_elems;
    const double* coords;
    const int32_t* conn;
    const double* mu;
    const double* lambda;
    double mu0;
    double lambda0;
    const uint8_t* dirichlet;
    int32_t tile_elems;
    int32_t reserved;
} fem_mesh_desc;

/* Partition statistics (fem_mesh_get_info / fem_plan_partition). */
typedef struct {
    int64_t n_nodes, n_elems;
    int32_t dim, n_en;
    int32_t n_tiles;          /* level-1 parts, one CTA each                    */
    int32_t max_tile_nodes;   /* largest local node set                         */
    int64_t n_rounds;         /* level-2 colour classes (<= 32 disjoint elems)  */
    int32_t max_rounds;       /* most rounds in one tile                        */
    int32_t n_shared;         /* nodes touched by more than one tile            */
    int64_t n_slots;          /* partial slots (sum over shared nodes of tiles) */
    int64_t n_local_nodes;    /* sum over tiles of local nodes                  */
    int64_t n_orphans;        /* nodes touched by no element                    */
    double round_fill;        /* elements / (32 * rounds)                       */
    int64_t device_bytes;     /* device memory held by the handle               */
} fem_mesh_info;

/*
 * fem_mesh_create -- validate the mesh, partition it (tiles of spatially
 * compact elements by recursive coordinate bisection; inside each tile,
 * element colouring into rounds of at most 32 node-disjoint elements), and
 * upload connectivity, precomputed P1 shape-function gradients and volumes
 * (Alg. 1: gathered det J and grad N), coordinates (Q1), moduli and the
 * Dirichlet mask.  Synchronous on `stream`.  Errors: FEM_ERR_ARG (null or
 * inconsistent sizes, node id out of range), FEM_ERR_BADMESH (a tile needs
 * more shared memory than the device offers, or a P1 element has det J <= 0),
 * FEM_ERR_CUDA.  On error *out is NULL and nothing is leaked.
 */
fem_status fem_mesh_create(const fem_mesh_desc* desc, fem_mesh** out, void* stream);

/* Release every device buffer of the handle (synchronises the device). */
fem_status fem_mesh_destroy(fem_mesh* mesh);

/* Fill *info (host) with the handle's partition statistics. */
fem_status fem_mesh_get_info(const fem_mesh* mesh, fem_mesh_info* info);

/*
 * Host-only partition planner (no GPU needed): runs the same partitioner as
 * fem_mesh_create and returns, per element (HOST arrays, any may be NULL), its
 * tile, its global round (colour) id and its lane in the round
 * ([n_elems] each), the element's node ids in the vertex order the kernels
 * use ([n_elems * n_en]; P1 vertices may be reordered to avoid shared-memory
 * bank conflicts), plus the statistics.  Used to check the plan on a CPU.
 */
fem_status fem_plan_partition(const fem_mesh_desc* desc, int32_t* elem_tile,
                              int64_t* elem_round, int32_t* elem_lane, int32_t* elem_nodes,
                              fem_mesh_info* info);

/*
 * fem_mesh_set_moduli -- replace the per-element moduli of a mesh created
 * with per-element arrays (desc.mu / desc.lambda non-NULL), as a design loop
 * does between solves (the moduli are the design variables of the adjoint
 * gradient).  The geometry, plan and every allocation are kept; the (mu,
 * lambda) slots of the round records of each precision are rewritten.
 *   mu, lambda  HOST double[n_elems], element order of the description;
 *               mu > 0, both finite (else FEM_ERR_ARG, nothing changed).
 * FEM_ERR_ARG for a mesh created with scalar moduli.  Synchronises `stream`.
 * Derived data that depend on the moduli (the learned preconditioner's node
 * statistics, the scatter-add ablation's element arrays) are rebuilt on
 * their next use; calls already enqueued on other streams must be complete.
 */
fem_status fem_mesh_set_moduli(fem_mesh* mesh, const double* mu, const double* lambda, void* stream);

/*
 * fem_energy -- Psi_h(u) (Eq. 2) with per-element densities in the call's
 * dtype and an FP64 Neumaier-compensated, deterministic (fixed-order) sum.
 *   out_dev  DEVICE double[4]: [0] Psi_h (+inf if some J <= 0), [1] the
 *            roundoff scale S = sum_q w detJ (mu/2 I1 + mu |ln J| +
 *            lam/2 ln^2 J) used by the line search, [2] the number of
 *            quadrature points with J <= 0, [3] reserved (0).
 */
fem_status fem_energy(fem_mesh* mesh, int dtype, const void* u, double* out_dev, void* stream);

/*
 * fem_energy_static -- fem_energy's result, bit for bit (same kernel, same
 * summation order), from a call that allocates nothing and uses none of the
 * handle's reduction workspace.  The paper has no counterpart: this is a
 * deployment variant for callers that may not allocate device memory after
 * start-up.  The energy reduction's arrival counter and per-tile partials live
 * in one file-scope device array of fixed size (a 256-byte line for the
 * counter, then FEM_STATIC_MAX_TILES x 4 doubles: 512 KiB + 256 B), one copy
 * per device and process.
 *   - A mesh with more than FEM_STATIC_MAX_TILES tiles (fem_mesh_info.n_tiles)
 *     is rejected with FEM_ERR_ARG and a message naming both numbers.  At the
 *     default tile sizes the limit is 16.7M P1 or 8.4M Q1 elements.  Every
 *     rejected call (tile limit, null or bad argument, FEM_F32 on a mesh
 *     without FP32 records) returns before it touches the shared array:
 *     nothing is enqueued.
 *   - Each call enqueues, on `stream`, a 4-byte memset that zeroes the counter,
 *     then the kernel; the partials need no clearing (each tile writes its own
 *     before the last CTA reads them).
 *   - Overlapping calls race: every handle on the device shares the one
 *     array, so two calls in flight at once (two streams, two threads, two
 *     handles) give wrong sums.  Order them on one stream or by events.
 *   - The first call in each CUDA context does one-time host-side setup
 *     (looks up the array's device address with cudaGetSymbolAddress, with
 *     that context's device current, sets the kernel's shared-memory limit,
 *     queries its occupancy); make that first call outside any stream
 *     capture.  The address is cached per context, so after a device reset
 *     the next call looks it up again.
 * Arguments, output and status bits as for fem_energy.
 */
#define FEM_STATIC_MAX_TILES 16384
fem_status fem_energy_static(fem_mesh* mesh, int dtype, const void* u, double* out_dev, void* stream);

/*
 * fem_residual -- r = grad Psi_h(u) (Eq. 1): per element P = dpsi/dF =
 * mu (F - F^-T) + lambda ln J F^-T, r_a += w detJ P grad N_a, scattered
 * deterministically.  flags & FEM_MASK_OUT zeroes prescribed components.
 * u and r must not alias.
 */
fem_status fem_residual(fem_mesh* mesh, int dtype, const void* u, void* r, unsigned flags,
                        void* stream);

/*
 * fem_hvp -- y = Mo K(u) Mi v, the matrix-free tangent action (Eq. 3):
 * dF = grad v, dP = mu dF + (mu - lambda ln J) F^-T dF^T F^-T +
 * lambda tr(F^-1 dF) F^-T, y_a += w detJ dP grad N_a.  Mi / Mo are the
 * Dirichlet masks selected by FEM_MASK_IN / FEM_MASK_OUT.
 *   vKv_dev  DEVICE double* or NULL: receives (Mi v)^T K (Mi v) summed
 *            element by element in FP64 in a fixed order.
 * y must alias neither u nor v.
 */
fem_status fem_hvp(fem_mesh* mesh, int dtype, const void* u, const void* v, void* y,
                   unsigned flags, double* vKv_dev, void* stream);

/*
 * fem_block_diag -- nodal diagonal blocks D_i = K_ii(u) (dim x dim, row
 * major, [n_nodes * dim * dim] of the call's dtype); rows/columns of
 * prescribed components are replaced by the identity.  Per element and node
 * a: K_aa = w detJ [mu |g0|^2 I + (mu - lambda ln J + lambda) g g^T] with
 * g0 = grad N_a and g = F^-T grad N_a.
 */
fem_status fem_block_diag(fem_mesh* mesh, int dtype, const void* u, void* D, void* stream);

/*
 * fem_param_vjp -- per-element sensitivities of a^T r(u) to the moduli:
 * g_mu[e] = a^T dr_e/dmu_e, g_lam[e] = a^T dr_e/dlambda_e (dP/dmu = F - F^-T,
 * dP/dlambda = ln J F^-T).  g_mu, g_lam: DEVICE double[n_elems] in the
 * caller's element order (either may be NULL).
 */
fem_status fem_param_vjp(fem_mesh* mesh, int dtype, const void* u, const void* a,
                         double* g_mu, double* g_lam, void* stream);

/* ------------------------------------------------------------------------
 * Matrix-free Newton-CG load stepping (Sec. 6.3.1 and 6.6 solve the
 * nonlinear problems by Newton-Krylov iterations on the residual and its
 * directional derivative; the paper fixes no further detail, so the
 * algorithm below is one fixed choice, shared step for step with the CPU
 * oracle):
 *   1. du_c = (s - s_prev) ubar on prescribed DOFs;
 *   2. predictor: t = M K(u) (I - M) du_c, r0 = ||t||; PCG on
 *      M K M du_f = -t to predictor_rtol r0; u += du_c + du_f; prescribed
 *      entries set to s ubar;
 *   3. Newton: r = M grad Psi(u), stop when ||r|| <= newton_rtol r0 (r0 =
 *      ||r|| when t = 0); PCG on M K M d = -r from 0 to eta ||r||,
 *      eta = min(eta_max, sqrt(||r|| / r0)), and on p^T K p <= 0 the current
 *      iterate (d = P r at the first iteration); backtracking Armijo line
 *      search on Psi (alpha = 1, 1/2, ... ls_max halvings; accept when
 *      Psi(u + a d) <= Psi(u) + armijo_c a r^T d, or when |dPsi| <= 16 eps S
 *      and the residual norm decreases, S the roundoff scale of fem_energy);
 *   4. an inverted state after the predictor, a non-SPD diagonal block, a
 *      failed line search or newton_max iterations restore u and bisect the
 *      increment, at most max_bisect levels deep.
 * M is the Dirichlet mask; the preconditioner P is block Jacobi (each nodal
 * diagonal block of fem_block_diag inverted through its Cholesky factor).
 * ------------------------------------------------------------------------ */
#define FEM_PC_BLOCK_JACOBI 0
#define FEM_PC_LEARNED 1 /* the learned block preconditioner (fem_lp_*); FP32 CG, 3D */

typedef struct {
    int32_t cg_dtype;      /* FEM_F64: the PCG, its HVPs and preconditioner in
                              FP64; FEM_F32: those in FP32 on an FP32 shadow of
                              u (mesh must be FEM_PREC_MIXED), dot products and
                              norms still FP64.  u, the Newton residual and the
                              line-search energies are FP64 in both modes.     */
    int32_t precond;       /* FEM_PC_BLOCK_JACOBI                            */
    double newton_rtol;    /* 1e-8                                           */
    int32_t newton_max;    /* 50                                             */
    int32_t ls_max;        /* 20                                             */
    double eta_max;        /* 0.1                                            */
    int64_t cg_max;        /* 0 = 10 * n_dofs                                */
    double predictor_rtol; /* 1e-2                                           */
    double armijo_c;       /* 1e-4                                           */
    int32_t max_bisect;    /* 5                                              */
    int32_t cg_batch;      /* CG iterations enqueued between host checks of
                              the device-side stop flag (0 = 8); iterations
                              past the stop are skipped on the device, so the
                              result does not depend on it                   */
    const void* learned;   /* fem_lp* when precond == FEM_PC_LEARNED, else NULL */
} fem_newton_opts;

typedef struct {
    int32_t status;       /* fem_status of the step                          */
    int32_t newton_iters; /* Newton iterations over all increments           */
    int64_t cg_iters;     /* HVPs inside PCG (predictors included)           */
    int32_t bisections;
    int32_t ls_halvings;
    double r0_norm;       /* reference norm of the last increment            */
    double r_norm;        /* final residual norm                             */
} fem_newton_stats;

/* Fill *opts with the defaults listed above. */
fem_status fem_newton_default_opts(fem_newton_opts* opts);

/*
 * fem_newton_step -- advance u from load factor s_prev to s (s >= s_prev).
 *   u     DEVICE double[n_nodes * dim]: on entry the state at s_prev, its
 *         prescribed entries equal to s_prev * ubar; on FEM_OK the converged
 *         state at s.  On failure u holds the last attempt of the deepest
 *         bisection (as the oracle leaves it).
 *   ubar  DEVICE double[n_nodes * dim]: prescribed displacement at s = 1
 *         (read on prescribed components only).
 *   opts  NULL for the defaults.  stats: HOST, always filled.
 * Unlike the element calls this one synchronises `stream` (the host decides
 * on convergence and line-search acceptance), and its first call on a handle
 * allocates the solver workspace (about 12 vectors and two block arrays),
 * kept until fem_mesh_destroy; a first bisection adds one save vector per
 * level.  The handle's status word is left as it was on entry.
 * Returns FEM_OK, FEM_ERR_INVERTED, FEM_ERR_NOT_SPD, FEM_ERR_NOT_CONVERGED or
 * FEM_ERR_LINESEARCH (after all bisections), FEM_ERR_ARG or FEM_ERR_CUDA.
 */
fem_status fem_newton_step(fem_mesh* mesh, double* u, const double* ubar, double s_prev, double s,
                           const fem_newton_opts* opts, fem_newton_stats* stats, void* stream);

/*
 * fem_tangent_solve -- the linear solve inside a Newton step, exposed for
 * adjoint (design-sensitivity) solves: block-Jacobi PCG on
 * M K(u) M x = M b from x = 0 until ||M b - M K M x|| <= rtol ||M b||, with
 * the same kernels, precisions and FP64 dot products as fem_newton_step.
 *   u  DEVICE double[n_nodes * dim], the linearisation state.
 *   b  DEVICE double[n_nodes * dim]; prescribed components are ignored.
 *   x  DEVICE double[n_nodes * dim] (out); prescribed components are 0.
 *   cg_max 0 = 10 * n_dofs; *iters (HOST, may be NULL) receives the HVP
 *   count.  Synchronises `stream`; allocates the solver workspace on first
 *   use like fem_newton_step.
 * Returns FEM_OK, FEM_ERR_NEG_CURVATURE (x = last iterate),
 * FEM_ERR_NOT_CONVERGED, FEM_ERR_NOT_SPD, FEM_ERR_ARG or FEM_ERR_CUDA.
 */
fem_status fem_tangent_solve(fem_mesh* mesh, int cg_dtype, const double* u, const double* b, double* x,
                             double rtol, int64_t cg_max, int64_t* iters, void* stream);

/*
 * fem_compliance_gradient -- the adjoint design gradient of the compliance
 * with respect to per-element shear moduli, the whole computation in the
 * library (the paper's design-sensitivity use of the residual's derivatives,
 * Sec. 2.1 with the inverse-design examples of Sec. 6).  Under pure
 * displacement loading the compliance is the work of the prescribed
 * displacements, c = u_c^T r_c(u*), r = grad Psi_h at the converged state u*;
 * with lambda_e = ratio * mu_e tied,
 *     dc/dmu_e = a^T (dr_e/dmu_e + ratio dr_e/dlambda_e),
 *     a = u_c on prescribed DOFs, -lam on free ones,  K_ff lam = K_fc u_c.
 * Steps (on `stream`): u_c from u and the mask; the unmasked FP64 residual
 * and c = u_c . r (FP64, fixed order); K_fc u_c as one HVP with u_c as the
 * direction (free rows); the adjoint PCG of fem_tangent_solve in cg_dtype
 * (FP64 dot products); a; the per-element pass of fem_param_vjp in
 * vjp_dtype; g_mu + ratio g_lam.
 *   u      DEVICE double[n_nodes * dim], the converged state (the checkpoint of
 *          the last load step: the law is hyperelastic, so the gradient
 *          depends on the final state only).
 *   dmu    DEVICE double[n_elems] (out), element order of the mesh description.
 *   c_dev  DEVICE double[1] (out): the compliance.
 *   iters  HOST (may be NULL): adjoint PCG iterations.
 * Uses the Newton-CG workspace (allocated on first use, as fem_newton_step,
 * plus one per-element array).  Synchronises `stream` (the PCG's stop test).
 * Returns FEM_OK, FEM_ERR_ARG, FEM_ERR_NOT_SPD, FEM_ERR_NEG_CURVATURE,
 * FEM_ERR_NOT_CONVERGED or FEM_ERR_CUDA.
 */
fem_status fem_compliance_gradient(fem_mesh* mesh, const double* u, double ratio, double rtol, int cg_dtype,
                                   int vjp_dtype, double* dmu, double* c_dev, int64_t* iters, void* stream);

/* ------------------------------------------------------------------------
 * Learned block preconditioner (3D meshes created FEM_PREC_MIXED; the PCG of
 * fem_newton_step with cg_dtype FEM_F32 and precond FEM_PC_LEARNED).
 *
 * The paper has no preconditioner of this kind; it is the learned part of
 * this implementation.  A per-node MLP 36 -> 64 -> 64 -> 6 (SiLU hidden
 * layers; BF16 weights and activations, FP32 accumulation, tensor cores)
 * corrects block Jacobi: with D_i the nodal diagonal block, s_i = tr(D_i)/3,
 * D_i / s_i = C C^T and F = C^-T, the preconditioner block is
 *     M_i = F A A^T F^T / s_i,
 * A lower-triangular from the 6 outputs (softplus(o) + 1e-4 on its
 * diagonal).  M_i is SPD for any weights and is block Jacobi D_i^-1 for
 * A = I, the network fem_lp_create starts from.  Prescribed components get
 * identity rows and columns.  Features per node (36): D_i / s_i (9); the mean
 * of the neighbours' D_j / s_i (9); their mean absolute deviation / s_i (9)
 * (these 27 compressed as sign(x) ln(1 + |x|));
 * ln of the mean incident mu, ln(mean lambda / mean mu), valence / 24 (3);
 * the Dirichlet bits (3); ln(D_i,cc / s_i) (3).  Neighbours share an element.
 * Training minimises ||H M r - r||^2 / ||r||^2 with H = M K(u) M (masked)
 * over states and residuals supplied by the caller (one Adam step per call;
 * the gradient needs a second HVP).  The first call on a mesh builds its node
 * graph (host) and allocates a workspace kept until fem_mesh_destroy.
 * Parameters (FEM_LP_PARAMS floats): W1[64][36], b1[64], W2[64][64], b2[64],
 * W3[6][64], b3[6], row-major W[out][in].
 * ------------------------------------------------------------------------ */
#define FEM_LP_FEATURES 36
#define FEM_LP_PARAMS 6918
typedef struct fem_lp fem_lp;

/* New network (W1, W2 ~ N(0, 1/fan_in) from a SplitMix64 stream of `seed`,
 * W3 = 0, biases giving A = I: block Jacobi). */
fem_status fem_lp_create(uint64_t seed, fem_lp** out);
fem_status fem_lp_destroy(fem_lp* lp);
/* Training loss: FEM_LP_LOSS_RESIDUAL (the default) ||H M r - r||^2 / ||r||^2,
 * whose gradient in z = M r is 2 H (H z - r) / ||r||^2 (a second HVP); or
 * FEM_LP_LOSS_ENERGY, the same residual measured in the H^-1 norm,
 * (r - H z)^T H^-1 (r - H z) / ||r||^2, reported shifted by the constant
 * r^T H^-1 r / ||r||^2 (1 + (z^T H z - 2 r^T z) / ||r||^2), gradient
 * 2 (H z - r) / ||r||^2.  For r with identity covariance the energy loss is
 * minimised over block-diagonal M exactly by block Jacobi. */
#define FEM_LP_LOSS_RESIDUAL 0
#define FEM_LP_LOSS_ENERGY 1
fem_status fem_lp_set_loss(fem_lp* lp, int kind);
/* Adam steps scale the gradient to at most this 2-norm (default 1; 0 = no
 * clipping). */
fem_status fem_lp_set_clip(fem_lp* lp, float max_grad_norm);
/* HOST float[FEM_LP_PARAMS] out / in (set also resets the Adam state). */
fem_status fem_lp_get_params(const fem_lp* lp, float* params);
fem_status fem_lp_set_params(fem_lp* lp, const float* params);
/* Features at the FP32 state u: X DEVICE bf16 [n_nodes * 48] (36 used, the
 * rest zero). */
fem_status fem_lp_features(fem_mesh* mesh, const float* u, void* X, void* stream);
/* Preconditioner blocks at the FP32 state u: Minv DEVICE float [n_nodes * 9]. */
fem_status fem_lp_blocks(const fem_lp* lp, fem_mesh* mesh, const float* u, float* Minv, void* stream);
/* Loss at (u, r) (DEVICE float [n_nodes * 3] each, r masked) and its
 * gradient in the parameters: grad HOST float[FEM_LP_PARAMS]; *loss HOST
 * (may be NULL).  Synchronises `stream`; changes nothing. */
fem_status fem_lp_gradient(fem_lp* lp, fem_mesh* mesh, const float* u, const float* r, float* grad,
                           double* loss, void* stream);
/* One Adam step (learning rate lr) on the loss at (u, r), both DEVICE float
 * [n_nodes * 3], r masked; *loss (HOST, may be NULL: no synchronisation)
 * receives the loss before the step. */
fem_status fem_lp_train_step(fem_lp* lp, fem_mesh* mesh, const float* u, const float* r, float lr,
                             double* loss, void* stream);

/*
 * fem_mesh_set_ncm -- the neural constitutive model (Sec. "Neural
 * Constitutive Modeling"): from this call on, the element operators of the
 * mesh (fem_energy, fem_energy_static, fem_residual, fem_hvp,
 * fem_block_diag, and through them fem_newton_step, fem_tangent_solve and
 * fem_sparse_assemble) evaluate
 *   psi = [NN(I1, J) - NN(3, 1)] + psi_NH(mu_e, lambda_e),
 * NN a 2 -> H -> H -> 1 MLP with softplus activations of the invariants
 * I1 = tr(F^T F) (+1 in plane strain) and J = det F, the same for every
 * element; the Neo-Hookean law with the element's moduli is the convex base.
 *   hidden  H = 8, 16 or 32; 0 removes the network (Neo-Hookean again).
 *   params  HOST double [H*H + 5H + 1]: W1 [H][2], b1 [H], W2 [H][H] (row m
 *           feeds unit m of the second layer), b2 [H], w3 [H], b3; copied.
 * Each operator call first evaluates the network at every element's (I1, J)
 * (an invariants pass of the element kernel and a network kernel, in the
 * call's precision); the PCG of the Newton solver evaluates it once per
 * solve.  The network does not depend on the moduli, so fem_param_vjp is
 * unchanged.  The arrays (8 + 2 values per element and precision) are
 * allocated here, so the operator calls allocate nothing.  P1 meshes only
 * (FEM_ERR_ARG for hexahedra); the atomic-scatter ablation refuses a mesh
 * with a network.  Synchronises the device.
 */
fem_status fem_mesh_set_ncm(fem_mesh* mesh, int hidden, const double* params);

/*
 * Sparse K by colouring -- the paper's second route to the tangent (Sec. 2.2,
 * Algorithm 2; App. A for the colouring, App. B for the pattern).
 *
 * Pattern: CSR over DOFs (dof = node * dim + component).  Entry (i, j) is
 * present when the nodes of DOFs i and j lie in a common element (a node with
 * itself included); the columns of every row ascend.  Colours: the greedy
 * distance-2 colouring of the columns -- columns in ascending order, each
 * takes the smallest colour not held by an earlier column that shares a row
 * with it -- so no two columns of one colour share a row.  Both are built on
 * the host by the first fem_sparse_* call on a mesh (time and host memory
 * O(nnz)) and kept, with device copies, until fem_mesh_destroy.
 *
 * fem_sparse_info: *nnz (entries) and *n_colors; either may be NULL.
 * fem_sparse_pattern: HOST copies; row_ptr int64 [n_dofs + 1], col_idx int32
 *   [nnz], colors int32 [n_dofs]; each may be NULL.
 * fem_sparse_assemble: Algorithm 2 on the device at the state u (DEVICE,
 *   dtype): for each colour c, the seed e_c (1 on the DOFs of colour c) and
 *   one HVP  Mo K(u) Mi e_c  (flags as fem_hvp), kept as column c of the
 *   compressed Jacobian [n_colors][n_dofs] (mesh workspace, allocated on first
 *   use per dtype); then values[k] = Jcomp[colour(col_idx[k])][row(k)].
 *   values: DEVICE [nnz] of dtype, in the pattern's order.  Status bits of
 *   the HVPs accumulate as for fem_hvp.
 * fem_sparse_spmv: y = K x with the mesh's pattern and `values`; x, y DEVICE
 *   [n_dofs] of dtype, not aliased.  Per row a fixed summation order.
 * Errors: FEM_ERR_ARG (null or bad arguments; FEM_F32 on an FP64 mesh),
 * FEM_ERR_BADMESH (more than 2^31 - 1 DOFs), FEM_ERR_CUDA.
 */
fem_status fem_sparse_info(fem_mesh* mesh, int64_t* nnz, int32_t* n_colors);
/* The same pattern and colouring from a mesh description alone, on the host
 * (no device, no handle): sizes in *nnz and *n_colors, arrays as for
 * fem_sparse_pattern; every output may be NULL (call once with NULL arrays
 * to size them). */
fem_status fem_sparse_pattern_desc(const fem_mesh_desc* desc, int64_t* nnz, int32_t* n_colors,
                                   int64_t* row_ptr, int32_t* col_idx, int32_t* colors);
fem_status fem_sparse_pattern(fem_mesh* mesh, int64_t* row_ptr, int32_t* col_idx, int32_t* colors);
fem_status fem_sparse_assemble(fem_mesh* mesh, int dtype, const void* u, unsigned flags, void* values,
                               void* stream);
fem_status fem_sparse_spmv(fem_mesh* mesh, int dtype, const void* values, const void* x, void* y,
                           void* stream);

/*
 * Ablation, not on the method's path: fem_residual / fem_hvp computed the
 * traditional way of Sec. 5's comparison with scatter-add assembly -- one
 * thread per element in mesh order, the element's nodal forces added into the
 * output with floating-point atomicAdd (the output is zeroed first on
 * `stream`).  Same constitutive code, arguments, flags and status bits as
 * fem_residual / fem_hvp; P1 elements only (FEM_ERR_ARG for hexahedra).
 * Results agree with the tiled kernels to rounding, but the order of the
 * atomic additions, and so the last bits, can change from run to run.  The
 * first call per precision builds per-element arrays in mesh order on the
 * host (connectivity, grad N, w det J, moduli) and keeps them on the device.
 */
fem_status fem_residual_atomic(fem_mesh* mesh, int dtype, const void* u, void* r, unsigned flags,
                               void* stream);
fem_status fem_hvp_atomic(fem_mesh* mesh, int dtype, const void* u, const void* v, void* y, unsigned flags,
                          void* stream);
/* The same ablation for the assembled K (the paper's "traditional scatter-add
 * assembly"): each element's stiffness, column by column from the same
 * tangent, added with atomicAdd into the CSR values of fem_sparse_pattern
 * (zeroed first).  Arguments and flags as fem_sparse_assemble; the values
 * agree with it to rounding, but not bit for bit from run to run. */
fem_status fem_sparse_assemble_atomic(fem_mesh* mesh, int dtype, const void* u, unsigned flags, void* values,
                                      void* stream);

/*
 * fem_fp32_fma_rate -- a measurement helper with no counterpart in the paper:
 * enqueues a kernel of `blocks` blocks of 256 threads, each thread running 8
 * independent FP32 FMA chains of `iters` steps, so that the caller can time
 * the GPU's FP32 FMA throughput (the roofline denominator of the ALU-bound
 * Q1 element kernels) with events on `stream`.
 *   out_dev  DEVICE float[blocks * 256], written (one value per thread, so
 *            that the chains are not removed); caller-owned.
 *   flops    HOST (may be NULL): the kernel's FP32 flops, FMA counted as 2.
 * FEM_ERR_ARG for non-positive sizes or a null out_dev.
 */
fem_status fem_fp32_fma_rate(int blocks, int iters, float* out_dev, double* flops, void* stream);

/* Synchronise `stream`, return the handle's status word (FEM_FLAG_*) in
 * *flags and clear it. */
fem_status fem_sync_status(fem_mesh* mesh, void* stream, int32_t* flags);

/* Message of the calling thread's last failing call ("" if none). */
const char* fem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FEM_B300_H */
