/*
 * shell.h -- C ABI of the GB300 (sm_103a) corotational hinge-based thin plate / shell library.
 *
 * The library advances triangle-mesh thin plates and shells in time under the six corotational bending
 * models of "Corotational Hinge-based Thin Plates/Shells" (Liang, arXiv 2502.10872): edge-based hinge
 * (EP/ES, Section 4.3), FVM hinge (FP/FS, Section 4.4) and smoothed hinge (SP/SS, Section 4.5), each as a
 * plate (rest-flat) and a shell (rest-curved) variant. One step is the linearised backward-Euler step of
 * the elastodynamic incremental potential (Section 5, Eq. 62-63) with the constant bending Hessian the
 * models share (Eq. 21, Eq. 41, Eq. 53):
 *
 *     (M + dt^2 K) v' = M v + dt (f(x) + f_ext),   x' = x + dt v',
 *
 * f = -grad(Psi_m + Psi_b) evaluated exactly at x (bending: Eq. 22, Eq. 25-26, Eq. 44-45, Eq. 56-57),
 * K = K_b + K_m constant and assembled once on the device at shell_create, M the lumped mass. The membrane
 * is the corotated linear constant-strain triangle (the paper adopts a constant-strain triangle membrane,
 * Section 3); its constant matrix block is 2 (mu + lam) A t grad(phi_a).grad(phi_b) per triangle, with
 * mu = E / (2 (1 + nu)) and lam = E nu / (1 - nu^2). The linear system is solved by preconditioned conjugate
 * gradients on the GPU (Jacobi, or a smoothed-aggregation multigrid cycle; the paper does not name its linear
 * solver), either in FP64 or in FP32 with FP64 iterative refinement of the residual.
 *
 * Every step of the path runs in CUDA kernels: rest-state precompute (FP64), matrix assembly (FP64),
 * per-stencil forces, right-hand side, PCG, state update. There is no CPU fallback: without a usable
 * CUDA device every entry point that needs one returns SHELL_ERR_CUDA or SHELL_ERR_NO_DEVICE.
 *
 * Conventions for every entry point:
 *   - Return value: SHELL_OK (0) on success, a negative SHELL_ERR_* code otherwise; shell_strerror()
 *     gives a message. On failure no output is written unless stated otherwise.
 *   - Host arrays passed in are copied; the caller keeps ownership and may free them after the call.
 *   - Output host buffers are allocated by the caller with the stated size.
 *   - Calls on one handle (or batch) must be externally serialised. Device work runs on the stream given
 *     in shell_options.cuda_stream (NULL = the legacy default stream); calls that return host data
 *     synchronise that stream.
 *   - Arrays of 3-vectors are row-major [n][3] (x, y, z interleaved) on the host.
 */
#ifndef SHELL_H_
#define SHELL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------------------------ codes */
#define SHELL_OK 0
#define SHELL_ERR_INVALID_ARG -1      /* NULL pointer, size out of range, bad enum, non-planar plate rest */
#define SHELL_ERR_NON_MANIFOLD -2     /* an edge is shared by more than two triangles */
#define SHELL_ERR_BAD_ORIENTATION -3  /* neighbouring triangles are not consistently oriented */
#define SHELL_ERR_DEGENERATE -4       /* a rest triangle or stencil height is (numerically) zero */
#define SHELL_ERR_SINGULAR_OPERATOR -5 /* L_p C_p of a smoothed hinge stencil is singular (Section 4.5) */
#define SHELL_ERR_OOM -6              /* device allocation failed */
#define SHELL_ERR_BUDGET -7           /* a batch's memory budget cannot hold the instance */
#define SHELL_ERR_NOT_CONVERGED -8    /* PCG / refinement hit its iteration cap; the step is not committed */
#define SHELL_ERR_NONFINITE -9        /* NaN or Inf met in the step; the step is not committed */
#define SHELL_ERR_TIMEOUT -10         /* a bounded device-side wait gave up; the launch was abandoned */
#define SHELL_ERR_CUDA -11            /* a CUDA runtime call failed */
#define SHELL_ERR_NO_DEVICE -12       /* no CUDA device of compute capability 10.3 is available */
#define SHELL_ERR_BUSY -13            /* the handle belongs to a batch and must be stepped through it */
#define SHELL_ERR_STATIC_LIMIT -14    /* the request needs more than shell_step_noalloc's static scratch */

/* ------------------------------------------------------------------------------------------ enums */
/* Bending model (Section 4.2): E/F/S = edge-based / FVM / smoothed hinge, P/S = plate / shell. */
typedef enum shell_model {
  SHELL_EP = 0,
  SHELL_ES = 1,
  SHELL_FP = 2,
  SHELL_FS = 3,
  SHELL_SP = 4,
  SHELL_SS = 5
} shell_model;

/* Arithmetic of the per-step force and linear solve. SHELL_FP64: everything in FP64.
 * SHELL_FP32_REFINE: forces and PCG in FP32, the right-hand side, the solution and the residual of an
 * outer iterative refinement in FP64 (positions and velocities are always held in FP64). */
typedef enum shell_precision { SHELL_FP64 = 0, SHELL_FP32_REFINE = 1 } shell_precision;

/* ------------------------------------------------------------------------------------------ inputs */
typedef struct shell_mesh {
  int32_t n_verts;          /* V >= 3 */
  int32_t n_tris;           /* T >= 1 */
  const int32_t *tris;      /* [T][3] vertex indices, consistently oriented, manifold */
  const double *rest_xyz;   /* [V][3] rest shape X (planar within 1e-9 * size for plate models) */
  const double *init_xyz;   /* [V][3] initial positions x, or NULL for x = X */
  const double *init_vel;   /* [V][3] initial velocities, or NULL for zero */
} shell_mesh;

typedef struct shell_material {
  double E;          /* Young's modulus > 0 */
  double nu;         /* Poisson's ratio in [0, 0.5) */
  double thickness;  /* t > 0 (bending rigidity k_b = E t^3 / (12 (1 - nu^2)), Section 4.3) */
  double density;    /* rho > 0 (lumped mass m_i = sum rho t A / 3 over incident triangles) */
} shell_material;

/* Boundary conditions (Section 4.3 "Boundary conditions", Eq. 30-31 and Eq. 58-61).
 * Boundary edges not listed as clamped are free (no edge stencil; the virtual node of a triangle
 * stencil is folded with w_L' = w_M + w_N - w_L). A clamped edge folds w_L' = w_L, measures transverse
 * displacement along the fixed rest normal of its stencil, and pins both end vertices. Pinned vertices
 * keep their position (zero velocity). Simply supported = free edges + pinned vertices.
 * Per-component constraints (fixed_dofs; the symmetry conditions of the Section 6.1 hemisphere): a fixed
 * component of a vertex keeps its position, the others move. All three bits set pins the vertex. The
 * assembled matrix is scalar (one entry per vertex pair, the same for x, y and z), so a vertex with fixed
 * and free components keeps its matrix row; the solves project instead (every product, right-hand side,
 * residual and preconditioned vector is zeroed at the fixed components: conjugate gradients on the free
 * components of the same system). An instance with such vertices runs in the step kernel's Newton-capable
 * variant, which carries the projection; shell_apply_matrix applies the assembled matrix without it. */
typedef struct shell_bc {
  const uint8_t *pinned;          /* [V] nonzero = fixed, or NULL */
  int32_t n_clamped;              /* number of clamped boundary edges */
  const int32_t *clamped_edges;   /* [n_clamped][2] vertex pairs of boundary edges */
  double gravity[3];              /* body acceleration; f_ext += m_i * gravity */
  int32_t n_loads;                /* point loads */
  const int32_t *load_vtx;        /* [n_loads] */
  const double *load_f;           /* [n_loads][3] newtons */
  const uint8_t *fixed_dofs;      /* [V] bit mask of fixed components (1 = x, 2 = y, 4 = z; 7 pins the
                                   * vertex), or NULL; bits above 4 are invalid (SHELL_ERR_INVALID_ARG) */
} shell_bc;

/* Device memory hooks: if alloc is NULL the library uses cudaMallocAsync / cudaFreeAsync on the handle's
 * stream. Hooks must return 256-byte aligned device memory (or NULL on failure). */
typedef void *(*shell_alloc_fn)(size_t bytes, void *cuda_stream, void *user);
typedef void (*shell_free_fn)(void *ptr, size_t bytes, void *cuda_stream, void *user);

/* Preconditioner of the PCG. AUTO: smoothed-aggregation multigrid when the step matrix is stiff
 * (median dt^2 K_ii / m_i > 30 and V >= 256), else Jacobi. AMG: the multigrid hierarchy is built once at
 * shell_create from the assembled matrix (it never changes) and applied as one V(1,1) cycle per
 * iteration. */
typedef enum shell_preconditioner { SHELL_PRECOND_AUTO = 0, SHELL_PRECOND_JACOBI = 1, SHELL_PRECOND_AMG = 2 }
    shell_preconditioner;

typedef struct shell_options {
  double dt;               /* time step > 0 */
  int32_t precision;       /* shell_precision */
  double pcg_rtol;         /* stop when ||r|| <= pcg_rtol ||b|| (FP64); inner relative tolerance (FP32; a
                            * round also stops once its residual is 0.7 refine_rtol ||b||) */
  double refine_rtol;      /* FP32_REFINE: stop when the FP64 residual ||b - A v|| <= refine_rtol ||b|| */
  int32_t pcg_max_it;      /* iteration cap per solve (per inner solve in FP32_REFINE) */
  int32_t refine_max;      /* FP32_REFINE: cap on refinement rounds */
  void *cuda_stream;       /* cudaStream_t, or NULL */
  shell_alloc_fn alloc;    /* optional device allocator */
  shell_free_fn free;
  void *alloc_user;
  int32_t preconditioner;  /* shell_preconditioner */
  int32_t no_staging;      /* 0 (default): FP32 products stage each 256-row block's gathered vector entries in
                            * shared memory when they fit; 1: gather from global memory. Results are bitwise
                            * identical either way (same values, same order of operations); for measurement. */
} shell_options;

/* Solver options of the step (Section 5; the paper names no linear solver or tolerance, so these are this
 * library's). Fills defaults: dt 1e-2, FP64, pcg_rtol 0 and refine_rtol 0 (= the precision's default: 1e-13 for the
 * FP64 PCG, 1e-6 for the inner FP32 PCG, 3e-7 for the refinement: at that target and below the FP32 force
 * rounding, not the solve, bounds the error against FP64), pcg_max_it 20000, refine_max 20,
 * preconditioner AUTO. */
void shell_default_options(shell_options *opt);

/* Statistics of the last shell_step / shell_batch_step call for one instance (solver counters of the step of
 * Section 5; no counterpart in the paper). */
typedef struct shell_step_stats {
  int32_t steps_done;          /* steps committed by this call */
  int32_t pcg_iterations;      /* PCG iterations of the last committed step (summed over rounds) */
  int32_t refine_rounds;       /* refinement rounds of the last committed step (0 in FP64) */
  int32_t status;              /* SHELL_OK or the error that stopped this instance */
  int64_t total_pcg_iterations;/* summed over the call's steps */
  double rel_residual;         /* ||b - A v'|| / ||b|| of the last committed step (recursive in FP64) */
  int64_t total_refine_rounds; /* summed over the call's steps */
  double last_solve_us;        /* device time of the last step's solve of this instance (rhs to commit) */
  int32_t team_ctas;           /* CTAs of the persistent launch that worked on this instance */
  int32_t nl_iterations;       /* exact backward Euler (shell_set_nonlinear): chord iterations (solves) of
                                * the last committed step; 0 for the linearised step */
} shell_step_stats;

/* ------------------------------------------------------------------------------------------ handle */
typedef struct shell_handle shell_handle;

/* Build one simulation (Section 4 rest-state precompute and the constant matrix, assembled once).
 * Validates the mesh (manifold, consistent orientation, non-degenerate), builds the stencils on the host,
 * uploads them and runs the FP64 precompute and assembly kernels. *out receives an owning handle.
 * Errors: INVALID_ARG, NON_MANIFOLD, BAD_ORIENTATION, DEGENERATE, SINGULAR_OPERATOR, OOM, CUDA, NO_DEVICE. */
int shell_create(const shell_mesh *mesh, const shell_material *mat, int32_t model, const shell_bc *bc,
                 const shell_options *opt, shell_handle **out);

/* Advance n_steps >= 0 linearised backward-Euler steps (Section 5, Eq. 62-63). Each step: per-stencil forces at
 * the current x, right-hand side, PCG (and refinement), v = v', x += dt v'. A step that fails (NOT_CONVERGED,
 * NONFINITE, TIMEOUT) is not committed and ends the call; the steps before it are committed. stats may be NULL
 * (else caller-owned). Synchronises the handle's stream. Errors: INVALID_ARG, BUSY (handle in a batch),
 * NOT_CONVERGED, NONFINITE, TIMEOUT, OOM, CUDA. */
int shell_step(shell_handle *h, int32_t n_steps, shell_step_stats *stats);

/* The same steps as shell_step, for callers that cannot allocate device memory once their handles exist:
 * for example a real-time loop whose device allocator is frozen after set-up, or a host framework that owns
 * the whole device-memory budget and forbids allocation inside its step callback. shell_step's first call
 * (and its first call after a batch retires the handle) allocates scheduling tables; this entry point never
 * allocates: its launch scratch (team schedule, barrier words, abort flag, status read-back) is a
 * file-scope static __device__ array of about 17 KB that every GPU loading the library holds until exit.
 * The paper has no counterpart to this; it is a deployment variant of shell_step.
 *   - Same arguments and results as shell_step (bit-identical states). It returns after its steps have
 *     finished on the GPU (it synchronises the handle's stream to read the status back).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current; make that first call before any stream capture.
 *   - The array is shared by every call in the process and keeps the last call's contents; the call clears
 *     the words that must start at zero. Calls that overlap on the GPU (other streams or threads) race on
 *     it: serialise them.
 *   - Limit: one team of at most 2048 CTAs (an instance may use up to 2048 x 256 rows per chunk pass);
 *     beyond that it returns SHELL_ERR_STATIC_LIMIT. */
int shell_step_noalloc(shell_handle *h, int32_t n_steps, shell_step_stats *stats);

/* Exact backward Euler (Section 5, Eq. 62-63 without the linearisation): the new velocity v' solves
 * M (v' - v) = dt (f(x + dt v') + f_ext) at free vertices (v' = 0 at pinned ones), i.e. it minimises the
 * incremental potential. Each step runs a chord iteration with the constant matrix A = M + dt^2 K: v_0 = 0,
 * v_{k+1} = v_k - A^-1 R(v_k) with R(v) = M (v - v_t) - dt (f(x_t + dt v) + f_ext), forces re-evaluated at
 * x_t + dt v_k for every iterate; its first iterate is the linearised step. The step commits the first iterate
 * with ||R(v_k)|| <= rtol ||R(0)||, or the last of max_iters solves (stats.nl_iterations = max_iters then).
 * max_iters <= 1 restores the linearised step (the default). Takes effect at the next step of the handle,
 * alone or in its batch (a batch issues as many force + solve launches per step as its largest max_iters;
 * finished instances skip the later ones). Errors: INVALID_ARG (max_iters < 0, rtol < 0 or NaN), CUDA. */
int shell_set_nonlinear(shell_handle *h, int32_t max_iters, double rtol);

/* Newton's method for the iterations of shell_set_nonlinear (Section 5: the incremental potential is minimised
 * by a Newton-type solver): with on != 0 each iteration solves with the tangent J(v_k) = M + dt^2 (K_b +
 * sum_t H_t(x_t + dt v_k)) instead of the constant matrix, K_b the constant bending Hessian (Eq. 21, 41, 53;
 * also for the shell models, so their iteration converges at a linear rate) and H_t the Hessian of triangle
 * t's corotated membrane energy at the iterate, in closed form with its two rotation terms clamped at zero
 * (positive semi-definite). The preconditioner stays that of the constant matrix. A batch holding a Newton
 * instance runs a solve variant that carries the tangent. Takes effect at the next step. Errors: INVALID_ARG,
 * CUDA. */
int shell_set_newton(shell_handle *h, int32_t on);

/* Quasi-static equilibrium (Section 5, Eq. 64): from the current positions, find x with f(x) + f_ext = 0 at the
 * free vertices (pinned ones stay) by Newton-Raphson in one load step: x_{k+1} = x_k + alpha dx with
 * (K_T(x_k) + M / dt^2) dx = f(x_k) + f_ext, K_T the tangent of shell_set_newton, alpha = min(1, eps_u /
 * max_i |dx_i|) (the incremental displacement limit; eps_u = 0: no limit), until ||f(x_k) + f_ext|| < eps_f
 * (2-norm over the free degrees of freedom). The mass shift M / dt^2 (the handle's dt and density) damps the
 * steps and leaves the equilibrium unchanged; a small density or a large dt makes it negligible. At most
 * max_iters Newton steps. On success x is the equilibrium and v = 0; stats (may be NULL): nl_iterations =
 * Newton steps, rel_residual = ||f + f_ext|| reached, pcg_iterations summed over the steps. If the residual
 * is still above eps_f after max_iters steps, nothing is committed and SHELL_ERR_NOT_CONVERGED is returned
 * (cleared by shell_set_state). The handle's settings of shell_set_nonlinear / shell_set_newton are kept.
 * Synchronises the handle's stream. Errors: INVALID_ARG (eps_f <= 0, eps_u < 0, max_iters < 1), BUSY (handle
 * in a batch), NOT_CONVERGED, NONFINITE, TIMEOUT, CUDA. */
int shell_solve_static(shell_handle *h, double eps_f, double eps_u, int32_t max_iters, shell_step_stats *stats);

/* Energies at the current state x, v in FP64, summed over stencils in a fixed order:
 *   out[0] membrane: corotated linear constant-strain triangles (Section 3), A t (mu |S - I|^2 + lam/2 tr(S - I)^2);
 *   out[1] bending: Eq. 16 (edge hinge, shell: Eq. 23), Eq. 39 (FVM hinge, shell: Eq. 42), Eq. 52 (smoothed
 *          hinge, shell: Eq. 54), per stencil 1/2 eps^T W eps, with the plate form of Eq. 20 / 41 / 53;
 *   out[2] kinetic 1/2 v^T M v (lumped mass); out[3] external potential -sum f_ext . (x - X)
 *          (the terms of the incremental potential of Section 5, Eq. 62).
 * out: caller-allocated host array of 4 doubles. Synchronises the handle's stream (also allowed while the
 * handle is in a batch, between batch steps). Errors: INVALID_ARG (NULL), CUDA. */
int shell_energy(shell_handle *h, double out[4]);

/* Elastic forces f = -grad(Psi_m + Psi_b) at the current x in FP64, the force of the step's right-hand side:
 * bending per stencil by Eq. 22 (edge hinge plate), Eq. 25-26 (edge hinge shell, normal derivative of App. B),
 * Eq. 44-45 (FVM hinge), Eq. 56-57 (smoothed hinge), clamped-edge stencils per Eq. 30-31 and Eq. 59; membrane
 * from the corotated constant-strain triangle (Section 3). Each vertex sums its stencils' contributions in a
 * fixed order. out_xyz: caller-allocated host buffer [V][3], row-major. Synchronises the handle's stream.
 * Errors: INVALID_ARG (NULL), CUDA. */
int shell_forces(shell_handle *h, double *out_xyz);

/* Apply the constant step matrix A = M + dt^2 (K_b + K_m) of the linearised step (Section 5, Eq. 62-63; K_b
 * the constant bending Hessian of Eq. 21 / 41 / 53, K_m the constant membrane block; identity rows / columns
 * at pinned vertices; the matrix is the scalar matrix (x) I_3) to in_xyz [V][3] in FP64: out_xyz = A in_xyz.
 * Both are caller-owned host buffers [V][3], row-major. Synchronises the handle's stream.
 * Errors: INVALID_ARG (NULL), CUDA. */
int shell_apply_matrix(shell_handle *h, const double *in_xyz, double *out_xyz);

/* The state of the time integration (Section 5, Eq. 62-63): positions x and velocities v, held in FP64 on the
 * device. Copy it to / from caller-owned host buffers [V][3], row-major (either pointer may be NULL to skip
 * it). Both synchronise the handle's stream before they return. Setting a state clears a previous step failure
 * of the handle. Errors: INVALID_ARG (h NULL), CUDA. Each step's solver
 * starts from the velocity extrapolated cubically from the last four committed steps
 * (4 (v + v_prev2) - 6 v_prev - v_prev3); setting a state keeps the three earlier velocities, since they
 * only shape the initial guess (results agree to the solve tolerance either way, and writing back an
 * unchanged state leaves the next step bitwise unchanged). */
int shell_get_state(shell_handle *h, double *x, double *v);
int shell_set_state(shell_handle *h, const double *x, const double *v);

/* Device-pointer variants of the state copies (Section 5's x and v): [V][3] row-major FP64 device buffers owned
 * by the caller, stream ordered on the handle's stream, no synchronisation. Errors: INVALID_ARG (h NULL), CUDA. */
int shell_get_state_device(shell_handle *h, double *d_x, double *d_v);
int shell_set_state_device(shell_handle *h, const double *d_x, const double *d_v);

/* Sizes: out[0] vertices, out[1] triangles, out[2] bending stencils, out[3] bytes of device memory the handle
 * holds, out[4] structural nonzeros of the scalar matrix, out[5] stored (SELL-padded) nonzeros, out[6]
 * force contribution slots, out[7] multigrid levels (0 = Jacobi preconditioner), out[8] algorithmic bytes
 * of one FP32 V-cycle (8 B per nonzero of each level operator above the dense level and of each transfer
 * operator with the smoother folded in, 136 B per level row, 4 B per entry of the dense coarse operator;
 * 0 without multigrid). */
int shell_info(shell_handle *h, int64_t out[9]);

/* Free the handle and all device memory it owns (after the handle's stream has finished its work). A handle in
 * a batch must be retired first. Errors: INVALID_ARG (NULL), BUSY (still in a batch). */
int shell_destroy(shell_handle *h);
/* Static message of a SHELL_* code (never NULL; unknown codes give a generic message). */
const char *shell_strerror(int code);

/* Host-only mesh check (needs no GPU): builds the stencils of Section 4 (edge stencils of Section 4.3, Eq. 9-10
 * and Eq. 31; triangle-centred stencils with virtual nodes of Section 4.4-4.5 and App. C, Eq. 78) and the matrix
 * structure shell_create would
 * build and checks every index they hold. out[0] interior edge stencils (edge hinge models), out[1]
 * clamped edge stencils, out[2] triangle stencils with a virtual neighbour, out[3] structural nonzeros of
 * the scalar matrix, out[4] stored (SELL-padded) nonzeros, out[5] force contribution slots, out[6] local
 * matrix entries assembled, out[7] 0 if every index is in range (else the number of bad indices).
 * Errors: INVALID_ARG, NON_MANIFOLD, BAD_ORIENTATION. */
int shell_topology_summary(int32_t n_verts, int32_t n_tris, const int32_t *tris, int32_t n_clamped,
                           const int32_t *clamped_edges, int32_t model, int64_t out[8]);

/* ------------------------------------------------------------------------------------------ batch */
/* The batch API has no counterpart in the paper: it runs the step of shell_step (Section 5, Eq. 62-63) for many
 * independent simulations at once. A batch steps many independent handles together: one persistent launch per
 * step for all resident instances (per-stencil forces, right-hand side, solve and commit; FP64 instances take
 * their forces from one force launch just before it), replayed from a CUDA graph. Instances are admitted while
 * the batch's
 * device-memory budget (bytes of the admitted handles) allows; each instance's result does not depend on
 * the other instances in the batch. A handle admitted to a batch cannot be stepped alone until retired. */
typedef struct shell_batch shell_batch;

int shell_batch_create(const shell_options *opt, size_t budget_bytes, shell_batch **out);
/* Admit a handle; *slot receives its slot id. Errors: BUDGET if it does not fit, BUSY if already in one. */
int shell_batch_admit(shell_batch *b, shell_handle *h, int32_t *slot);
int shell_batch_retire(shell_batch *b, int32_t slot);
/* Step every resident instance n_steps times. stats: NULL or an array indexed by slot with room for
 * shell_batch_capacity() entries. Instances that fail stop stepping; the others continue. Returns the
 * first error met, or SHELL_OK. */
int shell_batch_step(shell_batch *b, int32_t n_steps, shell_step_stats *stats);
int shell_batch_capacity(shell_batch *b);
/* Packed state transfer for every resident instance in one pass each way: x and v are host buffers of
 * [rows][3] FP64, the instances' rows concatenated in increasing slot order. Page-locked buffers (cudaHostAlloc,
 * cudaHostRegister) are read or written in place by the state kernel over the host link; pageable ones are
 * copied through a device staging buffer (two copies each way, slower). The values are the same either way.
 * shell_batch_state_layout returns the number of resident instances and fills (either may be NULL)
 * slots[k] (the k-th resident slot) and row_offsets[k] (its first row; row_offsets[count] = rows). */
int shell_batch_get_states(shell_batch *b, double *x, double *v);
int shell_batch_set_states(shell_batch *b, const double *x, const double *v);
int shell_batch_state_layout(shell_batch *b, int32_t *slots, int64_t *row_offsets);
/* shell_batch_set_states(x_in, v_in), shell_batch_step(n_steps) and shell_batch_get_states(x_out, v_out) in one
 * call: the copies in, the steps and the copies out are queued on the batch's stream behind one another and
 * the call waits once, at the end (the three calls wait after each). x_in, v_in: both NULL (keep the device
 * states) or both host buffers of the packed layout above; x_out, v_out likewise (NULL: no copy out; they may
 * be x_in, v_in). Results, stats and errors are those of the three calls; on an error the states copied out
 * are the committed ones. */
int shell_batch_step_states(shell_batch *b, int32_t n_steps, const double *x_in, const double *v_in, double *x_out,
                            double *v_out, shell_step_stats *stats);
/* Device time of the last shell_batch_step, per step, in milliseconds: out[k] for k < n (n <= steps). */
int shell_batch_step_times(shell_batch *b, float *out_ms, int32_t n);
/* Kernel timing of later shell_batch_step calls: with on != 0 every step is launched directly (not from
 * the graph) with CUDA events around the force launch of FP64 instances and the step launch (of every chord
 * iteration of an exact backward-Euler step). shell_batch_kernel_times then gives out_ms[0] = summed time of
 * the FP64 force launches (0 for a batch of FP32-refinement instances, whose forces are a phase of the step
 * launch) and out_ms[1] = summed time of the step launches of the last call, in milliseconds. */
int shell_batch_set_profiling(shell_batch *b, int32_t on);
/* Autotune the persistent solve launch of this batch: flat teams (any size, global barriers, cooperative
 * launch) with 3 occupancies (CTAs per SM: 1, half, the maximum) x 3 CTA shares for large instances (x0.5,
 * x1, x2), and one-cluster teams (8-CTA thread-block clusters, hardware cluster barrier) with the 3 shares;
 * steps_per_trial real (committed) steps each; keeps the fastest by device time, then runs 3 more calls of
 * steps_per_trial steps with it, re-planning the teams from that shape's own measured times (so a call takes
 * (trials that ran + 3) x steps_per_trial committed steps). A batch's results do not
 * depend on the launch shape, so tuning changes only speed. out_ms: NULL or [12] mean step time of each trial
 * (-1 if skipped, -2 if it ran but the cluster launch was refused); out_choice: NULL or [3] = {CTAs per SM, share x 100, 1 if clusters}. */
int shell_batch_autotune(shell_batch *b, int32_t steps_per_trial, double *out_ms, int32_t *out_choice);
/* Set the solve launch's shape without tuning, in the format of shell_batch_autotune's out_choice:
 * ctas_per_sm (capped at the kernel variant's occupancy), share_x100 (CTA share of large instances x 100),
 * clusters (1: one-cluster teams). For reusing a shape tuned earlier on the same workload. The teams are
 * re-planned at the next step; results do not depend on the shape. Errors: INVALID_ARG. */
int shell_batch_set_launch(shell_batch *b, int32_t ctas_per_sm, int32_t share_x100, int32_t clusters);
int shell_batch_kernel_times(shell_batch *b, double out_ms[2]);
/* Bound of every device-side wait at a team barrier of this batch's solve launches, in nanoseconds (ns <= 0
 * restores the default, 4 s). A CTA whose wait exceeds it raises the launch's abort flag and leaves; the other
 * CTAs leave at their next barrier or before they write any state, so the abandoned launch commits nothing
 * and shell_batch_step returns SHELL_ERR_TIMEOUT, with stats[k].steps_done the steps committed before it; the
 * batch resets its barrier words, and the next call steps normally. For callers that must bound the latency
 * of a stalled step (no counterpart in the paper). Errors: INVALID_ARG (NULL). */
int shell_batch_set_wait_limit(shell_batch *b, int64_t ns);
int shell_batch_destroy(shell_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* SHELL_H_ */
