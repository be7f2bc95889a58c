/*
 * mfg.h - C ABI of the GB300 solver for time-dependent variational mean field
 * games (Ljosheim, Kalise, Pearson, Silva: "Parallel-in-Time Preconditioning
 * for Time-Dependent Variational Mean Field Games", arXiv 2507.01958).
 *
 * The library solves problem (VMFG_h) of Sec. 2 (periodic torus or Neumann
 * rectangle, d = 1 or 2, quadratic Hamiltonian H = |p|^2/2) with the
 * accelerated Chambolle-Pock iteration of Sec. 3 and Sec. 5.  Each iteration
 * needs one solve with AAt = C C^T (eq. largeA), done by preconditioned CG with
 * the parallel-in-time preconditioner P of Sec. 4 (eq. prec / eq. pstrec:
 * time DCT-VIII (l = 1) or DST-I (l = 2), exact spatial diagonalisation per
 * time frequency, Alg. 1 and Alg. 2), and one per-cell proximal map of phi.
 *
 * Conventions shared by every entry point
 *   - All arrays are FP64 and live in DEVICE memory owned by the caller unless
 *     the entry point says otherwise (mfg_solve_host).  The library never
 *     frees or retains caller pointers past the call.
 *   - Grid layout: a spatial field is [Nx][Ny] (j fastest); a space-time field
 *     is [Nt][Nx][Ny], size n = Nt*Nx*Ny (Ny = 1 when dim = 1).  Plane k of a
 *     space-time field holds time level k+1 for m and level k for w, i.e. cell
 *     k pairs (m^{k+1}, w^k) as the scheme (MFG_T2h) of Sec. 2 does.
 *   - The primal y = (m, w) is c = 1 + 2*dim consecutive space-time planes
 *     (m, w1, w2[, w3, w4]); w1/w2 are the x-direction components of the
 *     cone K = [0,inf) x (-inf,0] (x [0,inf) x (-inf,0]) of Sec. 2, w3/w4 the
 *     y-direction ones.
 *   - Batched plans hold several instances; their arrays are concatenated in
 *     instance order at the offsets mfg_layout reports.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; entry points that report results on the host
 *     synchronise it before returning and say so.
 *   - Every function returns MFG_OK or an error code; mfg_last_error gives the
 *     text.  Nothing aborts or throws across this boundary.  A plan is not safe
 *     for concurrent use from two threads or two streams.
 */
#ifndef MFG_H
#define MFG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum mfg_status {
  MFG_OK = 0,
  MFG_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range          */
  MFG_ERR_UNSUPPORTED = 2,   /* valid in the paper, not built here (e.g. N_t > 256)   */
  MFG_ERR_CUDA = 3,          /* a CUDA runtime call failed                            */
  MFG_ERR_NOT_CONVERGED = 4, /* PCG hit max_cg before reaching its tolerance          */
  MFG_ERR_NONFINITE = 5,     /* NaN or Inf appeared in a residual or step             */
  MFG_ERR_TIMEOUT = 6        /* a bounded device-side wait ran out                    */
};

enum { MFG_PERIODIC = 0, MFG_NEUMANN = 1 };
/* MFG_FP64: every step in FP64.  MFG_MIXED: the preconditioner (transforms and
 * per-frequency division) in FP32 inside FP64 flexible PCG; AAt, residuals,
 * dot products and the prox stay FP64.  MFG_MIXED_DF: as MFG_MIXED, with the
 * AAt stencil evaluated in double-float arithmetic (pairs of FP32 numbers,
 * ~48 significant bits) from FP64 inputs to FP64 outputs; residuals, dot
 * products and the prox stay FP64.  MFG_MIXED_TC: as MFG_MIXED, with the
 * preconditioner's dense time transforms (DCT-VIII / DST-I products, Sec. 4.2)
 * on the tensor cores (tcgen05, TF32 operands split in three products for
 * ~FP32 accuracy) when N_t is 32, 64 or 128, on the CUDA cores otherwise.
 * GB300 issues FP32 at ~58x its FP64 rate. */
enum { MFG_FP64 = 0, MFG_MIXED = 1, MFG_MIXED_DF = 2, MFG_MIXED_TC = 3 };
/* PCG tolerance: fixed cg_tol, or the paper's rule
 * min{1e-4, max{1e-6, 1e-4 r}} with r the last CP step (Sec. 5). */
enum { MFG_CG_FIXED = 0, MFG_CG_ADAPTIVE = 1 };
/* What the PCG tolerance is relative to (the paper does not say, Sec. 5).
 * MFG_CG_REF_RHS: ||b||_2 of the system solved in eq. CC*,
 *   AAt z = C (x_l + sigma ybar_l) - sigma d, i.e. stop when
 *   ||b - AAt z|| <= tol ||b|| (the usual CG convention).  b = AAt z_l +
 *   sigma (C ybar_l - d): the plan keeps AAt z in an n-double vector, applied
 *   once per mfg_solve call to the caller's z and then carried by the CP loop
 *   (AAt z_{l+1} = b - r_final, r_final the recursive PCG residual).
 * MFG_CG_REF_RESID: the 2-norm of the residual of the warm start z_l,
 *   sigma (C ybar_l - d): a stricter stop that does not loosen as z_l grows. */
enum { MFG_CG_REF_RHS = 0, MFG_CG_REF_RESID = 1 };

/* One instance of (VMFG_h).  Paper symbols in brackets. */
typedef struct {
  int dim;           /* spatial dimension d: 1 or 2 (Sec. 2)                         */
  int n[2];          /* Nx, Ny grid points (Ny ignored, taken as 1, when dim = 1)    */
  double len[2];     /* domain lengths b-a, d-c (Sec. 2)                              */
  int bc[2];         /* MFG_PERIODIC | MFG_NEUMANN per axis (Alg. 2 allows mixed)    */
  int nt;            /* N_t >= 2 time steps                                           */
  double T;          /* horizon T > 0, dt = T/N_t                                      */
  double nu;         /* viscosity nu >= 0 (ignored when nu_field is set)               */
  double qprime;     /* Hamiltonian exponent q' of eq. power_hamiltonian, in [1.05, 20];
                        2 takes the fast prox, others a general FP64 root finder    */
  double f_a, f_b;   /* f(x,m) = f_a m + f_b m^2 + V(x); f_a, f_b >= 0 (monotone f)   */
  double g_a;        /* g(x,m) = g_a m + W(x); g_a >= 0                                */
  int l;             /* time preconditioner: 1 = DCT-VIII, 2 = DST-I (Sec. 4.1);
                        0 = no approximation in the first block (P = AAt): the time
                        blocks are solved exactly per spatial mode by tridiagonal
                        elimination (not in the paper; see mfg_apply_precond)      */
  double gamma;      /* acceleration constant gamma > 0 (Sec. 5)                       */
  double tau0, sigma0; /* initial step sizes (Sec. 5: 1 and 1)                         */
  int max_cp;        /* CP iterations per mfg_solve call                               */
  double cp_tol;     /* stop when ||m_{l+1} - m_l||_2 <= cp_tol; <= 0 disables (Sec. 5) */
  int cg_rule;       /* MFG_CG_FIXED | MFG_CG_ADAPTIVE                                 */
  double cg_tol;     /* relative PCG tolerance for MFG_CG_FIXED                        */
  int max_cg;        /* PCG iteration cap per solve                                    */
  int precision;     /* MFG_FP64 | MFG_MIXED | MFG_MIXED_DF | MFG_MIXED_TC             */
  int cg_ref;        /* MFG_CG_REF_RHS (0, the default) | MFG_CG_REF_RESID             */
  const double* nu_field; /* NULL: constant viscosity nu.  Otherwise a HOST array of
                        Nx*Ny node viscosities nu(x) >= 0 ([Nx][Ny], read during
                        mfg_plan only, never retained), which replaces nu; see
                        "Viscosity fields" below.                                    */
} mfg_problem;

/* Viscosity fields (nu_field != NULL).  The paper allows a non-constant
 * viscosity nu(x) (Sec. 4, before Sec. 4.1: the spatial matrices still repeat
 * at every time step) without fixing its discretisation.  Here nu K becomes
 *   K_nu = sum over the active axes of D^1 diag(nu_face) (D^1)^T / dx^2,
 * with the D^1 blocks of Sec. 4.3, face i of an axis between nodes i and i+1
 * (wrapping on a periodic axis) and nu_face the arithmetic mean of those two
 * node values: a symmetric conservative operator, so L = K_nu + I/dt is
 * symmetric, C = L^2 + B B^T, and eq. largeA and eq. prec keep their block
 * forms with C_hat = K_nu^2 + B B^T and L_hat = L/dt.  The constraint, its
 * transpose, AAt and the dual lift of the prox step use K_nu.
 * The preconditioner is Alg. 1 with an exact solve of every per-frequency
 * system (C_hat + lambda_k L_hat) x_k = y_k, the LU option of Sec. 4.1: a
 * banded Cholesky factorisation per time frequency, formed once in FP64 by
 * mfg_plan on the host (points ordered axis by axis, a periodic axis folded
 * 0, N-1, 1, N-2, ... so that the bandwidth stays ~2-4 Ny), stored on the
 * device in the plan's preconditioner precision (FP32 for the MIXED
 * precisions), and applied per frequency by forward and backward banded
 * substitution between the two time transforms.  Costs: factor storage
 * about 2 N_t Nx Ny (w+32) words, w the half-bandwidth (2 Ny on a Neumann x axis,
 * ~4 Ny + Ny on a periodic one), and O(N_t Nx Ny w^2) host work in mfg_plan.
 * Restrictions: l must be 1 or 2 (MFG_ERR_UNSUPPORTED for l = 0); w <= 4096
 * and factor storage <= 64 GiB (MFG_ERR_UNSUPPORTED beyond);
 * mfg_apply_precond_noalloc returns MFG_ERR_UNSUPPORTED; mfg_adjoint returns
 * the gradient with respect to nu(x) node by node; MFG_MIXED_DF runs its AAt
 * stencil in FP64 (as MFG_MIXED); the time transforms run on the CUDA cores in
 * every precision.  nu is ignored. */

/* Per-instance run record.  On entry to mfg_solve, `ell`, `tau`, `sigma` are
 * the resume state (ell = 0 starts from tau0, sigma0); on return all fields
 * describe the state after the call. */
typedef struct {
  int status;          /* mfg_status of this instance                                 */
  int ell;             /* CP iterations done in total (resume counter)                */
  int cp_iters;        /* CP iterations done by this call                             */
  int max_cg_in_solve; /* largest PCG count of one solve in this call                 */
  long long cg_iters;  /* PCG iterations done by this call                            */
  double r_last;       /* ||m_{l+1} - m_l||_2 of the last iteration                    */
  double tau, sigma;   /* step sizes for the next iteration                            */
} mfg_stats;

typedef struct mfg_plan_s* mfg_plan_t;

/* Validates `batch` problems, builds the eigenvalue tables (eq. eigs, Alg. 2)
 * and transform matrices on the host in FP64, uploads them and
 * allocates all device workspace on the current device.  Rejects q' outside
 * [1.05, 20] (MFG_ERR_UNSUPPORTED), N_t < 2, N < 2, T <= 0, nu < 0,
 * f_a/f_b/g_a < 0, l not in {0,1,2}, N_t > 256 (UNSUPPORTED), a viscosity
 * field with a negative or non-finite value (INVALID_ARG) or outside the
 * limits of "Viscosity fields" (UNSUPPORTED).  *out is NULL on failure. */
int mfg_plan(const mfg_problem* probs, int batch, mfg_plan_t* out);

/* Frees all plan-owned memory.  NULL is accepted. */
int mfg_destroy(mfg_plan_t plan);

/* Thread-local text of the last error raised in this thread ("" if none). */
const char* mfg_last_error(void);

/* Element offsets of instance b inside the concatenated batch arrays:
 * field (m0, V, W: Nx*Ny each), primal (y, ybar: c*n each), dual (z: n), plus
 * the instance sizes.  Any output pointer may be NULL. */
int mfg_layout(mfg_plan_t plan, int b, size_t* field_off, size_t* primal_off,
               size_t* dual_off, size_t* n, int* c);

/* Totals of the concatenated batch arrays (elements). */
int mfg_sizes(mfg_plan_t plan, size_t* field_total, size_t* primal_total,
              size_t* dual_total);

/* Runs up to max_cp accelerated Chambolle-Pock iterations (Sec. 3 eq.
 * pasosChamPock, step sizes of Sec. 5) on every instance of the plan.
 *   m0, V, W : fields [Nx][Ny] per instance (m0 = m^0, V and W of f and g)
 *   y        : in/out primal (m, w); caller sets m^k = m0, w = 0 (or any start)
 *   ybar     : in/out extrapolated primal; set ybar = y for a fresh start
 *   z        : in/out dual multiplier with x = C^T z; set z = 0 for a fresh start
 *   st       : array of `batch` records, in/out (resume state on entry)
 * The dual x = prox_{sigma psi*}(...) of eq. CC* is never stored: the library
 * keeps z and forms C^T z where needed.  The whole solve is one CUDA graph
 * launch; the call synchronises `stream` and fills `st` before returning.
 * Returns the first non-OK instance status, or MFG_OK (MFG_ERR_TIMEOUT: with
 * MFG_MIXED_TC, a tensor-core completion wait ran out; the instance stops and
 * its outputs are unspecified). */
int mfg_solve(mfg_plan_t plan, const double* m0, const double* V, const double* W,
              double* y, double* ybar, double* z, mfg_stats* st, void* stream);

/* Same as mfg_solve with HOST buffers: copies the inputs into plan-owned device
 * buffers, solves, and copies y, ybar, z back.  Synchronous. */
int mfg_solve_host(mfg_plan_t plan, const double* m0, const double* V,
                   const double* W, double* y, double* ybar, double* z,
                   mfg_stats* st, void* stream);

/* z = P^{-1} r for instance b (Alg. 1 with Alg. 2 for its per-frequency
 * spatial solves, eq. pstrec), in the plan's precision.  With l = 0 the time transform and the
 * per-frequency division are replaced by an exact tridiagonal solve in time per
 * spatial mode, so P = AAt (eq. largeA) up to rounding.  With a viscosity
 * field the per-frequency systems are solved by their banded Cholesky factors
 * (see "Viscosity fields").  r, z: n elements; must not alias. */
int mfg_apply_precond(mfg_plan_t plan, int b, const double* r, double* z, void* stream);

/* y = prox_{tau phi}(v) for instance b, cell by cell (Sec. 3; phi_ij = b_hat +
 * F, plus G/dt on the last plane; b_hat = |w|^q/(q m^{q-1}), q = q'/(q'-1),
 * Sec. 2).  v, y: c*n elements; y == v allowed.
 * V, W: the instance's fields. */
int mfg_prox(mfg_plan_t plan, int b, double tau, const double* v, const double* V,
             const double* W, double* y, void* stream);

/* One primal step of the CP iteration for instance b, with the kernel that
 * mfg_solve runs for it (Sec. 3 eq. pasosChamPock, step sizes of Sec. 5):
 * the dual lift x = C^T z, y <- prox_{tau phi}(y - tau x) cell by cell, and the
 * extrapolation ybar <- y_new + theta (y_new - y_old) with
 * theta = 1/sqrt(1 + 2 gamma tau).  z: n; y, ybar: c*n, updated in place;
 * V, W: the instance's fields.  Uses the plan's device scalars, so it must not
 * run concurrently with mfg_solve on the same plan.  Stream-ordered. */
int mfg_prox_step(mfg_plan_t plan, int b, double tau, const double* z, double* y, double* ybar,
                  const double* V, const double* W, void* stream);

/* q = C C^T p (eq. largeA) for instance b; p, q: n elements, no aliasing.
 * Two passes through 2n doubles of the plan's workspace, so it must not run
 * concurrently with mfg_solve or mfg_adjoint on the same plan (a plan is not
 * safe for concurrent use from two streams). */
int mfg_apply_AAt(mfg_plan_t plan, int b, const double* p, double* q, void* stream);

/* r = C v (eq. ABC, reduced: the m0 term excluded) for instance b; v: c*n, r: n. */
int mfg_apply_C(mfg_plan_t plan, int b, const double* v, double* r, void* stream);

/* x = C^T p for instance b; p: n, x: c*n. */
int mfg_apply_Ct(mfg_plan_t plan, int b, const double* p, double* x, void* stream);

/* Gradient of a loss on the converged equilibrium of instance b by implicit
 * differentiation of the optimality (KKT) conditions of (VMFG_h) (Sec. 2-3:
 * the fixed point y = prox_{tau phi}(y - tau C^T z), C y = d(m0)).
 *   y, z   : a converged solution from mfg_solve (c*n and n device doubles);
 *            the active set is read off y (m > 0, w components != 0)
 *   gy     : dloss/dy, c*n device doubles (same layout as y)
 *   dm0    : out, dloss/dm0, Nx*Ny           dV : out, dloss/dV(x), Nx*Ny
 *   dW     : out, dloss/dW(x), Nx*Ny or NULL dnu: out, dloss/dnu, 1 device double;
 *            with a viscosity field, Nx*Ny device doubles: dloss/dnu(x) at the
 *            nodes (nu_face = mean of its two nodes, so each face's term is
 *            split half and half between them)
 *   tol, max_iter: relative tolerance and cap of the adjoint PCG
 *   st     : out; cg_iters = adjoint PCG iterations, r_last = final relative residual
 * Built for q' = 2 (MFG_ERR_UNSUPPORTED otherwise).
 * The adjoint system is solved through its Schur complement
 * C_A H^{-1} C_A^T with the plan's preconditioner P (eq. prec) inside PCG,
 * H being the per-cell Hessian of phi.  The first call allocates a c*n + n
 * workspace owned by the plan.  Synchronises `stream`. */
int mfg_adjoint(mfg_plan_t plan, int b, const double* y, const double* z, const double* gy,
                double* dm0, double* dV, double* dW, double* dnu, double tol, int max_iter,
                mfg_stats* st, void* stream);

/* Number of kernel launches the library enqueued since the plan was made
 * (graph nodes executed by mfg_solve are counted per execution). */
long long mfg_kernel_launches(mfg_plan_t plan);

/* How mfg_solve issues its kernels.  MFG_LAUNCH_GRAPH (default): the whole
 * solve is one CUDA graph launch with device-side loop control.
 * MFG_LAUNCH_EAGER: the same kernels with the same launch shapes, issued one
 * by one on `stream`, the host reading the convergence flags after every PCG
 * iteration (slower; lets per-kernel profilers see each launch, which they
 * cannot inside graphs with conditional nodes). */
enum { MFG_LAUNCH_GRAPH = 0, MFG_LAUNCH_EAGER = 1 };
int mfg_set_launch_mode(mfg_plan_t plan, int mode);

/* Launch schedule of one instance.  A new plan uses fixed defaults; the
 * autotuner replaces them with the fastest of a set of measured candidates.
 * None of the choices changes the operators (results differ only by the
 * order of floating-point operations: reduction grids and transform
 * algorithms). */
enum { MFG_TIME_TENSOR_CORES = 0, MFG_TIME_CUDA_CORES = 1 };
typedef struct {
  int tuned;          /* 1: set by mfg_autotune (timed, or from its per-process cache)  */
  int measured;       /* 1: this plan's mfg_autotune timed the candidates itself        */
  int time_pass;      /* MFG_TIME_TENSOR_CORES | MFG_TIME_CUDA_CORES                    */
  int fft[2];         /* per problem axis: 1 = FFT spatial pass, 0 = dense transform   */
  int aat_blocks;     /* blocks of the AAt stencil launch                               */
  int vec_blocks;     /* grid cap of the vector and reduction kernels                   */
  double precond_us;  /* measured time of the chosen preconditioner step, 0 if none     */
  double aat_us;      /* measured time of the chosen AAt apply, 0 if none               */
} mfg_schedule;

/* Autotuner.  For every instance of the plan, times (CUDA events, on
 * `stream`) the candidate launch choices and keeps the fastest:
 *   - grid cap of the vector and reduction kernels: 152, 304 or 608 blocks;
 *   - the preconditioner step (Alg. 1/2 with the fused PCG vector work): time
 *     pass on the tensor cores or the CUDA cores (MFG_MIXED_TC with N_t in
 *     {32, 64, 128}), FFT or dense transform pass on each power-of-two axis;
 *   - AAt stencil launch: 152 x 4, 8 or 16 target blocks.
 * The choice is cached per process by instance shape (grid, N_t, boundary
 * conditions, precision, l): a later plan with the same shape takes it
 * without timing.  Uses the plan's workspace and a temporary n-double buffer
 * (allocated and freed here), overwrites the plan's device scalars, drops
 * the cached solve graph, and synchronises `stream`.  Call it before a
 * solve, not concurrently with one. */
int mfg_autotune(mfg_plan_t plan, void* stream);

/* The launch schedule instance b currently uses. */
int mfg_get_schedule(mfg_plan_t plan, int b, mfg_schedule* out);

/* Test hook for the failure-detection paths; MFG_INJECT_NONE in normal use.
 * MFG_INJECT_TC_NO_COMMIT: in the tensor-core time pass of mfg_solve
 * (MFG_MIXED_TC with N_t in {32, 64, 128}) the elected thread issues neither
 * the MMAs nor their completion commit, so no tensor-core work is in flight
 * and the bounded mbarrier wait (4096 polls under this hook) runs out: the
 * instance ends with MFG_ERR_TIMEOUT after its first CP iteration (outputs
 * unspecified, as for any timeout) and the call returns normally with the
 * context still usable.  MFG_INJECT_BAND_NO_COPY: in the banded substitutions
 * of a viscosity-field plan's mfg_solve, the copy warp issues neither a
 * stage's bulk copy nor its expected-bytes arrival, so the stage's bounded
 * mbarrier wait (4096 polls under this hook) runs out, with the same
 * outcome.  Either applies to the plan's later mfg_solve calls (no graph
 * rebuild).  Invalid `what`: MFG_ERR_INVALID_ARG. */
enum { MFG_INJECT_NONE = 0, MFG_INJECT_TC_NO_COMMIT = 1, MFG_INJECT_BAND_NO_COPY = 2 };
int mfg_set_fault_injection(mfg_plan_t plan, int what);

/* z = P^{-1} r for the single problem *p, like mfg_apply_precond, but with no
 * plan and no device memory allocation of any kind.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device
 * memory where they call it: work being recorded into a CUDA graph under
 * global stream capture (where cudaMalloc is not permitted), code whose memory
 * belongs to a pool or framework allocator it may not bypass, and latency-
 * critical paths that cannot risk an allocation's cost or failure.  Those
 * callers cannot use mfg_plan, which allocates.
 *   - Scratch: the transform tables and work buffers live in one static
 *     device array of 6.4 MB that every GPU loading this library holds until
 *     the process exits.  Limits: N_t*Nx*Ny <= 262144, Nx, Ny <= 256,
 *     N_t <= 128; larger problems return MFG_ERR_INVALID_ARG with a message.
 *   - The first call on each device resolves the array's device address and
 *     sets kernel attributes; make that first call before any stream capture.
 *     First calls from several host threads at once are safe (each resolves
 *     the same address).  The address is cached for the life of the process:
 *     after cudaDeviceReset on a device, do not call this entry point again
 *     there.
 *   - All calls share the array and each call rewrites all of it that it
 *     reads, so no state carries over; but calls whose work overlaps on the
 *     GPU (other streams or other threads) race and corrupt each other.
 *     Calls on one stream are ordered and safe.
 *   - r, z: n device doubles, caller-owned, must not alias.  Stream-ordered;
 *     returns after enqueueing.
 *   - Same passes as mfg_apply_precond: FFT spatial passes on power-of-two
 *     axes (twiddles are part of the static array), dense ones otherwise.
 *     p->precision: MFG_FP64 and MFG_MIXED as in a plan, MFG_MIXED_TC with the
 *     tensor-core time pass as in a plan; MFG_MIXED_DF runs as MFG_MIXED (the
 *     two differ only in the AAt stencil, which this apply does not use).
 *     l = 0 (the exact time solve) and viscosity fields need plan-built
 *     factors and return MFG_ERR_UNSUPPORTED. */
int mfg_apply_precond_noalloc(const mfg_problem* p, const double* r, double* z, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MFG_H */
