/*
 * dg.h -- C ABI of libdg, a single-GPU (sm_103a) implementation of the per-step
 * hot path of the nodal discontinuous Galerkin method of Kidder et al.,
 * "SpECTRE: A task-based discontinuous Galerkin code for relativistic
 * astrophysics", arXiv:1609.00098:
 *   primitive recovery (Sec. 2.1.1 closed form; Sec. 2.1.2 Newton con2prim),
 *   fluxes, tensor-product LGL differentiation and lifted face fluxes (Sec. 3.1,
 *   eq:411), LLF / HLL numerical fluxes (Sec. 3.2, eq:LLF, eq:HLL),
 *   SSP-RK3 (Sec. 3.4), the minmod-type troubled-cell limiter (Sec. 3.3.1-3.3.2)
 *   and the SR conserved-variable fix (Sec. 2.1.4), on periodic boxes of affine
 *   hexahedral elements (eq:AffineMap).
 *
 * Conventions shared by every call:
 *  - Every array argument is a DEVICE pointer on the current CUDA device unless
 *    the comment says "host".  The caller owns all arrays passed in.
 *  - State layout: U[e][v][k][j][i] (FP64), element-major, i fastest;
 *    e = ex + K0*(ey + K1*ez); v = 0..4 = (rho, S_x, S_y, S_z, E) for Newtonian
 *    Euler and (D, S_x, S_y, S_z, tau) for SR hydro.  dg_state_size() doubles.
 *  - Node order ("node index") is g = e*n^3 + (i + n*(j + n*k)).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work asynchronously; argument errors are returned synchronously.
 *  - Kernel-side failures (con2prim without a root, unphysical states) set a
 *    sticky per-mesh device status word; dg_sync_status() reads and clears it.
 *    No kernel traps, asserts or spins without bound.
 *  - On any error the thread-local message of dg_last_error() is set.
 */
#ifndef LIBDG_DG_H
#define LIBDG_DG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DG_OK = 0,
    DG_ERR_ARG = 1,          /* invalid argument (returned synchronously) */
    DG_ERR_CUDA = 2,         /* a CUDA call failed */
    DG_ERR_C2P = 3,          /* con2prim did not converge at some node */
    DG_ERR_UNPHYSICAL = 4,   /* conserved state with no physical primitive state */
    DG_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
    DG_ERR_NOMEM = 6         /* device allocation failed */
} dg_status;

enum { DG_SYSTEM_NEWTONIAN = 0, DG_SYSTEM_SR = 1 };
enum { DG_FLUX_LLF = 0, DG_FLUX_HLL = 1, DG_FLUX_ROE = 2 };
enum { DG_LIMITER_NONE = 0, DG_LIMITER_MINMODN = 1, DG_LIMITER_MINMOD = 2, DG_LIMITER_MRS = 3 };
enum { DG_PRECISION_FP64 = 0, DG_PRECISION_MIXED = 1 };

typedef struct {
    int system;      /* DG_SYSTEM_*: Newtonian Euler (Sec. 2.1.1) or flat-space SR hydro (Sec. 2.1.2) */
    int K[3];        /* elements per axis, >= 1 */
    int n;           /* LGL nodes per axis, 2..8 (degree N = n-1) */
    int flux;        /* DG_FLUX_*: eq:LLF, eq:HLL with Davis speeds, or eq:Roe (Newtonian only) */
    int limiter;     /* DG_LIMITER_*: none, generalized minmodB detector + limiter (Sec. 3.3.2), plain minmod
                        (Sec. 3.3.1), or the moment limiter of Moe, Rossmanith and Seal (Sec. 3.3.3, Newtonian) */
    int precision;   /* DG_PRECISION_* */
    double gamma;    /* ideal-gas adiabatic index, > 1 */
    double lo[3];    /* periodic box [lo, hi) */
    double hi[3];
    double tvb_M;    /* minmodB constant M (eq:MinModB), >= 0 */
    double beta;     /* slope-limiter beta (2 minmod, 1 MUSCL), > 0 */
    double d_atm;    /* SR fix: floor on D */
    double tau_atm;  /* SR fix: floor on tau as a fraction of D */
    double mrs_alpha; /* DG_LIMITER_MRS: alpha~ >= 0 of the bound widening alpha~ h^{3/2} */
    int bc[3];       /* DG_BC_* per axis: periodic, or analytic exterior states on the faces at lo and hi
                        (Sec. 3.4: the interior numerical flux with the exterior solution supplied) */
    int exact;       /* DG_EXACT_*: the analytic solution of analytic boundaries */
    double exact_par[6]; /* DG_EXACT_ISENTROPIC_VORTEX: beta, X0, Y0, U, V, W of eq:isen_vortex */
} dg_mesh_desc;

/* Analytic boundaries need the Newtonian system, DG_EXACT_ISENTROPIC_VORTEX and no
 * limiter.  The exterior state of a boundary face node is eq:isen_vortex (P = rho^gamma)
 * at the coordinates of the interior trace node and the stage time: SSP-RK3 takes
 * t, t + dt, t + dt/2 for its three stages, dg_rhs and Adams-Bashforth the mesh
 * time t.  Exterior states use CUDA's exp and pow, so FP64 results agree with a
 * libm evaluation to rounding rather than bit for bit. */
enum { DG_BC_PERIODIC = 0, DG_BC_ANALYTIC = 1 };
enum { DG_EXACT_NONE = 0, DG_EXACT_ISENTROPIC_VORTEX = 1 };

typedef struct dg_mesh dg_mesh;

/* Create a mesh on the current device.  Allocates the library's scratch (two
 * state copies, a primitive buffer, limiter summaries, flags) with cudaMalloc.
 * Returns DG_ERR_ARG for an invalid descriptor, DG_ERR_NOMEM if allocation fails. */
dg_status dg_mesh_create(const dg_mesh_desc *desc, dg_mesh **out);
/* Free a mesh and its scratch (synchronises the device first).  NULL is ignored. */
void dg_mesh_destroy(dg_mesh *mesh);
/* Number of doubles in one state vector: E * 5 * n^3. */
long long dg_state_size(const dg_mesh *mesh);
/* Number of nodes E * n^3. */
long long dg_num_nodes(const dg_mesh *mesh);

/* The 1D LGL tables the kernels use (Sec. 3.1), host arrays of n (x, w, row1)
 * and n*n (D) doubles: nodes x ascending, quadrature weights w, differentiation
 * matrix D[i*n+l] = ell_l'(x_i) (eq:405), and row1, the Legendre P1 coefficient
 * of the nodal interpolant (c1 = sum_i row1[i] u_i).  No GPU needed.
 * DG_ERR_ARG if n is outside 2..8 or a pointer is NULL. */
dg_status dg_lgl_tables(int n, double *x, double *w, double *D, double *row1);

/* Physical coordinates of every node, eq:AffineMap: xyz[a*N + g], a = 0..2,
 * N = dg_num_nodes(), g the node index. */
dg_status dg_node_coords(const dg_mesh *mesh, double *xyz, void *stream);

/* Primitive -> conserved (Sec. 2.1.1, 2.1.2): prim[v*N + g] with rows
 * (rho, vx, vy, vz, p) in node order, U in state layout.  Separate arrays. */
dg_status dg_prim2con(const dg_mesh *mesh, const double *prim, double *U, void *stream);

/* Primitive recovery for the whole mesh: P[e][c][node], c = (vx, vy, vz, p).
 * SR uses the safeguarded Newton con2prim of dg_con2prim. */
dg_status dg_primitives(dg_mesh *mesh, const double *U, double *P, void *stream);

/* Semi-discrete right-hand side dU/dt of eq:411 (volume term by tensor-product
 * differentiation, eq:405; surface term with the numerical flux lifted into the
 * boundary nodes).  U and dUdt must not alias.  Mixed-precision Newtonian meshes
 * move U in 16-byte pieces: U must be 16-byte aligned (cudaMalloc and PyTorch
 * allocations are), else DG_ERR_ARG. */
dg_status dg_rhs(dg_mesh *mesh, const double *U, double *dUdt, void *stream);

/* CFL step of Sec. 3.4: *dt = cfl * dx_min / lambda_max, dx_min the smallest
 * node gap min_a (dx_a/2)(xbar_1 - xbar_0), lambda_max the largest |wave speed|
 * over nodes and axes (an exact, order-independent maximum).  dt: device, 1 double. */
dg_status dg_compute_dt(dg_mesh *mesh, const double *U, double cfl, double *dt, void *stream);

/* One SSP-RK3 step (Shu-Osher form) in place on U, with the limiter and then the
 * SR fix after every stage (Sec. 3.3, 3.4):
 *   U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1)); Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2)).
 * cfl > 0: dt is the CFL step of Un, computed on the device inside the step;
 * cfl <= 0: the host value dt is used.  dt_used (device, 1 double, may be NULL)
 * receives the step taken.  troubled (device, E bytes, may be NULL) receives the
 * bitmask of limited variables of the last stage.  Mixed-precision Newtonian
 * meshes (other than with DG_LIMITER_MRS) run the step in the equivalent
 * difference form D_s = U_s - Un (FP32 differences, FP64 Un and Un+1) and need U
 * 16-byte aligned (else DG_ERR_ARG). */
dg_status dg_rk3_step(dg_mesh *mesh, double *U, double dt, double cfl, double *dt_used,
                      unsigned char *troubled, void *stream);

/* Mesh time t (device-resident; 0 at creation).  Every dg_rk3_step and
 * dg_ab3_step of a mesh with analytic boundaries advances it by the step taken
 * (on periodic meshes time enters nowhere and it stays put).  dg_mesh_set_time
 * is stream-ordered; dg_mesh_get_time synchronises `stream` and writes *t (host). */
dg_status dg_mesh_set_time(dg_mesh *mesh, double t, void *stream);
dg_status dg_mesh_get_time(dg_mesh *mesh, double *t, void *stream);

/* Limiter alone, in place (Sec. 3.3.1, 3.3.2, 3.3.3); troubled as in dg_rk3_step.
 * DG_LIMITER_MRS (Sec. 3.3.3, eq:MRSSol; Newtonian meshes): per element, w the
 * node primitives (rho, v, p) and w0 those of the cell average U0; with
 * [m, M] = [min, max] of w0 over the element and its six face neighbours, widened
 * to w0 -+ mrs_alpha h^{3/2} (h the largest element width), a scale
 * theta = min(1, |(M - w0)/(max w - w0)|, |(m - w0)/(min w - w0)|) over the five
 * primitives (a ratio counts 1 when its denominator is within 1e-12 |w0|) rescales
 * every variable, U -> U0 + theta (U - U0); troubled gets 0x1f where theta < 1. */
dg_status dg_limit(dg_mesh *mesh, double *U, unsigned char *troubled, void *stream);
/* SR conserved-variable fix alone, in place (Sec. 2.1.4); no-op for Newtonian meshes. */
dg_status dg_fix(dg_mesh *mesh, double *U, void *stream);
/* Third-order Adams-Bashforth step (Sec. 3.4, the paper's other third-order
 * integrator) with a fixed dt:
 *   U^{n+1} = U^n + dt (23/12 L^n - 16/12 L^{n-1} + 5/12 L^{n-2}),
 * then the limiter and (SR) the conserved fix, as after an SSP-RK3 stage.  The
 * mesh keeps the last three right-hand sides (library scratch, allocated on the
 * first call); the first two steps after mesh creation or dg_ab3_reset are
 * SSP-RK3 steps that record L(U) of the state they start from.  FP64 meshes
 * give the oracle's bits; mixed meshes evaluate L in mixed precision and
 * combine in FP64.  troubled (device, one byte per element, may be NULL) gets the
 * limiter's mask.  Errors: DG_ERR_ARG for dt <= 0 or a dt different from the
 * previous step's without a reset; DG_ERR_NOMEM/CUDA if the history cannot be
 * allocated. */
dg_status dg_ab3_step(dg_mesh *mesh, double *U, double dt, unsigned char *troubled, void *stream);
dg_status dg_ab3_reset(dg_mesh *mesh);

/* Limiter summaries S[e][v][10] = (cell mean, face means lo/hi for x, y, z,
 * Legendre P1 coefficients along x, y, z) of U. */
dg_status dg_limiter_summaries(dg_mesh *mesh, const double *U, double *S, void *stream);

/* Standalone SR con2prim (Sec. 2.1.2) of `count` nodes, FP64.
 * cons: 5 rows of `count` (D, S_x, S_y, S_z, tau); prim: 5 rows (rho, vx, vy, vz, p).
 * p_guess (may be NULL -> standard guess (gamma-1) tau, clamped into the bracket),
 * iters and status (may be NULL) have `count` entries.  status: 0 ok,
 * 1 unphysical input, 2 no convergence in 200 iterations. */
dg_status dg_con2prim(long long count, double gamma, const double *cons, double *prim,
                      const double *p_guess, int *iters, int *status, void *stream);

/* ---- Learned starting guess for SR con2prim (an addition to the method of Sec. 2.1.2; the paper has no counterpart) ----
 * A 3 -> 64 -> 64 -> 1 SiLU MLP maps three scaled invariants of (D, S, tau) to a
 * scaled log pressure; dg_con2prim's safeguarded Newton starts from it, so results
 * change only in iteration count.  Parameters are FP32, laid out flat as
 * W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3 (DG_C2P_NET_PARAMS floats;
 * W[j][i] maps input i to output j).  With E = tau + D and s = |S| the features are
 * x1 = 2 (log10(tau/D) - lo1)/(hi1 - lo1) - 1, x2 = 2 s/E - 1,
 * x3 = 2 (log10 D - lo3)/(hi3 - lo3) - 1, and the target y = (log10(p/E) - y_shift)/y_scale;
 * scales = (lo1, hi1, lo3, hi3, y_shift, y_scale).  The 64 x 64 layer runs on the
 * tensor cores in BF16 with FP32 accumulation (forward and backward). */
#define DG_C2P_NET_PARAMS 4481
typedef struct dg_c2p_net dg_c2p_net;
/* Create on the current device from host arrays params[DG_C2P_NET_PARAMS] and
 * scales[6] (copied).  Adam state starts at zero. */
dg_status dg_c2p_net_create(const float *params, const double *scales, dg_c2p_net **out);
void dg_c2p_net_destroy(dg_c2p_net *net);
/* Copy the current FP32 parameters to the host array params[DG_C2P_NET_PARAMS]. */
dg_status dg_c2p_net_get_params(const dg_c2p_net *net, float *params);
/* Pressure guesses E 10^(y y_scale + y_shift), clamped into [max(0, s-E), (gamma-1) tau],
 * for `count` conserved states (5 device rows as in dg_con2prim) into p_guess (device).
 * States whose features are not finite (D or tau not positive) get -1, which
 * dg_con2prim reads as "use the standard guess". */
dg_status dg_c2p_net_guess(dg_c2p_net *net, long long count, double gamma, const double *cons, double *p_guess,
                           void *stream);
/* Mean squared error of the scaled target over `count` states with true pressures p
 * (device), and its gradient: grad (device, DG_C2P_NET_PARAMS floats), loss (device, 1).
 * States whose features or target are not finite in FP32 (D or tau not positive,
 * p below the FP32 range) contribute zero to the loss and to the gradient. */
dg_status dg_c2p_net_grad(dg_c2p_net *net, long long count, const double *cons, const double *p, float *grad,
                          float *loss, void *stream);
/* `epochs` passes over the data in order, mini-batches of `batch`, one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) per mini-batch.
 * loss_per_epoch (device, `epochs` floats, may be NULL) gets each epoch's mean loss. */
dg_status dg_c2p_net_train(dg_c2p_net *net, long long count, const double *cons, const double *p, int epochs,
                           int batch, float lr, float *loss_per_epoch, void *stream);

/* dg_rhs without allocation (the paper has no counterpart: this serves callers that
 * cannot call cudaMalloc -- device memory owned by another allocator, or loops that
 * cannot afford the device synchronisation of cudaMalloc/cudaFree).  Same kernels
 * and result as dg_rhs on a mesh made from `desc` (FP64 only), but the node
 * primitives live in a static device array of DG_RHS_STATIC_MAX_NODES nodes
 * (4 doubles each, 4 MiB, held by every GPU that loads the library until exit)
 * and nothing is allocated.  U and dUdt are caller-owned device arrays in state
 * layout.  DG_ERR_ARG if the mesh has more than DG_RHS_STATIC_MAX_NODES nodes or
 * the descriptor is invalid.  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  The array is
 * shared by all calls and keeps the last call's contents; calls that overlap on
 * the GPU race on it.  A node without a physical primitive state gives non-finite
 * values in dUdt. */
#define DG_RHS_STATIC_MAX_NODES 131072
/* (periodic meshes only: DG_ERR_ARG for analytic boundaries) */
dg_status dg_rhs_static(const dg_mesh_desc *desc, const double *U, double *dUdt, void *stream);

/* Per-mesh options of the mixed-precision path (no effect on the FP64 path,
 * which always follows the oracle's arithmetic).
 *   DG_OPT_TENSOR_CORE_CONTRACTION (default 0): 1 evaluates the volume
 *     contraction sum_l D_il F_l (Sec. 3.1, eq:405) of the relativistic (and
 *     Newtonian MRS-limited) stage kernel on the tensor cores as split-BF16x3
 *     products accumulated in FP32; 0 uses FP32 FMA on the CUDA cores.  Both
 *     are FP32-accurate; FMA is the faster of the two for every n = 3..8 on
 *     this GPU.  The Newtonian stage kernel of the other limiters contracts
 *     with FMA only and ignores the option.
 *   DG_OPT_C2P_KAPPA_SWITCH (default 10): the conditioning estimate tau/(rho eps)
 *     above which the FP32 con2prim result is finished by FP64 Newton on the FP64
 *     state (it also bounds W^2 for the FP32 wave speeds); in [1, 1e30].
 *   DG_OPT_ELEMENTS_PER_CTA (default 1): elements per CTA of the mixed stage
 *     kernel, a power of two up to 256 / (n^3 rounded up to 32) (at least 1;
 *     for n = 5, which runs 160 threads per element, up to 2); the result does
 *     not depend on it.
 * Errors: DG_ERR_ARG for an unknown option or a value out of range. */
enum { DG_OPT_TENSOR_CORE_CONTRACTION = 1, DG_OPT_C2P_KAPPA_SWITCH = 2, DG_OPT_ELEMENTS_PER_CTA = 3 };
dg_status dg_mesh_set_option(dg_mesh *mesh, int option, double value);

/* Attach a learned-guess network to a mixed-precision SR mesh (net == NULL
 * detaches it).  With a network attached, every con2prim inside dg_rhs and
 * dg_rk3_step's stages starts its FP32 Newton from the network's guess, computed
 * in the stage kernel for the element's nodes and its neighbours' face nodes --
 * except the first stage of a CFL step, whose input U^n the CFL pass has just
 * solved with the network's guesses: it starts from those pressures.  Without a
 * network, con2prim starts from the pressure of the previous pass (carried in
 * library scratch).  Newton decides the result: the guess changes only the
 * iteration count and the result within the solver's stopping tolerance.  The
 * mesh does not own the network: it must stay alive while the mesh uses it, and
 * training it in place changes the guesses of later calls.  Errors: DG_ERR_ARG
 * when the mesh is not (mixed, SR) and net != NULL.  Not in the paper (an
 * addition to Sec. 2.1.2). */
dg_status dg_mesh_set_c2p_net(dg_mesh *mesh, const dg_c2p_net *net);

/* ---- Ragged ensemble (batching many independent meshes; the paper has no
 * counterpart on one device -- its task runtime spreads many small elements over
 * cores) ----
 * An ensemble advances `count` mixed-precision meshes together, each with its own
 * state U[i] (device, dg_state_size(meshes[i]) doubles) and its own CFL step.  The
 * ensemble keeps the mesh and state pointers: the caller keeps both alive and
 * must not destroy a mesh before the ensemble.  Meshes sharing n, system, flux,
 * limiter, gamma, fix bounds, options and learned-guess network form a group; a
 * step launches one CFL, one stage and one limiter kernel per group (per stage)
 * over the group's concatenated elements.  Per mesh the arithmetic is that of
 * dg_rk3_step(mesh, U, 0, cfl, ...), so results are bitwise those of stepping the
 * meshes one by one with the same per-group options.  Device-side failures set
 * each mesh's status word (dg_sync_status per mesh).
 * Errors: DG_ERR_ARG for NULL or repeated meshes/states, FP64 meshes, or meshes on
 * another device, meshes with the moment limiter (DG_LIMITER_MRS), Newtonian
 * states that are not 16-byte aligned; DG_ERR_CUDA for allocation failures. */
typedef struct dg_ensemble dg_ensemble;
dg_status dg_ensemble_create(dg_mesh *const *meshes, double *const *U, int count, dg_ensemble **out);
void dg_ensemble_destroy(dg_ensemble *ens);
/* Autotune: per group, time the stage kernel (right-hand side only, written to
 * library scratch; the states are not changed) for every elements-per-CTA choice
 * and both volume contractions, and keep the fastest.  Synchronises `stream`. */
dg_status dg_ensemble_tune(dg_ensemble *ens, void *stream);
/* One SSP-RK3 step of every mesh (Sec. 3.4) with dt = cfl dx_min / lambda_max of
 * that mesh.  use_graph = 0: direct launches on `stream`.  1: from the second step
 * on, the step's launches are captured once into a CUDA graph (again when cfl or
 * use_graph changes) and replayed.  2: as 1, but each group's launches run on a
 * stream of the ensemble's own, forked from `stream` and joined back to it (in the
 * graph: parallel branches), so that different groups' kernels overlap; the same
 * results (within about 1 % of the single chain on the GPUs measured).
 * Errors: DG_ERR_ARG for cfl <= 0 or use_graph outside 0..2. */
dg_status dg_ensemble_step(dg_ensemble *ens, double cfl, int use_graph, void *stream);
/* Groups and, for group g, info = (n, system, flux, limiter, meshes, elements,
 * elements per CTA, tensor-core contraction 0/1). */
int dg_ensemble_num_groups(const dg_ensemble *ens);
dg_status dg_ensemble_group_info(const dg_ensemble *ens, int g, long long info[8]);
/* Group of mesh i (-1 for a bad index or ensemble). */
int dg_ensemble_mesh_group(const dg_ensemble *ens, int i);
/* The last step's dt of every mesh into dt (device, count doubles). */
dg_status dg_ensemble_dt(const dg_ensemble *ens, double *dt, void *stream);

/* Synchronise `stream`, then read and clear the mesh's device status word.
 * Returns DG_OK, DG_ERR_C2P, DG_ERR_UNPHYSICAL or DG_ERR_TIMEOUT (a bounded wait
 * for the learned guess's weights ran out; first set), or DG_ERR_CUDA. */
dg_status dg_sync_status(dg_mesh *mesh, void *stream);

/* Per-kernel timing.  When enabled, the library records a CUDA event pair on the
 * call's stream around every kernel it launches for `mesh` and accumulates the
 * elapsed time per kernel class:
 *   0 primitive recovery (incl. SR con2prim and the fused fix), 1 fused RHS +
 *   RK stage, 2 limiter (decision passes of the Newtonian mixed step), 3 SR fix
 *   pass, 4 CFL step, 5 other, 6 the last pass of the Newtonian mixed step
 *   (limiter decisions and the write of U^{n+1}).
 * Calls made while `stream` is being captured into a CUDA graph record their
 * events as external event nodes of that graph; each replay records them again,
 * and each dg_profile_read reports the replay before it (those events stay
 * allocated until dg_mesh_destroy).  dg_profile_read synchronises the events,
 * writes ms[c] (total milliseconds) and launches[c] for c < min(nclass, 7) (host
 * arrays) and resets the counters of the eager launches. */
dg_status dg_profile_enable(dg_mesh *mesh, int on);
dg_status dg_profile_read(dg_mesh *mesh, double *ms, long long *launches, int nclass);

/* Thread-local message of the last failing call (never NULL). */
const char *dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
