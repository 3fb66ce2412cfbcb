/*
 * dg_oracle.h -- plain, slow FP64 CPU oracle for the nodal DG hot path of
 * Kidder et al., "SpECTRE: A task-based discontinuous Galerkin code for
 * relativistic astrophysics" (arXiv:1609.00098).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against an obviously correct restatement of the paper.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg may build, load or
 * call it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Layout of a state vector (same convention the paper's eqn:dgNodalInterpolation
 * expansion uses for U_{ijk}): U[e][v][k][j][i], element-major, i fastest,
 * e = ex + Kx*(ey + Ky*ez), v = 0..4 = (rho|D, S_x, S_y, S_z, E|tau).
 *
 * Axes at index >= dim are inactive: one node, one element, no derivative and
 * no faces.  This lets the same code run the paper's 1D tests (Sec. 6.1).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NV 5
#define OR_MAXN 12

typedef struct {
    int system;      /* 0 Newtonian Euler (Sec. 2.1.1), 1 SR hydro in flat space (Sec. 2.1.2) */
    int dim;         /* number of active axes, 1..3 */
    int K[3];        /* elements per axis (inactive axes: 1) */
    int n;           /* LGL nodes per active axis, 2..OR_MAXN */
    int flux;        /* 0 local Lax-Friedrichs (eq:LLF), 1 HLL with Davis speeds (eq:HLL),
                        2 Roe (eq:Roe, Newtonian only) */
    int limiter;     /* 0 none, 1 generalized minmodB troubled-cell limiter ("MinModN"), 2 plain minmod ("MinMod"),
                        3 moment limiter of Moe, Rossmanith and Seal ("MRS", Sec. 3.3.3, Newtonian only) */
    double gamma;    /* ideal-gas adiabatic index */
    double lo[3];    /* periodic box */
    double hi[3];
    double tvb_M;    /* minmodB constant M (eq:MinModB) */
    double beta;     /* slope limiter beta: 2 minmod, 1 MUSCL (Sec. 3.3.1) */
    double d_atm;    /* SR conserved fix: floor on D */
    double tau_atm;  /* SR conserved fix: floor on tau, as a fraction of D */
    double mrs_alpha; /* MRS: alpha~ of the bound widening alpha~ h^{3/2} */
    int bc[3];       /* per axis: 0 periodic, 1 analytic exterior state (Sec. 3.4, boundary faces) */
    int exact;       /* analytic solution supplying exterior states: 0 none, 1 isentropic vortex
                        (eq:isen_vortex; Newtonian, P = rho^gamma) */
    double exact_par[6]; /* isentropic vortex: beta, X0, Y0, U, V, W */
} or_desc;

typedef struct or_mesh or_mesh;

/* 1D LGL tables (Sec. 3.1): nodes x[0..n-1] ascending, weights w[], and the
 * differentiation matrix D[i*n+l] = d(ell_l)/dxbar at x_i (eq:405). */
int  or_lgl(int n, double *x, double *w);
int  or_diffmat(int n, const double *x, double *D);
/* Inverse of the Legendre Vandermonde V[i][m] = P_m(x_i): modal coefficients
 * c_m = sum_i Vinv[m*n+i] u_i.  Used for the limiter's linear part. */
int  or_legendre_vinv(int n, const double *x, double *Vinv);

or_mesh *or_mesh_create(const or_desc *d);
void     or_mesh_destroy(or_mesh *m);
long long or_num_elements(const or_mesh *m);
int      or_nodes_per_element(const or_mesh *m);
/* node coordinates in state order: xyz[0..N), xyz[N..2N), xyz[2N..3N), N = total nodes */
void or_node_coords(const or_mesh *m, double *xyz);

/* primitive (rho, vx, vy, vz, p) <-> conserved, count nodes, SoA rows of length count */
void or_prim2con(int system, double gamma, long long count, const double *prim, double *cons);
/* SR con2prim (Sec. 2.1.2) by safeguarded Newton on the pressure.
 * guess: NULL -> standard guess (gamma-1)*tau.  Returns number of failed nodes.
 * status per node: 0 ok, 1 unphysical input, 2 no convergence. */
long long or_con2prim(long long count, double gamma, const double *cons, double *prim,
                      const double *guess, int *iters, int *status);
/* Mesh-layout primitive recovery: P[e][0..3][node] = (vx, vy, vz, p).  Returns failures. */
long long or_primitives(const or_mesh *m, const double *U, double *P);

/* Point-wise numerical flux along +e_axis (LLF, HLL or Roe) for tests. */
int or_num_flux(int system, double gamma, int flux, int axis, const double *uL, const double *uR,
                double *Fs, double *FL, double *FR, double *speeds);
/* Semi-discrete right-hand side, eq:411, at the mesh time (which only enters
 * through analytic exterior states).  Returns number of con2prim failures. */
long long or_rhs(const or_mesh *m, const double *U, double *dUdt);
/* Mesh time t (0 at creation); or_rk3_step advances it by dt. */
void   or_set_time(or_mesh *m, double t);
double or_get_time(const or_mesh *m);
/* max over nodes and active axes of the largest |characteristic speed| */
double or_lambda_max(const or_mesh *m, const double *U);
/* CFL step Delta t = C * dx_min / lambda_max (Sec. 3.4) */
double or_cfl_dt(const or_mesh *m, const double *U, double cfl);
/* Limiter summaries for each element and variable: [e][v][10] =
 * (U0, face mean lo/hi for x, y, z, slope coefficient c1 for x, y, z) */
void or_limiter_summaries(const or_mesh *m, const double *U, double *S);
/* Apply the limiter in place; troubled[e] gets a bitmask of limited variables. */
long long or_limit(const or_mesh *m, double *U, unsigned char *troubled);
/* SR conserved-variable fix (Sec. 2.1.4), in place.  Returns the number of changed nodes. */
long long or_fix(const or_mesh *m, double *U);
/* One SSP-RK3 step with limiter and fix after each stage.  Returns con2prim failures. */
long long or_rk3_step(or_mesh *m, double *U, double dt, unsigned char *troubled_last);
/* L1 (eq:L1) and L2 norms of U - V per variable with LGL quadrature */
void or_norms(const or_mesh *m, const double *U, const double *V, double *l1, double *l2);
/* sum over the mesh of w J U per variable (discrete conserved totals) */
void or_totals(const or_mesh *m, const double *U, double *tot);

#ifdef __cplusplus
}
#endif
#endif
