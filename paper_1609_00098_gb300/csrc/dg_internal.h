// dg_internal.h -- host-side types shared by the translation units of libdg.
#pragma once

#include <cuda_runtime.h>

#include "../../include/dg.h"

namespace dg {

constexpr int MAXN = 8;  // largest LGL node count per axis

__host__ __device__ constexpr int round_up32(int v) { return (v + 31) / 32 * 32; }

// element coordinates of e (32-bit divisions while e fits, which 64-bit division
// on the GPU, a long software sequence, is not needed for)
__host__ __device__ inline void elem_coords(long long e, const int K[3], int ec[3])
{
    if (e <= 0x7fffffffLL) {
        const int ei = (int)e, q = ei / K[0];
        ec[0] = ei - q * K[0];
        ec[2] = q / K[1];
        ec[1] = q - ec[2] * K[1];
    } else {
        ec[0] = (int)(e % K[0]);
        ec[1] = (int)((e / K[0]) % K[1]);
        ec[2] = (int)(e / ((long long)K[0] * K[1]));
    }
}

// periodic neighbour of element e along axis a in direction s = +-1
__host__ __device__ inline long long elem_neighbour(long long e, const int K[3], int a, int s)
{
    int ec[3];
    elem_coords(e, K, ec);
    ec[a] = (ec[a] + s + K[a]) % K[a];
    return ec[0] + (long long)K[0] * (ec[1] + (long long)K[1] * ec[2]);
}

// Analytic outer boundaries: one ghost element per boundary face holds, on its
// face nodes facing the mesh, the exterior state (U in state layout, P the FP64
// primitives vx, vy, vz, p).  Ghosts of axis a, side s (0 lo, 1 hi) start at
// base[a][s] and are ordered by the face's element coordinates (b, c) =
// (a+1, a+2) mod 3, ec[b] fastest.
struct Ghosts {
    const double *U;
    const double *P;
    int mask;                // bit a: axis a analytic
    long long base[3][2];
};

// Neighbour of e along axis a in direction s: the periodic neighbour (>= 0), or on
// an analytic axis past the boundary -1 - (ghost index).
__host__ __device__ inline long long elem_neighbour_bc(long long e, const int K[3], int a, int s, const Ghosts &G)
{
    int ec[3];
    elem_coords(e, K, ec);
    const int c = ec[a] + s;
    if (((G.mask >> a) & 1) && (c < 0 || c >= K[a])) {
        const int b = (a + 1) % 3, d = (a + 2) % 3;
        return -1 - (G.base[a][s > 0 ? 1 : 0] + ec[b] + (long long)K[b] * ec[d]);
    }
    ec[a] = (c + K[a]) % K[a];
    return ec[0] + (long long)K[0] * (ec[1] + (long long)K[1] * ec[2]);
}

// 1D LGL tables for one n, as passed by value to the kernels.
struct Tables {
    double D[MAXN * MAXN];  // D[i*n+l] = ell_l'(xbar_i)
    double w[MAXN];         // quadrature weights
    double x[MAXN];         // nodes
    double row1[MAXN];      // Legendre P1 coefficient of the nodal interpolant: c1 = sum_i row1[i] u_i
};

// Per-launch arguments of the fused stage kernel (RHS of eq:411 + SSP-RK3 stage
// + limiter summaries).
struct StageArgs {
    const double *Us;      // state the RHS is evaluated on
    const double *Un;      // U^n (stages 2 and 3)
    const double *P;       // primitives (vx, vy, vz, p) of Us, [e][4][node]
    double *out;           // U_{s+1} (mode 1) or dU/dt (mode 0)
    double *S;             // limiter summaries [e][5][10] of out, or nullptr
    unsigned char *unphys; // SR: per-element unphysical flag of out, or nullptr
    const double *dt_ptr;  // device dt (CFL mode) or nullptr
    double dt;             // host dt when dt_ptr == nullptr
    double ca, cb;         // out = ca Un + cb (Us + dt R); first stage: out = Us + dt R
    int first;             // first stage flag
    int mode;              // 0 write RHS, 1 stage update
    int K[3];
    Ghosts gh;             // analytic boundaries (mask 0: periodic)
    double gamma;
    double g[3];           // 2/dx_a
    double lift0[3];       // (2/dx_a)/w_0
    double liftN[3];       // (2/dx_a)/w_N
    Tables T;
};

struct LimitArgs {
    double *U;
    const double *S;
    const unsigned char *unphys;
    unsigned char *troubled;
    long long E;
    int K[3];
    int limiter;
    double tvb_M, beta;
    double dx[3];
    Tables T;
};

struct SummaryArgs {
    const double *U;
    double *S;
    unsigned char *unphys;  // SR: per-element unphysical flag of U, or nullptr
    Tables T;
};

}  // namespace dg

struct dg_mesh {
    dg_mesh_desc d;
    int device;
    int nn;          // nodes per element
    long long E;     // elements
    double dx[3];
    double dxmin;    // smallest node gap
    dg::Tables T;
    // library-owned device scratch
    double *W1, *W2;         // stage states
    double *P;               // primitives [e][4][node]
    double *S;               // limiter summaries [e][5][10]
    unsigned char *unphys;   // per-element SR flags (bit 0: an unphysical node; mixed path bit 1: a node needs the fix)
    unsigned long long *lam; // max wave speed (bit pattern of a non-negative double)
    double *dt;              // device step
    unsigned int *err;       // sticky status word
    // mixed-precision scratch (precision == DG_PRECISION_MIXED)
    float *pbuf[2];          // SR pressures of the last two passes (con2prim warm starts)
    float *pfull;            // SR: the CFL pass's FP32 primitives [e][5][node] of U^n, for stage 1
    int pi, p_valid;         // index of the latest pressure buffer, and whether it holds one
    float kappa_sw;          // conditioning above which FP32 con2prim is polished in FP64
    const dg_c2p_net *net;   // attached learned-guess network (mixed SR path), or nullptr
    int tc_contract;         // mixed volume contraction on the tensor cores (split-BF16x3)
    int epb;                 // mixed stage kernel: elements per CTA
    // Newtonian mixed step in delta form (W1, W2 hold its FP32 stage differences;
    // S holds S(U^n)): FP32 summaries of the differences, the limiter's per-element
    // masks and replacement parameters
    float *ne_SD;            // [e][5][10]
    double *ne_M0;           // [e][5]
    float4 *ne_SH;           // [e][5]
    unsigned char *ne_mask;  // [e]
    // Adams-Bashforth state (dg_ab3_step): the last three right-hand sides (ring),
    // the steps taken since the last reset, and the fixed dt
    double *abL[3];
    long long ab_n;
    double ab_dt;
    double *mrsT;            // MRS limiter: per element U0, w0, w_max, w_min (20 doubles)
    double *t;               // mesh time (device, 1 double)
    dg::Ghosts gh;           // analytic boundaries: ghost exterior states (gh.mask 0: periodic)
    long long nghost;
    // optional per-kernel timing (dg_profile_enable)
    int prof_on;
    void *prof;              // host-side event log, owned by dg_api.cu
};

namespace dg {

// Kernel launchers (defined in the .cu files).
cudaError_t launch_stage_fp64(int n, int system, int flux, const StageArgs &a, long long E, cudaStream_t s);
cudaError_t launch_summaries(int n, const SummaryArgs &a, long long E, cudaStream_t s);
cudaError_t launch_limit(int n, const LimitArgs &a, cudaStream_t s);

cudaError_t launch_primitives(const dg_mesh *m, const double *U, double *P, int fix, double *Ufix,
                              unsigned long long *lam, cudaStream_t s);
cudaError_t launch_fix(const dg_mesh *m, double *U, cudaStream_t s);
cudaError_t launch_mrs(const dg_mesh *m, double *U, unsigned char *troubled, cudaStream_t s);
// Exterior states of the ghosts at time *t + ct * dt (dt = *dt_ptr if given).
cudaError_t launch_exterior(const dg_mesh *m, double ct, const double *dt_ptr, double dt, cudaStream_t s);
// *t += dt (dt = *dt_ptr if given).
cudaError_t launch_time_add(double *t, const double *dt_ptr, double dt, cudaStream_t s);
cudaError_t launch_ab3_combine(double *U, const double *L0, const double *L1, const double *L2, double dt,
                               long long count, cudaStream_t s);
cudaError_t launch_dt(const dg_mesh *m, double cfl, double *dt, cudaStream_t s);
cudaError_t launch_coords(const dg_mesh *m, double *xyz, cudaStream_t s);
cudaError_t launch_prim2con(const dg_mesh *m, const double *prim, double *U, cudaStream_t s);
cudaError_t launch_con2prim(long long count, double gamma, const double *cons, double *prim,
                            const double *guess, int *iters, int *status, cudaStream_t s);

struct MixedArgs;
struct LimitMixedArgs;
struct NeArgs;
struct NeDecideArgs;
struct NeSlot;
struct NeDecideSlot;
// Newtonian mixed step in delta form: stage kernel (stage 0 = right-hand side
// only) and the limiter's decision pass (final_pass: also writes U^{n+1}).
cudaError_t launch_ne_stage(int n, int flux, int stage, const NeArgs &a, cudaStream_t s);
cudaError_t launch_ne_decide(int n, int final_pass, const NeDecideArgs &a, cudaStream_t s);
NeSlot ne_slot(const dg_mesh *m);
NeArgs ne_args(const dg_mesh *m);
// Stage st (0, 1, 2) of the delta-form step on mesh m with state U, and the
// decision pass after it (st = 2: the last pass, which writes U^{n+1}).
NeArgs ne_stage_args(const dg_mesh *m, double *U, int st, bool lim, bool cflmode);
NeDecideSlot ne_decide_slot(const dg_mesh *m);
NeDecideSlot ne_decide_stage_slot(const dg_mesh *m, double *U, int st, bool cflmode, unsigned char *troubled);
NeDecideArgs ne_decide_args(const dg_mesh *m);
cudaError_t launch_stage_mixed(int n, int system, int flux, const MixedArgs &a, cudaStream_t s);
cudaError_t launch_limit_mixed(int n, int system, const LimitMixedArgs &a, cudaStream_t s);
cudaError_t launch_cfl_mixed(const dg_mesh *m, const double *Un, const float *pin, float *pout, float *Pout,
                             float kappa_sw,
                             cudaStream_t s);
struct CflArgs;
struct MeshSlot;
struct LimitSlot;
CflArgs cfl_args(const dg_mesh *m, float kappa_sw);
cudaError_t launch_cfl_batch(int system, const CflArgs &a, long long nchunks, cudaStream_t s);
MixedArgs mixed_args(const dg_mesh *m);
MeshSlot mixed_slot(const dg_mesh *m);
LimitMixedArgs limit_mixed_args(const dg_mesh *m, double *U, unsigned char *troubled);
LimitSlot limit_slot(const dg_mesh *m, double *U, unsigned char *troubled);

// Device view of a learned-guess network: the shared-memory image of its weights
// (a NetWeightsSmem in device memory), and its feature scales.
void net_device_view(const dg_c2p_net *n, const void **img, float sc[6]);

// Host LGL tables (long double Newton; closed-form LGL differentiation matrix).
void lgl_tables(int n, Tables &T);

// Set the thread-local message of dg_last_error and return `st`.
dg_status set_error(dg_status st, const char *msg);

}  // namespace dg
