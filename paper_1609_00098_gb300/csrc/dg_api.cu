// dg_api.cu -- the C ABI of libdg (declared in include/dg.h): argument checks,
// scratch ownership, LGL tables and the launch sequence of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "dg_mixed.cuh"
#include "dg_physics.cuh"

namespace {

thread_local char g_err[512] = "no error";

dg_status fail(dg_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define DG_CUDA(expr)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return fail(DG_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Per-kernel event log of dg_profile_enable.  Launches recorded while the stream
// is being captured into a CUDA graph get their events as external event nodes of
// the graph: every replay records them again, and each dg_profile_read reports the
// replay before it.  Those events live until the mesh is destroyed.
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    bool graph;
};
struct ProfLog {
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> recs;
};

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive;
}

void prof_record(cudaEvent_t e, cudaStream_t s, bool graph)
{
    if (graph) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
}

cudaEvent_t prof_event(ProfLog *L)
{
    if (!L->pool.empty()) {
        cudaEvent_t e = L->pool.back();
        L->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch `expr` (a cudaError_t expression) with optional event timing of class `cls`.
#define DG_LAUNCH(m, s, cls, expr)                                             \
    do {                                                                       \
        ProfLog *L_ = (m)->prof_on ? (ProfLog *)(m)->prof : nullptr;           \
        cudaEvent_t a_ = nullptr;                                              \
        const bool g_ = L_ && stream_capturing(s);                             \
        if (L_) {                                                              \
            a_ = prof_event(L_);                                               \
            prof_record(a_, (s), g_);                                          \
        }                                                                      \
        DG_CUDA(expr);                                                         \
        if (L_) {                                                              \
            cudaEvent_t b_ = prof_event(L_);                                   \
            prof_record(b_, (s), g_);                                          \
            L_->recs.push_back(ProfRec{(cls), a_, b_, g_});                    \
        }                                                                      \
    } while (0)

// Timing classes of dg_profile_read (PROFILE_CLASSES in the binding); FINAL is the
// last pass of the Newtonian delta-form step, which writes U^{n+1}.
enum { PROF_PRIM = 0, PROF_STAGE = 1, PROF_LIMIT = 2, PROF_FIX = 3, PROF_DT = 4, PROF_OTHER = 5, PROF_FINAL = 6 };

}  // namespace

namespace dg {

// error reporting shared with the other translation units of the library
dg_status set_error(dg_status st, const char *msg) { return fail(st, "%s", msg); }

// LGL tables (Sec. 3.1), computed on the host in FP64 with the textbook steps:
//  * Legendre P_m and P_m' by (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and
//    P'_{k+1} = P'_{k-1} + (2k+1) P_k;
//  * interior nodes = zeros of P_N', Newton from -cos(pi j/N) with P_N'' from
//    Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P, mirrored about 0;
//  * w_j = 2/(N(N+1) P_N(x_j)^2);
//  * D_il = (lambda_l/lambda_i)/(x_i - x_l), lambda_j = 1/prod_{k!=j}(x_j - x_k),
//    D_ii = -sum_{l!=i} D_il (eq:405; D annihilates constants);
//  * row1 = second row of the inverse Legendre Vandermonde V[i][m] = P_m(x_i)
//    (Gauss-Jordan with partial pivoting): c1 = sum_i row1[i] u_i.
// The FP64 kernels use these values directly, so every operation order here is
// fixed and written out.
static void legendre_and_slope(int N, double x, double &P, double &dP)
{
    if (N == 0) {
        P = 1.0;
        dP = 0.0;
        return;
    }
    double a = 1.0, b = x, da = 0.0, db = 1.0;  // P_{k-1}, P_k and their slopes
    for (int k = 1; k < N; ++k) {
        const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        const double dc = da + (2.0 * k + 1.0) * b;
        a = b;
        b = c;
        da = db;
        db = dc;
    }
    P = b;
    dP = db;
}

void lgl_tables(int n, Tables &T)
{
    std::memset(&T, 0, sizeof(T));
    const int N = n - 1;
    double *x = T.x;
    x[0] = -1.0;
    x[N] = 1.0;
    const int half = (N - 1) / 2 + ((N - 1) % 2);
    for (int j = 1; j <= half; ++j) {
        double t = -cos(M_PI * j / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre_and_slope(N, t, P, dP);
            const double d2P = (2.0 * t * dP - N * (N + 1.0) * P) / (1.0 - t * t);
            const double step = -dP / d2P;
            t += step;
            if (fabs(step) < 1e-16) break;
        }
        x[j] = t;
        x[N - j] = -t;
    }
    if (N % 2 == 0) x[N / 2] = 0.0;
    for (int j = 0; j <= N; ++j) {
        double P, dP;
        legendre_and_slope(N, x[j], P, dP);
        T.w[j] = 2.0 / (N * (N + 1.0) * P * P);
    }
    double lam[MAXN];
    for (int j = 0; j < n; ++j) {
        double prod = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) prod *= (x[j] - x[k]);
        lam[j] = 1.0 / prod;
    }
    for (int i = 0; i < n; ++i) {
        double off = 0.0;
        for (int l = 0; l < n; ++l) {
            if (l == i) continue;
            T.D[i * n + l] = (lam[l] / lam[i]) / (x[i] - x[l]);
            off += T.D[i * n + l];
        }
        T.D[i * n + i] = -off;
    }
    // [V | I] -> [I | V^-1]
    double M[MAXN][2 * MAXN];
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) {
            double P, dP;
            legendre_and_slope(m, x[i], P, dP);
            M[i][m] = P;
            M[i][n + m] = (i == m) ? 1.0 : 0.0;
        }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) {
                const double tmp = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = tmp;
            }
        const double inv = 1.0 / M[c][c];
        for (int k = 0; k < 2 * n; ++k) M[c][k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * n; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int i = 0; i < n; ++i) T.row1[i] = M[1][n + i];
}

cudaError_t launch_stage_fp64_n2(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n3(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n4(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n5(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n6(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n7(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_stage_fp64_n8(int, int, const StageArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n2(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n3(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n4(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n5(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n6(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n7(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_summaries_n8(const SummaryArgs &, long long, cudaStream_t);
cudaError_t launch_limit_n2(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n3(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n4(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n5(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n6(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n7(const LimitArgs &, cudaStream_t);
cudaError_t launch_limit_n8(const LimitArgs &, cudaStream_t);

cudaError_t launch_stage_fp64(int n, int system, int flux, const StageArgs &a, long long E, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_stage_fp64_n2(system, flux, a, E, s);
    case 3: return launch_stage_fp64_n3(system, flux, a, E, s);
    case 4: return launch_stage_fp64_n4(system, flux, a, E, s);
    case 5: return launch_stage_fp64_n5(system, flux, a, E, s);
    case 6: return launch_stage_fp64_n6(system, flux, a, E, s);
    case 7: return launch_stage_fp64_n7(system, flux, a, E, s);
    case 8: return launch_stage_fp64_n8(system, flux, a, E, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_summaries(int n, const SummaryArgs &a, long long E, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_summaries_n2(a, E, s);
    case 3: return launch_summaries_n3(a, E, s);
    case 4: return launch_summaries_n4(a, E, s);
    case 5: return launch_summaries_n5(a, E, s);
    case 6: return launch_summaries_n6(a, E, s);
    case 7: return launch_summaries_n7(a, E, s);
    case 8: return launch_summaries_n8(a, E, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_limit(int n, const LimitArgs &a, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_limit_n2(a, s);
    case 3: return launch_limit_n3(a, s);
    case 4: return launch_limit_n4(a, s);
    case 5: return launch_limit_n5(a, s);
    case 6: return launch_limit_n6(a, s);
    case 7: return launch_limit_n7(a, s);
    case 8: return launch_limit_n8(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_set(double *p, double v, cudaStream_t s);

#define DG_DECL_MIXED(NP)                                                                               \
    cudaError_t launch_stage_mixed_n##NP(int, int, const MixedArgs &, cudaStream_t);                    \
    cudaError_t launch_limit_mixed_n##NP(int, const LimitMixedArgs &, cudaStream_t);                    \
    cudaError_t launch_ne_stage_n##NP(int, int, const NeArgs &, cudaStream_t);                          \
    cudaError_t launch_ne_decide_n##NP(int, const NeDecideArgs &, cudaStream_t);
DG_DECL_MIXED(2)
DG_DECL_MIXED(3)
DG_DECL_MIXED(4)
DG_DECL_MIXED(5)
DG_DECL_MIXED(6)
DG_DECL_MIXED(7)
DG_DECL_MIXED(8)

cudaError_t launch_stage_mixed(int n, int system, int flux, const MixedArgs &a, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_stage_mixed_n2(system, flux, a, s);
    case 3: return launch_stage_mixed_n3(system, flux, a, s);
    case 4: return launch_stage_mixed_n4(system, flux, a, s);
    case 5: return launch_stage_mixed_n5(system, flux, a, s);
    case 6: return launch_stage_mixed_n6(system, flux, a, s);
    case 7: return launch_stage_mixed_n7(system, flux, a, s);
    case 8: return launch_stage_mixed_n8(system, flux, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_limit_mixed(int n, int system, const LimitMixedArgs &a, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_limit_mixed_n2(system, a, s);
    case 3: return launch_limit_mixed_n3(system, a, s);
    case 4: return launch_limit_mixed_n4(system, a, s);
    case 5: return launch_limit_mixed_n5(system, a, s);
    case 6: return launch_limit_mixed_n6(system, a, s);
    case 7: return launch_limit_mixed_n7(system, a, s);
    case 8: return launch_limit_mixed_n8(system, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_ne_stage(int n, int flux, int stage, const NeArgs &a, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_ne_stage_n2(flux, stage, a, s);
    case 3: return launch_ne_stage_n3(flux, stage, a, s);
    case 4: return launch_ne_stage_n4(flux, stage, a, s);
    case 5: return launch_ne_stage_n5(flux, stage, a, s);
    case 6: return launch_ne_stage_n6(flux, stage, a, s);
    case 7: return launch_ne_stage_n7(flux, stage, a, s);
    case 8: return launch_ne_stage_n8(flux, stage, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_ne_decide(int n, int final_pass, const NeDecideArgs &a, cudaStream_t s)
{
    switch (n) {
    case 2: return launch_ne_decide_n2(final_pass, a, s);
    case 3: return launch_ne_decide_n3(final_pass, a, s);
    case 4: return launch_ne_decide_n4(final_pass, a, s);
    case 5: return launch_ne_decide_n5(final_pass, a, s);
    case 6: return launch_ne_decide_n6(final_pass, a, s);
    case 7: return launch_ne_decide_n7(final_pass, a, s);
    case 8: return launch_ne_decide_n8(final_pass, a, s);
    }
    return cudaErrorInvalidValue;
}

// Per-mesh slot of the Newtonian delta-form stage kernel (pointers filled in by
// the caller) and the group-level arguments for meshes like m.
NeSlot ne_slot(const dg_mesh *m)
{
    NeSlot sl;
    std::memset(&sl, 0, sizeof(sl));
    sl.gh = m->gh;
    sl.err = m->err;
    const int n = m->d.n;
    for (int ax = 0; ax < 3; ++ax) {
        sl.K[ax] = m->d.K[ax];
        const double g = 2.0 / m->dx[ax];
        sl.g[ax] = (float)g;
        sl.lift0[ax] = (float)(g / m->T.w[0]);
        sl.liftN[ax] = (float)(g / m->T.w[n - 1]);
    }
    return sl;
}

NeArgs ne_args(const dg_mesh *m)
{
    NeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.one = ne_slot(m);
    a.nslots = 1;
    a.nelem = m->E;
    a.gamma = (float)m->d.gamma;
    for (int i = 0; i < MAXN * MAXN; ++i) a.D[i] = (float)m->T.D[i];
    const int n = m->d.n;
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) a.DT[l * n + i] = a.D[i * n + l];
    for (int i = 0; i < MAXN; ++i) {
        a.x[i] = (float)m->T.x[i];
        a.w[i] = (float)m->T.w[i];
        a.row1[i] = (float)m->T.row1[i];
        a.wh[i] = a.w[i];
        a.wl[i] = (float)(m->T.w[i] - (double)a.wh[i]);
    }
    return a;
}

// Stage st (0, 1, 2) of the delta-form step on mesh m with state U: the FP32
// stage differences live in W1 (D1, then D3) and W2 (D2); S holds S(U^n).
NeArgs ne_stage_args(const dg_mesh *m, double *U, int st, bool lim, bool cflmode)
{
    float *D1 = reinterpret_cast<float *>(m->W1), *D2 = reinterpret_cast<float *>(m->W2);
    static const float cb[3] = {1.0f, 0.25f, (float)(2.0 / 3.0)};
    NeArgs a = ne_args(m);
    a.one.Un = U;
    a.one.dt_ptr = cflmode ? m->dt : nullptr;
    a.one.Din = st == 1 ? D1 : st == 2 ? D2 : nullptr;
    a.one.Dout = st == 1 ? D2 : D1;
    a.cb = cb[st];
    a.one.mask = (lim && st > 0) ? m->ne_mask : nullptr;
    a.one.SH = m->ne_SH;
    a.one.M0 = m->ne_M0;
    a.one.SN = (lim && st == 0) ? m->S : nullptr;
    a.one.SD = lim ? m->ne_SD : nullptr;
    a.one.lam = (cflmode && st == 0) ? m->lam : nullptr;
    return a;
}

NeDecideSlot ne_decide_slot(const dg_mesh *m)
{
    NeDecideSlot sl;
    std::memset(&sl, 0, sizeof(sl));
    sl.SN = m->S;
    sl.SD = m->ne_SD;
    sl.mask = m->ne_mask;
    sl.M0 = m->ne_M0;
    sl.SH = m->ne_SH;
    for (int ax = 0; ax < 3; ++ax) {
        sl.K[ax] = m->d.K[ax];
        sl.tvb_f[ax] = (float)(m->d.tvb_M * m->dx[ax] * m->dx[ax]);
        sl.two_inv_dx_f[ax] = (float)(2.0 / m->dx[ax]);
        sl.beta_dx_f[ax] = (float)(m->d.beta / m->dx[ax]);
        sl.hdx_f[ax] = (float)(0.5 * m->dx[ax]);
    }
    return sl;
}

// Decision pass after stage st (0, 1: limiter only; 2: also writes U^{n+1}).
NeDecideSlot ne_decide_stage_slot(const dg_mesh *m, double *U, int st, bool cflmode, unsigned char *troubled)
{
    NeDecideSlot sl = ne_decide_slot(m);
    sl.dt_ptr = cflmode ? m->dt : nullptr;
    if (st == 2) {
        sl.U = U;
        sl.D3 = reinterpret_cast<const float *>(m->W1);
        sl.troubled = troubled;
    }
    return sl;
}

NeDecideArgs ne_decide_args(const dg_mesh *m)
{
    NeDecideArgs a;
    std::memset(&a, 0, sizeof(a));
    a.one = ne_decide_slot(m);
    a.nslots = 1;
    a.nelem = m->E;
    a.limiter = m->d.limiter;
    for (int i = 0; i < MAXN; ++i) a.x[i] = (float)m->T.x[i];
    return a;
}

// Per-mesh slot of a mixed stage launch (pointers filled in by the caller).
MeshSlot mixed_slot(const dg_mesh *m)
{
    MeshSlot sl;
    std::memset(&sl, 0, sizeof(sl));
    for (int ax = 0; ax < 3; ++ax) {
        sl.K[ax] = m->d.K[ax];
        const double g = 2.0 / m->dx[ax];
        sl.g[ax] = (float)g;
        sl.lift0[ax] = (float)(g / m->T.w[0]);
        sl.liftN[ax] = (float)(g / m->T.w[m->d.n - 1]);
    }
    sl.err = m->err;
    sl.gh = m->gh;
    return sl;
}

// Group-level arguments of a mixed stage launch for meshes like m (n, system,
// gamma, fix bounds, options, network); one element per CTA, no slot table.
MixedArgs mixed_args(const dg_mesh *m)
{
    MixedArgs a;
    std::memset(&a, 0, sizeof(a));
    a.one = mixed_slot(m);
    a.nslots = 1;
    a.nelem = m->E;
    a.epb = m->epb > 0 ? m->epb : 1;
    a.lim = m->d.limiter != 0;
    a.gamma = (float)m->d.gamma;
    a.gamma_d = m->d.gamma;
    a.kappa_sw = m->kappa_sw;
    a.tc = m->tc_contract;
    a.d_atm = m->d.d_atm;
    a.tau_atm = m->d.tau_atm;
    if (m->net && m->d.system == 1) {
        const void *img = nullptr;
        net_device_view(m->net, &img, a.net_sc);
        a.netImg = static_cast<const NetWeightsSmem *>(img);
    }
    for (int i = 0; i < MAXN * MAXN; ++i) a.D32[i] = (float)m->T.D[i];
    for (int i = 0; i < MAXN; ++i) {
        a.w64[i] = m->T.w[i];
        a.row1_64[i] = m->T.row1[i];
    }
    return a;
}

LimitSlot limit_slot(const dg_mesh *m, double *U, unsigned char *troubled)
{
    LimitSlot l;
    std::memset(&l, 0, sizeof(l));
    l.U = U;
    l.S = m->S;
    l.flags = (m->d.system == 1) ? m->unphys : nullptr;
    l.troubled = troubled;
    for (int ax = 0; ax < 3; ++ax) {
        l.K[ax] = m->d.K[ax];
        l.tvb[ax] = m->d.tvb_M * m->dx[ax] * m->dx[ax];
        l.inv_dx[ax] = 1.0 / m->dx[ax];
        l.beta_dx[ax] = m->d.beta / m->dx[ax];
        l.hdx[ax] = 0.5 * m->dx[ax];
    }
    return l;
}

LimitMixedArgs limit_mixed_args(const dg_mesh *m, double *U, unsigned char *troubled)
{
    LimitMixedArgs l;
    std::memset(&l, 0, sizeof(l));
    l.one = limit_slot(m, U, troubled);
    l.nslots = 1;
    l.E = m->E;
    l.limiter = m->d.limiter;
    l.d_atm = m->d.d_atm;
    l.tau_atm = m->d.tau_atm;
    for (int i = 0; i < MAXN; ++i) l.x[i] = m->T.x[i];
    return l;
}

}  // namespace dg

using namespace dg;

namespace {

StageArgs stage_args(const dg_mesh *m)
{
    StageArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int ax = 0; ax < 3; ++ax) {
        a.K[ax] = m->d.K[ax];
        a.g[ax] = 2.0 / m->dx[ax];
        a.lift0[ax] = a.g[ax] / m->T.w[0];
        a.liftN[ax] = a.g[ax] / m->T.w[m->d.n - 1];
    }
    a.gamma = m->d.gamma;
    a.gh = m->gh;
    a.T = m->T;
    return a;
}

LimitArgs limit_args(const dg_mesh *m, double *U, unsigned char *troubled)
{
    LimitArgs l;
    std::memset(&l, 0, sizeof(l));
    l.U = U;
    l.S = m->S;
    l.unphys = (m->d.system == 1) ? m->unphys : nullptr;
    l.troubled = troubled;
    l.E = m->E;
    for (int ax = 0; ax < 3; ++ax) {
        l.K[ax] = m->d.K[ax];
        l.dx[ax] = m->dx[ax];
    }
    l.limiter = m->d.limiter;
    l.tvb_M = m->d.tvb_M;
    l.beta = m->d.beta;
    l.T = m->T;
    return l;
}

dg_status check_mesh(const dg_mesh *m)
{
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
        return fail(DG_ERR_ARG, "mesh was created on device %d, current device is %d", m->device, dev);
    return DG_OK;
}

void free_scratch(dg_mesh *m)
{
    if (m->prof) {
        ProfLog *L = (ProfLog *)m->prof;
        for (auto &r : L->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : L->pool) cudaEventDestroy(e);
        delete L;
        m->prof = nullptr;
    }
    cudaFree(m->W1);
    cudaFree(m->W2);
    cudaFree(m->ne_SD);
    cudaFree(m->ne_M0);
    cudaFree(m->ne_SH);
    cudaFree(m->ne_mask);
    cudaFree(m->pbuf[0]);
    cudaFree(m->pbuf[1]);
    cudaFree(m->pfull);
    for (int i = 0; i < 3; ++i) cudaFree(m->abL[i]);
    cudaFree(m->P);
    cudaFree(m->S);
    cudaFree(m->mrsT);
    cudaFree(m->t);
    cudaFree(const_cast<double *>(m->gh.U));
    cudaFree(const_cast<double *>(m->gh.P));
    cudaFree(m->unphys);
    cudaFree(m->lam);
    cudaFree(m->dt);
    cudaFree(m->err);
}

}  // namespace

extern "C" {

const char *dg_last_error(void) { return g_err; }

dg_status dg_mesh_create(const dg_mesh_desc *d, dg_mesh **out)
{
    if (!d || !out) return fail(DG_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->system != 0 && d->system != 1) return fail(DG_ERR_ARG, "system must be 0 or 1");
    if (d->n < 2 || d->n > MAXN) return fail(DG_ERR_ARG, "n must be in 2..%d", MAXN);
    if (d->flux != 0 && d->flux != 1 && !(d->flux == 2 && d->system == 0))
        return fail(DG_ERR_ARG, "flux must be 0 (LLF), 1 (HLL) or, for the Newtonian system, 2 (Roe)");
    if (d->limiter < 0 || d->limiter > 3) return fail(DG_ERR_ARG, "limiter must be 0, 1, 2 or 3");
    if (d->limiter == DG_LIMITER_MRS && (d->system != 0 || !(d->mrs_alpha >= 0.0)))
        return fail(DG_ERR_ARG, "the moment limiter needs the Newtonian system and mrs_alpha >= 0");
    int analytic = 0;
    for (int a = 0; a < 3; ++a) {
        if (d->bc[a] != DG_BC_PERIODIC && d->bc[a] != DG_BC_ANALYTIC) return fail(DG_ERR_ARG, "bc[%d] must be 0 or 1", a);
        analytic |= d->bc[a];
    }
    if (d->exact != DG_EXACT_NONE && d->exact != DG_EXACT_ISENTROPIC_VORTEX) return fail(DG_ERR_ARG, "exact must be 0 or 1");
    if (analytic && (d->system != 0 || d->exact != DG_EXACT_ISENTROPIC_VORTEX || d->limiter != DG_LIMITER_NONE))
        return fail(DG_ERR_ARG, "analytic boundaries need the Newtonian system, the isentropic vortex and no limiter");
    if (d->precision != 0 && d->precision != 1) return fail(DG_ERR_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (!(d->gamma > 1.0)) return fail(DG_ERR_ARG, "gamma must be > 1");
    if (!(d->beta > 0.0) || !(d->tvb_M >= 0.0)) return fail(DG_ERR_ARG, "beta must be > 0 and tvb_M >= 0");
    long long E = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->K[a] < 1) return fail(DG_ERR_ARG, "K[%d] must be >= 1", a);
        if (!(d->hi[a] > d->lo[a])) return fail(DG_ERR_ARG, "hi[%d] must exceed lo[%d]", a, a);
        E *= d->K[a];
        if (E > (1LL << 40)) return fail(DG_ERR_ARG, "too many elements");
    }
    if (E > 0x7fffffffLL) return fail(DG_ERR_ARG, "at most 2^31-1 elements (one CTA per element)");
    dg_mesh *m = new dg_mesh;
    std::memset(m, 0, sizeof(*m));
    m->d = *d;
    cudaGetDevice(&m->device);
    m->nn = d->n * d->n * d->n;
    m->E = E;
    lgl_tables(d->n, m->T);
    m->dxmin = INFINITY;
    for (int a = 0; a < 3; ++a) {
        m->dx[a] = (d->hi[a] - d->lo[a]) / d->K[a];
        const double h = 0.5 * m->dx[a] * (m->T.x[1] - m->T.x[0]);
        if (h < m->dxmin) m->dxmin = h;
    }
    const size_t state = sizeof(double) * (size_t)E * 5 * m->nn;
    const bool mixed = d->precision == DG_PRECISION_MIXED;
    m->kappa_sw = 10.0f;
    m->tc_contract = 0;
    m->epb = 1;
    cudaError_t st = cudaSuccess;
    st = st ? st : cudaMalloc(&m->W1, state);
    st = st ? st : cudaMalloc(&m->W2, state);
    if (mixed && d->system == 0) {
        st = st ? st : cudaMalloc(&m->ne_SD, sizeof(float) * (size_t)E * 50);
        st = st ? st : cudaMalloc(&m->ne_M0, sizeof(double) * (size_t)E * 5);
        st = st ? st : cudaMalloc(&m->ne_SH, sizeof(float4) * (size_t)E * 5);
        st = st ? st : cudaMalloc(&m->ne_mask, (size_t)E);
    }
    if (mixed && d->system == 1) {
        st = st ? st : cudaMalloc(&m->pbuf[0], sizeof(float) * (size_t)E * m->nn);
        st = st ? st : cudaMalloc(&m->pbuf[1], sizeof(float) * (size_t)E * m->nn);
        st = st ? st : cudaMalloc(&m->pfull, sizeof(float) * 5 * (size_t)E * m->nn);
    }
    st = st ? st : cudaMalloc(&m->P, sizeof(double) * (size_t)E * 4 * m->nn);
    st = st ? st : cudaMalloc(&m->S, sizeof(double) * (size_t)E * 50);
    if (d->limiter == DG_LIMITER_MRS) st = st ? st : cudaMalloc(&m->mrsT, sizeof(double) * (size_t)E * 20);
    st = st ? st : cudaMalloc(&m->t, sizeof(double));
    if (st == cudaSuccess) st = cudaMemset(m->t, 0, sizeof(double));
    for (int a = 0; a < 3; ++a) {
        if (d->bc[a] != DG_BC_ANALYTIC) continue;
        const long long cnt = (long long)d->K[(a + 1) % 3] * d->K[(a + 2) % 3];
        m->gh.mask |= 1 << a;
        m->gh.base[a][0] = m->nghost;
        m->gh.base[a][1] = m->nghost + cnt;
        m->nghost += 2 * cnt;
    }
    if (m->nghost) {
        double *gU = nullptr, *gP = nullptr;
        st = st ? st : cudaMalloc(&gU, sizeof(double) * (size_t)m->nghost * 5 * m->nn);
        st = st ? st : cudaMalloc(&gP, sizeof(double) * (size_t)m->nghost * 4 * m->nn);
        m->gh.U = gU;
        m->gh.P = gP;
        if (st == cudaSuccess) st = cudaMemset(gU, 0, sizeof(double) * (size_t)m->nghost * 5 * m->nn);
        if (st == cudaSuccess) st = cudaMemset(gP, 0, sizeof(double) * (size_t)m->nghost * 4 * m->nn);
    }
    st = st ? st : cudaMalloc(&m->unphys, (size_t)E);
    st = st ? st : cudaMalloc(&m->lam, sizeof(unsigned long long));
    st = st ? st : cudaMalloc(&m->dt, sizeof(double));
    st = st ? st : cudaMalloc(&m->err, sizeof(unsigned int));
    if (st == cudaSuccess) st = cudaMemset(m->err, 0, sizeof(unsigned int));
    if (st == cudaSuccess) st = cudaMemset(m->unphys, 0, (size_t)E);
    if (st != cudaSuccess) {
        free_scratch(m);
        delete m;
        cudaGetLastError();
        return fail(st == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA, "mesh scratch: %s",
                    cudaGetErrorString(st));
    }
    *out = m;
    return DG_OK;
}

void dg_mesh_destroy(dg_mesh *m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    free_scratch(m);
    delete m;
}

dg_status dg_lgl_tables(int n, double *x, double *w, double *D, double *row1)
{
    if (n < 2 || n > MAXN) return fail(DG_ERR_ARG, "n must be in 2..%d", MAXN);
    if (!x || !w || !D || !row1) return fail(DG_ERR_ARG, "table pointers must not be NULL");
    Tables T;
    lgl_tables(n, T);
    for (int i = 0; i < n; ++i) {
        x[i] = T.x[i];
        w[i] = T.w[i];
        row1[i] = T.row1[i];
    }
    for (int i = 0; i < n * n; ++i) D[i] = T.D[i];
    return DG_OK;
}

long long dg_state_size(const dg_mesh *m) { return m ? m->E * 5 * m->nn : 0; }
long long dg_num_nodes(const dg_mesh *m) { return m ? m->E * m->nn : 0; }

dg_status dg_node_coords(const dg_mesh *m, double *xyz, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!xyz) return fail(DG_ERR_ARG, "xyz is NULL");
    DG_CUDA(launch_coords(m, xyz, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_prim2con(const dg_mesh *m, const double *prim, double *U, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!prim || !U || (const void *)prim == (const void *)U) return fail(DG_ERR_ARG, "prim and U must be distinct, non-NULL");
    DG_CUDA(launch_prim2con(m, prim, U, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_primitives(dg_mesh *m, const double *U, double *P, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U || !P) return fail(DG_ERR_ARG, "U and P must not be NULL");
    DG_CUDA(launch_primitives(m, U, P, 0, nullptr, nullptr, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_rhs(dg_mesh *m, const double *U, double *dUdt, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U || !dUdt || U == dUdt) return fail(DG_ERR_ARG, "U and dUdt must be distinct, non-NULL");
    const bool ne_mixed = m->d.precision == DG_PRECISION_MIXED && m->d.system == 0;
    if (ne_mixed && (reinterpret_cast<uintptr_t>(U) & 15u))
        return fail(DG_ERR_ARG, "the mixed Newtonian path needs U 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_exterior(m, 0.0, nullptr, 0.0, s));
    if (ne_mixed) {
        NeArgs a = ne_args(m);
        a.one.Un = U;
        a.one.rhs = dUdt;
        DG_LAUNCH(m, s, PROF_STAGE, launch_ne_stage(m->d.n, m->d.flux, 0, a, s));
        return DG_OK;
    }
    if (m->d.precision == DG_PRECISION_MIXED) {
        MixedArgs a = mixed_args(m);
        a.one.Us = U;
        a.one.Un = U;
        a.one.out = dUdt;
        a.mode = 0;
        a.lim = 0;
        DG_LAUNCH(m, s, PROF_STAGE, launch_stage_mixed(m->d.n, m->d.system, m->d.flux, a, s));
        return DG_OK;
    }
    DG_LAUNCH(m, s, PROF_PRIM, launch_primitives(m, U, m->P, 0, nullptr, nullptr, s));
    StageArgs a = stage_args(m);
    a.Us = U;
    a.Un = U;
    a.P = m->P;
    a.out = dUdt;
    a.mode = 0;
    DG_LAUNCH(m, s, PROF_STAGE, launch_stage_fp64(m->d.n, m->d.system, m->d.flux, a, m->E, s));
    return DG_OK;
}

dg_status dg_compute_dt(dg_mesh *m, const double *U, double cfl, double *dt, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U || !dt) return fail(DG_ERR_ARG, "U and dt must not be NULL");
    if (!(cfl > 0.0)) return fail(DG_ERR_ARG, "cfl must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    DG_CUDA(cudaMemsetAsync(m->lam, 0, sizeof(unsigned long long), s));
    DG_CUDA(launch_primitives(m, U, m->P, 0, nullptr, m->lam, s));
    DG_CUDA(launch_dt(m, cfl, dt, s));
    return DG_OK;
}

// Newtonian mixed-precision step in delta form (dg_ne_mixed.cuh): three stage
// kernels on FP32 stage differences D1 (in W1), D2 (in W2), D3 (in W1), the
// limiter's decision pass after stages 1 and 2, and a last pass that writes
// U^{n+1} = U^n + D3 in place (replaced where the stage-3 limiter acts).  Stage 1
// also takes the CFL maximum of U^n and S(U^n).
static dg_status rk3_step_ne(dg_mesh *m, double *U, double dt, double cfl, double *dt_used, unsigned char *troubled,
                             cudaStream_t s)
{
    const bool lim = m->d.limiter != 0;
    const bool cflmode = cfl > 0.0;
    const double *dtp = cflmode ? m->dt : nullptr;
    if (cflmode) DG_CUDA(cudaMemsetAsync(m->lam, 0, sizeof(unsigned long long), s));
    const double ct[3] = {0.0, 1.0, 0.5};  // stage times t + ct dt (analytic boundaries)
    for (int st = 0; st < 3; ++st) {
        if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_exterior(m, ct[st], dtp, dt, s));
        NeArgs a = ne_stage_args(m, U, st, lim, cflmode);
        a.one.dt = dt;
        DG_LAUNCH(m, s, PROF_STAGE, launch_ne_stage(m->d.n, m->d.flux, st + 1, a, s));
        if (st == 0 && cflmode) DG_LAUNCH(m, s, PROF_DT, launch_dt(m, cfl, m->dt, s));
        NeDecideArgs d = ne_decide_args(m);
        d.one = ne_decide_stage_slot(m, U, st, cflmode, st == 2 ? troubled : nullptr);
        d.one.dt = dt;
        d.scale_dt = st == 0;
        if (st < 2) {
            if (lim) DG_LAUNCH(m, s, PROF_LIMIT, launch_ne_decide(m->d.n, 0, d, s));
        } else {
            DG_LAUNCH(m, s, PROF_FINAL, launch_ne_decide(m->d.n, 1, d, s));
        }
    }
    if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_time_add(m->t, dtp, dt, s));
    if (dt_used) {
        if (cflmode) DG_CUDA(cudaMemcpyAsync(dt_used, m->dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
        else DG_CUDA(launch_set(dt_used, dt, s));
    }
    return DG_OK;
}

// Mixed-precision step: an optional CFL pass, then three fused stages on FP64
// stage states, U -> W1 -> W2 -> U, each followed by the limiter when one is
// selected (the limiter pass also applies the SR conserved fix).
static dg_status rk3_step_mixed(dg_mesh *m, double *U, double dt, double cfl, double *dt_used,
                                unsigned char *troubled, cudaStream_t s)
{
    const bool sr = m->d.system == 1;
    const bool lim = m->d.limiter != 0;
    const bool cflmode = cfl > 0.0;
    // with a learned guess attached, no pressures are carried between steps.  The
    // CFL pass solves con2prim on U^n, the very state stage 1 starts from, and
    // stage 1 takes those primitives (own and neighbour face nodes) instead of
    // solving again
    const bool carry = sr && m->net == nullptr;
    const bool pgiven = sr && cflmode;
    MixedArgs a = mixed_args(m);
    a.one.Un = U;
    a.one.dt = dt;
    a.one.dt_ptr = cflmode ? m->dt : nullptr;
    a.one.S = lim ? m->S : nullptr;
    a.one.flags = (lim && sr) ? m->unphys : nullptr;
    a.mode = 1;
    float *latest = (carry && m->p_valid) ? m->pbuf[m->pi] : nullptr;
    if (cflmode) {
        DG_CUDA(cudaMemsetAsync(m->lam, 0, sizeof(unsigned long long), s));
        DG_LAUNCH(m, s, PROF_PRIM,
                  launch_cfl_mixed(m, U, latest, carry ? m->pbuf[1 - m->pi] : nullptr, pgiven ? m->pfull : nullptr,
                                   m->kappa_sw, s));
        if (carry) {
            m->pi = 1 - m->pi;
            latest = m->pbuf[m->pi];
        }
        DG_LAUNCH(m, s, PROF_DT, launch_dt(m, cfl, m->dt, s));
    }
    double *ins[3] = {U, m->W1, m->W2};
    double *outs[3] = {m->W1, m->W2, U};
    const float ca[3] = {0.0f, 0.75f, (float)(1.0 / 3.0)};
    const float cb[3] = {1.0f, 0.25f, (float)(2.0 / 3.0)};
    const double ct[3] = {0.0, 1.0, 0.5};  // stage times t + ct dt (analytic boundaries)
    for (int st = 0; st < 3; ++st) {
        if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_exterior(m, ct[st], a.one.dt_ptr, dt, s));
        a.one.Us = ins[st];
        a.one.out = outs[st];
        a.first = st == 0;
        a.ca = ca[st];
        a.cb = cb[st];
        a.one.pin = latest;
        a.one.pout = carry ? m->pbuf[1 - m->pi] : nullptr;
        a.epb = m->epb > 0 ? m->epb : 1;
        MixedArgs as = a;
        if (pgiven && st == 0) {
            as.netImg = nullptr;
            as.one.Pin = m->pfull;
        }
        DG_LAUNCH(m, s, PROF_STAGE, launch_stage_mixed(m->d.n, m->d.system, m->d.flux, as, s));
        if (carry) {
            m->pi = 1 - m->pi;
            latest = m->pbuf[m->pi];
        }
        if (lim && m->d.limiter == DG_LIMITER_MRS) {
            DG_LAUNCH(m, s, PROF_LIMIT, launch_mrs(m, outs[st], st == 2 ? troubled : nullptr, s));
        } else if (lim) {
            LimitMixedArgs l = limit_mixed_args(m, outs[st], st == 2 ? troubled : nullptr);
            DG_LAUNCH(m, s, PROF_LIMIT, launch_limit_mixed(m->d.n, m->d.system, l, s));
        }
    }
    m->p_valid = carry ? 1 : 0;
    if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_time_add(m->t, a.one.dt_ptr, dt, s));
    if (dt_used) {
        if (cflmode) DG_CUDA(cudaMemcpyAsync(dt_used, m->dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
        else DG_CUDA(launch_set(dt_used, dt, s));
    }
    return DG_OK;
}

dg_status dg_rk3_step(dg_mesh *m, double *U, double dt, double cfl, double *dt_used, unsigned char *troubled,
                      void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U) return fail(DG_ERR_ARG, "U is NULL");
    const bool cflmode = cfl > 0.0;
    if (!cflmode && !(dt > 0.0)) return fail(DG_ERR_ARG, "need dt > 0 or cfl > 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->d.precision == DG_PRECISION_MIXED && m->d.system == 0 && m->d.limiter != DG_LIMITER_MRS) {
        if (reinterpret_cast<uintptr_t>(U) & 15u)
            return fail(DG_ERR_ARG, "the mixed Newtonian path needs U 16-byte aligned");
        return rk3_step_ne(m, U, dt, cfl, dt_used, troubled, s);
    }
    if (m->d.precision == DG_PRECISION_MIXED) return rk3_step_mixed(m, U, dt, cfl, dt_used, troubled, s);
    const bool sr = m->d.system == 1;
    const bool lim = m->d.limiter != 0;
    StageArgs a = stage_args(m);
    a.P = m->P;
    a.mode = 1;
    a.dt = dt;
    a.dt_ptr = cflmode ? m->dt : nullptr;
    a.S = lim ? m->S : nullptr;
    a.unphys = (lim && sr) ? m->unphys : nullptr;
    if (cflmode) DG_CUDA(cudaMemsetAsync(m->lam, 0, sizeof(unsigned long long), s));

    double *ins[3] = {U, m->W1, m->W2};
    double *outs[3] = {m->W1, m->W2, U};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const double ct[3] = {0.0, 1.0, 0.5};  // stage times t + ct dt (analytic boundaries)
    for (int st = 0; st < 3; ++st) {
        // the SR fix of the previous stage's result is fused into its primitive pass
        DG_LAUNCH(m, s, PROF_PRIM,
                  launch_primitives(m, ins[st], m->P, sr && st > 0, ins[st], (cflmode && st == 0) ? m->lam : nullptr, s));
        if (cflmode && st == 0) DG_LAUNCH(m, s, PROF_DT, launch_dt(m, cfl, m->dt, s));
        if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_exterior(m, ct[st], a.dt_ptr, dt, s));
        a.Us = ins[st];
        a.Un = U;
        a.out = outs[st];
        a.first = st == 0;
        a.ca = ca[st];
        a.cb = cb[st];
        DG_LAUNCH(m, s, PROF_STAGE, launch_stage_fp64(m->d.n, m->d.system, m->d.flux, a, m->E, s));
        if (lim && m->d.limiter == DG_LIMITER_MRS) {
            DG_LAUNCH(m, s, PROF_LIMIT, launch_mrs(m, outs[st], st == 2 ? troubled : nullptr, s));
        } else if (lim) {
            LimitArgs l = limit_args(m, outs[st], st == 2 ? troubled : nullptr);
            DG_LAUNCH(m, s, PROF_LIMIT, launch_limit(m->d.n, l, s));
        }
    }
    if (sr) DG_LAUNCH(m, s, PROF_FIX, launch_fix(m, U, s));
    if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_time_add(m->t, a.dt_ptr, dt, s));
    if (dt_used) {
        if (cflmode) DG_CUDA(cudaMemcpyAsync(dt_used, m->dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
        else DG_CUDA(launch_set(dt_used, dt, s));
    }
    return DG_OK;
}

dg_status dg_ab3_reset(dg_mesh *m)
{
    if (dg_status s = check_mesh(m)) return s;
    m->ab_n = 0;
    return DG_OK;
}

dg_status dg_ab3_step(dg_mesh *m, double *U, double dt, unsigned char *troubled, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U) return fail(DG_ERR_ARG, "U is NULL");
    if (!(dt > 0.0)) return fail(DG_ERR_ARG, "need dt > 0");
    if (m->ab_n > 0 && dt != m->ab_dt)
        return fail(DG_ERR_ARG, "Adams-Bashforth needs a fixed dt: call dg_ab3_reset before changing it");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t state = sizeof(double) * (size_t)m->E * 5 * m->nn;
    for (int i = 0; i < 3; ++i)
        if (!m->abL[i]) DG_CUDA(cudaMalloc(&m->abL[i], state));
    double *Ln = m->abL[m->ab_n % 3];
    if (dg_status st = dg_rhs(m, U, Ln, stream)) return st;
    if (m->ab_n < 2) {
        // start-up: SSP-RK3 steps record the right-hand sides AB3 needs
        if (dg_status st = dg_rk3_step(m, U, dt, 0.0, nullptr, troubled, stream)) return st;
    } else {
        const double *L1 = m->abL[(m->ab_n - 1) % 3], *L2 = m->abL[(m->ab_n - 2) % 3];
        DG_LAUNCH(m, s, PROF_OTHER, launch_ab3_combine(U, Ln, L1, L2, dt, m->E * 5 * m->nn, s));
        if (dg_status st = dg_limit(m, U, troubled, stream)) return st;
        if (m->d.system == 1)
            if (dg_status st = dg_fix(m, U, stream)) return st;
        if (m->gh.mask) DG_LAUNCH(m, s, PROF_OTHER, launch_time_add(m->t, nullptr, dt, s));
    }
    m->ab_n += 1;
    m->ab_dt = dt;
    return DG_OK;
}

dg_status dg_mesh_set_time(dg_mesh *m, double t, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    DG_CUDA(launch_set(m->t, t, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_mesh_get_time(dg_mesh *m, double *t, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!t) return fail(DG_ERR_ARG, "t is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    DG_CUDA(cudaMemcpyAsync(t, m->t, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    return DG_OK;
}

dg_status dg_limiter_summaries(dg_mesh *m, const double *U, double *S, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U || !S) return fail(DG_ERR_ARG, "U and S must not be NULL");
    SummaryArgs sa;
    sa.U = U;
    sa.S = S;
    sa.unphys = (m->d.system == 1) ? m->unphys : nullptr;
    sa.T = m->T;
    DG_CUDA(launch_summaries(m->d.n, sa, m->E, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_limit(dg_mesh *m, double *U, unsigned char *troubled, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U) return fail(DG_ERR_ARG, "U is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->d.limiter == 0) {
        if (troubled) DG_CUDA(cudaMemsetAsync(troubled, 0, (size_t)m->E, s));
        return DG_OK;
    }
    SummaryArgs sa;
    sa.U = U;
    sa.S = m->S;
    sa.unphys = (m->d.system == 1) ? m->unphys : nullptr;
    sa.T = m->T;
    DG_CUDA(launch_summaries(m->d.n, sa, m->E, s));
    if (m->d.limiter == DG_LIMITER_MRS) {
        DG_CUDA(launch_mrs(m, U, troubled, s));
        return DG_OK;
    }
    LimitArgs l = limit_args(m, U, troubled);
    DG_CUDA(launch_limit(m->d.n, l, s));
    return DG_OK;
}

dg_status dg_fix(dg_mesh *m, double *U, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!U) return fail(DG_ERR_ARG, "U is NULL");
    if (m->d.system == 1) DG_CUDA(launch_fix(m, U, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_con2prim(long long count, double gamma, const double *cons, double *prim, const double *p_guess,
                      int *iters, int *status, void *stream)
{
    if (count < 0) return fail(DG_ERR_ARG, "count must be >= 0");
    if (count == 0) return DG_OK;
    if (!cons || !prim) return fail(DG_ERR_ARG, "cons and prim must not be NULL");
    if (!(gamma > 1.0)) return fail(DG_ERR_ARG, "gamma must be > 1");
    DG_CUDA(launch_con2prim(count, gamma, cons, prim, p_guess, iters, status, (cudaStream_t)stream));
    return DG_OK;
}

dg_status dg_mesh_set_option(dg_mesh *m, int option, double value)
{
    if (dg_status s = check_mesh(m)) return s;
    switch (option) {
    case DG_OPT_TENSOR_CORE_CONTRACTION:
        if (value != 0.0 && value != 1.0) return fail(DG_ERR_ARG, "tensor-core contraction option takes 0 or 1");
        m->tc_contract = (int)value;
        return DG_OK;
    case DG_OPT_C2P_KAPPA_SWITCH:
        if (!(value >= 1.0 && value <= 1e30)) return fail(DG_ERR_ARG, "kappa switch must be in [1, 1e30]");
        m->kappa_sw = (float)value;
        return DG_OK;
    case DG_OPT_ELEMENTS_PER_CTA: {
        const int epb = (int)value;
        if ((double)epb != value || epb < 1 || epb > stage_max_epb(m->d.n) || (epb & (epb - 1)))
            return fail(DG_ERR_ARG, "elements per CTA must be a power of two in [1, %d] for n = %d",
                        stage_max_epb(m->d.n), m->d.n);
        m->epb = epb;
        return DG_OK;
    }
    default:
        return fail(DG_ERR_ARG, "unknown option %d", option);
    }
}

dg_status dg_mesh_set_c2p_net(dg_mesh *m, const dg_c2p_net *net)
{
    if (dg_status s = check_mesh(m)) return s;
    if (net && (m->d.system != 1 || m->d.precision != DG_PRECISION_MIXED))
        return fail(DG_ERR_ARG, "a learned guess can be attached to mixed-precision SR meshes only");
    m->net = net;
    m->p_valid = 0;
    return DG_OK;
}

dg_status dg_sync_status(dg_mesh *m, void *stream)
{
    if (dg_status s = check_mesh(m)) return s;
    DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int bits = 0;
    DG_CUDA(cudaMemcpy(&bits, m->err, sizeof(bits), cudaMemcpyDeviceToHost));
    DG_CUDA(cudaMemset(m->err, 0, sizeof(bits)));
    if (bits & ERRBIT_TIMEOUT) return fail(DG_ERR_TIMEOUT, "a bounded device wait ran out");
    if (bits & ERRBIT_C2P) return fail(DG_ERR_C2P, "con2prim failed at some node");
    if (bits & ERRBIT_UNPHYSICAL) return fail(DG_ERR_UNPHYSICAL, "unphysical conserved state");
    return DG_OK;
}

dg_status dg_profile_enable(dg_mesh *m, int on)
{
    if (dg_status s = check_mesh(m)) return s;
    if (!m->prof) {
        ProfLog *L = new ProfLog;
        // events made up front: none is created while a stream is being captured
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) break;
            L->pool.push_back(e);
        }
        m->prof = L;
    }
    m->prof_on = on ? 1 : 0;
    return DG_OK;
}

dg_status dg_profile_read(dg_mesh *m, double *ms, long long *launches, int nclass)
{
    if (dg_status s = check_mesh(m)) return s;
    if (nclass < 0 || (nclass > 0 && (!ms || !launches))) return fail(DG_ERR_ARG, "ms and launches must hold nclass entries");
    for (int c = 0; c < nclass; ++c) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    if (!m->prof) return DG_OK;
    ProfLog *L = (ProfLog *)m->prof;
    std::vector<ProfRec> keep;
    for (auto &r : L->recs) {
        DG_CUDA(cudaEventSynchronize(r.b));
        float t = 0.0f;
        DG_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.cls < nclass) {
            ms[r.cls] += t;
            launches[r.cls] += 1;
        }
        if (r.graph) {
            keep.push_back(r);
        } else {
            L->pool.push_back(r.a);
            L->pool.push_back(r.b);
        }
    }
    L->recs.swap(keep);
    return DG_OK;
}

}  // extern "C"
