// dg_ensemble.cu -- a ragged ensemble of independent mixed-precision meshes
// (different element counts, LGL orders and systems) advanced together.
//
// Meshes that can share kernels (same n, system, flux, limiter, gamma, fix
// bounds, options and learned-guess network) form a group.  A step launches,
// per SR group, one CFL kernel, and per stage one stage kernel and (limiter on)
// one limiter kernel over the concatenated element list of all its meshes; per
// Newtonian group, the delta-form step's three stage kernels and decision passes
// (dg_ne_mixed.cuh) over the same concatenation.  Each CTA finds its mesh by
// binary search over the group's element offsets.  With a few
// groups in place of hundreds of meshes, a step is a few dozen launches; they are
// captured once into a CUDA graph and replayed.  dg_ensemble_tune picks, per
// group, the elements per CTA and the volume contraction (tensor cores or FP32
// FMA) by timing the stage kernel on the ensemble's own states.
//
// The arithmetic per element is that of dg_rk3_step on each mesh, so a step of
// the ensemble gives the same bits as stepping every mesh on its own with the
// same per-group options.
#include <algorithm>
#include <cstring>
#include <vector>

#include "dg_mixed.cuh"

namespace dg {

cudaError_t launch_stage_mixed(int n, int system, int flux, const MixedArgs &a, cudaStream_t s);
cudaError_t launch_limit_mixed(int n, int system, const LimitMixedArgs &a, cudaStream_t s);

namespace {

struct DtSlot {
    unsigned long long *lam;
    double *dt;
    double dxmin;
};

__global__ void k_lam_zero(const DtSlot *slots, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) *slots[i].lam = 0ull;
}

// dt = C dx_min / lambda_max per mesh (Sec. 3.4), the same operations as k_dt.
__global__ void k_dt_batch(const DtSlot *slots, int count, double cfl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double l = __longlong_as_double((long long)*slots[i].lam);
    *slots[i].dt = cfl * slots[i].dxmin / l;
}

__global__ void k_dt_gather(const DtSlot *slots, int count, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = *slots[i].dt;
}

}  // namespace

struct EnsGroup {
    int n = 0, system = 0, flux = 0, limiter = 0;
    std::vector<int> members;
    long long nelem = 0, nchunks = 0;
    int epb = 1, tc = 1;
    bool pgiven = false;         // SR: stage 1 takes the CFL pass's primitives
    MixedArgs proto;             // group-level stage arguments (members[0])
    CflArgs cproto;
    LimitMixedArgs lproto;
    MeshSlot *d_stage[3] = {nullptr, nullptr, nullptr};
    MeshSlot *d_stage_first = nullptr;   // stage 1 of the very first step (no pressure guesses yet)
    MeshSlot *d_rhs = nullptr;           // RHS into W1 (tuning)
    LimitSlot *d_limit[3] = {nullptr, nullptr, nullptr};
    CflSlot *d_cfl = nullptr, *d_cfl_first = nullptr;
    long long *d_elem0 = nullptr, *d_chunk0 = nullptr;
    // Newtonian groups: the delta-form step's stage and decision slots per stage
    NeArgs ne_proto[3];
    NeDecideArgs ne_dproto[3];
    NeSlot *d_ne[3] = {nullptr, nullptr, nullptr};
    NeDecideSlot *d_ned[3] = {nullptr, nullptr, nullptr};
};

}  // namespace dg

struct dg_ensemble {
    int device = 0;
    std::vector<dg_mesh *> meshes;
    std::vector<double *> U;
    std::vector<dg::EnsGroup> groups;
    dg::DtSlot *d_dt = nullptr;
    long long steps = 0;
    cudaGraphExec_t exec = nullptr;
    double graph_cfl = 0.0;
    int graph_mode = 0;                  // use_graph of the captured graph
    std::vector<cudaStream_t> branch;    // one stream per group: its launches run beside the other groups'
    std::vector<cudaEvent_t> done;       // per group: end of its part of a phase
    cudaEvent_t fork = nullptr;          // start of a phase on the step's stream
};

using namespace dg;

namespace {

bool same_group(const dg_mesh *a, const dg_mesh *b)
{
    return a->d.n == b->d.n && a->d.system == b->d.system && a->d.flux == b->d.flux &&
           a->d.limiter == b->d.limiter && a->d.gamma == b->d.gamma && a->d.d_atm == b->d.d_atm &&
           a->d.tau_atm == b->d.tau_atm && a->kappa_sw == b->kappa_sw && a->tc_contract == b->tc_contract &&
           a->net == b->net;
}

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src)
{
    cudaError_t e = cudaMalloc(dst, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

void free_group(EnsGroup &g)
{
    for (int s = 0; s < 3; ++s) {
        cudaFree(g.d_stage[s]);
        cudaFree(g.d_limit[s]);
    }
    cudaFree(g.d_stage_first);
    cudaFree(g.d_rhs);
    cudaFree(g.d_cfl);
    cudaFree(g.d_cfl_first);
    cudaFree(g.d_elem0);
    cudaFree(g.d_chunk0);
    for (int s = 0; s < 3; ++s) {
        cudaFree(g.d_ne[s]);
        cudaFree(g.d_ned[s]);
    }
}

// Slot tables of a Newtonian group: the delta-form step of dg_rk3_step on each
// member, its stage kernels and decision passes batched over the members.
cudaError_t build_ne_group(dg_ensemble *en, EnsGroup &g)
{
    const dg_mesh *m0 = en->meshes[g.members[0]];
    const bool lim = m0->d.limiter != 0;
    std::vector<NeSlot> st[3];
    std::vector<NeDecideSlot> de[3];
    std::vector<long long> elem0;
    long long e0 = 0;
    for (int idx : g.members) {
        dg_mesh *m = en->meshes[idx];
        double *U = en->U[idx];
        for (int s = 0; s < 3; ++s) {
            st[s].push_back(ne_stage_args(m, U, s, lim, true).one);
            de[s].push_back(ne_decide_stage_slot(m, U, s, true, nullptr));
        }
        elem0.push_back(e0);
        e0 += m->E;
    }
    g.nelem = e0;
    g.epb = ne_epb(g.n);
    g.tc = 0;
    cudaError_t e = upload(&g.d_elem0, elem0);
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = upload(&g.d_ne[s], st[s]);
        if (e == cudaSuccess) e = upload(&g.d_ned[s], de[s]);
    }
    if (e != cudaSuccess) return e;
    for (int s = 0; s < 3; ++s) {
        NeArgs a = ne_stage_args(m0, en->U[g.members[0]], s, lim, true);
        a.slots = g.d_ne[s];
        a.elem0 = g.d_elem0;
        a.nslots = (int)g.members.size();
        a.nelem = g.nelem;
        g.ne_proto[s] = a;
        NeDecideArgs d = ne_decide_args(m0);
        d.slots = g.d_ned[s];
        d.elem0 = g.d_elem0;
        d.nslots = (int)g.members.size();
        d.nelem = g.nelem;
        d.scale_dt = s == 0;
        g.ne_dproto[s] = d;
    }
    return cudaSuccess;
}

// Slot tables of a group: the pointers of every member for each pass of a step.
// Pressure buffers (warm start, no network) follow the same alternation as
// dg_rk3_step: CFL reads pbuf[0] and writes pbuf[1], stage 1 reads pbuf[1] and
// writes pbuf[0], stage 2 the reverse, stage 3 as stage 1.  For SR meshes the CFL
// pass also writes its primitives of U^n (pfull), which stage 1 takes instead of
// solving con2prim, as in dg_rk3_step.
cudaError_t build_group(dg_ensemble *en, EnsGroup &g)
{
    const dg_mesh *m0 = en->meshes[g.members[0]];
    const bool carry = m0->d.system == 1 && m0->net == nullptr;
    const bool pgiven = m0->d.system == 1;
    g.pgiven = pgiven;
    std::vector<MeshSlot> st[3], first, rhs;
    std::vector<LimitSlot> li[3];
    std::vector<CflSlot> cf, cf1;
    std::vector<long long> elem0, chunk0;
    long long e0 = 0, c0 = 0;
    for (int idx : g.members) {
        dg_mesh *m = en->meshes[idx];
        double *U = en->U[idx];
        double *ins[3] = {U, m->W1, m->W2};
        double *outs[3] = {m->W1, m->W2, U};
        float *pr[2] = {carry ? m->pbuf[0] : nullptr, carry ? m->pbuf[1] : nullptr};
        for (int s = 0; s < 3; ++s) {
            MeshSlot sl = mixed_slot(m);
            sl.Us = ins[s];
            sl.Un = U;
            sl.out = outs[s];
            sl.pin = (s == 1) ? pr[0] : pr[1];
            sl.pout = (s == 1) ? pr[1] : pr[0];
            if (pgiven && s == 0) sl.Pin = m->pfull;
            sl.S = m->d.limiter ? m->S : nullptr;
            sl.flags = (m->d.limiter && m->d.system == 1) ? m->unphys : nullptr;
            sl.dt_ptr = m->dt;
            st[s].push_back(sl);
            if (s == 0) first.push_back(sl);
            li[s].push_back(limit_slot(m, outs[s], nullptr));
        }
        MeshSlot r = mixed_slot(m);
        r.Us = U;
        r.Un = U;
        r.out = m->W1;
        rhs.push_back(r);
        CflSlot c;
        std::memset(&c, 0, sizeof(c));
        c.Un = U;
        c.pin = pr[0];
        c.pout = pr[1];
        c.Pout = pgiven ? m->pfull : nullptr;
        c.lam = m->lam;
        c.err = m->err;
        c.nodes = m->E * m->nn;
        cf.push_back(c);
        c.pin = nullptr;
        cf1.push_back(c);
        elem0.push_back(e0);
        chunk0.push_back(c0);
        e0 += m->E;
        c0 += (c.nodes + CFL_CHUNK - 1) / CFL_CHUNK;
    }
    g.nelem = e0;
    g.nchunks = c0;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = upload(&g.d_stage[s], st[s]);
        if (e == cudaSuccess) e = upload(&g.d_limit[s], li[s]);
    }
    if (e == cudaSuccess) e = upload(&g.d_stage_first, first);
    if (e == cudaSuccess) e = upload(&g.d_rhs, rhs);
    if (e == cudaSuccess) e = upload(&g.d_cfl, cf);
    if (e == cudaSuccess) e = upload(&g.d_cfl_first, cf1);
    if (e == cudaSuccess) e = upload(&g.d_elem0, elem0);
    if (e == cudaSuccess) e = upload(&g.d_chunk0, chunk0);
    if (e != cudaSuccess) return e;
    g.proto = mixed_args(m0);
    g.proto.slots = nullptr;
    g.proto.elem0 = g.d_elem0;
    g.proto.nslots = (int)g.members.size();
    g.proto.nelem = g.nelem;
    g.proto.mode = 1;
    g.tc = m0->tc_contract;
    g.cproto = cfl_args(m0, m0->kappa_sw);
    g.cproto.chunk0 = g.d_chunk0;
    g.cproto.nslots = (int)g.members.size();
    g.lproto = limit_mixed_args(m0, nullptr, nullptr);
    g.lproto.elem0 = g.d_elem0;
    g.lproto.nslots = (int)g.members.size();
    g.lproto.E = g.nelem;
    return cudaSuccess;
}

MixedArgs stage_args_for(const EnsGroup &g, const MeshSlot *slots, int stage)
{
    static const float ca[3] = {0.0f, 0.75f, (float)(1.0 / 3.0)};
    static const float cb[3] = {1.0f, 0.25f, (float)(2.0 / 3.0)};
    MixedArgs a = g.proto;
    a.slots = slots;
    a.first = stage == 0;
    a.ca = ca[stage];
    a.cb = cb[stage];
    a.epb = g.epb;
    a.tc = g.tc;
    return a;
}

// The two phases of a group's step.  Before the batched dt: the SR CFL pass, or the
// Newtonian delta-form stage 1 (which takes the CFL maximum itself).  After it:
// SR: per stage the stage kernel and the limiter; Newtonian: the decision pass
// after stage 1, then stages 2 and 3 with their decision passes (the last one
// writes U^{n+1}).  A group's launches touch only its own meshes.
cudaError_t group_pre_dt(EnsGroup &g, bool first, cudaStream_t s)
{
    if (g.system == 0) return launch_ne_stage(g.n, g.flux, 1, g.ne_proto[0], s);
    CflArgs c = g.cproto;
    c.slots = first ? g.d_cfl_first : g.d_cfl;
    return launch_cfl_batch(g.system, c, g.nchunks, s);
}

cudaError_t group_stage(EnsGroup &g, bool first, int st, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (g.system == 0) {
        if (st > 0) e = launch_ne_stage(g.n, g.flux, st + 1, g.ne_proto[st], s);
        if (e == cudaSuccess && (st == 2 || g.limiter)) e = launch_ne_decide(g.n, st == 2, g.ne_dproto[st], s);
        return e;
    }
    MixedArgs a = stage_args_for(g, (first && st == 0) ? g.d_stage_first : g.d_stage[st], st);
    if (g.pgiven && st == 0) a.netImg = nullptr;  // stage 1 takes the CFL pass's primitives
    e = launch_stage_mixed(g.n, g.system, g.flux, a, s);
    if (e == cudaSuccess && g.limiter) {
        LimitMixedArgs l = g.lproto;
        l.slots = g.d_limit[st];
        e = launch_limit_mixed(g.n, g.system, l, s);
    }
    return e;
}

// One step of the ensemble: the per-mesh lambda reset, every group's pre-dt
// phase, the batched dt, every group's stages, all on s, stage by stage across
// the groups.  concurrent: each group's phase runs on its own stream instead,
// forked from and joined back to s by events (in a captured graph: parallel
// branches), so that the groups' launches overlap.  Both orders give the same
// bits: no data crosses groups.  (On the 256-mesh recipe the two orders run within
// about 1 % of each other: the launches' tails that the branches overlap are a
// small part of a step.)
cudaError_t launch_step(dg_ensemble *en, double cfl, bool first, bool concurrent, cudaStream_t s)
{
    const int count = (int)en->meshes.size();
    const unsigned blocks = (unsigned)((count + 127) / 128);
    const int G = (int)en->groups.size();
    k_lam_zero<<<blocks, 128, 0, s>>>(en->d_dt, count);
    cudaError_t e = cudaGetLastError();
    auto fan_out = [&](auto &&body) -> cudaError_t {
        cudaError_t r = cudaEventRecord(en->fork, s);
        for (int i = 0; i < G && r == cudaSuccess; ++i) {
            r = cudaStreamWaitEvent(en->branch[i], en->fork, 0);
            if (r == cudaSuccess) r = body(en->groups[i], en->branch[i]);
            if (r == cudaSuccess) r = cudaEventRecord(en->done[i], en->branch[i]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(s, en->done[i], 0);
        }
        return r;
    };
    if (e == cudaSuccess) {
        if (concurrent) {
            e = fan_out([&](EnsGroup &g, cudaStream_t b) { return group_pre_dt(g, first, b); });
        } else {
            for (int i = 0; i < G && e == cudaSuccess; ++i) e = group_pre_dt(en->groups[i], first, s);
        }
    }
    if (e != cudaSuccess) return e;
    k_dt_batch<<<blocks, 128, 0, s>>>(en->d_dt, count, cfl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (concurrent)
        return fan_out([&](EnsGroup &g, cudaStream_t b) {
            cudaError_t r = cudaSuccess;
            for (int st = 0; st < 3 && r == cudaSuccess; ++st) r = group_stage(g, first, st, b);
            return r;
        });
    for (int st = 0; st < 3 && e == cudaSuccess; ++st)
        for (int i = 0; i < G && e == cudaSuccess; ++i) e = group_stage(en->groups[i], first, st, s);
    return e;
}

dg_status cuda_fail(cudaError_t e) { return set_error(DG_ERR_CUDA, cudaGetErrorString(e)); }

}  // namespace

extern "C" {

dg_status dg_ensemble_create(dg_mesh *const *meshes, double *const *U, int count, dg_ensemble **out)
{
    if (!meshes || !U || !out || count < 1) return set_error(DG_ERR_ARG, "need meshes, states, out and count >= 1");
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(DG_ERR_CUDA, "no current CUDA device");
    for (int i = 0; i < count; ++i) {
        if (!meshes[i] || !U[i]) return set_error(DG_ERR_ARG, "NULL mesh or state in the ensemble");
        if (meshes[i]->device != dev) return set_error(DG_ERR_ARG, "every mesh must live on the current device");
        if (meshes[i]->d.precision != DG_PRECISION_MIXED)
            return set_error(DG_ERR_ARG, "the ensemble advances mixed-precision meshes only");
        if (meshes[i]->gh.mask) return set_error(DG_ERR_ARG, "the ensemble advances periodic meshes only");
        if (meshes[i]->d.limiter == DG_LIMITER_MRS)
            return set_error(DG_ERR_ARG, "the ensemble runs the minmod limiters only, not the moment limiter");
        if (meshes[i]->d.system == 0 && (reinterpret_cast<uintptr_t>(U[i]) & 15u))
            return set_error(DG_ERR_ARG, "the mixed Newtonian path needs U 16-byte aligned");
        for (int j = 0; j < i; ++j)
            if (meshes[j] == meshes[i] || U[j] == U[i]) return set_error(DG_ERR_ARG, "meshes and states must be distinct");
    }
    dg_ensemble *en = new dg_ensemble;
    en->device = dev;
    en->meshes.assign(meshes, meshes + count);
    en->U.assign(U, U + count);
    for (int i = 0; i < count; ++i) {
        bool placed = false;
        for (EnsGroup &g : en->groups)
            if (same_group(en->meshes[g.members[0]], meshes[i])) {
                g.members.push_back(i);
                placed = true;
                break;
            }
        if (!placed) {
            EnsGroup g;
            g.n = meshes[i]->d.n;
            g.system = meshes[i]->d.system;
            g.flux = meshes[i]->d.flux;
            g.limiter = meshes[i]->d.limiter;
            g.members.push_back(i);
            en->groups.push_back(g);
        }
    }
    cudaError_t e = cudaSuccess;
    for (EnsGroup &g : en->groups)
        if (e == cudaSuccess) e = g.system == 0 ? build_ne_group(en, g) : build_group(en, g);
    std::vector<DtSlot> dts;
    for (dg_mesh *m : en->meshes) dts.push_back(DtSlot{m->lam, m->dt, m->dxmin});
    if (e == cudaSuccess) e = upload(&en->d_dt, dts);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&en->fork, cudaEventDisableTiming);
    for (size_t i = 0; i < en->groups.size() && e == cudaSuccess; ++i) {
        cudaStream_t b = nullptr;
        cudaEvent_t d = nullptr;
        e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
        if (e == cudaSuccess) en->branch.push_back(b);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
        if (e == cudaSuccess) en->done.push_back(d);
    }
    if (e != cudaSuccess) {
        dg_ensemble_destroy(en);
        return cuda_fail(e);
    }
    *out = en;
    return DG_OK;
}

void dg_ensemble_destroy(dg_ensemble *en)
{
    if (!en) return;
    if (en->exec) cudaGraphExecDestroy(en->exec);
    for (cudaStream_t b : en->branch) cudaStreamDestroy(b);
    for (cudaEvent_t d : en->done) cudaEventDestroy(d);
    if (en->fork) cudaEventDestroy(en->fork);
    for (EnsGroup &g : en->groups) free_group(g);
    cudaFree(en->d_dt);
    delete en;
}

dg_status dg_ensemble_tune(dg_ensemble *en, void *stream)
{
    if (!en) return set_error(DG_ERR_ARG, "ensemble is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        return set_error(DG_ERR_CUDA, "event creation failed");
    dg_status st = DG_OK;
    for (EnsGroup &g : en->groups) {
        if (g.system == 0) continue;  // the Newtonian step has no launch-shape options
        float best = 1e30f;
        int best_epb = g.epb, best_tc = g.tc;
        for (int tc = 1; tc >= 0; --tc)
            for (int epb = 1; epb <= stage_max_epb(g.n); epb *= 2) {
                MixedArgs a = g.proto;
                a.slots = g.d_rhs;
                a.mode = 0;
                a.lim = 0;
                a.epb = epb;
                a.tc = tc;
                cudaError_t e = launch_stage_mixed(g.n, g.system, g.flux, a, s);  // warm-up
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventRecord(t0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_stage_mixed(g.n, g.system, g.flux, a, s);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) {
                    st = cuda_fail(e);
                    break;
                }
                if (ms < best) {
                    best = ms;
                    best_epb = epb;
                    best_tc = tc;
                }
            }
        if (st != DG_OK) break;
        g.epb = best_epb;
        g.tc = best_tc;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (en->exec) {
        cudaGraphExecDestroy(en->exec);
        en->exec = nullptr;
    }
    return st;
}

dg_status dg_ensemble_step(dg_ensemble *en, double cfl, int use_graph, void *stream)
{
    if (!en) return set_error(DG_ERR_ARG, "ensemble is NULL");
    if (!(cfl > 0.0)) return set_error(DG_ERR_ARG, "cfl must be > 0");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != en->device)
        return set_error(DG_ERR_ARG, "the ensemble was created on another device");
    cudaStream_t s = (cudaStream_t)stream;
    const bool first = en->steps == 0;
    cudaError_t e = cudaSuccess;
    if (use_graph < 0 || use_graph > 2) return set_error(DG_ERR_ARG, "use_graph must be 0, 1 or 2");
    if (!use_graph || first) {
        // the first step has no pressure guesses yet and runs directly
        e = launch_step(en, cfl, first, use_graph == 2, s);
    } else {
        if (en->exec && (en->graph_cfl != cfl || en->graph_mode != use_graph)) {
            cudaGraphExecDestroy(en->exec);
            en->exec = nullptr;
        }
        if (!en->exec) {
            // launch sequences are captured on a private stream: the legacy
            // default stream cannot be captured
            cudaStream_t cap;
            cudaGraph_t graph = nullptr;
            e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e);
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                const cudaError_t el = launch_step(en, cfl, false, use_graph == 2, cap);
                e = cudaStreamEndCapture(cap, &graph);
                if (e == cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&en->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) return cuda_fail(e);
            en->graph_cfl = cfl;
            en->graph_mode = use_graph;
        }
        e = cudaGraphLaunch(en->exec, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    for (dg_mesh *m : en->meshes) m->p_valid = 0;  // the meshes' own pressure carry is not the ensemble's
    en->steps += 1;
    return DG_OK;
}

int dg_ensemble_num_groups(const dg_ensemble *en) { return en ? (int)en->groups.size() : 0; }

dg_status dg_ensemble_group_info(const dg_ensemble *en, int g, long long info[8])
{
    if (!en || !info || g < 0 || g >= (int)en->groups.size()) return set_error(DG_ERR_ARG, "bad ensemble or group");
    const EnsGroup &G = en->groups[g];
    info[0] = G.n;
    info[1] = G.system;
    info[2] = G.flux;
    info[3] = G.limiter;
    info[4] = (long long)G.members.size();
    info[5] = G.nelem;
    info[6] = G.epb;
    info[7] = G.tc;
    return DG_OK;
}

int dg_ensemble_mesh_group(const dg_ensemble *en, int i)
{
    if (!en || i < 0 || i >= (int)en->meshes.size()) return -1;
    for (int g = 0; g < (int)en->groups.size(); ++g)
        for (int m : en->groups[g].members)
            if (m == i) return g;
    return -1;
}

dg_status dg_ensemble_dt(const dg_ensemble *en, double *dt, void *stream)
{
    if (!en || !dt) return set_error(DG_ERR_ARG, "ensemble and dt must not be NULL");
    const int count = (int)en->meshes.size();
    k_dt_gather<<<(count + 127) / 128, 128, 0, (cudaStream_t)stream>>>(en->d_dt, count, dt);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DG_OK : cuda_fail(e);
}

}  // extern "C"
