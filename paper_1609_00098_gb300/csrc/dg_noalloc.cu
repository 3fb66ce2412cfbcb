// dg_noalloc.cu -- dg_rhs_static: the FP64 right-hand side of dg_rhs for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: host codes whose device memory is
// owned by another allocator (a framework pool that has reserved the free
// memory, so a cudaMalloc would fail or fragment it), or time-critical loops
// where the implicit device synchronisation of cudaMalloc / cudaFree is not
// acceptable.  dg_rhs needs a dg_mesh, whose creation allocates the library's
// scratch; this entry point instead keeps its one scratch buffer (the node
// primitives) in a file-scope static device array of fixed size, takes the mesh
// descriptor directly, and allocates nothing.  The caller still owns U and dUdt.
//
// The array is global to the process on each device that loads the library and
// keeps the last call's contents.  Calls that overlap on the GPU (two streams,
// or two host threads) race on it and must be serialised by the caller.
#include <cstring>
#include <mutex>

#include "dg_internal.h"

namespace {

constexpr long long kStaticMaxNodes = DG_RHS_STATIC_MAX_NODES;

// Node primitives (vx, vy, vz, p), [e][4][node]; overwritten in full by each call.
static __device__ __align__(256) double g_static_P[4 * kStaticMaxNodes];
// Device status word of the primitive recovery; cleared at the start of each call.
static __device__ __align__(256) unsigned int g_static_err;

// Device addresses of the two arrays, looked up once per device with that device
// current (in host code the symbols are host-side stand-ins, not device addresses).
struct StaticSlots {
    double *P = nullptr;
    unsigned int *err = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
StaticSlots g_slots[kMaxDevices];
std::mutex g_slots_mu;

dg_status static_slots(int dev, StaticSlots &out)
{
    if (dev < 0 || dev >= kMaxDevices) return dg::set_error(DG_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_slots_mu);
    StaticSlots &s = g_slots[dev];
    if (!s.ready) {
        cudaError_t e = cudaGetSymbolAddress((void **)&s.P, g_static_P);
        if (e != cudaSuccess) return dg::set_error(DG_ERR_CUDA, cudaGetErrorString(e));
        e = cudaGetSymbolAddress((void **)&s.err, g_static_err);
        if (e != cudaSuccess) return dg::set_error(DG_ERR_CUDA, cudaGetErrorString(e));
        s.ready = true;
    }
    out = s;
    return DG_OK;
}

}  // namespace

extern "C" dg_status dg_rhs_static(const dg_mesh_desc *d, const double *U, double *dUdt, void *stream)
{
    using namespace dg;
    if (!d || !U || !dUdt || U == dUdt) return set_error(DG_ERR_ARG, "desc, U and dUdt must be non-NULL and distinct");
    if (d->system != 0 && d->system != 1) return set_error(DG_ERR_ARG, "system must be 0 or 1");
    if (d->n < 2 || d->n > MAXN) return set_error(DG_ERR_ARG, "n must be in 2..8");
    if (d->flux != 0 && d->flux != 1 && !(d->flux == 2 && d->system == 0))
        return set_error(DG_ERR_ARG, "flux must be 0 (LLF), 1 (HLL) or, for the Newtonian system, 2 (Roe)");
    if (d->precision != DG_PRECISION_FP64) return set_error(DG_ERR_ARG, "dg_rhs_static computes the FP64 path only");
    if (d->bc[0] || d->bc[1] || d->bc[2]) return set_error(DG_ERR_ARG, "dg_rhs_static takes periodic meshes only");
    if (!(d->gamma > 1.0)) return set_error(DG_ERR_ARG, "gamma must be > 1");
    long long E = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->K[a] < 1) return set_error(DG_ERR_ARG, "K must be >= 1");
        if (!(d->hi[a] > d->lo[a])) return set_error(DG_ERR_ARG, "hi must exceed lo");
        E *= d->K[a];
        if (E > kStaticMaxNodes) break;
    }
    const long long nn = (long long)d->n * d->n * d->n;
    if (E > kStaticMaxNodes || E * nn > kStaticMaxNodes)
        return set_error(DG_ERR_ARG, "mesh exceeds the static scratch of dg_rhs_static (DG_RHS_STATIC_MAX_NODES nodes)");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(DG_ERR_CUDA, "no current CUDA device");
    StaticSlots slots;
    if (dg_status st = static_slots(dev, slots)) return st;

    // a mesh view on the host stack; its only device buffers are the static arrays
    dg_mesh m;
    std::memset(&m, 0, sizeof(m));
    m.d = *d;
    m.device = dev;
    m.nn = (int)nn;
    m.E = E;
    lgl_tables(d->n, m.T);
    for (int a = 0; a < 3; ++a) m.dx[a] = (d->hi[a] - d->lo[a]) / d->K[a];
    m.P = slots.P;
    m.err = slots.err;

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(slots.err, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = launch_primitives(&m, U, slots.P, 0, nullptr, nullptr, s);
    if (e == cudaSuccess) {
        StageArgs a;
        std::memset(&a, 0, sizeof(a));
        for (int ax = 0; ax < 3; ++ax) {
            a.K[ax] = d->K[ax];
            a.g[ax] = 2.0 / m.dx[ax];
            a.lift0[ax] = a.g[ax] / m.T.w[0];
            a.liftN[ax] = a.g[ax] / m.T.w[d->n - 1];
        }
        a.gamma = d->gamma;
        a.T = m.T;
        a.Us = U;
        a.Un = U;
        a.P = slots.P;
        a.out = dUdt;
        a.mode = 0;
        e = launch_stage_fp64(d->n, d->system, d->flux, a, E, s);
    }
    if (e != cudaSuccess) return set_error(DG_ERR_CUDA, cudaGetErrorString(e));
    return DG_OK;
}
