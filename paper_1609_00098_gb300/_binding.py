"""ctypes binding of libdg (include/dg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
device pointers taken from torch CUDA tensors plus the current torch stream.
All computation happens in libdg's CUDA kernels; if the library cannot be
loaded this module raises instead of computing anything elsewhere.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdg.so")

DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_C2P, DG_ERR_UNPHYSICAL, DG_ERR_TIMEOUT, DG_ERR_NOMEM = range(7)
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_CUDA", 3: "DG_ERR_C2P", 4: "DG_ERR_UNPHYSICAL",
                5: "DG_ERR_TIMEOUT", 6: "DG_ERR_NOMEM"}


class DGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class dg_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int),
        ("K", ctypes.c_int * 3),
        ("n", ctypes.c_int),
        ("flux", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("tvb_M", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("d_atm", ctypes.c_double),
        ("tau_atm", ctypes.c_double),
        ("mrs_alpha", ctypes.c_double),
        ("bc", ctypes.c_int * 3),
        ("exact", ctypes.c_int),
        ("exact_par", ctypes.c_double * 6),
    ]


_vp = ctypes.c_void_p
_ll = ctypes.c_longlong
_d = ctypes.c_double
_i = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "dg_mesh_create": (_i, [ctypes.POINTER(dg_mesh_desc), ctypes.POINTER(_vp)]),
    "dg_mesh_destroy": (None, [_vp]),
    "dg_state_size": (_ll, [_vp]),
    "dg_num_nodes": (_ll, [_vp]),
    "dg_lgl_tables": (_i, [_i, _vp, _vp, _vp, _vp]),
    "dg_node_coords": (_i, [_vp, _vp, _vp]),
    "dg_prim2con": (_i, [_vp, _vp, _vp, _vp]),
    "dg_primitives": (_i, [_vp, _vp, _vp, _vp]),
    "dg_rhs": (_i, [_vp, _vp, _vp, _vp]),
    "dg_rhs_static": (_i, [ctypes.POINTER(dg_mesh_desc), _vp, _vp, _vp]),
    "dg_compute_dt": (_i, [_vp, _vp, _d, _vp, _vp]),
    "dg_rk3_step": (_i, [_vp, _vp, _d, _d, _vp, _vp, _vp]),
    "dg_limit": (_i, [_vp, _vp, _vp, _vp]),
    "dg_fix": (_i, [_vp, _vp, _vp]),
    "dg_limiter_summaries": (_i, [_vp, _vp, _vp, _vp]),
    "dg_con2prim": (_i, [_ll, _d, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dg_sync_status": (_i, [_vp, _vp]),
    "dg_mesh_set_c2p_net": (_i, [_vp, _vp]),
    "dg_mesh_set_option": (_i, [_vp, _i, _d]),
    "dg_ab3_step": (_i, [_vp, _vp, _d, _vp, _vp]),
    "dg_ab3_reset": (_i, [_vp]),
    "dg_mesh_set_time": (_i, [_vp, _d, _vp]),
    "dg_mesh_get_time": (_i, [_vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "dg_ensemble_create": (_i, [_vp, _vp, _i, ctypes.POINTER(_vp)]),
    "dg_ensemble_destroy": (None, [_vp]),
    "dg_ensemble_tune": (_i, [_vp, _vp]),
    "dg_ensemble_step": (_i, [_vp, _d, _i, _vp]),
    "dg_ensemble_num_groups": (_i, [_vp]),
    "dg_ensemble_group_info": (_i, [_vp, _i, _vp]),
    "dg_ensemble_mesh_group": (_i, [_vp, _i]),
    "dg_ensemble_dt": (_i, [_vp, _vp, _vp]),
    "dg_c2p_net_create": (_i, [_vp, _vp, ctypes.POINTER(_vp)]),
    "dg_c2p_net_destroy": (None, [_vp]),
    "dg_c2p_net_get_params": (_i, [_vp, _vp]),
    "dg_c2p_net_guess": (_i, [_vp, _ll, _d, _vp, _vp, _vp]),
    "dg_c2p_net_grad": (_i, [_vp, _ll, _vp, _vp, _vp, _vp, _vp]),
    "dg_c2p_net_train": (_i, [_vp, _ll, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp]),
    "dg_profile_enable": (_i, [_vp, _i]),
    "dg_profile_read": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_ll), _i]),
    "dg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(build_if_missing: bool = False):
    """Load libdg.so (optionally building it first).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdg is not built ({LIB_PATH} missing): run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != DG_OK:
        raise DGError(status, load().dg_last_error().decode())


def _stream(stream=None):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, numel: int | None = None, dtype=None, name: str = "tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def make_desc(system=0, K=(4, 4, 4), n=4, flux=0, limiter=0, precision=0, gamma=1.4,
              lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), tvb_M=0.0, beta=2.0, d_atm=1e-12,
              tau_atm=1e-14, mrs_alpha=0.0, bc=(0, 0, 0), exact=0, exact_par=(0.0,) * 6) -> dg_mesh_desc:
    d = dg_mesh_desc()
    d.system, d.n, d.flux, d.limiter, d.precision = system, n, flux, limiter, precision
    d.gamma, d.tvb_M, d.beta, d.d_atm, d.tau_atm = gamma, tvb_M, beta, d_atm, tau_atm
    d.mrs_alpha = mrs_alpha
    for a in range(3):
        d.K[a], d.lo[a], d.hi[a] = K[a], lo[a], hi[a]
        d.bc[a] = bc[a]
    d.exact = exact
    for i in range(6):
        d.exact_par[i] = exact_par[i]
    return d


# --- one function per entry point -------------------------------------------

def dg_mesh_create(desc: dg_mesh_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().dg_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def dg_mesh_destroy(mesh) -> None:
    load().dg_mesh_destroy(mesh)


def dg_state_size(mesh) -> int:
    return load().dg_state_size(mesh)


def dg_num_nodes(mesh) -> int:
    return load().dg_num_nodes(mesh)


def dg_lgl_tables(n: int):
    """Host LGL tables of the library: (x, w, D (n, n), row1) as numpy arrays."""
    import numpy as np
    x, w, r1 = np.zeros(n), np.zeros(n), np.zeros(n)
    D = np.zeros((n, n))
    _check(load().dg_lgl_tables(n, x.ctypes.data, w.ctypes.data, D.ctypes.data, r1.ctypes.data))
    return x, w, D, r1


def dg_node_coords(mesh, xyz, stream=None):
    import torch
    _check(load().dg_node_coords(mesh, _ptr(xyz, 3 * dg_num_nodes(mesh), torch.float64, "xyz"), _stream(stream)))


def dg_prim2con(mesh, prim, U, stream=None):
    import torch
    N = dg_num_nodes(mesh)
    _check(load().dg_prim2con(mesh, _ptr(prim, 5 * N, torch.float64, "prim"),
                              _ptr(U, 5 * N, torch.float64, "U"), _stream(stream)))


def dg_primitives(mesh, U, P, stream=None):
    import torch
    N = dg_num_nodes(mesh)
    _check(load().dg_primitives(mesh, _ptr(U, 5 * N, torch.float64, "U"), _ptr(P, 4 * N, torch.float64, "P"),
                                _stream(stream)))


def dg_rhs(mesh, U, dUdt, stream=None):
    import torch
    n = dg_state_size(mesh)
    _check(load().dg_rhs(mesh, _ptr(U, n, torch.float64, "U"), _ptr(dUdt, n, torch.float64, "dUdt"),
                         _stream(stream)))


RHS_STATIC_MAX_NODES = 131072


def dg_rhs_static(desc: "dg_mesh_desc", U, dUdt, stream=None):
    """dg_rhs of a mesh described by `desc`, with no device allocation."""
    import torch
    n = desc.K[0] * desc.K[1] * desc.K[2] * desc.n ** 3 * 5
    _check(load().dg_rhs_static(ctypes.byref(desc), _ptr(U, n, torch.float64, "U"),
                                _ptr(dUdt, n, torch.float64, "dUdt"), _stream(stream)))


def dg_compute_dt(mesh, U, cfl, dt, stream=None):
    import torch
    _check(load().dg_compute_dt(mesh, _ptr(U, dg_state_size(mesh), torch.float64, "U"), float(cfl),
                                _ptr(dt, 1, torch.float64, "dt"), _stream(stream)))


def dg_rk3_step(mesh, U, dt=0.0, cfl=0.0, dt_used=None, troubled=None, stream=None):
    import torch
    _check(load().dg_rk3_step(mesh, _ptr(U, dg_state_size(mesh), torch.float64, "U"), float(dt), float(cfl),
                              _ptr(dt_used, 1, torch.float64, "dt_used"),
                              _ptr(troubled, None, torch.uint8, "troubled"), _stream(stream)))


def dg_limit(mesh, U, troubled=None, stream=None):
    import torch
    _check(load().dg_limit(mesh, _ptr(U, dg_state_size(mesh), torch.float64, "U"),
                           _ptr(troubled, None, torch.uint8, "troubled"), _stream(stream)))


def dg_fix(mesh, U, stream=None):
    import torch
    _check(load().dg_fix(mesh, _ptr(U, dg_state_size(mesh), torch.float64, "U"), _stream(stream)))


def dg_limiter_summaries(mesh, U, S, stream=None):
    import torch
    _check(load().dg_limiter_summaries(mesh, _ptr(U, dg_state_size(mesh), torch.float64, "U"),
                                       _ptr(S, None, torch.float64, "S"), _stream(stream)))


def dg_con2prim(count, gamma, cons, prim, p_guess=None, iters=None, status=None, stream=None):
    import torch
    _check(load().dg_con2prim(int(count), float(gamma), _ptr(cons, 5 * count, torch.float64, "cons"),
                              _ptr(prim, 5 * count, torch.float64, "prim"),
                              _ptr(p_guess, count, torch.float64, "p_guess"),
                              _ptr(iters, count, torch.int32, "iters"),
                              _ptr(status, count, torch.int32, "status"), _stream(stream)))


def dg_sync_status(mesh, stream=None) -> int:
    """Returns the status code (does not raise for kernel-side failures)."""
    return load().dg_sync_status(mesh, _stream(stream))


def dg_ensemble_create(meshes, states):
    """meshes: Mesh handles (c_void_p); states: matching device float64 tensors."""
    import torch
    n = len(meshes)
    if n != len(states) or n < 1:
        raise ValueError("need as many states as meshes, at least one")
    mh = (ctypes.c_void_p * n)(*[m.value if isinstance(m, ctypes.c_void_p) else m for m in meshes])
    sp = (ctypes.c_void_p * n)(*[_ptr(U, U.numel(), torch.float64, "U") for U in states])
    h = ctypes.c_void_p()
    _check(load().dg_ensemble_create(ctypes.addressof(mh), ctypes.addressof(sp), n, ctypes.byref(h)))
    return h


def dg_ensemble_destroy(ens):
    load().dg_ensemble_destroy(ens)


def dg_ensemble_tune(ens, stream=None):
    _check(load().dg_ensemble_tune(ens, _stream(stream)))


def dg_ensemble_step(ens, cfl, use_graph=True, stream=None):
    """use_graph: False/0 direct launches, True/1 graph with the groups one after the
    other, 2 graph with the groups on parallel branches."""
    g = int(use_graph) if not isinstance(use_graph, bool) else (1 if use_graph else 0)
    _check(load().dg_ensemble_step(ens, float(cfl), g, _stream(stream)))


def dg_ensemble_num_groups(ens) -> int:
    return int(load().dg_ensemble_num_groups(ens))


def dg_ensemble_group_info(ens, g):
    """(n, system, flux, limiter, meshes, elements, elements per CTA, tensor-core contraction)."""
    info = (ctypes.c_longlong * 8)()
    _check(load().dg_ensemble_group_info(ens, int(g), ctypes.addressof(info)))
    return tuple(info)


def dg_ensemble_mesh_group(ens, i) -> int:
    return int(load().dg_ensemble_mesh_group(ens, int(i)))


def dg_ensemble_groups(ens):
    """List of dicts (n, system, flux, limiter, meshes, elements, epb, tc) per group."""
    keys = ("n", "system", "flux", "limiter", "meshes", "elements", "epb", "tc")
    groups = [dict(zip(keys, dg_ensemble_group_info(ens, g))) for g in range(dg_ensemble_num_groups(ens))]
    count = sum(g["meshes"] for g in groups)
    for g in groups:
        g["members"] = []
    for i in range(count):
        groups[dg_ensemble_mesh_group(ens, i)]["members"].append(i)
    return groups


def dg_ensemble_dt(ens, dt, stream=None):
    import torch
    _check(load().dg_ensemble_dt(ens, _ptr(dt, dt.numel(), torch.float64, "dt"), _stream(stream)))


OPT_TENSOR_CORE_CONTRACTION = 1
OPT_C2P_KAPPA_SWITCH = 2
OPT_ELEMENTS_PER_CTA = 3


def dg_mesh_set_option(mesh, option, value):
    """Set a mixed-path option (OPT_TENSOR_CORE_CONTRACTION, OPT_C2P_KAPPA_SWITCH)."""
    _check(load().dg_mesh_set_option(mesh, int(option), float(value)))


def dg_ab3_step(mesh, U, dt, troubled=None, stream=None):
    import torch
    _check(load().dg_ab3_step(mesh, _ptr(U, None, torch.float64, "U"), float(dt),
                              _ptr(troubled, None, torch.uint8, "troubled"), _stream(stream)))


def dg_ab3_reset(mesh):
    _check(load().dg_ab3_reset(mesh))


def dg_mesh_set_time(mesh, t, stream=None):
    _check(load().dg_mesh_set_time(mesh, float(t), _stream(stream)))


def dg_mesh_get_time(mesh, stream=None) -> float:
    t = ctypes.c_double(0.0)
    _check(load().dg_mesh_get_time(mesh, ctypes.byref(t), _stream(stream)))
    return t.value


def dg_mesh_set_c2p_net(mesh, net):
    """Attach a learned-guess network to a mixed SR mesh (None detaches)."""
    _check(load().dg_mesh_set_c2p_net(mesh, net))


N_NET_PARAMS = 4481


def dg_c2p_net_create(params, scales):
    """params: host float32 array of 4481; scales: 6 floats (host)."""
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    sc = np.ascontiguousarray(scales, dtype=np.float64)
    if p.size != N_NET_PARAMS or sc.size != 6:
        raise ValueError("need 4481 parameters and 6 scales")
    h = ctypes.c_void_p()
    _check(load().dg_c2p_net_create(p.ctypes.data, sc.ctypes.data, ctypes.byref(h)))
    return h


def dg_c2p_net_destroy(net):
    load().dg_c2p_net_destroy(net)


def dg_c2p_net_get_params(net):
    import numpy as np
    p = np.zeros(N_NET_PARAMS, dtype=np.float32)
    _check(load().dg_c2p_net_get_params(net, p.ctypes.data))
    return p


def dg_c2p_net_guess(net, count, gamma, cons, p_guess, stream=None):
    import torch
    _check(load().dg_c2p_net_guess(net, int(count), float(gamma), _ptr(cons, 5 * count, torch.float64, "cons"),
                                   _ptr(p_guess, count, torch.float64, "p_guess"), _stream(stream)))


def dg_c2p_net_grad(net, count, cons, p, grad, loss, stream=None):
    import torch
    _check(load().dg_c2p_net_grad(net, int(count), _ptr(cons, 5 * count, torch.float64, "cons"),
                                  _ptr(p, count, torch.float64, "p"), _ptr(grad, N_NET_PARAMS, torch.float32, "grad"),
                                  _ptr(loss, 1, torch.float32, "loss"), _stream(stream)))


def dg_c2p_net_train(net, count, cons, p, epochs, batch, lr, loss_per_epoch=None, stream=None):
    import torch
    _check(load().dg_c2p_net_train(net, int(count), _ptr(cons, 5 * count, torch.float64, "cons"),
                                   _ptr(p, count, torch.float64, "p"), int(epochs), int(batch), float(lr),
                                   _ptr(loss_per_epoch, epochs, torch.float32, "loss_per_epoch"), _stream(stream)))


PROFILE_CLASSES = ("primitives", "stage", "limit", "fix", "dt", "other", "final")


def dg_profile_enable(mesh, on: bool = True):
    _check(load().dg_profile_enable(mesh, 1 if on else 0))


def dg_profile_read(mesh) -> dict:
    """{class: (total_ms, launches)} accumulated since the last read."""
    n = len(PROFILE_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(load().dg_profile_read(mesh, ms, cnt, n))
    return {c: (ms[i], cnt[i]) for i, c in enumerate(PROFILE_CLASSES)}


def dg_last_error() -> str:
    return load().dg_last_error().decode()
