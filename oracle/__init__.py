"""FP64 CPU oracle for the nodal DG hot path of arXiv:1609.00098.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the C source here is compiled
with gcc, loaded with ctypes and never linked with anything under the product
package.

The C routines live in ``dg_oracle.c``; each cites the section or equation of
the paper it restates.  ``build()`` compiles them (``-O2 -ffp-contract=off
-fopenmp``) into ``oracle/_build/libdg_oracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_HDR = os.path.join(_HERE, "dg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdg_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Desc(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int),
        ("dim", ctypes.c_int),
        ("K", ctypes.c_int * 3),
        ("n", ctypes.c_int),
        ("flux", ctypes.c_int),
        ("limiter", ctypes.c_int),
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


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # DG_ORACLE_LIB names another build of this same source (the planted-mistake
    # tests load copies with one deliberate error through it)
    lib = ctypes.CDLL(os.environ.get("DG_ORACLE_LIB") or build())
    vp = ctypes.c_void_p
    ll = ctypes.c_longlong
    sig = {
        "or_lgl": (ctypes.c_int, [ctypes.c_int, _dp, _dp]),
        "or_diffmat": (ctypes.c_int, [ctypes.c_int, _dp, _dp]),
        "or_legendre_vinv": (ctypes.c_int, [ctypes.c_int, _dp, _dp]),
        "or_mesh_create": (vp, [ctypes.POINTER(Desc)]),
        "or_mesh_destroy": (None, [vp]),
        "or_num_elements": (ll, [vp]),
        "or_nodes_per_element": (ctypes.c_int, [vp]),
        "or_node_coords": (None, [vp, _dp]),
        "or_prim2con": (None, [ctypes.c_int, ctypes.c_double, ll, _dp, _dp]),
        "or_con2prim": (ll, [ll, ctypes.c_double, _dp, _dp, _dp, _ip, _ip]),
        "or_primitives": (ll, [vp, _dp, _dp]),
        "or_rhs": (ll, [vp, _dp, _dp]),
        "or_lambda_max": (ctypes.c_double, [vp, _dp]),
        "or_cfl_dt": (ctypes.c_double, [vp, _dp, ctypes.c_double]),
        "or_limiter_summaries": (None, [vp, _dp, _dp]),
        "or_limit": (ll, [vp, _dp, _up]),
        "or_fix": (ll, [vp, _dp]),
        "or_rk3_step": (ll, [vp, _dp, ctypes.c_double, _up]),
        "or_set_time": (None, [vp, ctypes.c_double]),
        "or_get_time": (ctypes.c_double, [vp]),
        "or_norms": (None, [vp, _dp, _dp, _dp, _dp]),
        "or_totals": (None, [vp, _dp, _dp]),
        "or_num_flux": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       _dp, _dp, _dp, _dp, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# LGL tables

def lgl(n: int):
    """LGL nodes and weights (Sec. 3.1)."""
    lib = _load()
    x = np.zeros(n)
    w = np.zeros(n)
    if lib.or_lgl(n, _ptr(x), _ptr(w)):
        raise ValueError(f"bad n={n}")
    return x, w


def diffmat(n: int) -> np.ndarray:
    """Differentiation matrix D[i, l] = ell_l'(x_i) (eq:405)."""
    lib = _load()
    x, _ = lgl(n)
    D = np.zeros(n * n)
    lib.or_diffmat(n, _ptr(x), _ptr(D))
    return D.reshape(n, n)


def legendre_vinv(n: int) -> np.ndarray:
    lib = _load()
    x, _ = lgl(n)
    V = np.zeros(n * n)
    if lib.or_legendre_vinv(n, _ptr(x), _ptr(V)):
        raise ValueError("singular Vandermonde")
    return V.reshape(n, n)


# ---------------------------------------------------------------------------
# point-wise physics

def prim2con(system: int, gamma: float, prim: np.ndarray) -> np.ndarray:
    """prim: (5, N) rows rho, vx, vy, vz, p -> conserved (5, N)."""
    lib = _load()
    prim = _f64(prim)
    N = prim.shape[1]
    out = np.zeros((5, N))
    lib.or_prim2con(system, gamma, N, _ptr(prim), _ptr(out))
    return out


def con2prim(gamma: float, cons: np.ndarray, guess: np.ndarray | None = None):
    """SR con2prim.  Returns (prim (5, N), iterations (N,), status (N,))."""
    lib = _load()
    cons = _f64(cons)
    N = cons.shape[1]
    prim = np.zeros((5, N))
    it = np.zeros(N, dtype=np.int32)
    st = np.zeros(N, dtype=np.int32)
    g = None if guess is None else _f64(guess)
    lib.or_con2prim(N, gamma, _ptr(cons), _ptr(prim), None if g is None else _ptr(g),
                    _ptr(it, _ip), _ptr(st, _ip))
    return prim, it, st


def num_flux(system: int, gamma: float, flux: int, axis: int, uL, uR):
    """Numerical flux along +e_axis between conserved states uL, uR (Sec. 3.2).
    Returns (F*, F(uL), F(uR), speeds (lmin_L, lmax_L, lmin_R, lmax_R))."""
    lib = _load()
    uL = _f64(uL)
    uR = _f64(uR)
    Fs, FL, FR, sp = np.zeros(5), np.zeros(5), np.zeros(5), np.zeros(4)
    lib.or_num_flux(system, gamma, flux, axis, _ptr(uL), _ptr(uR), _ptr(Fs), _ptr(FL), _ptr(FR), _ptr(sp))
    return Fs, FL, FR, sp


# ---------------------------------------------------------------------------
# mesh-level operations

@dataclass
class MeshSpec:
    system: int = 0
    dim: int = 3
    K: tuple = (4, 4, 4)
    n: int = 4
    flux: int = 0
    limiter: int = 0
    gamma: float = 1.4
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    tvb_M: float = 0.0
    beta: float = 2.0
    d_atm: float = 1e-12
    tau_atm: float = 1e-14
    mrs_alpha: float = 0.0
    bc: tuple = (0, 0, 0)          # per axis: 0 periodic, 1 analytic exterior state
    exact: int = 0                 # 1: isentropic vortex (eq:isen_vortex) supplies exterior states
    exact_par: tuple = (0.0,) * 6  # isentropic vortex: beta, X0, Y0, U, V, W
    extra: dict = field(default_factory=dict)


class Mesh:
    """Owns an oracle mesh handle; arrays are numpy FP64 in the layout
    U[e][v][k][j][i]."""

    def __init__(self, spec: MeshSpec):
        lib = _load()
        self.spec = spec
        d = Desc()
        d.system = spec.system
        d.dim = spec.dim
        for a in range(3):
            d.K[a] = spec.K[a]
            d.lo[a] = spec.lo[a]
            d.hi[a] = spec.hi[a]
        d.n = spec.n
        d.flux = spec.flux
        d.limiter = spec.limiter
        d.gamma = spec.gamma
        d.tvb_M = spec.tvb_M
        d.beta = spec.beta
        d.d_atm = spec.d_atm
        d.tau_atm = spec.tau_atm
        d.mrs_alpha = spec.mrs_alpha
        for a in range(3):
            d.bc[a] = spec.bc[a]
        d.exact = spec.exact
        for i in range(6):
            d.exact_par[i] = spec.exact_par[i]
        self._d = d
        self.h = lib.or_mesh_create(ctypes.byref(d))
        if not self.h:
            raise ValueError(f"bad mesh spec {spec}")
        self.E = lib.or_num_elements(self.h)
        self.nn = lib.or_nodes_per_element(self.h)
        self.lib = lib

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_mesh_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (self.E, 5, self.nn)

    def coords(self) -> np.ndarray:
        """(3, E*nn) node coordinates in state order."""
        xyz = np.zeros(3 * self.E * self.nn)
        self.lib.or_node_coords(self.h, _ptr(xyz))
        return xyz.reshape(3, self.E * self.nn)

    def from_prim(self, prim: np.ndarray) -> np.ndarray:
        """prim (5, E*nn) in node order -> U (E, 5, nn)."""
        cons = prim2con(self.spec.system, self.spec.gamma, prim)
        return np.ascontiguousarray(cons.reshape(5, self.E, self.nn).transpose(1, 0, 2))

    def primitives(self, U) -> np.ndarray:
        U = _f64(U)
        P = np.zeros((self.E, 4, self.nn))
        self.lib.or_primitives(self.h, _ptr(U), _ptr(P))
        return P

    def rhs(self, U) -> np.ndarray:
        U = _f64(U)
        R = np.zeros_like(U)
        self.lib.or_rhs(self.h, _ptr(U), _ptr(R))
        return R

    def lambda_max(self, U) -> float:
        return self.lib.or_lambda_max(self.h, _ptr(_f64(U)))

    def cfl_dt(self, U, cfl: float) -> float:
        return self.lib.or_cfl_dt(self.h, _ptr(_f64(U)), cfl)

    def summaries(self, U) -> np.ndarray:
        U = _f64(U)
        S = np.zeros((self.E, 5, 10))
        self.lib.or_limiter_summaries(self.h, _ptr(U), _ptr(S))
        return S

    def limit(self, U):
        """Returns (limited copy, troubled bitmask per element)."""
        U = _f64(U).copy()
        t = np.zeros(self.E, dtype=np.uint8)
        self.lib.or_limit(self.h, _ptr(U), _ptr(t, _up))
        return U, t

    def fix(self, U):
        U = _f64(U).copy()
        n = self.lib.or_fix(self.h, _ptr(U))
        return U, n

    @property
    def t(self) -> float:
        """Mesh time; enters the method only through analytic exterior states."""
        return self.lib.or_get_time(self.h)

    @t.setter
    def t(self, value: float):
        self.lib.or_set_time(self.h, value)

    def rk3_step(self, U, dt: float, troubled: np.ndarray | None = None) -> np.ndarray:
        U = _f64(U).copy()
        self.lib.or_rk3_step(self.h, _ptr(U), dt, None if troubled is None else _ptr(troubled, _up))
        return U

    def run(self, U, steps: int, dt: float | None = None, cfl: float | None = None,
            t_end: float | None = None):
        """Advance `steps` SSP-RK3 steps (fixed dt, or CFL dt from the state at the
        start of each step).  With t_end, the last step is shortened to land on it."""
        U = _f64(U).copy()
        t = 0.0
        for s in range(steps):
            h = dt if dt is not None else self.cfl_dt(U, cfl)
            if t_end is not None:
                if t >= t_end:
                    break
                h = min(h, t_end - t)
            self.lib.or_rk3_step(self.h, _ptr(U), h, None)
            t += h
        return U, t

    def ab3_run(self, U, steps: int, dt: float):
        """Third-order Adams-Bashforth with a fixed dt (Sec. 3.4, the paper's other
        third-order integrator):
            U^{n+1} = U^n + dt (23/12 L^n - 16/12 L^{n-1} + 5/12 L^{n-2}),
        followed by the limiter and (SR) the conserved fix, as after an SSP-RK3
        stage.  The two right-hand sides missing at the start come from two
        SSP-RK3 steps, each recording L(U) of the state it starts from."""
        U = _f64(U).copy()
        hist = []
        for _ in range(steps):
            L = self.rhs(U)
            if len(hist) < 2:
                hist.append(L)
                U = self.rk3_step(U, dt)
                continue
            U = U + dt * ((23.0 / 12.0 * L - 16.0 / 12.0 * hist[-1]) + 5.0 / 12.0 * hist[-2])
            self.t = self.t + dt
            hist = [hist[-1], L]
            U, _ = self.limit(U)
            if self.spec.system == 1:
                U, _ = self.fix(U)
        return U

    def norms(self, U, V):
        l1 = np.zeros(5)
        l2 = np.zeros(5)
        self.lib.or_norms(self.h, _ptr(_f64(U)), _ptr(_f64(V)), _ptr(l1), _ptr(l2))
        return l1, l2

    def totals(self, U) -> np.ndarray:
        t = np.zeros(5)
        self.lib.or_totals(self.h, _ptr(_f64(U)), _ptr(t))
        return t
