"""GB300 (sm_103a) nodal DG hot path of arXiv:1609.00098 behind the libdg C ABI.

``_binding`` exposes one Python function per C entry point of include/dg.h
(argument marshalling only); ``Mesh`` is a small owner of a ``dg_mesh*`` for
convenience.  Importing this package loads libdg.so and raises if it is not
built; nothing here computes on the CPU.
"""
from __future__ import annotations

from . import _binding as abi
from ._binding import DGError, make_desc

__all__ = ["abi", "DGError", "make_desc", "Mesh"]


class Mesh:
    """Owns a dg_mesh created on the current CUDA device."""

    def __init__(self, system=0, K=(4, 4, 4), n=4, flux=0, limiter=0, precision=0, gamma=1.4,
                 lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), tvb_M=0.0, beta=2.0, d_atm=1e-12, tau_atm=1e-14,
                 mrs_alpha=0.0, bc=(0, 0, 0), exact=0, exact_par=(0.0,) * 6):
        abi.load()
        self.desc = make_desc(system, K, n, flux, limiter, precision, gamma, lo, hi, tvb_M, beta, d_atm, tau_atm,
                              mrs_alpha, bc, exact, exact_par)
        self.h = abi.dg_mesh_create(self.desc)
        self.K, self.n = tuple(K), n
        self.E = K[0] * K[1] * K[2]
        self.nn = n ** 3
        self.system = system

    def close(self):
        if getattr(self, "h", None):
            abi.dg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.E, 5, self.nn)

    def state(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def coords(self):
        import torch
        xyz = torch.empty((3, self.E * self.nn), dtype=torch.float64, device="cuda")
        abi.dg_node_coords(self.h, xyz)
        return xyz

    def from_prim(self, prim):
        U = self.state()
        abi.dg_prim2con(self.h, prim.contiguous(), U)
        return U

    def primitives(self, U):
        import torch
        P = torch.empty((self.E, 4, self.nn), dtype=torch.float64, device="cuda")
        abi.dg_primitives(self.h, U, P)
        return P

    def rhs(self, U):
        R = self.state()
        abi.dg_rhs(self.h, U, R)
        return R

    def cfl_dt(self, U, cfl):
        import torch
        dt = torch.empty(1, dtype=torch.float64, device="cuda")
        abi.dg_compute_dt(self.h, U, cfl, dt)
        return dt

    def rk3_step(self, U, dt=0.0, cfl=0.0, dt_used=None, troubled=None):
        abi.dg_rk3_step(self.h, U, dt, cfl, dt_used, troubled)
        return U

    def limit(self, U, troubled=None):
        abi.dg_limit(self.h, U, troubled)
        return U

    def fix(self, U):
        abi.dg_fix(self.h, U)
        return U

    def summaries(self, U):
        import torch
        S = torch.empty((self.E, 5, 10), dtype=torch.float64, device="cuda")
        abi.dg_limiter_summaries(self.h, U, S)
        return S

    def sync_status(self) -> int:
        return abi.dg_sync_status(self.h)

    def ab3_step(self, U, dt, troubled=None):
        """Third-order Adams-Bashforth step with a fixed dt (two SSP-RK3 start-up steps)."""
        abi.dg_ab3_step(self.h, U, dt, troubled)
        return U

    def ab3_reset(self):
        abi.dg_ab3_reset(self.h)

    @property
    def t(self) -> float:
        """Mesh time (advanced by steps of meshes with analytic boundaries)."""
        return abi.dg_mesh_get_time(self.h)

    @t.setter
    def t(self, value):
        abi.dg_mesh_set_time(self.h, value)

    def set_option(self, option, value):
        """Mixed-path option: abi.OPT_TENSOR_CORE_CONTRACTION or abi.OPT_C2P_KAPPA_SWITCH."""
        abi.dg_mesh_set_option(self.h, option, value)

    def set_c2p_net(self, net):
        """Attach (or with None detach) a learned con2prim guess network."""
        abi.dg_mesh_set_c2p_net(self.h, net)
