"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1609_00098_gb300 import build as b
    return b.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("dg_mesh_create", "dg_rhs", "dg_rk3_step", "dg_limit", "dg_con2prim"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dg_[a-z0-9_]+)$", out, flags=re.M))
    assert _declared() <= exported


def test_binding_covers_every_entry_point(lib_path):
    from paper_1609_00098_gb300 import _binding
    assert _declared() <= set(_binding.SIGNATURES)
    for name in _declared():
        if name != "dg_mesh_desc":
            assert callable(getattr(_binding, name)), name


def test_argument_errors_need_no_gpu(lib_path):
    """Invalid descriptors are rejected synchronously, before any CUDA call."""
    import paper_1609_00098_gb300 as pkg
    for bad in (dict(n=1), dict(n=9), dict(system=2), dict(flux=3), dict(limiter=5), dict(gamma=1.0),
                dict(K=(0, 1, 1)), dict(hi=(0.0, 1.0, 1.0)), dict(beta=0.0), dict(tvb_M=-1.0),
                dict(precision=2), dict(gamma=float("nan")),
                dict(system=1, flux=2),                                   # Roe is Newtonian only
                dict(system=1, limiter=3), dict(limiter=3, mrs_alpha=-1.0),  # MRS: Newtonian, alpha >= 0
                dict(bc=(2, 0, 0)), dict(exact=2),
                dict(bc=(1, 0, 0)),                                       # analytic faces need an exact solution
                dict(bc=(1, 0, 0), exact=1, system=1),                    # ... the Newtonian system
                dict(bc=(0, 1, 0), exact=1, limiter=1)):                  # ... and no limiter
        with pytest.raises(pkg.DGError) as ei:
            pkg.abi.dg_mesh_create(pkg.make_desc(**bad))
        assert ei.value.status == pkg.abi.DG_ERR_ARG
    with pytest.raises(pkg.DGError):
        pkg.abi.dg_con2prim(-1, 1.4, None, None, stream=0)


@pytest.mark.parametrize("n", range(2, 9))
def test_library_tables_match_closed_forms_and_oracle(lib_path, n):
    """The library's LGL tables (host call, no GPU) satisfy the closed forms and
    identities of Sec. 3.1 and equal the oracle's bit for bit, which the FP64
    path needs to reproduce the oracle operation for operation."""
    import numpy as np
    import oracle
    from paper_1609_00098_gb300 import _binding as abi
    x, w, D, r1 = abi.dg_lgl_tables(n)
    xo, wo = oracle.lgl(n)
    assert np.array_equal(x, xo) and np.array_equal(w, wo)
    assert np.array_equal(D, oracle.diffmat(n))
    assert np.array_equal(r1, oracle.legendre_vinv(n)[1])
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.max(np.abs(D @ x - 1.0)) < 1e-12
