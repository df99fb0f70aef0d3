"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point include/lbm.h declares, and rejects invalid arguments before any
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_01628_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_fields", "lbm_init_fields", "lbm_reduce", "lbm_destroy",
                     "lbm_last_error", "lbm_get_populations", "lbm_set_populations"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.lbm_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert lib.lbm_status_string(s)


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_2010_01628_gb300 import binding as L
    ctx = ctypes.c_void_p()

    def create(nx=8, ny=8, nz=8, omega=1.2, ob=1.0, physics=0, precision=1, lattice=0):
        g = L.lbm_grid(nx, ny, nz, 7)
        r = L.lbm_relax(omega, ob, 1.0, 1.0)
        f = L.lbm_forcing()
        p = L.lbm_physparams()
        p.tau_m = 1.0
        return L._lib.lbm_create(ctypes.byref(ctx), ctypes.byref(g), lattice, ctypes.byref(r), ctypes.byref(f),
                                 physics, ctypes.byref(p), precision, None)

    assert create(nx=0) == L.LBM_ERR_ARG
    assert create(ny=70000) == L.LBM_ERR_ARG
    assert create(nx=2048, ny=2048, nz=1024) == L.LBM_ERR_ARG  # >= 2^31 nodes
    assert create(omega=2.0) == L.LBM_ERR_ARG
    assert create(omega=0.0) == L.LBM_ERR_ARG
    assert create(ob=1.2) == L.LBM_ERR_UNSUPPORTED
    assert create(lattice=2) == L.LBM_ERR_UNSUPPORTED
    assert create(lattice=1, precision=2) == L.LBM_ERR_UNSUPPORTED  # D3Q27: FP32/FP64 only
    assert create(lattice=1, physics=2) == L.LBM_ERR_UNSUPPORTED  # D3Q27: single phase only
    assert create(physics=1, precision=2) == L.LBM_ERR_UNSUPPORTED
    assert create(precision=9) == L.LBM_ERR_ARG
    assert L._lib.lbm_step(None, 1) == L.LBM_ERR_ARG
    assert L._lib.lbm_fields(None, None, None, None, None) == L.LBM_ERR_ARG


def test_dipole_initial_energy_and_enstrophy():
    """Sec. III.D states E(0) = 2 and Psi(0) = 800 for the dipole of w_e = 299.56,
    r0 = 0.1 in [-1, 1]^2: the input recipe reproduces both (second-order
    central differences, D_lb = 512)."""
    import numpy as np
    from paper_2010_01628_gb300 import inputs
    D = 512
    _, u = inputs.dipole(D, 1.0)
    h = 1.0 / D
    E = 0.5 * (u[0] ** 2 + u[1] ** 2).sum() * h * h
    w = np.gradient(u[1, 0], h, axis=1) - np.gradient(u[0, 0], h, axis=0)
    P = 0.5 * (w ** 2).sum() * h * h
    assert abs(E - 2.0) < 1e-3
    assert abs(P - 800.0) < 1.0
