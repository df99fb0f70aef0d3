"""D3Q27 single-phase step (App. D) on the GPU against the FP64 numpy oracle."""
import math

import numpy as np
import pytest

from helpers import rel_l2
from oracle import q27_oracle as Q
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def oracle(shape, omega, steps, rho, u, collision="factorised", **kw):
    d = Q.Domain27(shape, omega, collision=collision, **kw)
    d.init(rho, u)
    d.step(steps)
    return d.fields()


def gpu(shape, omega, steps, rho, u, precision, collision="cm", **kw):
    from paper_2010_01628_gb300 import binding as L
    ctx = L.lbm_create(shape, omega, precision=precision, lattice="d3q27", collision=collision, **kw)
    try:
        L.lbm_init_fields(ctx, np.ascontiguousarray(rho), np.ascontiguousarray(u))
        L.lbm_step(ctx, steps)
        out = L.lbm_fields(ctx, shape)
    finally:
        L.lbm_destroy(ctx)
    return out["rho"], out["u"]


def check(g, o, tol):
    errs = (rel_l2(g[0], o[0]), rel_l2(g[1], o[1]))
    assert max(errs) <= tol, errs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("collision", ["cm", "rm"])
def test_taylor_green_32(precision, collision):
    """Sec. III.E 3D Taylor-Green (the App. D timing case), u0 = 0.05, tau = 0.53, 60 steps."""
    rho, u = inputs.taylor_green_3d(32, u0=0.05)
    o = oracle((32, 32, 32), 1 / 0.53, 60, rho, u, collision="factorised" if collision == "cm" else "rm")
    g = gpu((32, 32, 32), 1 / 0.53, 60, rho, u, precision, collision)
    check(g, o, TOL[precision])


@pytest.mark.parametrize("shape,periodic", [((13, 9, 7), (True, False, False)), ((5, 6, 4), (False, False, False)),
                                            ((40, 3, 2), (True, True, True))])
@pytest.mark.parametrize("collision", ["cm", "rm"])
def test_walls_lid_force_against_dense_oracle_fp64(shape, periodic, collision):
    """Half-way bounce-back, a moving lid and a body force; the GPU against the
    oracle's definitional (dense) collision; nx = 13 and 40 leave ragged blocks."""
    rho, u = inputs.random_fields(shape, seed=81, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.04, 0.0, 0.01), g=(2e-5, -1e-5, 5e-6))
    o = oracle(shape, 1.35, 10, rho, u, collision="dense" if collision == "cm" else "dense_rm", **kw)
    g = gpu(shape, 1.35, 10, rho, u, "fp64", collision, **kw)
    check(g, o, 1e-12)


def test_reductions_and_configurations():
    from paper_2010_01628_gb300 import binding as L
    shape = (20, 12, 10)
    rho, u = inputs.random_fields(shape, seed=82, u_amp=0.02)
    d = Q.Domain27(shape, 1.4, periodic=(True, False, True), g=(1e-5, 0.0, 0.0))
    d.init(rho, u)
    d.step(7)
    ro, uo = d.fields()
    ctx = L.lbm_create(shape, 1.4, precision="fp64", lattice="d3q27", periodic=(True, False, True), g=(1e-5, 0.0, 0.0))
    try:
        L.lbm_init_fields(ctx, rho, u)
        L.lbm_step(ctx, 7)
        m, p, _ = L.lbm_reduce(ctx)
        with pytest.raises(Exception):
            L.lbm_set_launch_shape(ctx, 1, 64, 2, 1)
        L.lbm_autotune(ctx, None)
        assert L.lbm_get_launch_shape(ctx)["variant"] == "direct"
    finally:
        L.lbm_destroy(ctx)
    assert math.isclose(m, ro.sum(), rel_tol=1e-13)
    np.testing.assert_allclose(p, (ro * uo).sum(axis=(1, 2, 3)), rtol=0, atol=1e-12 * m)
    for kw in (dict(physics="mhd"), dict(precision="bf16"), dict(periodic=(True, False, True), wall_model="regularized")):
        with pytest.raises(Exception):
            L.lbm_create((8, 8, 8), 1.2, lattice="d3q27", **kw)
