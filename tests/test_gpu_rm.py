"""Raw-moment variant (App. C, N = I) on the GPU against the FP64 oracle."""
import pytest

from helpers import gpu_run, oracle_run, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 4e-3}


def compare(g, o, tol):
    errs = {k: rel_l2(g[k], o[k]) for k in ("rho", "u")}
    assert max(errs.values()) <= tol, errs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_taylor_green_32_raw_moments(precision):
    """Sec. III.E 3D Taylor-Green (the App. D timing case), u0 = 0.05, 200 steps."""
    rho, u = inputs.taylor_green_3d(32, u0=0.05)
    o = oracle_run((32, 32, 32), 1 / 0.53, 200, rho, u, collision="rm")
    r = gpu_run((32, 32, 32), 1 / 0.53, 200, rho, u, precision=precision, collision="rm")
    compare(r, o, TOL[precision])


@pytest.mark.parametrize("shape,periodic", [((37, 9, 5), (True, False, False)), ((6, 5, 7), (False, False, False)),
                                            ((70, 4, 3), (True, True, True))])
def test_walls_lid_and_force_fp64(shape, periodic):
    """Walls, a moving lid and a body force (the printed forcing of App. C)."""
    rho, u = inputs.random_fields(shape, seed=71, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.04, 0.0, 0.01), g=(2e-5, -1e-5, 5e-6), collision="rm")
    o = oracle_run(shape, 1.45, 20, rho, u, **kw)
    r = gpu_run(shape, 1.45, 20, rho, u, precision="fp64", **kw)
    compare(r, o, 1e-12)


def test_unforced_matches_the_mrt_definition_fp64():
    """Without a force the printed list is the raw-moment MRT: the GPU against
    the oracle's dense (definition) collision."""
    shape = (9, 8, 7)
    rho, u = inputs.random_fields(shape, seed=72, u_amp=0.05)
    o = oracle_run(shape, 1.2, 15, rho, u, collision="rm", closed_form=False)
    r = gpu_run(shape, 1.2, 15, rho, u, precision="fp64", collision="rm")
    compare(r, o, 1e-12)


def test_launch_shapes_and_configurations():
    from paper_2010_01628_gb300 import binding as L
    ctx = L.lbm_create((64, 8, 4), 1.2, precision="bf16", collision="rm")
    try:
        with pytest.raises(Exception):
            L.lbm_set_launch_shape(ctx, 1, 64, 2, 1)
        with pytest.raises(Exception):
            L.lbm_set_launch_shape(ctx, 2, 128, 0, 1)
        with pytest.raises(Exception):
            L.lbm_set_launch_shape(ctx, 4, 128, 0, 1)
        L.lbm_autotune(ctx, None)
        assert L.lbm_get_launch_shape(ctx)["variant"] == "direct"
    finally:
        L.lbm_destroy(ctx)
    for kw in (dict(physics="sc", G=-5.0), dict(periodic=(True, False, True), wall_model="regularized")):
        with pytest.raises(Exception):
            L.lbm_create((8, 8, 8), 1.2, collision="rm", **kw)
