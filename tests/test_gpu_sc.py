"""Shan-Chen pseudopotential multiphase (Sec. III.G) on the GPU against the
FP64 oracle, plus the static-bubble physics at the paper's full size."""
import math

import numpy as np
import pytest

from helpers import gpu_run, oracle_run, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

G = -5.0
NU = 0.0333
OMEGA = 1.0 / (3.0 * NU + 0.5)
# FP32: both phases sit at O(1) density deviations, where FP32 arithmetic
# rounds at eps32 * rho per population and step.  The FP64 oracle perturbed by
# noise of that size moves u by 0.85e-5 to 1.15e-5 on these cases (three seeds
# each), and the GPU lands on the same values; the bound is twice that.
TOL = {"fp64": 1e-12, "fp32": 2e-5}
FIELDS = ("rho", "u", "phase")


def compare(g, o, tol, fields=FIELDS):
    errs = {k: rel_l2(g[k], o[k]) for k in fields}
    for k, e in errs.items():
        assert e <= tol, (k, errs)
    return errs


def pressure(rho):
    psi = 1.0 - np.exp(-rho)
    return rho / 3.0 + G / 6.0 * psi * psi


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_bubble_parity_ragged(precision):
    """Sharp 1.95 / 0.15 droplet (the paper's start), periodic box with
    nx = 40 (one block of 32 and a ragged tail of 8), 60 steps."""
    shape = (40, 36, 34)
    rho, u = inputs.static_bubble(shape, 9.0, noise=1e-3, seed=5)
    o = oracle_run(shape, OMEGA, 60, rho, u, physics="sc", G=G)
    r = gpu_run(shape, OMEGA, 60, rho, u, physics="sc", G=G, precision=precision)
    compare(r, o, TOL[precision])


def test_fields_before_any_step_fp64():
    """psi, rho and u (with +F/2) of the initial state."""
    shape = (12, 10, 9)
    rho, u = inputs.static_bubble(shape, 3.0, width=1.0, noise=1e-3, seed=7)
    o = oracle_run(shape, OMEGA, 0, rho, u, physics="sc", G=G)
    r = gpu_run(shape, OMEGA, 0, rho, u, physics="sc", G=G, precision="fp64")
    compare(r, o, 1e-13)


@pytest.mark.parametrize("shape", [(5, 6, 7), (1, 8, 1), (33, 4, 3)])
def test_brute_force_walls_lid_force_dense_oracle(shape):
    """Tiny boxes with walls on y and z, a moving lid and a body force,
    against the definitional dense-solve oracle."""
    rho, u = inputs.static_bubble(shape, 2.0, width=1.0, noise=2e-2, seed=11)
    kw = dict(periodic=(True, False, False), lid_u=(0.03, 0.0, 0.01), g=(1e-4, -2e-4, 0.0), G=G)
    o = oracle_run(shape, 1.3, 12, rho, u, physics="sc", closed_form=False, **kw)
    r = gpu_run(shape, 1.3, 12, rho, u, physics="sc", precision="fp64", **kw)
    compare(r, o, 1e-12)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True), (False, True, True)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_walls_and_gravity(periodic, precision):
    """A droplet next to a wall under gravity: the wall rule for psi (own value)
    and the body force added to the interaction force."""
    shape = (13, 11, 9)
    rho, u = inputs.static_bubble(shape, 3.5, width=1.0, centre=(6.0, 3.0, 4.0), noise=1e-3, seed=6)
    kw = dict(periodic=periodic, lid_u=(0.02, 0.0, 0.0), g=(0.0, -1e-4, 0.0), G=G)
    o = oracle_run(shape, 1.2, 25, rho, u, physics="sc", **kw)
    r = gpu_run(shape, 1.2, 25, rho, u, physics="sc", precision=precision, **kw)
    compare(r, o, TOL[precision])


def test_reductions_conserve_mass_and_momentum_fp64():
    """lbm_reduce's FP64 sums against the oracle's fields; the pair force keeps
    the periodic box's momentum."""
    from paper_2010_01628_gb300 import binding as L
    shape = (24, 20, 18)
    rho, u = inputs.static_bubble(shape, 6.0, noise=1e-3, seed=8)
    o = oracle_run(shape, OMEGA, 30, rho, u, physics="sc", G=G)
    ctx = L.lbm_create(shape, OMEGA, physics="sc", G=G, precision="fp64")
    try:
        L.lbm_init_fields(ctx, rho, u)
        m0, p0, _ = L.lbm_reduce(ctx)
        L.lbm_step(ctx, 30)
        m1, p1, res = L.lbm_reduce(ctx)
    finally:
        L.lbm_destroy(ctx)
    assert math.isclose(m1, o["rho"].sum(), rel_tol=1e-13)
    assert math.isclose(m1, m0, rel_tol=1e-13)
    mom = (o["rho"] * o["u"]).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(p1, mom, rtol=0, atol=1e-12 * m1)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-12 * m1)
    assert res > 0


def test_create_rejects_unsupported_sc_configurations():
    from paper_2010_01628_gb300 import binding as L
    with pytest.raises(Exception):
        L.lbm_create((8, 8, 8), OMEGA, physics="sc", G=G, precision="fp16")
    with pytest.raises(Exception):
        L.lbm_create((8, 8, 8), OMEGA, physics="sc", G=float("nan"))


@pytest.mark.parametrize("radius", [20.0, 30.0])
def test_full_size_static_bubble_fp32(radius):
    """The paper's configuration (100^3 periodic, nu = 0.0333, G = -5, sharp
    1.95 / 0.15 droplet) for 12 steps: every node against the oracle."""
    shape = (100, 100, 100)
    rho, u = inputs.static_bubble(shape, radius)
    o = oracle_run(shape, OMEGA, 12, rho, u, physics="sc", G=G)
    r = gpu_run(shape, OMEGA, 12, rho, u, physics="sc", G=G, precision="fp32")
    compare(r, o, TOL["fp32"])


def test_flat_interface_coexistence_fp32():
    """FP32 slab converges to the oracle's coexistence densities (1.88847 /
    0.119443 at G = -5, nu = 0.1) to FP32 accuracy."""
    from paper_2010_01628_gb300 import binding as L
    ny = 64
    rho, u = inputs.static_bubble((1, ny, 1), ny / 4.0, width=2.0, axes=(1,))
    ctx = L.lbm_create((1, ny, 1), 1.0 / (0.3 + 0.5), physics="sc", G=G, precision="fp32")
    try:
        L.lbm_init_fields(ctx, rho, u)
        L.lbm_step(ctx, 12000)
        out = L.lbm_fields(ctx, (1, ny, 1))
    finally:
        L.lbm_destroy(ctx)
    o = oracle_run((1, ny, 1), 1.0 / (0.3 + 0.5), 12000, rho, u, physics="sc", G=G)
    r = out["rho"]
    assert abs(r[0, ny // 2, 0] - o["rho"][0, ny // 2, 0]) < 1e-5
    assert abs(r[0, 0, 0] - o["rho"][0, 0, 0]) < 1e-5


def test_laplace_law_paper_configuration_fp32():
    """Fig. 11: on 100^3 with R in [15, 30] the pressure jump (equation of
    state p = rho/3 + (G/6) psi^2, droplet centre against the far corner) is
    linear in 1/R: a straight line explains >= 98 % of the variance and no
    point is off it by more than 4 %.  With the interface's finite width the
    jump follows dp = 2 sigma / R + b / R^2 (a Tolman-type first correction)
    to 1 %, sigma > 0.  12000 steps per radius (converged to 0.1 % by then)."""
    from paper_2010_01628_gb300 import binding as L
    shape = (100, 100, 100)
    radii = np.array([15.0, 20.0, 25.0, 30.0])
    dp = []
    for R in radii:
        rho, u = inputs.static_bubble(shape, R)
        ctx = L.lbm_create(shape, OMEGA, physics="sc", G=G, precision="fp32")
        try:
            L.lbm_init_fields(ctx, rho, u)
            L.lbm_step(ctx, 12000)
            out = L.lbm_fields(ctx, shape)
        finally:
            L.lbm_destroy(ctx)
        r = out["rho"]
        dp.append(pressure(r[50, 50, 50]) - pressure(r[0, 0, 0]))
    dp = np.array(dp)
    assert np.all(dp > 0) and np.all(np.diff(dp) < 0)
    A = np.vstack([1.0 / radii, np.ones_like(radii)]).T
    coef, *_ = np.linalg.lstsq(A, dp, rcond=None)
    resid = dp - A @ coef
    r2 = 1.0 - (resid ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert r2 >= 0.98 and np.abs(resid / dp).max() <= 0.04, (dp, coef, r2)
    B = np.vstack([1.0 / radii, 1.0 / radii ** 2]).T
    (two_sigma, b), *_ = np.linalg.lstsq(B, dp, rcond=None)
    assert two_sigma > 0 and np.abs((dp - B @ np.array([two_sigma, b])) / dp).max() <= 0.01, (dp, two_sigma, b)


@pytest.mark.parametrize("precision,threads,lz", [("fp64", 256, 7), ("fp32", 256, 16), ("fp32", 512, 32)])
@pytest.mark.parametrize("shape,periodic", [((40, 36, 34), (True, True, True)), ((13, 11, 9), (False, False, False)),
                                            ((70, 5, 6), (True, False, True)), ((1, 30, 20), (True, True, True))])
def test_fused_kernel_against_oracle(precision, threads, lz, shape, periodic):
    """The fused step (psi in a shared-memory ring, z-chunks of lz planes with
    ragged last chunks and tiles) against the oracle: periodic, all walls with a
    lid and gravity, mixed, and a one-node-thick slab."""
    rho, u = inputs.static_bubble(shape, min(shape[1:]) / 4.0, width=1.5, noise=1e-3, seed=13)
    # gravity only where a wall carries it (in a periodic box it accelerates the whole box)
    g = (0.0, 0.0, 0.0) if periodic[1] else (0.0, -5e-5, 0.0)
    kw = dict(periodic=periodic, G=G, g=g, lid_u=(0.02, 0.0, 0.0))
    o = oracle_run(shape, OMEGA, 25, rho, u, physics="sc", **kw)
    r = gpu_run(shape, OMEGA, 25, rho, u, physics="sc", precision=precision, launch=(3, threads, lz, 1), **kw)
    compare(r, o, TOL[precision])


def test_fused_and_two_pass_agree_fp64():
    from paper_2010_01628_gb300 import binding as L
    shape = (40, 36, 34)
    rho, u = inputs.static_bubble(shape, 9.0, noise=1e-3, seed=5)
    out = []
    for launch in ((0, 64, 0, 1), (3, 256, 32, 1)):
        r = gpu_run(shape, OMEGA, 40, rho, u, physics="sc", G=G, precision="fp64", launch=launch)
        out.append(r)
    for k in ("rho", "u", "phase"):
        np.testing.assert_allclose(out[0][k], out[1][k], rtol=0, atol=1e-14)


def test_fused_and_two_pass_agree_fp32():
    """FP32: the fused step reproduces the two-pass step on the same case (the
    two paths take the same psi, force sum and collision in the same order)."""
    shape = (40, 36, 34)
    rho, u = inputs.static_bubble(shape, 8.5, width=1.5, noise=1e-3, seed=13)
    out = [gpu_run(shape, OMEGA, 25, rho, u, physics="sc", G=G, precision="fp32", launch=launch)
           for launch in ((0, 64, 0, 1), (3, 256, 16, 1), (3, 512, 32, 1))]
    for other in out[1:]:
        for k in ("rho", "u", "phase"):
            assert rel_l2(other[k], out[0][k]) < 1e-6, k
