"""Rayleigh-Taylor instability with the colour-gradient step (Sec. III.H) on
the GPU: parity against the FP64 oracle and the spike positions of Table 6."""
import numpy as np
import pytest

from helpers import gpu_run, oracle_run, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

# Table 6, D3Q19-CGM-CM column: spike position / W at t/t0 = 0, 0.5, ..., 4.
PAPER_Q19 = [1.897, 1.897, 1.753, 1.592, 1.381, 1.126, 0.844, 0.546, 0.242]


def rt_setup(W):
    """sqrt(g W) = 0.04, Re = W sqrt(g W)/nu = 512, At = 0.5 (rho 3 over 1),
    alpha_b = 1/3 and alpha_r = 7/9 for the density ratio 3, no surface tension
    (A = 0), walls at the bottom and top, F = (rho - 2) g with g = (0, -g, 0)."""
    g = 0.04 ** 2 / W
    nu = W * 0.04 / 512.0
    omega = 1.0 / (3.0 * nu + 0.5)
    kw = dict(periodic=(True, False, True), g=(0.0, -g, 0.0), rho_ref=2.0, physics="cgm", alpha_r=7.0 / 9.0,
              alpha_b=1.0 / 3.0, A=0.0, beta=0.7)
    return omega, kw, (W / g) ** 0.5


def errors(r, o, W):
    """rho and phase: relative L2.  u: L2 error over max(||u||, sqrt(N) U) with
    U = sqrt(g W) = 0.04, the problem's velocity scale: the flow starts at rest,
    so early on ||u|| is far below the rounding of populations of size ~rho/3."""
    n = o["rho"].size
    du = np.linalg.norm(r["u"] - o["u"]) / max(np.linalg.norm(o["u"]), np.sqrt(n) * 0.04)
    return {"rho": rel_l2(r["rho"], o["rho"]), "u": du, "phase": rel_l2(r["phase"], o["phase"])}


def spike(phase, W):
    """Lowest zero of the order parameter on the column x = z = W/2 (where the
    initial interface dips deepest), linearly interpolated, in units of W."""
    col = phase[W // 2, :, W // 2]
    for y in range(len(col) - 1):
        if col[y] < 0 <= col[y + 1]:
            return (y + col[y] / (col[y] - col[y + 1])) / W
    return float("nan")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_rt_parity_w32(precision, tol):
    """W = 32 (32 x 128 x 32), 400 steps = t/t0 0.5: every node."""
    W = 32
    omega, kw, _ = rt_setup(W)
    rho, u, ph = inputs.rayleigh_taylor(W)
    shape = (W, 4 * W, W)
    o = oracle_run(shape, omega, 400, rho, u, phase=ph, **kw)
    r = gpu_run(shape, omega, 400, rho, u, phase=ph, precision=precision, **kw)
    errs = errors(r, o, W)
    assert max(errs.values()) <= tol, errs


def test_rt_full_size_first_steps_fp32():
    """The paper's 64 x 256 x 64 box, 8 steps, every node."""
    W = 64
    omega, kw, _ = rt_setup(W)
    rho, u, ph = inputs.rayleigh_taylor(W)
    shape = (W, 4 * W, W)
    o = oracle_run(shape, omega, 8, rho, u, phase=ph, **kw)
    r = gpu_run(shape, omega, 8, rho, u, phase=ph, precision="fp32", **kw)
    errs = errors(r, o, W)
    assert max(errs.values()) <= 1e-5, errs


def test_rt_spike_positions_against_table6_fp32():
    """Spike position at t/t0 = 0 .. 4 (t0 = sqrt(W/g) = 1600 steps) against the
    paper's own D3Q19 column, within 0.02 W.  At t/t0 = 0.5 the printed value
    repeats the t = 0 one while every other column of Table 6 has moved to
    1.84-1.87; there the band is 0.06 W."""
    from paper_2010_01628_gb300 import binding as L
    W = 64
    omega, kw, t0 = rt_setup(W)
    rho, u, ph = inputs.rayleigh_taylor(W)
    shape = (W, 4 * W, W)
    phys = kw.pop("physics")
    ctx = L.lbm_create(shape, omega, physics=phys, precision="fp32", **kw)
    got = []
    try:
        L.lbm_init_fields(ctx, rho, u, phase=ph)
        done = 0
        for k in range(9):
            target = int(round(0.5 * k * t0))
            L.lbm_step(ctx, target - done)
            done = target
            got.append(spike(L.lbm_fields(ctx, shape, want=("phase",))["phase"], W))
    finally:
        L.lbm_destroy(ctx)
    got = np.array(got)
    assert np.all(np.diff(got) < 0), got
    band = np.full(9, 0.02)
    band[1] = 0.06
    assert np.all(np.abs(got - np.array(PAPER_Q19)) <= band), (got, PAPER_Q19)
