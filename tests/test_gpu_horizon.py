"""Precision over the configurations' own horizons, per field, against the
FP64 oracle.

- Periodic body-force flow (g = 1e-6 along x, velocity noise 1e-3, tau = 0.6)
  for its full 1000 steps on a 96^3 box, in every storage precision.
- Colour-gradient droplets (density ratio 10, sigma = 1e-4, interface width 4,
  beta = 0.7, tau = 0.8, 10 % volume fraction) for their full 5000 steps on a
  48^3 box with radii 5-9 (the 256^3 recipe's radii 8-24 do not fit 48^3).

Fields are compared separately (relative L2 over the box): u, and the density
as its deviation from the reference state (rho - 1 for the single-phase flow,
rho(t) - rho(0) for the droplets), each against its own norm, beside the plain
relative L2 of rho.  A density near 1 makes the plain measure weak: an error
of 1e-5 in rho ~ 1 is a large error in a deviation of 1e-4.

Bounds: the stated targets (1e-12 FP64, 1e-5 FP32, 1e-3 FP16) on rho and u
where they hold, else what bounds the precision, measured:
- rho - 1 of the body-force flow has decayed to ~5e-7 (rms) by step 1000.  The
  oracle holds unshifted populations whose sum rounds at ulp(1) = 2.2e-16, so
  the FP64 comparison of rho - 1 stops near 1e-7 of its norm (bound 1e-6); the
  16-bit formats round the stored (f - w)/w at 2^-11 (FP16) and 2^-8 (BF16) of
  values ~1e-3, far above that deviation (no bound).
- In FP32 that rho - 1 follows the velocity error acoustically: u is within
  5e-6 of its norm (~5e-9 absolute), rho - 1 within ~3e-2 of its ~5e-7
  (bound 5e-2).
- BF16 storage of that flow: the oracle with exact arithmetic and its
  populations rounded to BF16 after every step already misses u by 1.4-1.9e-2
  (test_bf16_floor_of_the_body_force_flow); the GPU lands on that floor.
- The droplets' velocity is the spurious current, |u| <= 4e-4, against FP32
  rounding of unshifted colour populations of size up to rho/3 = 3.3: a few
  ulp of 3.3 (2.4e-7 each) per step put the FP32 u at ~1e-3 of its norm
  (bound 2e-3); FP64 at ~1e-12 (bound 1e-11).
"""
import numpy as np
import pytest

from helpers import gpu_run, oracle_run, oracle_run_stored, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

C2_N, C2_STEPS = 96, 1000
C4_N, C4_STEPS = 48, 5000

# relative L2 bounds per field
C2_BOUND = {
    "fp64": {"rho": 1e-12, "u": 1e-12, "drho": 1e-6},
    "fp32": {"rho": 1e-5, "u": 1e-5, "drho": 5e-2},
    "fp16": {"rho": 1e-3, "u": 1e-3},
    "bf16": {"rho": 4e-3, "u": 2e-2},
}
C4_BOUND = {
    "fp64": {"rho": 1e-12, "u": 1e-11, "drho": 1e-12, "phase": 1e-12},
    "fp32": {"rho": 1e-5, "u": 2e-3, "drho": 1e-4, "phase": 1e-5},
}


def errors(g, o, ref_rho, fields):
    e = {"rho": rel_l2(g["rho"], o["rho"]), "drho": rel_l2(g["rho"] - ref_rho, o["rho"] - ref_rho),
         "u": rel_l2(g["u"], o["u"])}
    for a, name in enumerate("xyz"):
        e["u" + name] = rel_l2(g["u"][a], o["u"][a])
    if "phase" in fields:
        e["phase"] = rel_l2(g["phase"], o["phase"])
    return e


@pytest.fixture(scope="module")
def c2_case():
    shape = (C2_N,) * 3
    rho, u = inputs.noise_box(shape, amp=1e-3, seed=1)
    o = oracle_run(shape, 1 / 0.6, C2_STEPS, rho, u, g=(1e-6, 0.0, 0.0))
    return rho, u, o


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_body_force_flow_full_horizon(c2_case, precision):
    rho, u, o = c2_case
    shape = (C2_N,) * 3
    g = gpu_run(shape, 1 / 0.6, C2_STEPS, rho, u, g=(1e-6, 0.0, 0.0), precision=precision)
    e = errors(g, o, 1.0, ())
    print(f"\nHORIZON body-force {C2_N}^3 x {C2_STEPS} {precision}: "
          + " ".join(f"{k}={v:.3e}" for k, v in e.items()))
    for k, b in C2_BOUND[precision].items():
        assert e[k] <= b, (k, e)


@pytest.fixture(scope="module")
def c4_case():
    n = C4_N
    rho, u, phase, _, _ = inputs.droplets(n, seed=3, r_min=5.0, r_max=9.0)
    sigma, tau, rho_r0, rho_b0 = 1e-4, 0.8, 10.0, 1.0
    alpha_b = 1.0 / 3.0
    alpha_r = 1.0 - (1.0 - alpha_b) * rho_b0 / rho_r0
    omega = 1.0 / tau
    kw = dict(alpha_r=alpha_r, alpha_b=alpha_b, A=9.0 * sigma * omega / 4.0, beta=0.7)
    o = oracle_run((n, n, n), omega, C4_STEPS, rho, u, phase=phase, physics="cgm", **kw)
    return rho, u, phase, omega, kw, o


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_droplets_full_horizon(c4_case, precision):
    rho, u, phase, omega, kw, o = c4_case
    n = C4_N
    g = gpu_run((n, n, n), omega, C4_STEPS, rho, u, phase=phase, physics="cgm", precision=precision, **kw)
    e = errors(g, o, rho, ("phase",))
    print(f"\nHORIZON droplets {n}^3 x {C4_STEPS} {precision}: " + " ".join(f"{k}={v:.3e}" for k, v in e.items())
          + f" |u|max={np.abs(o['u']).max():.3e}")
    for k, b in C4_BOUND[precision].items():
        assert e[k] <= b, (k, e)


def test_bf16_floor_of_the_body_force_flow():
    """The BF16 floor of the body-force flow's full horizon on a 32^3 box: the
    oracle with exact arithmetic and BF16-rounded storage misses u by more than
    1e-2 (the format, not the kernels), and the GPU stays within 1.6x of it."""
    shape = (32, 32, 32)
    rho, u = inputs.noise_box(shape, amp=1e-3, seed=1)
    kw = dict(g=(1e-6, 0.0, 0.0))
    o = oracle_run(shape, 1 / 0.6, C2_STEPS, rho, u, **kw)
    floor = oracle_run_stored(shape, 1 / 0.6, C2_STEPS, rho, u, "bf16", **kw)
    g = gpu_run(shape, 1 / 0.6, C2_STEPS, rho, u, precision="bf16", **kw)
    f_u, g_u = rel_l2(floor["u"], o["u"]), rel_l2(g["u"], o["u"])
    print(f"\nHORIZON bf16 floor 32^3 x {C2_STEPS}: emulated u={f_u:.3e} gpu u={g_u:.3e}")
    assert f_u > 1e-2
    assert g_u <= 1.6 * f_u
