"""Pins of the oracle's raw-moment variant (App. C, N = I; CPU only).

The printed post-collision list is pinned to the raw-moment MRT it stands for
(k = M f relaxed with the same K, solved back), to the central-moment step at
rest, and to the flow physics the variant must share with it.
"""
import math

import numpy as np

import oracle as O
from paper_2010_01628_gb300 import inputs

CS2 = 1.0 / 3.0
C, W = O.lattice()


def random_state(rng, u_amp=0.08):
    rho = rng.uniform(0.8, 1.2)
    u = u_amp * rng.standard_normal(3)
    f = O.feq(rho, u) + 0.01 * W * rng.standard_normal(19)
    rho = f.sum()
    return f, rho


def test_printed_list_is_the_raw_moment_mrt_unforced():
    """F = 0: the printed list equals the MRT definition with M = T(0) on 200
    random non-equilibrium states."""
    rng = np.random.default_rng(21)
    for _ in range(200):
        f, rho = random_state(rng)
        u = C.T @ f / rho
        om = rng.uniform(0.2, 1.95)
        a = O.collide_rm(f, rho, u, (0.0, 0.0, 0.0), om)
        b = O.collide_rm(f, rho, u, (0.0, 0.0, 0.0), om, dense=True)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_forced_list_conserves_mass_and_adds_f():
    """With a force the printed list still gives Sum f* = rho and
    Sum f* c = Sum f c + F (u = (Sum f c + F/2)/rho); it then differs from the
    MRT definition only at second and higher order (the printed list omits the
    velocity-dependent forcing moments there)."""
    rng = np.random.default_rng(22)
    for _ in range(50):
        f, rho = random_state(rng)
        F = 1e-3 * rng.standard_normal(3)
        j = C.T @ f
        u = (j + F / 2) / rho
        a = O.collide_rm(f, rho, u, F, 1.3)
        b = O.collide_rm(f, rho, u, F, 1.3, dense=True)
        assert abs(a.sum() - rho) < 1e-14
        np.testing.assert_allclose(C.T @ a, j + F, rtol=0, atol=1e-15)
        np.testing.assert_allclose(C.T @ b, j + F, rtol=0, atol=1e-15)
        assert np.abs(a - b).max() > 1e-9


def test_raw_and_central_collisions_agree_at_rest():
    """T(0) = M: at u = 0 and F = 0 the two variants are one collision."""
    rng = np.random.default_rng(23)
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        d = rng.standard_normal(19)
        d[10:] = d[1:10]  # opp(i) = i + 9: a symmetric perturbation carries no momentum
        f = W * rho * (1.0 + 0.01 * d)
        rho = f.sum()
        assert np.abs(C.T @ f).max() < 1e-15
        a = O.collide_rm(f, rho, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.4)
        b = O.collide_closed(f, rho, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.4)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_equilibrium_is_a_fixed_point():
    rng = np.random.default_rng(24)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = 0.1 * rng.standard_normal(3)
        feq = O.feq(rho, u)
        np.testing.assert_allclose(O.collide_rm(feq, rho, u, (0.0, 0.0, 0.0), 1.7), feq, rtol=0, atol=1e-15)


def test_rm_viscosity_and_galilean_defect():
    """Both steps give the viscosity c_s^2 (1/omega - 1/2) to a shear wave
    u_x(y) at rest.  Seen from a frame moving along x at U = 0.2 the central-
    moment step decays at exactly the same rate (to 1e-9), while the raw-moment
    step's rate drifts at O(U^2): the Galilean invariance the paper attributes
    to central moments (Sec. I)."""
    n, omega, steps = 32, 1.25, 400
    nu = CS2 * (1 / omega - 0.5)
    k = 2 * math.pi / n
    _, y, _ = inputs.grid(1, n, 1)
    s = np.sin(k * y)
    rates = {}
    for coll in ("rm", "cm"):
        for U in (0.0, 0.2):
            u = np.zeros((3, 1, n, 1))
            u[0] = 1e-4 * s + U
            d = O.Domain((1, n, 1), omega, collision=coll)
            d.init(np.ones((1, n, 1)), u)
            d.step(steps)
            _, un, _, _ = d.fields()
            amp = ((un[0] - un[0].mean()) * s).sum() / (s * s).sum()
            rates[coll, U] = -math.log(amp / 1e-4) / (k * k * steps)
    assert abs(rates["rm", 0.0] / nu - 1) < 1e-2
    assert abs(rates["cm", 0.0] / nu - 1) < 1e-2
    assert abs(rates["cm", 0.2] / rates["cm", 0.0] - 1) < 1e-9
    assert abs(rates["rm", 0.2] / rates["rm", 0.0] - 1) > 1e-6
