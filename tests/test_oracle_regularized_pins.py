"""Pins of the oracle's regularized on-node walls (CPU only).

The paper imposes walls "by the regularized technique" of Latt, Chopard,
Malaspinas, Deville and Michler, Phys. Rev. E 77, 056703 (2008) (Sec. III
opening paragraph) without defining it; the oracle restates that method for
straight walls on the y axis.  Pinned to closed-form channel flows, to the
second-order convergence the method has for a parabolic profile, and to
properties of one reconstruction that do not restate its formula.
"""
import numpy as np
import pytest

import oracle as O

C, W = O.lattice()


def channel(ny, omega, steps, g=(0.0, 0.0, 0.0), lid=(0.0, 0.0, 0.0)):
    d = O.Domain((1, ny, 1), omega, periodic=(True, False, True), g=g, lid_u=lid, wall_model="regularized")
    d.init(np.ones((1, ny, 1)), np.zeros((3, 1, ny, 1)))
    d.step(steps)
    r, u, _, _ = d.fields()
    return r[0, :, 0], u[:, 0, :, 0]


def test_poiseuille_exact_at_unit_relaxation():
    """On-node walls at y = 0 and y = H = ny - 1: with omega = 1 the steady
    body-force channel flow is the parabola u = g y (H - y) / (2 nu) to rounding,
    at uniform density, with no wall-normal velocity."""
    ny, gx = 17, 1e-5
    nu = (1.0 - 0.5) / 3.0
    rho, u = channel(ny, 1.0, 60000, g=(gx, 0.0, 0.0))
    y = np.arange(ny)
    exact = gx / (2 * nu) * y * (ny - 1 - y)
    assert np.abs(u[0] - exact).max() <= 1e-12 * exact.max()
    assert np.abs(u[1]).max() < 1e-15 and np.abs(u[2]).max() < 1e-15
    assert np.abs(rho - 1.0).max() < 1e-12


@pytest.mark.parametrize("omega", [1.0, 1.0 / 0.6])
def test_couette_linear_profile(omega):
    """Lid (y = ny - 1) moving at U along x, wall at rest at y = 0: the linear
    profile U y / H, exact to rounding at omega = 1 and to the method's
    second-order error otherwise."""
    ny, U = 17, 0.05
    rho, u = channel(ny, omega, 60000, lid=(U, 0.0, 0.0))
    exact = U * np.arange(ny) / (ny - 1)
    tol = 1e-13 if omega == 1.0 else 1e-4
    assert np.abs(u[0] - exact).max() <= tol * U
    assert u[0][0] == pytest.approx(0.0, abs=1e-15) and u[0][-1] == pytest.approx(U, abs=1e-15)


def test_poiseuille_converges_at_second_order():
    """tau = 0.6: the maximum relative error of the parabola falls by 4 per
    halving of the grid spacing (H = 8, 16, 32)."""
    tau, gx = 0.6, 1e-6
    nu = (tau - 0.5) / 3.0
    err = []
    for ny in (9, 17, 33):
        H = ny - 1
        _, u = channel(ny, 1.0 / tau, int(2 * H * H / nu), g=(gx, 0.0, 0.0))
        y = np.arange(ny)
        exact = gx / (2 * nu) * y * (H - y)
        err.append(np.abs(u[0] - exact).max() / exact.max())
    for a, b in zip(err, err[1:]):
        assert 3.8 < a / b < 4.2, err
    assert err[-1] < 2e-3


def moments(f):
    rho = f.sum()
    j = C.T @ f
    pi = np.einsum("i,ia,ib->ab", f, C, C)
    return rho, j, pi


@pytest.mark.parametrize("sgn", [1, -1])
def test_reconstruction_depends_on_known_populations_only(sgn):
    """The five populations entering from the wall side are overwritten:
    arbitrary values in those slots give the same result."""
    rng = np.random.default_rng(3)
    f = W * (1.0 + 0.1 * rng.standard_normal(19))
    g = rng.standard_normal(19)
    unknown = C[:, 1] == sgn
    f2 = f.copy()
    f2[unknown] = g[unknown]
    uw = (0.03, 0.0, -0.01)
    a = O.regularize(f, sgn, uw, g=(1e-4, 2e-4, 0.0))
    b = O.regularize(f2, sgn, uw, g=(1e-4, 2e-4, 0.0))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("sgn", [1, -1])
def test_reconstruction_moments(sgn):
    """Mass from the known populations, rho (1 - u_n + g_n/2) = rho_0 + 2
    rho_out (the missing mass enters through the wall); momentum rho u_w - F/2,
    so that the corrected velocity is the wall's; zero third-order
    non-equilibrium content: the result is f_eq plus a second-order Hermite term,
    so it is fixed by its first three moments (a second reconstruction returns it)."""
    rng = np.random.default_rng(4)
    f = W * (1.0 + 0.05 * rng.standard_normal(19))
    uw = np.array([0.04, 0.0, 0.02])
    gv = np.array([2e-4, -3e-4, 1e-4])
    out = O.regularize(f, sgn, uw, g=gv)
    rho0 = f[C[:, 1] == 0].sum()
    rout = f[C[:, 1] == -sgn].sum()
    gn = sgn * gv[1]
    rho_expect = (rho0 + 2 * rout) / (1 + 0.5 * gn)
    rho, j, _ = moments(out)
    assert rho == pytest.approx(rho_expect, rel=1e-14)
    np.testing.assert_allclose(j, rho * uw - 0.5 * rho * gv, rtol=0, atol=1e-15)
    again = O.regularize(out, sgn, uw, g=gv)
    np.testing.assert_allclose(again, out, rtol=0, atol=1e-15)


def test_equilibrium_wall_node_is_a_fixed_point():
    """Populations at the equilibrium of (rho, u_w) are returned unchanged."""
    uw = (0.05, 0.0, -0.02)
    f = O.feq(1.1, uw)
    for sgn in (1, -1):
        np.testing.assert_allclose(O.regularize(f, sgn, uw), f, rtol=0, atol=1e-15)
