"""Pins of the oracle's Shan-Chen pseudopotential multiphase step (CPU only).

Sec. III.G (static bubble): psi = 1 - exp(-rho), F(x) = -G psi(x) sum_i w_i
c_i psi(x + c_i), G = -5, nu = 0.0333, droplet density 1.95 in 0.15.

The force is pinned to a closed form of the lattice sum; the step to exact
conservation laws, to the mechanical-stability coexistence densities of the
equation of state p = rho c_s^2 + (G c_s^2 / 2) psi^2, to Young-Laplace's law
and to the paper's observation that the central-moment collision carries
smaller spurious currents than BGK with the same equilibrium.
"""
import numpy as np
import pytest

import oracle as O

G = -5.0
CS2 = 1.0 / 3.0


def omega_of(nu):
    return 1.0 / (3.0 * nu + 0.5)


def pressure(rho):
    """Bulk equation of state of the pseudopotential fluid (Shan & Chen 1993)."""
    psi = 1.0 - np.exp(-rho)
    return rho * CS2 + 0.5 * G * CS2 * psi * psi


def test_sc_force_matches_discrete_closed_form_for_a_plane_wave():
    """For psi = psi0 + e sin(k.x) on a periodic box the D3Q19 lattice sum is
    exact: sum_i w_i c_ia sin(k.(x+c_i)) = cos(k.x) (sin k_a / 9)(1 + sum_(b!=a)
    cos k_b) (axis links w = 1/18, edge links w = 1/36).  A dropped link family,
    a wrong weight, sign or neighbour direction breaks it."""
    nx, ny, nz = 8, 6, 10
    k = 2 * np.pi * np.array([1 / nx, 2 / ny, 3 / nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    psi0, e = 0.6, 0.25
    psi = psi0 + e * np.sin(ph)
    d = O.Domain((nx, ny, nz), 1.0, physics=O.SC, G=G)
    F = d.sc_force(psi)
    for a in range(3):
        lat = np.sin(k[a]) / 9.0 * (1.0 + sum(np.cos(k[b]) for b in range(3) if b != a))
        expect = -G * psi * e * np.cos(ph) * lat
        np.testing.assert_allclose(F[a], expect, rtol=0, atol=1e-14)


def test_sc_force_vanishes_for_uniform_psi_between_walls():
    """A neighbour behind a wall contributes the node's own psi (neutral
    wetting), so a uniform field carries no force anywhere, wall nodes included."""
    d = O.Domain((5, 4, 6), 1.0, physics=O.SC, G=G, periodic=(False, False, False))
    F = d.sc_force(np.full((6, 4, 5), 0.7))
    assert np.abs(F).max() < 1e-16


def test_sc_step_conserves_mass_and_momentum_exactly():
    """The pair force is antisymmetric (link x->x+c_i and x+c_i->x with c_opp
    = -c_i), so sum_x F = 0 and a periodic box keeps total mass and momentum
    to rounding, also with a moving bulk."""
    shape = (10, 8, 6)
    rng = np.random.default_rng(5)
    rho0 = rng.uniform(0.1, 2.0, size=shape[::-1])
    u0 = 0.02 * rng.standard_normal((3,) + shape[::-1]) + np.array([0.03, -0.01, 0.02])[:, None, None, None]
    d = O.Domain(shape, omega_of(0.1), physics=O.SC, G=G)
    d.init(rho0, u0)
    r, u, _, _ = d.fields()
    m0, p0 = r.sum(), (r * u).sum(axis=(1, 2, 3))
    for _ in range(5):
        d.step(10)
        r, u, _, _ = d.fields()
        assert abs(r.sum() - m0) <= 1e-12 * m0
        np.testing.assert_allclose((r * u).sum(axis=(1, 2, 3)), p0, rtol=0, atol=1e-11 * m0)


def test_sc_uniform_state_stays_at_rest():
    d = O.Domain((6, 5, 4), omega_of(0.0333), physics=O.SC, G=G)
    d.init(np.full((4, 5, 6), 0.5), np.zeros((3, 4, 5, 6)))
    d.step(20)
    r, u, psi, _ = d.fields()
    assert np.abs(u).max() < 1e-15 and np.abs(r - 0.5).max() < 1e-14
    np.testing.assert_allclose(psi, 1.0 - np.exp(-0.5), rtol=0, atol=1e-15)


def coexistence(eps):
    """Densities with p(rho_v) = p(rho_l) = p0 and the mechanical-stability
    integral of (p0 - p) psi' / psi^(1+eps) over [rho_v, rho_l] equal to zero
    (Shan, PRE 77, 066702 (2008))."""
    integrate = pytest.importorskip("scipy.integrate")
    optimize = pytest.importorskip("scipy.optimize")

    def eqs(v):
        rv, rl = v
        p0 = pressure(rl)
        f = lambda r: (p0 - pressure(r)) * np.exp(-r) / (1.0 - np.exp(-r)) ** (1.0 + eps)
        return [pressure(rv) - p0, integrate.quad(f, rv, rl, epsabs=1e-14, epsrel=1e-12)[0]]

    return optimize.fsolve(eqs, [0.15, 1.9], xtol=1e-13)


def flat_slab(nu, ny=64, steps=12000, **kw):
    y = np.arange(ny)
    rho = 0.15 + 1.8 * 0.5 * (1 + np.tanh((ny / 4 - np.abs(y - (ny - 1) / 2)) / 2.0))
    d = O.Domain((1, ny, 1), omega_of(nu), physics=O.SC, G=G, **kw)
    d.init(rho[None, :, None], np.zeros((3, 1, ny, 1)))
    d.step(steps)
    r, u, _, _ = d.fields()
    return r[0, ny // 2, 0], r[0, 0, 0], np.abs(u).max()


def test_sc_flat_interface_reaches_mechanical_stability_coexistence():
    """G = -5 separates the paper's 1.95 / 0.15 start into liquid and vapour at
    the densities of the mechanical-stability condition with eps = 0, the member
    of Shan's family that a second-order forcing with u = (sum f c + F/2)/rho
    lands on (within the interface's discretisation error); the eps = 1 member
    is 2 % away and excluded.  The result is independent of the viscosity."""
    rv0, rl0 = coexistence(0.0)
    rv1, rl1 = coexistence(1.0)
    assert abs(rl1 - rl0) > 0.02
    for nu in (0.1, 1.0 / 6.0):
        rl, rv, umax = flat_slab(nu)
        assert umax < 1e-4
        assert abs(rl - rl0) < 2e-4 * rl0, (rl, rl0)
        assert abs(rv - rv0) < 1e-3 * rv0, (rv, rv0)


def test_sc_spinodal_threshold_is_minus_four():
    """The equation of state has dp/drho = c_s^2 (1 + G psi psi'), and psi psi'
    peaks at 1/4 (psi = 1/2, rho = ln 2): a uniform state at rho = ln 2 is
    unstable for G < -4 and stable above.  A small long-wave perturbation
    grows at G = -4.2 and does not at G = -3.8; an extra c_s^2 in the force, or
    a wrong weight, moves the threshold."""
    ny = 64
    y = np.arange(ny)
    a0 = 1e-3
    rho = np.log(2.0) + a0 * np.cos(2 * np.pi * y / ny)
    amp = {}
    for g in (-3.8, -4.2):
        d = O.Domain((1, ny, 1), omega_of(0.1), physics=O.SC, G=g)
        d.init(rho[None, :, None], np.zeros((3, 1, ny, 1)))
        hist = []
        for _ in range(10):
            d.step(100)
            r, _, _, _ = d.fields()
            hist.append(0.5 * (r.max() - r.min()))
        amp[g] = max(hist)
    assert amp[-3.8] < a0
    assert amp[-4.2] > 100 * a0


def droplet(shape, R, nu=0.0333, steps=6000, **kw):
    """Liquid droplet (1.95) of radius R centred in vapour (0.15), tanh profile
    of width 2; a cylinder along x when nx == 1.  Returns (dp, max |u|)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d2 = (y - (ny - 1) / 2) ** 2 + (z - (nz - 1) / 2) ** 2
    if nx > 1:
        d2 = d2 + (x - (nx - 1) / 2) ** 2
    rho = 0.15 + 1.8 * 0.5 * (1 + np.tanh((R - np.sqrt(d2)) / 2.0))
    d = O.Domain(shape, omega_of(nu), physics=O.SC, G=G, **kw)
    d.init(rho, np.zeros((3,) + rho.shape))
    d.step(steps)
    r, u, _, _ = d.fields()
    c = (nz // 2, ny // 2, nx // 2)
    return pressure(r[c]) - pressure(r[0, 0, 0]), np.sqrt((u * u).sum(axis=0)).max()


def test_sc_laplace_law_on_cylinders():
    """Young-Laplace for a cylinder: dp = sigma / R, linear in 1/R (the
    paper's Fig. 11 test, on 2D cylinders for CPU time)."""
    R = np.array([8.0, 12.0, 16.0])
    dp = np.array([droplet((1, 64, 64), r)[0] for r in R])
    assert np.all(dp > 0) and np.all(np.diff(dp) < 0)
    A = np.vstack([1.0 / R, np.ones_like(R)]).T
    (sigma, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    resid = dp - A @ np.array([sigma, c])
    assert np.abs(resid).max() < 0.02 * dp.min()
    # the intercept is a finite-interface-width correction, small against dp
    assert abs(c) < 0.25 * dp.min()
    assert 0.01 < sigma < 0.05


def test_sc_sphere_jump_is_twice_the_cylinder_jump():
    """Young-Laplace curvature: a sphere (two principal radii R) carries twice
    the pressure jump of a cylinder of the same radius and interface."""
    R = 8.0
    dp_cyl, _ = droplet((1, 48, 48), R, steps=4000)
    dp_sph, _ = droplet((32, 32, 32), R, steps=2500)
    assert abs(dp_sph / dp_cyl - 2.0) < 0.06, dp_sph / dp_cyl


def test_central_moments_reduce_spurious_currents_against_bgk():
    """Sec. III.G, Fig. 12: relaxing the high-order central moments to
    equilibrium (and omega_b = 1) leaves markedly weaker spurious currents at
    the interface than BGK toward the same extended equilibrium (every moment
    at omega)."""
    nu = 0.0333
    om = omega_of(nu)
    _, u_cm = droplet((1, 48, 48), 10.0, nu=nu, steps=3000, closed_form=False)
    _, u_bgk = droplet((1, 48, 48), 10.0, nu=nu, steps=3000, closed_form=False, omega_b=om, omega_3=om, omega_4=om)
    assert u_cm < 0.5 * u_bgk, (u_cm, u_bgk)
