"""Pins of the FP64 oracle to the paper and to mathematics (CPU only).

Each test ties one part of the oracle to something other than itself: a matrix
the paper prints, a second printed formula for the same quantity, a closed
form, an invariant, a special case, or an exact analytic flow.  The oracle's
own formulas are never retyped here as the expected value.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2010_01628_gb300 import inputs

CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_state(rng, u_amp=0.1, F_amp=1e-3, spread=0.05):
    rho = 1.0 + 0.1 * rng.standard_normal()
    u = u_amp * rng.uniform(-1, 1, 3)
    f = O.feq(rho, u) * (1.0 + spread * rng.uniform(-1, 1, 19))
    F = F_amp * rng.standard_normal(3)
    c, _ = O.lattice()
    rho = f.sum()
    u = (f @ c + 0.5 * F) / rho
    return f, rho, u, F


# --- lattice (Sec. II.A) -------------------------------------------------------

def test_lattice_isotropy_and_pairs():
    c, w = O.lattice()
    assert c.shape == (19, 3)
    # D3Q19 = the rest vector, 6 axis and 12 face-diagonal vectors, each once.
    n2 = (c * c).sum(1)
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert len({tuple(v) for v in c}) == 19
    assert math.isclose(w.sum(), 1.0, abs_tol=1e-15)
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(3), atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    assert math.isclose((w * c[:, 0] ** 4).sum(), 1.0 / 3.0, rel_tol=1e-14)
    assert math.isclose((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum(), 1.0 / 9.0, rel_tol=1e-14)
    # the swap-trick ordering: opposite(i) = i + 9 for i = 1..9
    for i in range(1, 10):
        np.testing.assert_array_equal(c[i + 9], -c[i])
        assert w[i] == w[i + 9]


def test_T_at_rest_equals_printed_matrix_M():
    """App. C prints M numerically; T(u = 0) must reproduce it entry by entry."""
    M = np.loadtxt(os.path.join(GOLDEN, "M_matrix_appC.txt"))
    assert M.shape == (19, 19)
    np.testing.assert_array_equal(O.T([0.0, 0.0, 0.0]), M)


def test_shift_matrix_is_unit_lower_triangular():
    """App. C: N = T M^-1 maps raw to central moments and is lower-triangular."""
    M = O.T([0.0, 0.0, 0.0])
    rng = np.random.default_rng(7)
    for _ in range(5):
        u = 0.2 * rng.uniform(-1, 1, 3)
        N = O.T(u) @ np.linalg.inv(M)
        np.testing.assert_allclose(np.triu(N, 1), 0.0, atol=1e-13)
        np.testing.assert_allclose(np.diag(N), 1.0, atol=1e-13)


# --- equilibrium (Eq. eq:EqQ19RM) ---------------------------------------------

def keq_central(rho):
    """Sec. II.B: the equilibrium central moments printed after Eq. (13)."""
    k = np.zeros(19)
    k[0] = rho
    k[4] = 3 * rho * CS2
    k[16:19] = rho * CS2 * CS2
    return k


def keq_raw(rho, u):
    """App. C: the equilibrium raw moments printed for N = I."""
    ux, uy, uz = u
    return rho * np.array([
        1, ux, uy, uz, 3 * CS2 + ux * ux + uy * uy + uz * uz, ux * ux - uy * uy, uy * uy - uz * uz,
        ux * uy, ux * uz, uy * uz,
        uy * (ux * ux + CS2), ux * (uy * uy + CS2), uz * (ux * ux + CS2), ux * (uz * uz + CS2),
        uz * (uy * uy + CS2), uy * (uz * uz + CS2),
        (ux * ux + CS2) * (uy * uy + CS2), (ux * ux + CS2) * (uz * uz + CS2), (uy * uy + CS2) * (uz * uz + CS2)])


def test_feq_has_the_printed_central_moments():
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1 + 0.3 * rng.uniform(-1, 1)
        u = 0.3 * rng.uniform(-1, 1, 3)
        np.testing.assert_allclose(O.T(u) @ O.feq(rho, u), keq_central(rho), atol=2e-15)
        # and the inverse: T^-1 k_eq reproduces every one of the 19 printed f_eq
        np.testing.assert_allclose(O.solve19(O.T(u), keq_central(rho)), O.feq(rho, u), atol=2e-15)


def test_feq_has_the_printed_raw_moments():
    M = np.loadtxt(os.path.join(GOLDEN, "M_matrix_appC.txt"))
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = 1 + 0.3 * rng.uniform(-1, 1)
        u = 0.3 * rng.uniform(-1, 1, 3)
        np.testing.assert_allclose(M @ O.feq(rho, u), keq_raw(rho, u), atol=2e-15)


def test_feq_hydrodynamic_moments():
    c, _ = O.lattice()
    rho, u = 1.07, np.array([0.04, -0.02, 0.03])
    f = O.feq(rho, u)
    assert math.isclose(f.sum(), rho, rel_tol=1e-15)
    np.testing.assert_allclose(f @ c, rho * u, atol=1e-16)
    Pi = np.einsum("i,ia,ib->ab", f, c, c)
    np.testing.assert_allclose(Pi, rho * (np.outer(u, u) + CS2 * np.eye(3)), atol=1e-16)


def test_feq_at_rest_is_weights():
    _, w = O.lattice()
    np.testing.assert_allclose(O.feq(1.3, [0, 0, 0]), 1.3 * w, atol=1e-16)


# --- collision (Eqs. eq:posColl, eq:posColl0, rawQ19, pdfQ19) ------------------

def forced_kstar_printed(rho, F, k59, omega):
    """Sec. II.B: the post-collision CM list printed after Eq. (eq:posColl0)."""
    Fx, Fy, Fz = F
    k = np.zeros(19)
    k[0] = rho
    k[1:4] = np.array(F) / 2
    k[4] = 3 * rho * CS2
    k[5:10] = (1 - omega) * np.asarray(k59)
    k[10:16] = np.array([Fy, Fx, Fz, Fx, Fz, Fy]) * CS2 / 2
    k[16:19] = rho * CS2 * CS2
    return k


def test_dense_collision_lands_on_printed_kstar():
    """T(u) f*_dense equals the printed forced post-collision list."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        f, rho, u, F = rand_state(rng)
        omega = rng.uniform(0.5, 1.95)
        k = O.T(u) @ f
        fs = O.collide_dense(f, rho, u, F, omega)
        np.testing.assert_allclose(O.T(u) @ fs, forced_kstar_printed(rho, F, k[5:10], omega), atol=1e-14)


def test_closed_form_equals_dense_solve():
    """Oracle-B (two-step closed form with the documented corrections) equals
    Oracle-A (dense solve) on random forced states, single phase and CGM."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        f, rho, u, F = rand_state(rng, u_amp=0.2)
        omega = rng.uniform(0.5, 1.99)
        np.testing.assert_allclose(O.collide_closed(f, rho, u, F, omega), O.collide_dense(f, rho, u, F, omega),
                                   rtol=0, atol=1e-13)
        alpha = rng.uniform(1 / 3, 0.95)
        np.testing.assert_allclose(O.collide_closed(f, rho, u, F, omega, cgm=True, alpha=alpha),
                                   O.collide_dense(f, rho, u, F, omega, cgm=True, alpha=alpha), rtol=0, atol=1e-13)


def test_conservation_and_momentum_gain():
    c, _ = O.lattice()
    rng = np.random.default_rng(5)
    for _ in range(50):
        f, rho, u, F = rand_state(rng)
        for fs in (O.collide_dense(f, rho, u, F, 1.7), O.collide_closed(f, rho, u, F, 1.7)):
            assert abs(fs.sum() - f.sum()) < 1e-14
            np.testing.assert_allclose(fs @ c, f @ c + F, atol=1e-15)


def test_equilibrium_is_a_fixed_point():
    rng = np.random.default_rng(6)
    for _ in range(20):
        rho = 1 + 0.2 * rng.uniform(-1, 1)
        u = 0.2 * rng.uniform(-1, 1, 3)
        fe = O.feq(rho, u)
        for omega in (0.6, 1.0, 1.5, 1.95):
            np.testing.assert_allclose(O.collide_dense(fe, rho, u, [0, 0, 0], omega), fe, atol=1e-15)
            np.testing.assert_allclose(O.collide_closed(fe, rho, u, [0, 0, 0], omega), fe, atol=1e-15)


def test_omega_one_unforced_returns_equilibrium():
    """With K = I the collision is a projection onto f_eq(rho, u) (BGK at omega = 1)."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        f, rho, u, _ = rand_state(rng, F_amp=0.0)
        np.testing.assert_allclose(O.collide_closed(f, rho, u, [0, 0, 0], 1.0), O.feq(rho, u), atol=1e-15)


def test_rest_frame_cm_equals_raw_mrt():
    """At u = 0, T = M: the CM collision is the raw-moment MRT of App. C (N = I)."""
    rng = np.random.default_rng(9)
    M = O.T([0, 0, 0])
    _, w = O.lattice()
    for _ in range(10):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        f = rho * w * (1 + 0.05 * rng.uniform(-1, 1, 19))
        c, _ = O.lattice()
        f = f - w * (f @ c)[None, :].dot(c.T).ravel() * 3  # remove momentum so that u = 0
        rho = f.sum()
        assert np.abs(f @ c).max() < 1e-15
        k = M @ f
        omega = 1.4
        ks = np.zeros(19)
        ks[0] = rho
        ks[4] = rho * 3 * CS2
        ks[5:10] = (1 - omega) * k[5:10]
        ks[10:16] = rho * 0.0
        ks[16:19] = rho * CS2 * CS2
        np.testing.assert_allclose(O.collide_closed(f, rho, [0, 0, 0], [0, 0, 0], omega), np.linalg.solve(M, ks),
                                   atol=1e-15)


# --- forcing (App. B) ----------------------------------------------------------

def test_forcing_central_moments_match_printed_CM_list():
    """T(u) F_i (F_i from the printed raw forcing moments) equals the printed
    central forcing moments R^CM: two printed lists of App. B agree."""
    rng = np.random.default_rng(10)
    for _ in range(20):
        u = 0.2 * rng.uniform(-1, 1, 3)
        F = rng.standard_normal(3)
        Fx, Fy, Fz = F
        Rcm = np.zeros(19)
        Rcm[1:4] = F
        Rcm[10:16] = CS2 * np.array([Fy, Fx, Fz, Fx, Fz, Fy])
        np.testing.assert_allclose(O.T(u) @ O.forcing_pop(u, F), Rcm, atol=1e-14)


def test_forcing_hermite_limit():
    """App. B: R^HM is R^RM without the c_s-proportional terms; at rest the
    forcing reduces to Guo's first-order term 3 w_i c_i . F."""
    c, w = O.lattice()
    F = np.array([0.3, -0.2, 0.1])
    np.testing.assert_allclose(O.forcing_pop([0, 0, 0], F), 3 * w * (c @ F), atol=1e-15)


# --- colour gradient (App. E) ---------------------------------------------------

def test_cgm_weights_and_sound_speed():
    c, w = O.lattice()
    for alpha in (1 / 3, 0.5, 14 / 15):
        h = O.heq(1.0, [0, 0, 0], alpha)
        assert math.isclose(h.sum(), 1.0, rel_tol=1e-15)
        # p = rho (c_s^k)^2 = rho (1 - alpha)/2 for D3Q19 (Eq. eq:press)
        assert math.isclose((h * c[:, 0] ** 2).sum(), (1 - alpha) / 2, rel_tol=1e-14)
    # alpha = 1/3 gives back the single-phase equilibrium
    u = [0.05, -0.02, 0.01]
    np.testing.assert_allclose(O.heq(1.2, u, 1 / 3), O.feq(1.2, u), atol=1e-16)


def test_cgm_equilibrium_central_moments():
    """T h_eq reproduces App. E's post-collision list at F = 0 for the
    equilibrated moments (k4, k10..15), and k16..18 with the factor 1/6."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        rho = 1 + rng.uniform(0, 5)
        u = 0.1 * rng.uniform(-1, 1, 3)
        alpha = rng.uniform(1 / 3, 0.95)
        ux, uy, uz = u
        k = O.T(u) @ O.heq(rho, u, alpha)
        a3 = (3 * alpha - 1) / 6
        assert math.isclose(k[0], rho, rel_tol=1e-14)
        assert math.isclose(k[4], 3 * rho * (1 - alpha) / 2, rel_tol=1e-13)
        np.testing.assert_allclose(k[10:16], rho * a3 * np.array([uy, ux, uz, ux, uz, uy]), atol=1e-14)
        exp16 = [rho * (1 + a * a + b * b - alpha * (1 + 3 * a * a + 3 * b * b)) / 6
                 for a, b in ((ux, uy), (ux, uz), (uy, uz))]
        np.testing.assert_allclose(k[16:19], exp16, atol=1e-14)
        np.testing.assert_allclose(k[5:10], 0.0, atol=1e-14)


def test_cgm_perturbation_conserves_mass_and_momentum():
    c, _ = O.lattice()
    rng = np.random.default_rng(12)
    for _ in range(20):
        grad = rng.standard_normal(3)
        f0 = rng.uniform(0.01, 0.1, 19)
        f1 = O.cgm_perturb(f0, grad, 1e-3)
        scale = np.abs(f1 - f0).max()
        assert abs((f1 - f0).sum()) < 1e-12 * scale
        np.testing.assert_allclose((f1 - f0) @ c, 0.0, atol=1e-12 * scale)
        assert np.abs(f1 - f0).max() > 0


def test_cgm_recolouring_conserves_each_colour():
    rng = np.random.default_rng(13)
    for _ in range(20):
        grad = rng.standard_normal(3)
        rr, rb = rng.uniform(0.1, 10), rng.uniform(0.1, 10)
        f = O.feq(rr + rb, 0.05 * rng.uniform(-1, 1, 3))
        alpha = (rr * 0.9 + rb / 3) / (rr + rb)
        fr, fb = O.cgm_recolour(f, grad, rr, rb, alpha, 0.7)
        assert math.isclose(fr.sum(), rr, rel_tol=1e-13)
        assert math.isclose(fb.sum(), rb, rel_tol=1e-13)
        np.testing.assert_allclose(fr + fb, f, atol=1e-14)


# --- domain-level: streaming, boundaries, flows ---------------------------------

@pytest.mark.parametrize("closed", [False, True])
@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 6, 7)])
def test_uniform_acceleration_exact_momentum(shape, closed):
    """Periodic box, F = rho g: total reported momentum grows by M g per step
    exactly (streaming conserves totals, each collision adds F)."""
    g = np.array([1e-4, -2e-5, 3e-5])
    rho, u = inputs.random_fields(shape, seed=21, u_amp=0.02)
    d = O.Domain(shape, 1.4, g=g, closed_form=closed)
    d.init(rho, u)
    r0, u0, _, _ = d.fields()
    P0 = (r0[None] * u0).reshape(3, -1).sum(1)
    mass = r0.sum()
    for t in range(1, 6):
        d.step(1)
        r, uu, _, _ = d.fields()
        assert abs(r.sum() - mass) < 1e-12
        P = (r[None] * uu).reshape(3, -1).sum(1)
        np.testing.assert_allclose(P, P0 + t * mass * g, atol=1e-13)


def test_dense_and_closed_domains_agree_with_walls_and_lid():
    shape = (5, 6, 4)
    rho, u = inputs.random_fields(shape, seed=22)
    a = O.Domain(shape, 1.2, periodic=(True, False, False), lid_u=(0.05, 0, 0), g=(1e-4, 0, 0), closed_form=False)
    b = O.Domain(shape, 1.2, periodic=(True, False, False), lid_u=(0.05, 0, 0), g=(1e-4, 0, 0), closed_form=True)
    a.init(rho, u)
    b.init(rho, u)
    a.step(10)
    b.step(10)
    np.testing.assert_allclose(a.f, b.f, atol=1e-13)
    ra, ua, _, _ = a.fields()
    rb_, ub, _, _ = b.fields()
    np.testing.assert_allclose(ra, rb_, atol=1e-13)
    np.testing.assert_allclose(ua, ub, atol=1e-13)


def test_bounce_back_conserves_mass_with_moving_lid():
    shape = (6, 6, 6)
    rho, u = inputs.cavity_rest(6)
    d = O.Domain(shape, 1.5, periodic=(False, False, False), lid_u=(0.1, 0, 0))
    d.init(rho, u)
    m0 = d.fields()[0].sum()
    d.step(50)
    r, uu, _, _ = d.fields()
    assert abs(r.sum() - m0) < 1e-11
    # the lid drags the top layer in +x
    assert uu[0, :, -1, :].mean() > 0.01


def tg2d_error(n, u0=0.01, re=1000.0):
    nu = u0 * n / re
    omega = 1.0 / (nu / CS2 + 0.5)
    k = 2 * math.pi / n
    T = 1.0 / (2 * k * k * nu)
    steps = int(round(T))
    rho, u = inputs.taylor_green_2d(n, u0)
    d = O.Domain((n, n, 1), omega)
    d.init(rho, u)
    d.step(steps)
    _, un, _, _ = d.fields()
    ua = u * math.exp(-steps / T)
    return np.linalg.norm(ua[:2] - un[:2]) / np.linalg.norm(ua[:2])


def test_taylor_green_2d_decay_second_order():
    """Sec. III.A: decay exp(-2 xi^2 nu t); error eq. (error) falls at order 2
    at u0 = 0.01, Re = 1000."""
    e = [tg2d_error(n) for n in (8, 16, 32)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert e[-1] < 2e-2
    assert orders[-1] > 1.7, (e, orders)


def test_viscosity_from_shear_wave_decay():
    """nu = c_s^2 (1/omega - 1/2): a sinusoidal shear wave decays at nu k^2."""
    n = 32
    omega = 1.25
    nu = CS2 * (1 / omega - 0.5)
    k = 2 * math.pi / n
    x, y, z = inputs.grid(1, n, 1)
    u = np.zeros((3, 1, n, 1))
    u[0] = 1e-4 * np.sin(k * y)
    d = O.Domain((1, n, 1), omega)
    d.init(np.ones((1, n, 1)), u)
    steps = 400
    d.step(steps)
    _, un, _, _ = d.fields()
    amp = (un[0] * np.sin(k * y)).sum() / (np.sin(k * y) ** 2).sum()
    nu_meas = -math.log(amp / 1e-4) / (k * k * steps)
    assert abs(nu_meas / nu - 1) < 1e-2


def poiseuille_error(ny, omega=1.0 / 0.8, umax=1e-3):
    nu = CS2 * (1 / omega - 0.5)
    g = 8 * nu * umax / ny ** 2
    d = O.Domain((1, ny, 1), omega, periodic=(True, False, True), g=(g, 0, 0))
    d.init(np.ones((1, ny, 1)), np.zeros((3, 1, ny, 1)))
    d.step(int(8 * ny * ny / nu))
    _, un, _, _ = d.fields()
    y = np.arange(ny) + 0.5
    ua = g / (2 * nu) * y * (ny - y)
    return np.linalg.norm(un[0].ravel() - ua) / np.linalg.norm(ua)


def test_poiseuille_with_halfway_bounce_back():
    e8, e16 = poiseuille_error(8), poiseuille_error(16)
    assert e16 < 5e-3
    assert e16 < e8


def hartmann_profile(ny, ha, nu=0.1, u0=1e-3):
    L = ny
    g = 8 * nu * u0 / L ** 2
    b0 = 2 * ha * nu / L
    tau_m = 0.5 + nu / 0.25  # eta = nu with cs_m^2 = 1/4
    omega = 1.0 / (nu / CS2 + 0.5)
    d = O.Domain((1, ny, 1), omega, periodic=(True, False, True), g=(g, 0, 0), physics=O.MHD, tau_m=tau_m,
                 b_wall=(0, b0, 0))
    rho, u, B = inputs.hartmann(ny, b0)
    d.init(rho, u, B=B)
    d.step(int(10 * ny * ny / nu))
    _, un, _, Bn = d.fields()
    s = (2 * (np.arange(ny) + 0.5) - L) / L
    ua = 2 * u0 / (ha * math.tanh(ha)) * (1 - np.cosh(ha * s) / math.cosh(ha))
    return un[0].ravel(), ua, Bn


def test_hartmann_profile_matches_analytic():
    """Sec. III.F: u_x = (4 nu u0 / (L b tanh Ha)) [1 - cosh(Ha y'/L)/cosh Ha],
    with Ha = b L / sqrt(4 rho nu eta) and the driving g = 8 nu u0 / L^2."""
    errs = []
    for ny in (16, 32):
        un, ua, Bn = hartmann_profile(ny, 3.0)
        errs.append(np.linalg.norm(un - ua) / np.linalg.norm(ua))
        # b_y stays uniform (div b = 0 in a channel), b_x is induced and odd in y
        np.testing.assert_allclose(Bn[1], Bn[1].mean(), rtol=1e-8)
        bx = Bn[0].ravel()
        np.testing.assert_allclose(bx, -bx[::-1], atol=1e-9 * max(1e-30, np.abs(bx).max()) + 1e-15)
    assert errs[1] < 1e-2, errs
    assert math.log2(errs[0] / errs[1]) > 1.5, errs


def test_hartmann_small_ha_is_poiseuille():
    un, ua, _ = hartmann_profile(16, 0.05)
    y = np.arange(16) + 0.5
    pois = 1e-3 * 4 * y * (16 - y) / 256
    assert np.linalg.norm(un - pois) / np.linalg.norm(pois) < 1e-2


def test_magnetic_diffusivity():
    """Reading of the magnetic scheme: b diffuses with eta = cs_m^2 (tau_m - 1/2),
    cs_m^2 = 1/4, at rest (u = 0, no coupling since b_x(y) gives j x b along y
    only at second order in the amplitude)."""
    n = 32
    tau_m = 0.9
    eta = 0.25 * (tau_m - 0.5)
    k = 2 * math.pi / n
    x, y, z = inputs.grid(1, n, 1)
    B = np.zeros((3, 1, n, 1))
    B[0] = 1e-6 * np.sin(k * y)
    d = O.Domain((1, n, 1), 1.0, physics=O.MHD, tau_m=tau_m)
    d.init(np.ones((1, n, 1)), np.zeros((3, 1, n, 1)), B=B)
    steps = 300
    d.step(steps)
    _, _, _, Bn = d.fields()
    amp = (Bn[0] * np.sin(k * y)).sum() / (np.sin(k * y) ** 2).sum()
    eta_meas = -math.log(amp / 1e-6) / (k * k * steps)
    assert abs(eta_meas / eta - 1) < 1e-2


def test_current_from_nonequilibrium_flux_is_curl_b():
    """j from the antisymmetric non-equilibrium flux equals curl b (central
    differences) on a relaxed smooth field."""
    n = 64
    tau_m = 0.8
    k = 2 * math.pi / n
    x, y, z = inputs.grid(1, n, 1)
    B = np.zeros((3, 1, n, 1))
    B[0] = 1e-6 * np.sin(k * y)
    d = O.Domain((1, n, 1), 1.0, physics=O.MHD, tau_m=tau_m)
    d.init(np.ones((1, n, 1)), np.zeros((3, 1, n, 1)), B=B)
    d.step(40)
    # gather the populations of one node by hand through the public fields:
    # compare j_z computed by the oracle's current() on the post-stream g with
    # -d b_x / d y from the fields.
    _, _, _, Bn = d.fields()
    bx = Bn[0].ravel()
    dbx = (np.roll(bx, -1) - np.roll(bx, 1)) / 2
    g = d.g.reshape(n, 7, 3)
    # post-stream populations at node j: g_m(j) = g*_m(j - c_m) (periodic)
    jz = np.zeros(n)
    mdir = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    for j in range(n):
        gin = np.array([g[(j - cy) % n, m] for m, (_, cy, _) in enumerate(mdir)])
        _, jj = O.current(gin, [0, 0, 0], tau_m)
        jz[j] = jj[2]
    np.testing.assert_allclose(jz, -dbx, rtol=0, atol=0.02 * np.abs(dbx).max())


def test_cgm_flat_interface_stays_put():
    """A flat red/blue layer pair in a periodic box: colours conserved, the
    interface stays where it started, spurious velocity stays tiny."""
    ny = 32
    y = np.arange(ny)
    phase = np.tanh((8 - np.abs(y - 15.5)) / 2.0)[None, :, None] * np.ones((1, ny, 1))
    rho_r0, rho_b0 = 4.0, 1.0
    alpha_b = 1 / 3
    alpha_r = 1 - (1 - alpha_b) * rho_b0 / rho_r0
    rho = rho_r0 * (1 + phase) / 2 + rho_b0 * (1 - phase) / 2
    omega = 1 / 0.8
    d = O.Domain((1, ny, 1), omega, physics=O.CGM, alpha_r=alpha_r, alpha_b=alpha_b, A=9 * 1e-3 * omega / 4,
                 beta=0.7)
    d.init(rho, np.zeros((3, 1, ny, 1)), phase=phase)
    r0 = d.fr.reshape(-1, 19).sum(), d.fb.reshape(-1, 19).sum()
    d.step(300)
    r1 = d.fr.reshape(-1, 19).sum(), d.fb.reshape(-1, 19).sum()
    assert abs(r1[0] - r0[0]) < 1e-10 * r0[0]
    assert abs(r1[1] - r0[1]) < 1e-10 * r0[1]
    rho_n, un, ph, _ = d.fields()
    u300 = np.abs(un).max()
    assert u300 < 1e-2
    d.step(700)
    rho_n, un, ph, _ = d.fields()
    assert np.abs(un).max() < u300  # the start-up transient decays
    # interface positions (phase zero crossings) unchanged within a cell
    zc0 = np.where(np.diff(np.sign(phase.ravel())))[0]
    zc1 = np.where(np.diff(np.sign(ph.ravel())))[0]
    np.testing.assert_array_equal(zc0, zc1)


def test_reference_density_force_momentum_growth():
    """F = (rho - rho_ref) g: on a periodic box the total momentum grows by
    exactly (M - N rho_ref) g per step (Eq. eq:posColl0 adds F to rho u), for
    the single-phase, colour-gradient and Shan-Chen steps alike."""
    shape = (6, 5, 4)
    n = 6 * 5 * 4
    rng = np.random.default_rng(12)
    rho = rng.uniform(0.8, 1.4, size=shape[::-1])
    u = 0.01 * rng.standard_normal((3,) + shape[::-1])
    g = np.array([2e-5, -3e-5, 1e-5])
    for phys, extra in ((O.FLUID, {}), (O.CGM, {"alpha_r": 7 / 9, "alpha_b": 1 / 3, "A": 1e-4}),
                        (O.SC, {"G": -1.0})):
        d = O.Domain(shape, 1.3, physics=phys, g=tuple(g), rho_ref=1.1, **extra)
        d.init(rho, u, phase=np.where(rho > 1.1, 1.0, -1.0) if phys == O.CGM else None)
        r0, u0, _, _ = d.fields()
        M = r0.sum()
        p0 = (r0 * u0).sum(axis=(1, 2, 3))
        d.step(7)
        r1, u1, _, _ = d.fields()
        p1 = (r1 * u1).sum(axis=(1, 2, 3))
        assert abs(r1.sum() - M) < 1e-12 * M
        np.testing.assert_allclose(p1 - p0, 7 * (M - n * 1.1) * g, rtol=1e-9, atol=1e-15)


def cgm_cylinder_jump(R, n=64, sigma=5e-3, tau=1.0, steps=3000, width=2.0):
    """Pressure jump of a red cylinder (along x) in blue, equal densities, after
    `steps`; the phase pressure is rho (1 - alpha)/2 (Eq. eq:press)."""
    ab = 1.0 / 3.0
    ar = ab
    om = 1.0 / tau
    y, z = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    d = np.sqrt((y - (n - 1) / 2) ** 2 + (z - (n - 1) / 2) ** 2)
    ph = np.tanh((R - d) / width).T[:, :, None]
    d_ = O.Domain((1, n, n), om, physics=O.CGM, alpha_r=ar, alpha_b=ab, A=9 * sigma * om / 4, beta=0.7)
    d_.init(np.ones_like(ph), np.zeros((3, n, n, 1)), phase=ph)
    d_.step(steps)
    r, _, _, _ = d_.fields()
    c = n // 2
    return (r[c, c, 0] - r[0, 0, 0]) * (1 - ab) / 2


def test_cgm_laplace_law_with_the_stated_surface_tension():
    """App. E: each colour's perturbation carries A_k/2 and
    sigma = (2/9)(A_r + A_b)/omega = (4/9) A/omega.  A cylinder's pressure jump
    then equals sigma/R: within 3 % at R = 10 and 1 % at R = 18 (the
    interface's finite width fades with R).  Half the amplitude, or a wrong
    projection, misses by a factor."""
    sigma = 5e-3
    ratios = [cgm_cylinder_jump(R, sigma=sigma) * R / sigma for R in (10.0, 14.0, 18.0)]
    assert abs(ratios[0] - 1) < 0.03, ratios
    assert abs(ratios[2] - 1) < 0.01, ratios
    assert abs(ratios[2] - 1) <= abs(ratios[0] - 1)


@pytest.mark.parametrize("tau", [0.6, 1.3])
@pytest.mark.parametrize("axis", [0, 2])
def test_couette_moving_lid_is_the_exact_line(tau, axis):
    """Half-way bounce-back with the moving-wall term 2 w_i c_i.u_w / c_s^2
    (Sec. III opening paragraph): plane Couette flow between a wall at rest
    half a cell below y = 0 and the +y wall half a cell above y = ny - 1,
    moving at U along x (or z), x and z periodic, no force.  The steady
    velocity is the straight line u(y) = U (y + 1/2)/ny, with no slip at either
    wall, for every relaxation time.  Starting from rest the oracle converges
    onto it to round-off; a halved (or doubled) wall term moves the slope to
    U/2 (2U), a wrong sign reverses it."""
    ny, U = 8, 0.05
    lid = [0.0, 0.0, 0.0]
    lid[axis] = U
    d = O.Domain((1, ny, 1), 1.0 / tau, periodic=(True, False, True), lid_u=tuple(lid))
    d.init(np.ones((1, ny, 1)), np.zeros((3, 1, ny, 1)))
    d.step(6000)
    _, u, _, _ = d.fields()
    y = np.arange(ny)
    exact = U * (y + 0.5) / ny
    np.testing.assert_allclose(u[axis, 0, :, 0], exact, rtol=0, atol=1e-12)
    for other in {0, 1, 2} - {axis}:
        assert np.abs(u[other]).max() < 1e-12


@pytest.mark.parametrize("alpha,beta,rho0,steps", [(0.6, 0.12, 1.5, 8000), (0.6, 0.2, 1.0, 3000),
                                                    (1 / 3, 0.1, 1.0, 6000)])
def test_cgm_recolouring_sets_the_interface_width(alpha, beta, rho0, steps):
    """The magnitude of the recolouring separation (App. E, Eqs. eq:op3r and
    eq:op3b, with g_eq(rho, 0) = rho phi_i(alpha) and cos(theta_i) =
    c_i.n / |c_i|) fixes the width of a flat interface at rest.

    Derivation (equal colour densities, so alpha is uniform; A = 0, so the
    total populations stay at f_eq(rho, 0) = rho phi_i(alpha)).  With the
    interface normal along x and a = rho_r/rho, the red density after
    streaming is Sum_i phi_i [a + beta a(1 - a) cos(theta_i)](x - c_ix).
    Grouping directions by c_ix, with P = Sum_{c_ix = 1} phi_i = (1 - alpha)/4
    and S = Sum_{c_ix = 1} phi_i / |c_i| = (1 - alpha)(1/12 + 1/(6 sqrt 2)),
    a steady profile satisfies
        P [a(x+1) + a(x-1) - 2 a(x)] = beta S [h(x+1) - h(x-1)],  h = a(1 - a).
    Its continuum limit a' = k h, k = 2 beta S / P, is the logistic profile,
    phi = 2a - 1 = tanh(k x / 2); the next order of the shift operators gives
    a' = k h + (k/12) h'', so across the centre cell atanh(phi) rises by
    (k/2)(1 - k^2/24) + O(k^5).  k is independent of alpha and of rho0.

    A halved beta halves the rise; cos(theta_i) without the 1/|c_i| moves it by
    24 %; the plain weights w_i in place of phi_i(alpha) move it by 67 % at
    alpha = 0.6; a factor rho_r rho_b / rho instead of / rho^2 moves it by
    50 % at rho0 = 1.5."""
    nx = 64 if beta < 0.15 else 48
    S = (1 - alpha) * (1.0 / 12.0 + 1.0 / (6.0 * math.sqrt(2.0)))
    P = (1 - alpha) / 4.0
    k = 2.0 * beta * S / P
    d = O.Domain((nx, 1, 1), 1.0 / 0.8, physics=O.CGM, alpha_r=alpha, alpha_b=alpha, A=0.0, beta=beta)
    x = np.arange(nx)
    phase = np.where((x >= nx // 4) & (x < 3 * nx // 4), 1.0, -1.0).reshape(1, 1, nx)
    d.init(rho0 * np.ones((1, 1, nx)), np.zeros((3, 1, 1, nx)), phase=phase)
    d.step(steps)
    _, u, ph, _ = d.fields()
    assert np.abs(u).max() < 1e-12  # the total populations stay at rest
    a = np.arctanh(ph.ravel())
    c = nx // 4  # the interface sits between nodes c - 1 and c (and, mirrored, 3c - 1 and 3c)
    predicted = 0.5 * k * (1.0 - k * k / 24.0)
    assert abs((a[c] - a[c - 1]) / predicted - 1.0) < 3e-4
    assert abs((a[3 * c - 1] - a[3 * c]) / predicted - 1.0) < 3e-4
