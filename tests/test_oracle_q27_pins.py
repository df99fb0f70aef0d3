"""Pins of the D3Q27 central-moment oracle (App. D; CPU only)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import q27_oracle as Q
import oracle as O
from paper_2010_01628_gb300 import inputs

CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pdfQ27_appD.txt")
CVEC = np.array([Q.CX, Q.CY, Q.CZ])


def printed_minv():
    rows = np.zeros((27, 27))
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            i, terms = line.split(":")
            for t in terms.split():
                c, r = t.split("*r")
                rows[int(i), int(r)] += float(Fraction(c))
    return rows


def test_printed_back_transform_is_m_inverse():
    """Eq. (pdfQ27) as printed equals M^-1 of the App. D basis and lattice in
    24 of 27 rows, which fixes the lattice order and the row order of M.  The
    other three carry misprints, read as:
      f17: (r4/4 - r22 - ...)/4  ->  (r4 - r22 - r23 - r24 - r26)/4,
      f19: (r5/4 - r21 - ...)/4  ->  (r5 - r21 - r23 - r25 - r26)/4,
      f20: (r10 - r12 + r13 + r15 + r19)/8  ->  (r10 - r12 - r13 - r15 - r19)/8."""
    P = printed_minv()
    P[17, 4] = 0.25
    P[19, 5] = 0.25
    P[20, 13] = P[20, 15] = P[20, 19] = -0.125
    np.testing.assert_allclose(P, np.linalg.inv(Q.M), rtol=0, atol=1e-13)
    assert Q.OPP.tolist() == [0] + list(range(14, 27)) + list(range(1, 14))
    np.testing.assert_array_equal(CVEC[:, Q.OPP], -CVEC)


def test_equilibrium_moments():
    """Central moments rho prod(1, 0, c_s^2) at any velocity (the Galilean-
    invariant equilibrium); raw moments rho prod(1, u, u^2 + c_s^2)."""
    rng = np.random.default_rng(31)
    for _ in range(20):
        rho = rng.uniform(0.7, 1.3)
        u = 0.15 * rng.standard_normal(3)
        fe = Q.feq(rho, u)
        np.testing.assert_allclose(Q.T(u) @ fe, Q.central_eq(rho), rtol=0, atol=1e-15)
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    raw = (fe * Q.CX ** a * Q.CY ** b * Q.CZ ** c).sum()
                    m = [(1.0, u[d], u[d] ** 2 + CS2)[e] for d, e in enumerate((a, b, c))]
                    assert raw == pytest.approx(rho * m[0] * m[1] * m[2], abs=1e-15)


def test_force_has_only_first_order_central_hermite_moments():
    """App. B: the central Hermite moments of the force term vanish except the
    first-order ones (= F).  The Hermite polynomials 1, cbar, cbar^2 - c_s^2
    per axis applied to central_force give exactly that."""
    rng = np.random.default_rng(32)
    F = rng.standard_normal(3)
    Rb = Q.central_force(F)
    mono = np.linalg.solve(Q.P_MONO, Rb)  # monomial central moments
    cube = np.zeros((3, 3, 3))
    for v, (a, b, c) in zip(mono, Q.MONO):
        cube[a, b, c] = v
    H = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-CS2, 0.0, 1.0]])  # H_n in terms of cbar^m
    chm = np.einsum("ia,jb,kc,abc->ijk", H, H, H, cube)
    expect = np.zeros((3, 3, 3))
    expect[1, 0, 0], expect[0, 1, 0], expect[0, 0, 1] = F
    np.testing.assert_allclose(chm, expect, rtol=0, atol=1e-14)


def random_states(rng, n=200):
    f = np.array([Q.feq(rng.uniform(0.85, 1.15), 0.08 * rng.standard_normal(3)) for _ in range(n)])
    f += 0.01 * Q.W * rng.standard_normal((n, 27))
    rho = f.sum(axis=1)
    F = 1e-3 * rng.standard_normal((n, 3))
    j = f @ CVEC.T
    u = (j + F / 2) / rho[:, None]
    return f, rho, j, u, F


def test_dense_and_factorised_collisions_agree():
    rng = np.random.default_rng(33)
    f, rho, _, u, F = random_states(rng)
    for om in (0.6, 1.0, 1.9):
        a = Q.collide_dense(f, rho, u, F, om)
        b = Q.collide_factorised(f, rho, u, F, om)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_conservation_and_fixed_point():
    rng = np.random.default_rng(34)
    f, rho, j, u, F = random_states(rng, 50)
    out = Q.collide_factorised(f, rho, u, F, 1.4)
    np.testing.assert_allclose(out.sum(axis=1), rho, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out @ CVEC.T, j + F, rtol=0, atol=1e-15)
    fe = Q.feq(1.07, (0.04, -0.03, 0.02))
    np.testing.assert_allclose(Q.collide_factorised(fe, fe.sum(), np.array([0.04, -0.03, 0.02]), np.zeros(3), 1.4),
                               fe, rtol=0, atol=1e-15)


def shear_rate(make, U_axis=None, U=0.0, n=32, omega=1.25, steps=400):
    k = 2 * math.pi / n
    _, y, _ = inputs.grid(1, n, 1)
    s = np.sin(k * y)
    u = np.zeros((3, 1, n, 1))
    u[0] = 1e-4 * s
    if U_axis is not None:
        u[U_axis] += U
    d = make((1, n, 1), omega)
    d.init(np.ones((1, n, 1)), u)
    d.step(steps)
    out = d.fields()
    ux = out[1][0] - out[1][0].mean()
    return -math.log(((ux * s).sum() / (s * s).sum()) / 1e-4) / (k * k * steps)


def test_viscosity_and_frame_independence():
    """Shear wave u_x(y): decay rate nu k^2 with nu = c_s^2 (1/omega - 1/2);
    the same rate, to rounding, as the D3Q19 step (both relax the deviatoric
    second moments alike); unchanged in frames moving along x or z."""
    nu = CS2 * (1 / 1.25 - 0.5)
    r27 = shear_rate(Q.Domain27)
    r19 = shear_rate(O.Domain)
    assert abs(r27 / nu - 1) < 1e-2
    assert abs(r27 / r19 - 1) < 1e-9
    for axis in (0, 2):
        assert abs(shear_rate(Q.Domain27, axis, 0.2) / r27 - 1) < 1e-9


def test_walls_lid_force_dense_against_factorised_domain():
    """Streaming with half-way bounce-back, the moving lid and a body force:
    the two collision paths through whole steps."""
    shape = (5, 6, 4)
    rho, u = inputs.random_fields(shape, seed=35, u_amp=0.03)
    out = []
    for coll in ("dense", "factorised"):
        d = Q.Domain27(shape, 1.3, periodic=(True, False, False), lid_u=(0.04, 0.0, 0.01), g=(1e-4, -2e-5, 0.0),
                       collision=coll)
        d.init(rho, u)
        d.step(6)
        out.append(d.fields())
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=0, atol=1e-13)


def test_raw_moment_variant():
    """D3Q27 with raw moments (T = M): the factorised path equals the MRT
    definition; mass exact, momentum gains F; one collision with the central
    variant at rest (u = 0, F = 0)."""
    rng = np.random.default_rng(36)
    f, rho, j, u, F = random_states(rng, 60)
    a = Q.collide_dense_rm(f, rho, u, F, 1.3)
    b = Q.collide_factorised_rm(f, rho, u, F, 1.3)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
    np.testing.assert_allclose(b.sum(axis=1), rho, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b @ CVEC.T, j + F, rtol=0, atol=1e-15)
    z = np.zeros(3)
    f0 = Q.W * (1 + 0.01 * rng.standard_normal(27))
    f0 = 0.5 * (f0 + f0[Q.OPP])
    np.testing.assert_allclose(Q.collide_factorised_rm(f0, f0.sum(), z, z, 1.3),
                               Q.collide_factorised(f0, f0.sum(), z, z, 1.3), rtol=0, atol=1e-15)
