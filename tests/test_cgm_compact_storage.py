"""The colour-gradient step on the GPU stores the total populations with each
node's red fraction a = rho_r / rho and recolouring vector
V = beta (rho_r rho_b / rho)(1 - alpha) grad phi / |grad phi|, and rebuilds a
moving red population as a f_i + kappa_i c_i . V (kappa = 1/12 on the axes,
1/(24 sqrt 2) on the diagonals), the red rest population from the colour mass
balance, blue as the total minus red.  This checks that identity against the
oracle's recolouring (App. E, Eqs. eq:op3r and eq:op3b) on random states,
including a vanishing gradient (no recolouring term).  CPU only."""
import numpy as np

import oracle as O


def compact_red(f, grad, rho_r, rho_b, alpha, beta, c):
    rho = rho_r + rho_b
    norm = np.linalg.norm(grad)
    inv_norm = 1.0 / norm if norm > 1e-12 else 0.0
    a = rho_r / rho
    V = beta * rho_r * rho_b / rho * (1.0 - alpha) * inv_norm * np.asarray(grad)
    c2 = (c ** 2).sum(axis=1)
    kappa = np.where(c2 == 1, 1.0 / 12.0, 1.0 / (24.0 * np.sqrt(2.0)))
    red = a * f + kappa * (c @ V)
    red[0] = rho_r - red[1:].sum()  # the colour mass balance of the rest direction
    return red


def test_compact_red_populations_equal_the_recolouring():
    c, w = O.lattice()
    rng = np.random.default_rng(17)
    for trial in range(300):
        f = w * rng.uniform(0.2, 3.0, 19)
        rho = f.sum()
        rho_r = rho * rng.uniform(0.0, 1.0)
        rho_b = rho - rho_r
        alpha, beta = rng.uniform(0.2, 0.95), rng.uniform(0.1, 0.99)
        grad = rng.normal(size=3) * 10.0 ** rng.uniform(-6, 0)
        if trial % 50 == 0:
            grad = np.zeros(3)
        fr, fb = O.cgm_recolour(f, grad, rho_r, rho_b, alpha, beta)
        red = compact_red(f, grad, rho_r, rho_b, alpha, beta, c)
        np.testing.assert_allclose(red, fr, rtol=0, atol=1e-14 * rho)
        np.testing.assert_allclose(f - red, fb, rtol=0, atol=1e-14 * rho)
        # the stored quantities reproduce both colour densities
        assert abs(red.sum() - rho_r) <= 1e-14 * rho and abs((f - red).sum() - rho_b) <= 1e-14 * rho


def test_recolouring_terms_cancel_over_opposite_directions():
    """The red rest population of the balance equals a f_0 because the
    recolouring terms of opposite directions cancel (c_opp = -c, same kappa)."""
    c, _ = O.lattice()
    opp = [0] + [i + 9 for i in range(1, 10)] + [i - 9 for i in range(10, 19)]
    assert all((c[opp[i]] == -c[i]).all() for i in range(19))
    rng = np.random.default_rng(3)
    V = rng.normal(size=3)
    c2 = (c ** 2).sum(axis=1)
    kappa = np.where(c2 == 1, 1.0 / 12.0, 1.0 / (24.0 * np.sqrt(2.0)))
    assert abs((kappa * (c @ V))[1:].sum()) < 1e-15
