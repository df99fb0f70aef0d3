"""The seeded synthetic workloads match the recipes the design notes state
(CPU): sizes, ranges, node counts, volume fractions and the phase and density
profiles the configurations name."""
import math

import numpy as np

from paper_2010_01628_gb300 import inputs


def test_body_force_noise_box():
    rho, u = inputs.noise_box((24, 16, 8), amp=1e-3, seed=1)
    assert rho.shape == (8, 16, 24) and u.shape == (3, 8, 16, 24)
    assert np.all(rho == 1.0) and np.abs(u).max() <= 1e-3 and np.abs(u).max() > 0.9e-3
    # seeded: the same call gives the same field, another seed another one
    assert np.array_equal(u, inputs.noise_box((24, 16, 8), seed=1)[1])
    assert not np.array_equal(u, inputs.noise_box((24, 16, 8), seed=2)[1])


def _check_sweep(sweep, lo, hi, nodes):
    assert len(sweep) == 64
    assert {n for n, _ in sweep} <= {32, 48, 64, 96}
    assert all(lo <= v <= hi for _, v in sweep)
    assert sum(n ** 3 for n, _ in sweep) == nodes


def test_parameter_sweeps():
    _check_sweep(inputs.hartmann_batch(64, seed=2), 1.0, 20.0, 21_651_456)  # Hartmann numbers
    _check_sweep(inputs.droplet_sweep(64, seed=5), 2.0, 10.0, 21_581_824)  # density ratios
    _check_sweep(inputs.bubble_sweep(64, seed=6), -5.5, -4.5, 22_269_952)  # interaction strengths G


def test_cavity_reynolds_split():
    re = inputs.cavity_reynolds(512 + 32, seed=4)
    assert re.min() >= 100.0 and re.max() <= 1000.0
    train, held = re[:512], re[512:]
    assert len(held) == 32 and not set(np.round(held, 9)) & set(np.round(train, 9))


def test_droplets_recipe_small_box():
    """The C4 recipe on a 96^3 box: non-overlapping spheres with surface gaps
    of at least 4 (periodic distances), radii in [8, 24], volume fraction at
    or just past 10%, phase = tanh(2 (R - r)/4) of the nearest sphere, red
    density 10 inside and blue 1 outside."""
    n = 96
    rho, u, phase, spheres, frac = inputs.droplets(n, seed=3)
    assert 0.10 <= frac < 0.10 + 4.0 / 3.0 * math.pi * 24 ** 3 / n ** 3
    assert all(8.0 <= r <= 24.0 for _, r in spheres)
    for i, (c1, r1) in enumerate(spheres):
        for c2, r2 in spheres[i + 1:]:
            d = np.abs(c1 - c2)
            d = np.minimum(d, n - d)
            assert math.sqrt(float((d * d).sum())) >= r1 + r2 + 4.0
    assert np.all(u == 0) and phase.min() >= -1.0 and phase.max() <= 1.0
    np.testing.assert_allclose(rho, 10.0 * (1 + phase) / 2 + 1.0 * (1 - phase) / 2, rtol=0, atol=1e-12)
    c, r = spheres[0]
    x = int(round(c[0] + r)) % n, int(round(c[1])) % n, int(round(c[2])) % n  # a node near the first interface
    dist = math.sqrt(sum(min(abs(v - cv), n - abs(v - cv)) ** 2 for v, cv in zip(x, c)))
    assert abs(phase[x[2], x[1], x[0]] - math.tanh(2.0 * (r - dist) / 4.0)) < 1e-12
    # the droplets' volume matches the phase field's red volume to a few per cent
    red = float(((1 + phase) / 2).sum()) / n ** 3
    assert abs(red - frac) < 0.1 * frac


def test_static_bubble_and_rayleigh_taylor():
    rho, u = inputs.static_bubble((40, 40, 40), 10.0)[:2]
    assert rho[20, 20, 20] == 1.95 and rho[0, 0, 0] == 0.15 and np.all(u == 0)
    out = inputs.rayleigh_taylor(W=16)
    rho = out[0]
    nz, ny, nx = rho.shape
    assert (nx, ny, nz) == (16, 64, 16)
    assert np.all(rho[:, -1, :] == 3.0) and np.all(rho[:, 0, :] == 1.0)
    # the interface sits at y = 2W + 0.05 W (cos(2 pi x/W) + cos(2 pi z/W)): heavy fluid above it
    y_top = 2 * 16 + 0.05 * 16 * 2  # at x = z = 0 the perturbation is largest
    assert rho[0, int(math.ceil(y_top)) + 1, 0] == 3.0 and rho[0, int(y_top) - 1, 0] == 1.0
