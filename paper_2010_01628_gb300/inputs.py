"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the oracle.

This module holds none of the method's arithmetic: it only draws random numbers
and evaluates the initial-condition formulas of the workloads (fields rho, u,
phase, B in the layout [nz][ny][nx], x fastest; vectors as [3, nz, ny, nx]).
Both sides turn these fields into populations with their own code.

Workloads (all in lattice units):

* 3D Taylor-Green vortex (Sec. III.E initial field, x -> 2 pi x / n on node
  centres, rho = 1).
* 2D Taylor-Green mode (Sec. III.A initial field; density from the pressure of
  the exact solution, u_y with the sign that makes the field divergence-free).
* Periodic box with uniform seeded velocity noise (body-force-driven flow).
* Hartmann channel (Sec. III.F): walls in y, uniform b = (0, b_y0, 0).
* Colour-gradient droplets: non-overlapping spheres with a tanh profile.
* Lid-driven cavity at rest.
"""
from __future__ import annotations

import math

import numpy as np


def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def taylor_green_3d(n, u0=0.05, rho0=1.0):
    x, y, z = grid(n, n, n)
    k = 2.0 * math.pi / n
    X, Y, Z = k * x, k * y, k * z
    u = np.stack([u0 * np.cos(X) * np.sin(Y) * np.sin(Z),
                  -0.5 * u0 * np.sin(X) * np.cos(Y) * np.sin(Z),
                  -0.5 * u0 * np.sin(X) * np.sin(Y) * np.cos(Z)])
    rho = np.full((n, n, n), rho0)
    return rho, u


def taylor_green_2d(n, u0=0.01, rho0=1.0, nz=1):
    """Shear-wave pair in the x-y plane, uniform along z (nz nodes)."""
    x, y, _ = grid(n, n, nz)
    k = 2.0 * math.pi / n
    u = np.stack([u0 * np.cos(k * x) * np.sin(k * y),
                  -u0 * np.sin(k * x) * np.cos(k * y),
                  np.zeros_like(x)])
    rho = rho0 * (1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * k * y)))
    return rho, u


def noise_box(shape, amp=1e-3, seed=1, rho0=1.0):
    """Uniform density, velocity components i.i.d. U(-amp, amp)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    u = rng.uniform(-amp, amp, size=(3, nz, ny, nx))
    rho = np.full((nz, ny, nx), rho0)
    return rho, u


def random_fields(shape, seed, rho_amp=0.02, u_amp=0.05):
    """Smooth-free random fields for brute-force parity on tiny grids."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rho = 1.0 + rng.uniform(-rho_amp, rho_amp, size=(nz, ny, nx))
    u = rng.uniform(-u_amp, u_amp, size=(3, nz, ny, nx))
    return rho, u


def random_populations(n_cells, seed, spread=0.1):
    """Arbitrary positive populations, cell-major [n_cells, 19]."""
    rng = np.random.default_rng(seed)
    return (1.0 / 19.0) * (1.0 + spread * rng.uniform(-1.0, 1.0, size=(n_cells, 19)))


def hartmann(ny, b_y0, nx=1, nz=1):
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    B = np.zeros((3, nz, ny, nx))
    B[1] = b_y0
    return rho, u, B


def droplets(n, seed=3, r_min=8.0, r_max=24.0, fraction=0.10, width=4.0, gap=4.0, rho_r0=10.0, rho_b0=1.0,
             max_tries=100000):
    """Seeded non-overlapping spheres (radius U[r_min, r_max], surface gap >= gap)
    added until their volume fraction reaches ``fraction`` (the last sphere may
    overshoot).  phase = tanh(2 (R - r) / width) of the nearest sphere;
    rho = rho_r0 (1 + phase)/2 + rho_b0 (1 - phase)/2.  Returns (rho, u, phase,
    spheres, actual_fraction)."""
    rng = np.random.default_rng(seed)
    spheres = []
    vol = 0.0
    total = float(n) ** 3
    tries = 0
    while vol / total < fraction and tries < max_tries:
        tries += 1
        r = rng.uniform(r_min, r_max)
        c = rng.uniform(0, n, size=3)
        ok = True
        for (c2, r2) in spheres:
            d = np.abs(c - c2)
            d = np.minimum(d, n - d)
            if math.sqrt(float((d * d).sum())) < r + r2 + gap:
                ok = False
                break
        if ok:
            spheres.append((c, r))
            vol += 4.0 / 3.0 * math.pi * r ** 3
    phase = np.full((n, n, n), -1.0)
    for (c, r) in spheres:
        # the tanh profile is -1 to double precision beyond r + 10 w; work on
        # the periodic bounding box of that radius
        reach = int(math.ceil(r + 10.0 * width))
        idx = [np.arange(int(math.floor(c[a])) - reach, int(math.floor(c[a])) + reach + 2) for a in range(3)]
        d = [np.abs(idx[a] - c[a]) for a in range(3)]
        d = [np.minimum(d[a] % n, n - d[a] % n) for a in range(3)]
        dist = np.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
        prof = np.tanh(2.0 * (r - dist) / width)
        zi, yi, xi = (idx[2] % n), (idx[1] % n), (idx[0] % n)
        sub = phase[np.ix_(zi, yi, xi)]
        phase[np.ix_(zi, yi, xi)] = np.maximum(sub, prof)
    rho = rho_r0 * (1.0 + phase) / 2.0 + rho_b0 * (1.0 - phase) / 2.0
    u = np.zeros((3, n, n, n))
    return rho, u, phase, spheres, vol / total


def static_bubble(shape, radius, rho_l=1.95, rho_v=0.15, width=0.0, centre=None, axes=(0, 1, 2), noise=0.0,
                  seed=0):
    """Liquid droplet of density rho_l and radius ``radius`` in vapour rho_v,
    at rest (the static-bubble workload: 100^3, R in [15, 30], 1.95 / 0.15).
    width = 0 is the sharp step; width > 0 a tanh profile of that width.
    ``axes`` lists the axes the distance is taken over (two axes: a cylinder
    along the third).  ``noise`` adds i.i.d. U(-noise, noise) to u."""
    nx, ny, nz = shape
    x, y, z = grid(nx, ny, nz)
    c = [(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0] if centre is None else list(centre)
    d2 = np.zeros_like(x)
    for a, v in zip((0, 1, 2), (x, y, z)):
        if a in axes:
            d2 += (v - c[a]) ** 2
    d = np.sqrt(d2)
    if width > 0:
        rho = rho_v + (rho_l - rho_v) * 0.5 * (1.0 + np.tanh((radius - d) / width))
    else:
        rho = np.where(d <= radius, rho_l, rho_v)
    u = np.zeros((3, nz, ny, nx))
    if noise > 0:
        u += np.random.default_rng(seed).uniform(-noise, noise, size=u.shape)
    return rho, u


def rayleigh_taylor(W=64, rho_h=3.0, rho_l=1.0, amp=0.05, ny_factor=4):
    """Rayleigh-Taylor start (Sec. III.H): a W x 4W x W box at rest, heavy
    fluid (rho_h, order parameter +1) where y > 2W + amp W [cos(2 pi x/W) +
    cos(2 pi z/W)], light fluid (rho_l, -1) below; node coordinates 0..n-1.
    Returns (rho, u, phase) with the [nz][ny][nx] layout."""
    nx, ny, nz = W, ny_factor * W, W
    x, y, z = grid(nx, ny, nz)
    surface = 0.5 * ny_factor * W + amp * W * (np.cos(2.0 * math.pi * x / W) + np.cos(2.0 * math.pi * z / W))
    heavy = y > surface
    rho = np.where(heavy, rho_h, rho_l)
    phase = np.where(heavy, 1.0, -1.0)
    return rho, np.zeros((3, nz, ny, nx)), phase


def double_shear_layer(L=256, u0=0.57 / math.sqrt(3.0), kappa=80.0, delta=0.05):
    """Double shear layer (Sec. III.B) on a periodic L x L x 1 box, nodes at
    x, y = 0 .. L-1: u_x = u0 tanh(kappa (y/L - 1/4)) for y/L <= 1/2, else
    u0 tanh(kappa (3/4 - y/L)); u_y = u0 delta sin(2 pi (x/L + 1/4)); rho = 1."""
    x, y, _ = grid(L, L, 1)
    ux = np.where(y / L <= 0.5, u0 * np.tanh(kappa * (y / L - 0.25)), u0 * np.tanh(kappa * (0.75 - y / L)))
    uy = u0 * delta * np.sin(2.0 * math.pi * (x / L + 0.25))
    u = np.stack([ux, uy, np.zeros_like(ux)])
    return np.ones_like(ux), u


def dipole(D_lb, U_lb, inclined=False, w_e=299.56, r0=0.1):
    """Dipole in the box [-1, 1]^2 (Sec. III.D), 2 D_lb x 2 D_lb x 1 nodes at
    cell centres x_i = -1 + (i + 1/2)/D_lb (half-way walls lie on x, y = +-1).
    Monopoles at (0, 0.1) and (0, -0.1), or rotated by 30 degrees at
    (0.0839, 0.0866) and (0.1839, -0.0866); velocity in lattice units, the
    physical field (rms 1) times U_lb; rho = 1."""
    n = 2 * D_lb
    i, j, _ = grid(n, n, 1)
    x = -1.0 + (i + 0.5) / D_lb
    y = -1.0 + (j + 0.5) / D_lb
    (x1, y1), (x2, y2) = ((0.0839, 0.0866), (0.1839, -0.0866)) if inclined else ((0.0, 0.1), (0.0, -0.1))
    e1 = np.exp(-((x - x1) ** 2 + (y - y1) ** 2) / r0 ** 2)
    e2 = np.exp(-((x - x2) ** 2 + (y - y2) ** 2) / r0 ** 2)
    a = 0.5 * abs(w_e)
    ux = -a * (y - y1) * e1 + a * (y - y2) * e2
    uy = a * (x - x1) * e1 - a * (x - x2) * e2
    u = U_lb * np.stack([ux, uy, np.zeros_like(ux)])
    return np.ones_like(ux), u


def cavity_rest(n):
    return np.ones((n, n, n)), np.zeros((3, n, n, n))


def hartmann_batch(ndomains=64, seed=2, sizes=(32, 48, 64, 96), ha_range=(1.0, 20.0)):
    """Parameter sweep of cubic Hartmann channels: (n_d, Ha_d) pairs."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(sizes), size=ndomains)
    ha = rng.uniform(ha_range[0], ha_range[1], size=ndomains)
    return [(int(a), float(b)) for a, b in zip(n, ha)]


def droplet_sweep(ndomains=64, seed=5, sizes=(32, 48, 64, 96), ratio_range=(2.0, 10.0)):
    """Parameter sweep of cubic droplet boxes: (n_d, density ratio_d) pairs.
    Each box is filled by droplets(n_d, seed + d, r_min = max(4, n_d/16),
    r_max = max(6, n_d/8), rho_r0 = ratio_d, rho_b0 = 1) (the 256^3 recipe's
    radii 8-24 scaled to the box)."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(sizes), size=ndomains)
    ratio = rng.uniform(ratio_range[0], ratio_range[1], size=ndomains)
    return [(int(a), float(b)) for a, b in zip(n, ratio)]


def bubble_sweep(ndomains=64, seed=6, sizes=(32, 48, 64, 96), g_range=(-5.5, -4.5)):
    """Shan-Chen sweep: (n_d, G_d) pairs; box d holds a centred static bubble
    (static_bubble, sharp 1.95 / 0.15 start) of radius n_d / 4."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(sizes), size=ndomains)
    G = rng.uniform(g_range[0], g_range[1], size=ndomains)
    return [(int(a), float(b)) for a, b in zip(n, G)]


def sweep_droplets(n, ratio, index, seed=5):
    """Fields (rho, u, phase) of domain `index` of droplet_sweep."""
    rho, u, phase, _, _ = droplets(n, seed=seed + index, r_min=max(4.0, n / 16.0), r_max=max(6.0, n / 8.0),
                                   rho_r0=ratio, rho_b0=1.0)
    return rho, u, phase


def cavity_reynolds(count, seed=4, lo=100.0, hi=1000.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=count)
