"""Two-dimensional validation cases of Sec. III on the GPU: the double shear
layer (Sec. III.B) and the dipole-wall collision (Sec. III.D, Tables 2-4).

The paper's printed values are its own FP64 runs with regularized walls; here
the walls are half-way bounce-back (on all four sides, which the regularized
channel walls do not cover), so the comparison bands are loose and stated per
quantity."""
import math
import os

import numpy as np
import pytest

from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dipole_tables_appIII_D.txt")
U_LB = 0.06 / math.sqrt(3.0)  # Ma ~ 0.06


def golden():
    t2, t3, t4 = {}, {}, {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            v = [float(a) for a in v]
            if k == "table2":
                t2[(int(v[0]), v[1])] = (v[2], v[3])
            elif k == "table3":
                t3[(int(v[0]), v[1])] = v[2]
            else:
                t4[int(v[0])] = (v[1], v[2])
    return t2, t3, t4


def d_wall(f, h, axis):
    """Derivative with no-slip walls half a cell beyond both end nodes:
    central inside, three-point (wall, node, next node) at the ends."""
    f = np.moveaxis(f, axis, 0)
    d = np.empty_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (2 * h)
    a, b = h / 2, h
    d[0] = (a * a * f[1] - (a * a - b * b) * f[0]) / (a * b * (a + b))
    d[-1] = (-a * a * f[-2] - (b * b - a * a) * f[-1]) / (a * b * (a + b))
    return np.moveaxis(d, 0, axis)


def dipole_history(Re, D, inclined, times):
    """E(t) = 1/2 int |u|^2 and Psi(t) = 1/2 int w^2 in the paper's units
    (D = 1, rms velocity 1) at the given times."""
    from paper_2010_01628_gb300 import binding as L
    nu = U_LB * D / Re
    n = 2 * D
    rho, u = inputs.dipole(D, U_LB, inclined)
    ctx = L.lbm_create((n, n, 1), 1.0 / (3 * nu + 0.5), precision="fp32", periodic=(False, False, True))
    out, done, h = [], 0, 1.0 / D
    try:
        L.lbm_init_fields(ctx, rho, u)
        for t in times:
            target = int(round(t * D / U_LB))
            L.lbm_step(ctx, target - done)
            done = target
            up = L.lbm_fields(ctx, (n, n, 1))["u"] / U_LB
            E = 0.5 * float((up[0] ** 2 + up[1] ** 2).sum()) * h * h
            w = d_wall(up[1, 0], h, 1) - d_wall(up[0, 0], h, 0)
            out.append((t, E, 0.5 * float((w * w).sum()) * h * h))
    finally:
        L.lbm_destroy(ctx)
    return out


CASES = [(625, 512), (1250, 768), (2500, 1024)]


@pytest.mark.parametrize("Re,D", CASES)
def test_dipole_normal_collision_table2(Re, D):
    """Energy within 2 % of the paper's D3Q19 values at t = 0.25, 0.5, 0.75
    (measured: 0.2 to 1.6 %); enstrophy within 10 % (measured: up to 8 %;
    it changes fast around the collision and depends on how the wall vorticity
    is taken)."""
    t2, _, _ = golden()
    for t, E, P in dipole_history(Re, D, False, (0.25, 0.5, 0.75)):
        E_p, P_p = t2[(Re, t)]
        assert abs(E / E_p - 1) < 0.02, (Re, t, E, E_p)
        assert abs(P / P_p - 1) < 0.10, (Re, t, P, P_p)


@pytest.mark.parametrize("Re,D", CASES)
def test_dipole_inclined_collision_tables3_4(Re, D):
    """Table 3: energy within 3.5 % at t = 0.3, 0.5, 2.0.  Table 4: the first
    enstrophy maximum (largest in t in [0.25, 0.48], enstrophy smoothed over
    0.02 to remove the acoustic ripple of the uniform-density start) within
    0.03 of the paper's time."""
    _, t3, t4 = golden()
    times = sorted(set([0.3, 0.5, 2.0] + [round(0.2 + 0.002 * k, 6) for k in range(141)]))
    hist = dipole_history(Re, D, True, times)
    vals = {round(t, 6): (E, P) for t, E, P in hist}
    for t in (0.3, 0.5, 2.0):
        assert abs(vals[t][0] / t3[(Re, t)] - 1) < 0.035, (Re, t, vals[t][0], t3[(Re, t)])
    ts = np.array(sorted(t for t in vals if 0.2 <= t <= 0.48 + 1e-9))
    P = np.array([vals[t][1] for t in ts])
    Ps = np.convolve(P, np.ones(11) / 11, mode="same")
    inner = (ts > 0.25) & (ts < 0.47)
    t1 = ts[inner][np.argmax(Ps[inner])]
    assert abs(t1 - t4[Re][0]) < 0.03, (Re, t1, t4[Re][0])


def dsl_history(lattice, precision, Ma, points):
    from paper_2010_01628_gb300 import binding as L
    Lb = 256
    u0 = Ma / math.sqrt(3.0)
    nu = u0 * Lb / 3e4
    t0 = Lb / u0
    rho, u = inputs.double_shear_layer(Lb, u0=u0)
    ctx = L.lbm_create((Lb, Lb, 1), 1.0 / (3 * nu + 0.5), precision=precision, lattice=lattice)
    out, done = [], 0
    try:
        L.lbm_init_fields(ctx, rho, u)
        for k in range(points + 1):
            target = int(round(k * t0 / points))
            L.lbm_step(ctx, target - done)
            done = target
            uu = L.lbm_fields(ctx, (Lb, Lb, 1))["u"]
            w = np.gradient(uu[1, 0], axis=1) - np.gradient(uu[0, 0], axis=0)
            out.append((float((uu[0] ** 2 + uu[1] ** 2).sum()), float((w * w).sum())))
    finally:
        L.lbm_destroy(ctx)
    E = np.array([o[0] for o in out])
    P = np.array([o[1] for o in out])
    return E / E[0], P / P[0]


def test_double_shear_layer_d3q19_d3q27_agree_fp64():
    """Sec. III.B at Ma = 0.57, Re = 3e4, L = 256, to t/t0 = 1 (t0 = L/u0): both
    lattices stay stable, and their normalised kinetic energy agrees to 1e-4
    (the paper: about 0.009 %; measured 6e-6) and their enstrophy to 1e-3."""
    E19, P19 = dsl_history("d3q19", "fp64", 0.57, 10)
    E27, P27 = dsl_history("d3q27", "fp64", 0.57, 10)
    assert np.all(np.isfinite(E19)) and np.all(np.isfinite(E27))
    assert np.abs(E19 - E27).max() < 1e-4
    assert np.abs(P19 - P27).max() < 1e-3 * P27.max()
    assert 0.9 < E19[-1] < 1.0


def test_double_shear_layer_fp32_tracks_fp64_at_ma_035():
    """FP32 storage follows FP64 to 1e-5 in normalised energy at Ma = 0.35 (at
    Ma = 0.57 it tracks FP64 to 1e-6 until t/t0 = 0.8 and then rounding noise
    seeds an instability the FP64 run does not reach)."""
    E64, _ = dsl_history("d3q19", "fp64", 0.35, 10)
    E32, _ = dsl_history("d3q19", "fp32", 0.35, 10)
    assert np.abs(E64 - E32).max() < 1e-5
