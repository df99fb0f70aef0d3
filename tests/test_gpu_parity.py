"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (relative L2 of rho and of u after the same number of steps) are
the stated targets: 1e-12 for FP64 storage, 1e-5 for FP32, 1e-3 for FP16
storage.  BF16 storage (8-bit significand, unit roundoff 2^-9) does not meet
1e-3 on the Taylor-Green case (2.4e-3 measured for u after 200 steps); its
bound here is 4e-3 ~ 2^-8, two roundings of the stored (f - w)/w per step.
"""
import math

import numpy as np
import pytest

from helpers import gpu_run, oracle_run, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 4e-3}
# The density deviation rho - 1 against its own norm: rho ~ 1 makes the plain
# relative error of rho weak.  rho - 1 is 1e-3 to 1e-2 of rho on these cases,
# so an error at the rho bound is 1e2 to 1e3 times larger relative to rho - 1;
# the bounds sit between (measured on the GB300: FP64 <= 3e-11, FP32 <= 8e-5,
# FP16 <= 5e-3, BF16 <= 6e-2).
DRHO_TOL = {1e-12: 1e-10, 1e-5: 2e-4, 1e-3: 2e-2, 4e-3: 1e-1}


def compare(g, o, tol, fields=("rho", "u")):
    errs = {k: rel_l2(g[k], o[k]) for k in fields}
    errs["drho"] = rel_l2(g["rho"] - 1.0, o["rho"] - 1.0)
    for k in fields:
        assert errs[k] <= tol, (k, errs)
    if tol in DRHO_TOL:
        assert errs["drho"] <= DRHO_TOL[tol], ("drho", errs)
    return errs


# --- single phase --------------------------------------------------------------

@pytest.fixture(scope="module")
def tg32_oracle():
    """Taylor-Green vortex 32^3, u0 = 0.05, tau = 0.53, 200 steps (FP64 oracle)."""
    rho, u = inputs.taylor_green_3d(32, u0=0.05)
    return rho, u, oracle_run((32, 32, 32), 1 / 0.53, 200, rho, u)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_taylor_green_32(tg32_oracle, precision):
    rho, u, o = tg32_oracle
    g = gpu_run((32, 32, 32), 1 / 0.53, 200, rho, u, precision=precision)
    compare(g, o, TOL[precision])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_16bit_error_is_the_storage_floor(tg32_oracle, precision):
    """What bounds the 16-bit storage: the FP64 oracle with its populations
    rounded to the storage format after every step (exact arithmetic in
    between) already carries the format's floor.  The GPU (FP32 arithmetic,
    same storage) stays within 1.6x of that floor for u, so the kernels add
    little to it; for BF16 the floor itself exceeds 1e-3 on this case."""
    from helpers import oracle_run_stored
    rho, u, o = tg32_oracle
    floor = oracle_run_stored((32, 32, 32), 1 / 0.53, 200, rho, u, precision)
    g = gpu_run((32, 32, 32), 1 / 0.53, 200, rho, u, precision=precision)
    f_u = rel_l2(floor["u"], o["u"])
    g_u = rel_l2(g["u"], o["u"])
    assert g_u <= 1.6 * f_u, (g_u, f_u)
    if precision == "bf16":
        assert f_u > 1e-3, f_u


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_body_force_ragged_box(precision):
    """Periodic box, nx = 70 (two blocks + a ragged tail), uniform g.  The
    velocity noise is 1e-2: at 1e-3 the oracle's own FP64 summation of
    unshifted populations (terms ~ 1/18 cancelling to ~1e-3) already puts
    ~1e-12 relative error on u after 30 steps."""
    shape = (70, 9, 5)
    rho, u = inputs.noise_box(shape, amp=1e-2, seed=1)
    g = (1e-6, 2e-7, -3e-7)
    o = oracle_run(shape, 1 / 0.6, 30, rho, u, g=g)
    r = gpu_run(shape, 1 / 0.6, 30, rho, u, g=g, precision=precision)
    compare(r, o, TOL[precision])


@pytest.mark.parametrize("shape", [(5, 6, 7), (37, 4, 3), (1, 8, 1), (1, 1, 1)])
def test_brute_force_walls_and_lid_dense_oracle(shape):
    """Random fields on tiny boxes, walls on y and z, moving lid, body force:
    FP64 GPU against the definitional dense-solve oracle."""
    rho, u = inputs.random_fields(shape, seed=31)
    kw = dict(periodic=(True, False, False), lid_u=(0.05, 0.0, 0.02), g=(1e-4, -2e-5, 0.0))
    o = oracle_run(shape, 1.3, 12, rho, u, closed_form=False, **kw)
    r = gpu_run(shape, 1.3, 12, rho, u, precision="fp64", **kw)
    compare(r, o, 1e-12)


@pytest.mark.parametrize("periodic", [(False, False, False), (False, True, True), (True, True, False)])
def test_all_wall_combinations_fp64(periodic):
    shape = (9, 7, 6)
    rho, u = inputs.random_fields(shape, seed=32, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.04, 0.0, 0.0), g=(0.0, 0.0, 1e-5))
    o = oracle_run(shape, 1.7, 15, rho, u, **kw)
    r = gpu_run(shape, 1.7, 15, rho, u, precision="fp64", **kw)
    compare(r, o, 1e-12)


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("shape,periodic", [((36, 10, 6), (False, False, True)), ((2, 4, 3), (False, False, False)),
                                            ((70, 3, 4), (True, True, True))])
def test_16bit_two_cell_kernel(precision, shape, periodic):
    """The 16-bit path handles two x-cells per thread (even nx); walls in x,
    the lid, a two-node row and ragged rows against the FP64 oracle."""
    rho, u = inputs.random_fields(shape, seed=33, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.05, 0.0, 0.01), g=(1e-5, 0.0, 0.0))
    o = oracle_run(shape, 1.4, 20, rho, u, **kw)
    r = gpu_run(shape, 1.4, 20, rho, u, precision=precision, launch=(2, 64, 0, 1), **kw)
    compare(r, o, TOL[precision])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("shape,periodic", [((37, 10, 7), (False, False, False)), ((5, 4, 1), (False, False, False)),
                                            ((70, 3, 4), (True, True, True)), ((33, 6, 9), (True, False, True))])
def test_16bit_z_pair_kernel(precision, shape, periodic):
    """Two z-neighbour nodes per thread (launch variant 4): odd nz (the last
    thread updates one node), a single plane, walls on every side with the lid,
    and ragged rows against the FP64 oracle."""
    rho, u = inputs.random_fields(shape, seed=34, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.05, 0.0, 0.01), g=(1e-5, 0.0, 2e-6))
    o = oracle_run(shape, 1.4, 20, rho, u, **kw)
    r = gpu_run(shape, 1.4, 20, rho, u, precision=precision, launch=(4, 64, 0, 1), **kw)
    compare(r, o, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape,periodic,stages,ctas", [((64, 9, 7), (False, False, False), 3, 1),
                                                        ((32, 5, 6), (True, True, True), 2, 2),
                                                        ((48, 11, 4), (True, False, True), 4, 1)])
def test_tma_staged_kernel(precision, shape, periodic, stages, ctas):
    """The TMA-staged single-phase kernel (rows of 19 planes in shared memory,
    several rows in flight per CTA) against the FP64 oracle, walls and lid
    included; rows outnumber CTAs so every stage is reused."""
    rho, u = inputs.random_fields(shape, seed=35, u_amp=0.03)
    kw = dict(periodic=periodic, lid_u=(0.04, 0.0, 0.01), g=(1e-5, 0.0, -1e-5))
    o = oracle_run(shape, 1.45, 16, rho, u, **kw)
    r = gpu_run(shape, 1.45, 16, rho, u, precision=precision, launch=(1, 64, stages, ctas), **kw)
    compare(r, o, TOL[precision])


def test_tma_wait_limit_reports_timeout_and_device_stays_usable():
    """The bounded mbarrier wait of the TMA-staged kernels: with no arrival the
    wait gives up after its limit and the kernel reports LBM_ERR_TIMEOUT; with
    the arrival it succeeds at once; a staged step still matches the oracle
    afterwards."""
    import time
    from paper_2010_01628_gb300 import binding as L
    t = time.perf_counter()
    assert L.lbm_mbarrier_selftest(0.2, arrive=False) == L.LBM_ERR_TIMEOUT
    assert time.perf_counter() - t >= 0.2
    assert L.lbm_mbarrier_selftest(0.2, arrive=True) == L.LBM_OK
    shape = (32, 5, 6)
    rho, u = inputs.random_fields(shape, seed=36, u_amp=0.03)
    o = oracle_run(shape, 1.45, 8, rho, u)
    r = gpu_run(shape, 1.45, 8, rho, u, precision="fp32", launch=(1, 64, 2, 1))
    compare(r, o, TOL["fp32"])


def test_launch_shapes_agree_bitwise_fp64():
    """Direct-pull and TMA-staged kernels compute the same arithmetic."""
    shape = (40, 12, 10)
    rho, u = inputs.random_fields(shape, seed=36, u_amp=0.03)
    kw = dict(periodic=(True, False, True), lid_u=(0.03, 0.0, 0.0), g=(1e-5, 0.0, 0.0))
    a = gpu_run(shape, 1.3, 10, rho, u, precision="fp64", launch=(0, 128, 0, 1), **kw)
    b = gpu_run(shape, 1.3, 10, rho, u, precision="fp64", launch=(1, 64, 3, 1), **kw)
    assert rel_l2(a["u"], b["u"]) < 1e-14 and rel_l2(a["rho"], b["rho"]) < 1e-15


def test_uniform_acceleration_momentum_fp32_256():
    """At 256^3 (C2 size, FP32), total momentum grows by exactly M g per step:
    checked with the library's FP64 reductions after 50 steps."""
    from paper_2010_01628_gb300 import binding as L
    n = 256
    rho, u = inputs.noise_box((n, n, n), amp=1e-3, seed=1)
    gx = 1e-6
    ctx = L.lbm_create((n, n, n), 1 / 0.6, g=(gx, 0, 0), precision="fp32")
    try:
        L.lbm_init_fields(ctx, rho, u)
        m0, p0, _ = L.lbm_reduce(ctx)
        L.lbm_step(ctx, 50)
        m1, p1, _ = L.lbm_reduce(ctx)
    finally:
        L.lbm_destroy(ctx)
    assert abs(m1 - m0) / m0 < 1e-6
    # mean u_x(t) = mean u_x(0) + g t (momentum per unit mass)
    assert abs((p1[0] - p0[0]) / m0 - 50 * gx) < 1e-3 * 50 * gx


def sampled_oracle(u_full, rho_full, centre, k, omega, g):
    """Oracle value at one node after k steps.  The reported fields gather
    once more after the k-th collision, so they depend on the initial fields
    within Chebyshev radius k + 1: a periodic (2k+3)^3 box around the node
    reproduces them exactly."""
    n = rho_full.shape[0]
    r = k + 1
    idx = [(np.arange(-r, r + 1) + c) % n for c in centre]  # x, y, z
    sub_rho = rho_full[np.ix_(idx[2], idx[1], idx[0])]
    sub_u = u_full[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    L = 2 * r + 1
    o = oracle_run((L, L, L), omega, k, np.ascontiguousarray(sub_rho), np.ascontiguousarray(sub_u), g=g)
    return o["rho"][r, r, r], o["u"][:, r, r, r]


@pytest.mark.parametrize("precision,launch", [("fp32", "auto"), ("fp16", None), ("fp16", "auto"), ("bf16", None),
                                              ("bf16", "auto"), ("bf16", (4, 128, 0, 1))])
def test_full_size_512_sampled(precision, launch):
    """512^3 body-force box in the benchmark's launch configuration (the
    autotuner's choice, as bench.py runs it; for 16-bit storage also the
    default one-node kernel and the z-pair kernel): sampled nodes (corners and
    edges included) against the oracle's dependency cone."""
    from paper_2010_01628_gb300 import binding as L
    n, k = 512, 4
    omega, g = 1 / 0.6, (1e-6, 0.0, 0.0)
    rho, u = inputs.noise_box((n, n, n), amp=1e-3, seed=1)
    ctx = L.lbm_create((n, n, n), omega, g=g, precision=precision)
    try:
        if launch == "auto":
            L.lbm_autotune(ctx, None)
        elif launch is not None:
            L.lbm_set_launch_shape(ctx, *launch)
        L.lbm_init_fields(ctx, rho, u)
        L.lbm_step(ctx, k)
        out = L.lbm_fields(ctx, (n, n, n))
    finally:
        L.lbm_destroy(ctx)
    rng = np.random.default_rng(5)
    centres = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 7), (n - 1, 3, 0)] + [
        tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(8)]
    ug, uo, rg, ro = [], [], [], []
    for c in centres:
        r_o, u_o = sampled_oracle(u, rho, c, k, omega, g)
        x, y, z = c
        rg.append(out["rho"][z, y, x])
        ro.append(r_o)
        ug.append(out["u"][:, z, y, x])
        uo.append(u_o)
    assert rel_l2(rg, ro) <= TOL[precision]
    assert rel_l2(ug, uo) <= TOL[precision]


# --- magnetohydrodynamics ------------------------------------------------------

def hartmann_kw(ny, ha, nu=0.1, u0=1e-3):
    L_ = ny
    b0 = 2 * ha * nu / L_
    return dict(periodic=(True, False, True), g=(8 * nu * u0 / L_ ** 2, 0, 0), tau_m=0.5 + nu / 0.25,
                b_wall=(0.0, b0, 0.0)), b0, 1.0 / (nu / (1 / 3) + 0.5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_channel_parity(precision):
    shape = (6, 16, 5)
    kw, b0, omega = hartmann_kw(16, 5.0)
    rho, u = inputs.random_fields(shape, seed=41, u_amp=0.01)
    B = np.zeros((3,) + rho.shape)
    B[1] = b0
    B[0] = 1e-3 * np.sin(np.arange(16) * 2 * math.pi / 16)[None, :, None]
    o = oracle_run(shape, omega, 40, rho, u, B=B, physics="mhd", **kw)
    r = gpu_run(shape, omega, 40, rho, u, B=B, physics="mhd", precision=precision, **kw)
    compare(r, o, TOL[precision], fields=("rho", "u", "B"))


def test_mhd_hartmann_profile_gpu():
    """Steady Hartmann profile on the GPU (FP64) against the closed form."""
    ny, ha, nu, u0 = 32, 3.0, 0.1, 1e-3
    kw, b0, omega = hartmann_kw(ny, ha, nu, u0)
    rho, u, B = inputs.hartmann(ny, b0, nx=4, nz=4)
    r = gpu_run((4, ny, 4), omega, int(10 * ny * ny / nu), rho, u, B=B, physics="mhd", precision="fp64", **kw)
    s = (2 * (np.arange(ny) + 0.5) - ny) / ny
    ua = 2 * u0 / (ha * math.tanh(ha)) * (1 - np.cosh(ha * s) / math.cosh(ha))
    prof = r["u"][0].mean(axis=(0, 2))
    assert rel_l2(prof, ua) < 1e-2


# --- colour gradient -----------------------------------------------------------

def cgm_setup(n, seed=3, rho_r0=10.0, rho_b0=1.0, sigma=1e-4, tau=0.8):
    rho, u, phase, spheres, frac = inputs.droplets(n, seed=seed, r_min=3.0, r_max=5.0, fraction=0.1, width=4.0,
                                                   gap=2.0, rho_r0=rho_r0, rho_b0=rho_b0)
    alpha_b = 1.0 / 3.0
    alpha_r = 1.0 - (1.0 - alpha_b) * rho_b0 / rho_r0
    omega = 1.0 / tau
    kw = dict(alpha_r=alpha_r, alpha_b=alpha_b, A=9.0 * sigma * omega / 4.0, beta=0.7)
    return rho, u, phase, omega, kw


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cgm_droplets_parity(precision):
    n = 20
    rho, u, phase, omega, kw = cgm_setup(n)
    u = u + inputs.noise_box((n, n, n), amp=1e-2, seed=9)[1]
    o = oracle_run((n, n, n), omega, 20, rho, u, phase=phase, physics="cgm", **kw)
    r = gpu_run((n, n, n), omega, 20, rho, u, phase=phase, physics="cgm", precision=precision, **kw)
    compare(r, o, TOL[precision], fields=("rho", "u", "phase"))


def test_cgm_walls_fp64():
    shape = (7, 10, 6)
    rho, u, phase, omega, kw = cgm_setup(10)
    rho, phase = rho[:6, :10, :7].copy(), phase[:6, :10, :7].copy()
    u = inputs.random_fields(shape, seed=8, u_amp=0.01)[1]
    kw.update(periodic=(True, False, False))
    o = oracle_run(shape, omega, 10, rho, u, phase=phase, physics="cgm", **kw)
    r = gpu_run(shape, omega, 10, rho, u, phase=phase, physics="cgm", precision="fp64", **kw)
    compare(r, o, 1e-12, fields=("rho", "u", "phase"))


# --- reductions, residual, checkpoint, errors -------------------------------------

def test_reductions_match_oracle_fields():
    from paper_2010_01628_gb300 import binding as L
    shape = (24, 10, 6)
    rho, u = inputs.random_fields(shape, seed=51, u_amp=0.02)
    kw = dict(periodic=(True, False, True), g=(1e-5, 0, 0))
    o1 = oracle_run(shape, 1.4, 7, rho, u, **kw)
    o2 = oracle_run(shape, 1.4, 8, rho, u, **kw)
    ctx = L.lbm_create(shape, 1.4, precision="fp64", **kw)
    try:
        L.lbm_init_fields(ctx, rho, u)
        L.lbm_step(ctx, 7)
        m1, p1, r1 = L.lbm_reduce(ctx)
        L.lbm_step(ctx, 1)
        m2, p2, r2 = L.lbm_reduce(ctx)
    finally:
        L.lbm_destroy(ctx)
    assert r1 == -1.0
    assert math.isclose(m2, o2["rho"].sum(), rel_tol=1e-13)
    np.testing.assert_allclose(p2, (o2["rho"][None] * o2["u"]).reshape(3, -1).sum(1), rtol=1e-12, atol=1e-16)
    res = np.linalg.norm(o2["u"] - o1["u"]) / np.linalg.norm(o2["u"])
    assert math.isclose(r2, res, rel_tol=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_checkpoint_restart_is_bitwise(precision):
    from paper_2010_01628_gb300 import binding as L
    shape = (33, 12, 8)
    rho, u = inputs.random_fields(shape, seed=61, u_amp=0.02)
    kw = dict(periodic=(True, True, False), g=(1e-5, 0, 0))
    a = L.lbm_create(shape, 1.5, precision=precision, **kw)
    b = L.lbm_create(shape, 1.5, precision=precision, **kw)
    try:
        L.lbm_init_fields(a, rho, u)
        L.lbm_step(a, 10)
        snap = L.lbm_get_populations(a)
        L.lbm_step(a, 10)
        L.lbm_set_populations(b, snap)
        L.lbm_step(b, 10)
        np.testing.assert_array_equal(L.lbm_get_populations(a), L.lbm_get_populations(b))
    finally:
        L.lbm_destroy(a)
        L.lbm_destroy(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cgm_checkpoint_restart_is_bitwise(precision):
    """The colour-gradient state (total populations, red fraction, recolouring
    vector, red rest population) restarts exactly: phi and rho_r are rebuilt
    from it every step, so 2n steps equal n, save, load into a fresh context,
    n; the restored state also reads back the same fields."""
    from paper_2010_01628_gb300 import binding as L
    n = 16
    rho, u, phase, omega, kw = cgm_setup(n)
    shape = (n, n, n)
    kw = dict(kw, periodic=(True, False, True), g=(0.0, -1e-6, 0.0), rho_ref=5.0)
    a = L.lbm_create(shape, omega, physics="cgm", precision=precision, **kw)
    b = L.lbm_create(shape, omega, physics="cgm", precision=precision, **kw)
    try:
        L.lbm_init_fields(a, rho, u, phase)
        L.lbm_step(a, 10)
        snap = L.lbm_get_populations(a)
        L.lbm_set_populations(b, snap)
        fa = L.lbm_fields(a, shape, want=("rho", "u", "phase"))
        fb = L.lbm_fields(b, shape, want=("rho", "u", "phase"))
        for k in ("rho", "u", "phase"):
            np.testing.assert_array_equal(fa[k], fb[k])
        L.lbm_step(a, 10)
        L.lbm_step(b, 10)
        np.testing.assert_array_equal(L.lbm_get_populations(a), L.lbm_get_populations(b))
    finally:
        L.lbm_destroy(a)
        L.lbm_destroy(b)


def test_divergence_is_reported_not_trapped():
    """A NaN planted in the input fields comes back as LBM_ERR_DIVERGED from
    the reduction, and the context stays usable."""
    from paper_2010_01628_gb300 import binding as L
    shape = (16, 8, 4)
    rho, u = inputs.random_fields(shape, seed=71)
    rho[2, 3, 4] = float("nan")
    ctx = L.lbm_create(shape, 1.2, precision="fp32")
    try:
        L.lbm_init_fields(ctx, rho, u)
        L.lbm_step(ctx, 3)
        with pytest.raises(L.LBMError) as ei:
            L.lbm_reduce(ctx)
        assert ei.value.status == L.LBM_ERR_DIVERGED
        rho2, u2 = inputs.random_fields(shape, seed=72)
        L.lbm_init_fields(ctx, rho2, u2)
        L.lbm_step(ctx, 3)
        L.lbm_reduce(ctx)
    finally:
        L.lbm_destroy(ctx)


def test_run_to_steady_poiseuille():
    from paper_2010_01628_gb300 import binding as L
    ny = 16
    nu = (1 / 3) * (0.8 - 0.5)
    gx = 8 * nu * 1e-3 / ny ** 2
    ctx = L.lbm_create((4, ny, 4), 1 / 0.8, periodic=(True, False, True), g=(gx, 0, 0), precision="fp64")
    try:
        steps, res = L.lbm_run_to_steady(ctx, 200000, check_every=100, tol=1e-8)
        out = L.lbm_fields(ctx, (4, ny, 4))
    finally:
        L.lbm_destroy(ctx)
    assert 0 <= res <= 1e-8 and steps < 200000
    y = np.arange(ny) + 0.5
    ua = gx / (2 * nu) * y * (ny - y)
    assert rel_l2(out["u"][0].mean(axis=(0, 2)), ua) < 5e-3


def test_device_pointer_fields_roundtrip():
    """lbm_init_fields / lbm_fields accept device (torch CUDA) buffers too."""
    import torch
    from paper_2010_01628_gb300 import binding as L
    shape = (20, 6, 5)
    rho, u = inputs.random_fields(shape, seed=81)
    ctx = L.lbm_create(shape, 1.1, precision="fp64")
    try:
        L.lbm_init_fields(ctx, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        r_d = torch.empty(rho.shape, dtype=torch.float64, device="cuda")
        u_d = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        L.lbm_fields(ctx, shape, rho=r_d, u=u_d)
        host = L.lbm_fields(ctx, shape)
    finally:
        L.lbm_destroy(ctx)
    np.testing.assert_array_equal(r_d.cpu().numpy(), host["rho"])
    np.testing.assert_array_equal(u_d.cpu().numpy(), host["u"])


def test_cgm_sphere_laplace_law_fp32():
    """App. E surface tension sigma = (4/9) A/omega: spheres of radius 12, 16, 20
    in a 96^3 box (density ratio 1) carry dp = 2 sigma / R within 4 %."""
    from paper_2010_01628_gb300 import binding as L
    n, sigma, tau = 96, 5e-3, 1.0
    ab = 1.0 / 3.0
    for R in (12.0, 16.0, 20.0):
        z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
        d = np.sqrt((x - (n - 1) / 2) ** 2 + (y - (n - 1) / 2) ** 2 + (z - (n - 1) / 2) ** 2)
        ph = np.tanh((R - d) / 2.0)
        ctx = L.lbm_create((n, n, n), 1 / tau, physics="cgm", precision="fp32", alpha_r=ab, alpha_b=ab,
                           A=9 * sigma / tau / 4, beta=0.7)
        try:
            L.lbm_init_fields(ctx, np.ones_like(ph), np.zeros((3, n, n, n)), phase=ph)
            L.lbm_step(ctx, 4000)
            rho = L.lbm_fields(ctx, (n, n, n))["rho"]
        finally:
            L.lbm_destroy(ctx)
        dp = (rho[n // 2, n // 2, n // 2] - rho[0, 0, 0]) * (1 - ab) / 2
        assert abs(dp * R / (2 * sigma) - 1) < 0.04, (R, dp * R / (2 * sigma))
