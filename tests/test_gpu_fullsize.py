"""Parity at the full workload sizes, in the launch configurations the
benchmark times: the 64-domain Hartmann batch and the 64-domain droplet
(density-ratio) batch (one persistent graph-captured launch per call,
autotuned shape), the 256^3 colour-gradient droplets and the warm-start
network at 128^3.
Outputs are checked on sampled domains or nodes the oracle can compute alone.
"""
import numpy as np
import pytest

from helpers import oracle_run, rel_l2
from paper_2010_01628_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_mhd_batch_64_domains_sampled():
    from paper_2010_01628_gb300 import binding as L
    sweep = inputs.hartmann_batch(64, seed=2)
    nu = 0.1
    omega = 1 / (nu / (1 / 3) + 0.5)
    tau_m = 0.5 + nu / 0.25
    shapes = [(n, n, n) for n, _ in sweep]
    b0s = [2 * ha * nu / n for n, ha in sweep]
    gs = [(8 * nu * 0.01 / n ** 2, 0.0, 0.0) for n, _ in sweep]
    batch = L.lbm_batch_create(shapes, omega, periodic=(True, False, True), physics="mhd", precision="fp32",
                               tau_m=tau_m, g=gs, b_wall=[(0.0, b, 0.0) for b in b0s])
    steps = 5
    # smallest domain of each size is compared in full
    pick = {}
    for k, (n, _) in enumerate(sweep):
        pick.setdefault(n, k)
    init = {}
    try:
        for k, (n, _) in enumerate(sweep):
            rho, u = inputs.random_fields((n, n, n), seed=100 + k, u_amp=0.01)
            B = np.zeros((3, n, n, n))
            B[1] = b0s[k]
            if k in pick.values():
                init[k] = (rho, u, B)
            L.lbm_init_fields(L.lbm_batch_domain(batch, k), rho, u, B=B)
        L.lbm_autotune(batch, None)
        L.lbm_batch_step(batch, 2)
        L.lbm_batch_step(batch, 3)
        L.lbm_sync(batch)
        outs = {k: L.lbm_fields(L.lbm_batch_domain(batch, k), shapes[k], want=("rho", "u", "B")) for k in init}
    finally:
        L.lbm_destroy(batch)
    for k, (rho, u, B) in init.items():
        o = oracle_run(shapes[k], omega, steps, rho, u, B=B, physics="mhd", periodic=(True, False, True), g=gs[k],
                       b_wall=(0.0, b0s[k], 0.0), tau_m=tau_m, threads=None)
        for f in ("rho", "u", "B"):
            assert rel_l2(outs[k][f], o[f]) <= 1e-5, (shapes[k], f)


def test_cgm_batch_64_domains_sampled():
    """The density-ratio sweep of the benchmark (64 droplet boxes, sizes
    {32,48,64,96}^3, ratio U[2, 10]), FP32, autotuned, 5 steps; the first
    domain of each size compared in full with the oracle.  Velocity noise of
    1e-2 is added so that u is not the (tiny) spurious current alone."""
    from paper_2010_01628_gb300 import binding as L
    sweep = inputs.droplet_sweep(64, seed=5)
    tau, sigma, alpha_b = 0.8, 1e-4, 1.0 / 3.0
    om = 1.0 / tau
    alpha_r = [1.0 - (1.0 - alpha_b) / r for _, r in sweep]
    A = 9.0 * sigma * om / 4.0
    shapes = [(n, n, n) for n, _ in sweep]
    batch = L.lbm_batch_create(shapes, om, physics="cgm", precision="fp32", alpha_b=alpha_b, alpha_r=alpha_r, A=A,
                               beta=0.7)
    pick = {}
    for k, (n, _) in enumerate(sweep):
        pick.setdefault(n, k)
    init = {}
    try:
        for k, (n, ratio) in enumerate(sweep):
            rho, u, ph = inputs.sweep_droplets(n, ratio, k)
            u = u + inputs.noise_box((n, n, n), amp=1e-2, seed=200 + k)[1]
            if k in pick.values():
                init[k] = (rho, u, ph)
            L.lbm_init_fields(L.lbm_batch_domain(batch, k), rho, u, phase=ph)
        L.lbm_autotune(batch, None)
        L.lbm_batch_step(batch, 2)
        L.lbm_batch_step(batch, 3)
        L.lbm_sync(batch)
        outs = {k: L.lbm_fields(L.lbm_batch_domain(batch, k), shapes[k], want=("rho", "u", "phase")) for k in init}
    finally:
        L.lbm_destroy(batch)
    for k, (rho, u, ph) in init.items():
        o = oracle_run(shapes[k], om, 5, rho, u, phase=ph, physics="cgm", alpha_r=alpha_r[k], alpha_b=alpha_b, A=A,
                       beta=0.7)
        for f in ("rho", "u", "phase"):
            assert rel_l2(outs[k][f], o[f]) <= 1e-5, (shapes[k], f)


def test_cgm_droplets_256_sampled():
    """256^3 droplets, FP32, 3 steps: nodes sampled inside, outside and on the
    interfaces against the oracle run on their dependency cone (radius 2 per
    step, +1 for the reported fields' gather)."""
    from paper_2010_01628_gb300 import binding as L
    n, k = 256, 3
    rho, u, phase, spheres, _ = inputs.droplets(n, seed=3)
    u = u + inputs.noise_box((n, n, n), amp=1e-2, seed=7)[1]
    sigma, tau = 1e-4, 0.8
    alpha_b = 1 / 3
    alpha_r = 1 - (1 - alpha_b) / 10.0
    kw = dict(alpha_r=alpha_r, alpha_b=alpha_b, A=9 * sigma / tau / 4, beta=0.7)
    ctx = L.lbm_create((n, n, n), 1 / tau, physics="cgm", precision="fp32", **kw)
    try:
        L.lbm_init_fields(ctx, rho, u, phase=phase)
        L.lbm_step(ctx, k)
        out = L.lbm_fields(ctx, (n, n, n), want=("rho", "u", "phase"))
    finally:
        L.lbm_destroy(ctx)
    r = 2 * k + 1
    rng = np.random.default_rng(11)
    centres = [(0, 0, 0), (n - 1, 5, n - 1)]
    for (c, rad) in spheres[:4]:  # centre of a droplet and a point on its interface
        ci = [int(round(v)) % n for v in c]
        centres.append(tuple(ci))
        centres.append(((ci[0] + int(round(rad))) % n, ci[1], ci[2]))
    centres += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(4)]
    got, ref = {"rho": [], "u": [], "phase": []}, {"rho": [], "u": [], "phase": []}
    for (x, y, z) in centres:
        idx = [(np.arange(-r, r + 1) + c) % n for c in (x, y, z)]
        sub = lambda a: np.ascontiguousarray(a[np.ix_(idx[2], idx[1], idx[0])])
        su = np.ascontiguousarray(u[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])
        L_ = 2 * r + 1
        o = oracle_run((L_, L_, L_), 1 / tau, k, sub(rho), su, phase=sub(phase), physics="cgm", **kw)
        got["rho"].append(out["rho"][z, y, x])
        ref["rho"].append(o["rho"][r, r, r])
        got["u"].append(out["u"][:, z, y, x])
        ref["u"].append(o["u"][:, r, r, r])
        got["phase"].append(out["phase"][z, y, x])
        ref["phase"].append(o["phase"][r, r, r])
    for f in ("rho", "u", "phase"):
        assert rel_l2(got[f], ref[f]) <= 1e-5, f


def test_cnn_forward_128_sampled():
    """The warm-start network at the study's 128^3 grid with the committed
    weights, as lbm_cnn_warm_start and the benchmark run it: outputs at
    sampled nodes (corners, edges, faces, interior) against the FP64 numpy
    network run on each node's receptive field, the 9^3 nodes around it
    clipped to the grid. The clipped faces then carry the grid's own zero
    padding, and the patch's other faces lie too far out to reach the centre
    through four 3x3x3 layers. Bound: the BF16 forward bound, 3e-2."""
    import os

    from oracle import cnn_oracle as C
    from paper_2010_01628_gb300 import binding as L
    from paper_2010_01628_gb300 import surrogate as S
    n, re = 128, 600.0
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    w, _ = S.load_weights(os.path.join(root, "paper_2010_01628_gb300", "weights", "cavity128_warmstart.npz"))
    net = L.lbm_cnn_create((n, n, n), w)
    try:
        L.lbm_cnn_set_input(net, re)
        got = L.lbm_cnn_forward(net, n ** 3).reshape(n, n, n, 4)  # [z][y][x][4]
    finally:
        L.lbm_cnn_destroy(net)
    X = C.features((n, n, n), re)  # [z][y][x][16]
    rng = np.random.default_rng(12)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 0, 64), (64, n - 1, 64), (3, 64, n - 2)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(6)]
    g, r = [], []
    for (x, y, z) in pts:
        lo = [max(c - 4, 0) for c in (z, y, x)]
        hi = [min(c + 5, n) for c in (z, y, x)]
        out = C.forward(w.astype(np.float64), X[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])[-1]
        r.append(out[z - lo[0], y - lo[1], x - lo[2]])
        g.append(got[z, y, x])
    assert rel_l2(np.array(g), np.array(r)) < 3e-2
