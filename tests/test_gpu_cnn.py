"""Warm-start network on the GPU (tcgen05 BF16 tensor-core kernels with TMEM
accumulators; rows staged by bulk copies) against the FP64 numpy oracle, and
the warm start's gain over a cold start.

Shapes cover the staging cases of the kernels: rows that fit one tile (nx <=
128: halo cells zeroed once, cells past a short row left stale), rows of two
tiles (nx = 130: halo cells written per row, a ragged second tile whose
weight-gradient K-steps stop early), staged rows outside the grid at every
y and z face, and more CTAs than tiles (empty weight-gradient CTAs).

Tolerances: activations and kernel weights are BF16 (unit roundoff 2^-9 ~
2e-3); four layers of rounded inputs, weights and activations put the output
within ~1e-2 relative: forward 3e-2 and gradients 5e-2 (relative L2).
"""

import numpy as np
import pytest

from helpers import rel_l2
from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu


def params(seed, scale=0.12):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(C.param_count())).astype(np.float32)


def test_param_layout_matches_oracle():
    from paper_2010_01628_gb300 import binding as L
    assert L.lbm_cnn_param_count() == C.param_count()


@pytest.mark.parametrize("shape", [(13, 9, 11), (16, 16, 16), (130, 5, 4)])
def test_forward_matches_oracle(shape):
    from paper_2010_01628_gb300 import binding as L
    nx, ny, nz = shape
    p = params(1)
    x = np.random.default_rng(2).uniform(-1, 1, (nz, ny, nx, C.CH[0]))
    net = L.lbm_cnn_create(shape, p)
    try:
        L.lbm_cnn_set_input_raw(net, x.reshape(-1, C.CH[0]))
        got = L.lbm_cnn_forward(net, nx * ny * nz)
    finally:
        L.lbm_cnn_destroy(net)
    ref = C.forward(p.astype(np.float64), x)[-1].reshape(-1, 4)
    assert rel_l2(got, ref) < 3e-2


def test_features_and_forward_for_reynolds():
    from paper_2010_01628_gb300 import binding as L
    shape = (12, 10, 8)
    p = params(3)
    net = L.lbm_cnn_create(shape, p)
    try:
        L.lbm_cnn_set_input(net, 730.0)
        got = L.lbm_cnn_forward(net, 12 * 10 * 8)
    finally:
        L.lbm_cnn_destroy(net)
    ref = C.forward(p.astype(np.float64), C.features(shape, 730.0))[-1].reshape(-1, 4)
    assert rel_l2(got, ref) < 3e-2


@pytest.mark.parametrize("shape", [(10, 12, 9), (130, 4, 3)])
def test_gradient_matches_oracle(shape):
    from paper_2010_01628_gb300 import binding as L
    nx, ny, nz = shape
    p = params(4)
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.01 * rng.standard_normal((nz, ny, nx))
    u = 0.05 * rng.standard_normal((3, nz, ny, nx))
    net = L.lbm_cnn_create(shape, p)
    try:
        L.lbm_cnn_set_input(net, 300.0)
        loss, g = L.lbm_cnn_gradient(net, rho, u)
    finally:
        L.lbm_cnn_destroy(net)
    lref, gref = C.loss_and_grad(p.astype(np.float64), C.features(shape, 300.0), rho, u)
    assert abs(loss - lref) <= 2e-2 * lref
    o = 0
    for l, size in enumerate(C.layer_sizes()):
        assert rel_l2(g[o:o + size], gref[o:o + size]) < 5e-2, l
        o += size


def test_adam_step_on_own_gradient():
    """One train step = forward/backward + Adam: the first Adam update is
    lr * g / (|g| + eps) elementwise on the gradient the kernels produce."""
    from paper_2010_01628_gb300 import binding as L
    shape = (8, 8, 8)
    p = params(6)
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.01 * rng.standard_normal((8, 8, 8))
    u = 0.05 * rng.standard_normal((3, 8, 8, 8))
    net = L.lbm_cnn_create(shape, p)
    try:
        L.lbm_cnn_set_input(net, 500.0)
        _, g = L.lbm_cnn_gradient(net, rho, u)
        lr = 1e-3
        L.lbm_cnn_train_step(net, rho, u, lr)
        w = L.lbm_cnn_get_weights(net)
    finally:
        L.lbm_cnn_destroy(net)
    g = g.astype(np.float64)
    m_hat = g
    v_hat = g * g
    expect = p - lr * m_hat / (np.sqrt(v_hat) + 1e-8)
    np.testing.assert_allclose(w, expect, rtol=1e-5, atol=1e-6)


def test_warm_start_reaches_steady_state_sooner():
    """Train on a few solver steady states of a small cavity, then compare the
    steps to a 1e-6 residual from rest and from the network's prediction for
    held-out Reynolds numbers, and let the solver judge the network.

    The residual is the mean per-step change over the check interval, so a run
    stops at a distance of about r / lambda from the fixed point (lambda the
    slowest decay rate per step, ~1e-3 on this cavity): the warm and cold runs
    end on the same steady state only to that distance, ~1e-3 relative in u.
    Bounds: warm vs cold final u within 2e-2 (measured 4e-3) and rho - 1
    within 5e-2 of its norm (measured 1e-2); the prediction closer to the
    converged u than the rest state is (relative error < 0.5; rest = 1)."""
    from paper_2010_01628_gb300 import surrogate as S
    n = 24
    train_re = np.linspace(100, 300, 8)
    data = S.steady_states(n, train_re, tol=1e-6, check_every=100, continuation=True)
    assert all(d["converged"] for d in data)
    net = S.train(n, data, epochs=80, lr=3e-3)
    try:
        rep = S.evaluate(net, n, [170.0, 260.0], tol=1e-6, check_every=100, max_steps=200000)
    finally:
        from paper_2010_01628_gb300 import binding as L
        L.lbm_cnn_destroy(net)
    for r in rep["cases"]:
        assert r["warm_steps"] < r["cold_steps"], r
        assert r["warm_vs_cold_u"] < 2e-2, r
        assert r["warm_vs_cold_rho"] < 5e-2, r
        assert r["net_err_u"] < 0.5, r
