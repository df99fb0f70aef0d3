"""Pins of the warm-start network's FP64 oracle (CPU only)."""
import numpy as np

from oracle import cnn_oracle as C


def small_params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(C.param_count())


def test_conv_matches_brute_force_sums():
    """The sliced convolution equals the scalar triple sum of its definition
    (zero outside the box) at sampled voxels, corners included."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 5, 6, 3))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    Y = C.conv(X, W, b)
    nz, ny, nx = X.shape[:3]
    for (z, y, x) in [(0, 0, 0), (3, 4, 5), (1, 2, 3), (0, 4, 2)]:
        for o in range(2):
            s = b[o]
            for tap in range(27):
                dx, dy, dz = tap % 3 - 1, (tap // 3) % 3 - 1, tap // 9 - 1
                zz, yy, xx = z + dz, y + dy, x + dx
                if 0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx:
                    for c in range(3):
                        s += X[zz, yy, xx, c] * W[o, c, tap]
            assert abs(Y[z, y, x, o] - s) < 1e-12


def test_single_tap_kernel_shifts_the_input():
    """A kernel with one tap (dx, dy, dz) reads the node at +(dx, dy, dz)."""
    X = np.random.default_rng(2).standard_normal((5, 6, 7, 1))
    tap = 2 * 9 + 0 * 3 + 1  # dz = +1, dy = -1, dx = 0
    W = np.zeros((1, 1, 27))
    W[0, 0, tap] = 1.0
    Y = C.conv(X, W, np.zeros(1))
    np.testing.assert_array_equal(Y[:-1, 1:, :, 0], X[1:, :-1, :, 0])
    assert np.all(Y[-1, :, :, 0] == 0) and np.all(Y[:, 0, :, 0] == 0)


def test_gradient_matches_finite_differences():
    shape = (4, 3, 3)  # nx, ny, nz
    p = small_params(3)
    X0 = C.features(shape, 400.0)
    rng = np.random.default_rng(4)
    rho = 1.0 + 0.01 * rng.standard_normal((3, 3, 4))
    u = 0.05 * rng.standard_normal((3, 3, 3, 4))
    loss, g = C.loss_and_grad(p, X0, rho, u)
    idx = rng.choice(p.size, 40, replace=False)
    # include biases of the last layer and the first layer's weights
    idx = np.concatenate([idx, [p.size - 1, 0, 10]])
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp, _ = C.loss_and_grad(q, X0, rho, u)
        q[i] -= 2 * h
        lm, _ = C.loss_and_grad(q, X0, rho, u)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_features_layout():
    f = C.features((4, 3, 2), 1000.0)
    assert f.shape == (2, 3, 4, 16)
    assert np.allclose(f[..., 0], 1.0) and np.allclose(f[..., 14], 1.0)
    assert f[0, 0, 0, 1] == -0.75 and f[0, 0, 3, 1] == 0.75
    assert np.all(f[:, 2, :, 4] == 1) and np.all(f[:, :2, :, 4] == 0)
    # the wall-vanishing and periodic coordinate functions at x = -0.75
    assert abs(f[0, 0, 0, 5] - np.cos(-0.375 * np.pi)) < 1e-15
    assert abs(f[0, 0, 0, 8] - np.sin(-0.75 * np.pi)) < 1e-15
    assert abs(f[0, 0, 0, 11] - np.cos(-0.75 * np.pi)) < 1e-15
    # r (y + 1)/2: r at the top node centre y = 2/3
    assert abs(f[0, 2, 0, 15] - 1.0 * (2.0 / 3.0 + 1.0) / 2.0) < 1e-15


def test_receptive_field_is_nine_nodes():
    """Four zero-padded 3x3x3 layers: an output depends on exactly the 9^3
    inputs around it. The network run on that neighbourhood (clipped to the
    grid) reproduces the full-grid output; on the 7^3 neighbourhood it does
    not."""
    n = 14
    p = small_params(7)
    X = C.features((n, n, n), 600.0)
    full = C.forward(p, X)[-1]
    for (x, y, z) in [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (7, 7, 7), (3, 6, n - 2)]:
        for r, same in ((4, True), (3, False)):
            lo = [max(c - r, 0) for c in (z, y, x)]
            hi = [min(c + r + 1, n) for c in (z, y, x)]
            out = C.forward(p, X[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])[-1][z - lo[0], y - lo[1], x - lo[2]]
            if same:
                np.testing.assert_array_equal(out, full[z, y, x])
            else:
                assert np.abs(out - full[z, y, x]).max() > 1e-8
