"""FP64 numpy oracle of the warm-start network (test infrastructure only).

Architecture: 4 layers of 3x3x3 zero-padded convolutions, channels
16 -> 32 -> 32 -> 32 -> 4, ReLU after the first three.  Volume layout
[nz, ny, nx, channels] (node p = x + nx (y + ny z)); weights per layer
[C_out, C_in, 27] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), then biases [C_out];
all layers' parameters back to back.

Loss: mean over nodes and the 4 outputs of (y - t)^2 with the targets
t = [(rho - 1) * 30, u * 10] (the library's output scaling).

Parity is pinned by tests/test_cnn_oracle.py: a brute-force scalar
convolution at sampled voxels, the tap convention of a single-tap kernel, and a
finite-difference check of the analytic gradient.
"""
import numpy as np

CH = [16, 32, 32, 32, 4]
NL = len(CH) - 1
RHO_SCALE, U_SCALE = 30.0, 10.0


def taps():
    for tap in range(27):
        yield tap, tap % 3 - 1, (tap // 3) % 3 - 1, tap // 9 - 1


def layer_sizes():
    return [27 * CH[l + 1] * CH[l] + CH[l + 1] for l in range(NL)]


def param_count():
    return sum(layer_sizes())


def split(params):
    out, o = [], 0
    for l in range(NL):
        nw = 27 * CH[l + 1] * CH[l]
        W = params[o:o + nw].reshape(CH[l + 1], CH[l], 27)
        b = params[o + nw:o + nw + CH[l + 1]]
        out.append((W, b))
        o += nw + CH[l + 1]
    return out


def shifted(Xp, dx, dy, dz, shape):
    """View of the zero-padded volume at node + (dx, dy, dz)."""
    nz, ny, nx = shape
    return Xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]


def conv(X, W, b):
    """Y[z,y,x,o] = b[o] + sum_tap sum_c X[z+dz, y+dy, x+dx, c] W[o, c, tap]."""
    shape = X.shape[:3]
    Xp = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
    Y = np.broadcast_to(b, shape + (W.shape[0],)).astype(np.float64).copy()
    for tap, dx, dy, dz in taps():
        Y += shifted(Xp, dx, dy, dz, shape) @ W[:, :, tap].T
    return Y


def forward(params, X0):
    acts = [X0]
    x = X0
    for l, (W, b) in enumerate(split(params)):
        y = conv(x, W, b)
        if l < NL - 1:
            y = np.maximum(y, 0.0)
        acts.append(y)
        x = y
    return acts


def targets(rho, u):
    """rho [nz,ny,nx], u [3,nz,ny,nx] -> [nz,ny,nx,4] scaled targets."""
    return np.stack([(rho - 1.0) * RHO_SCALE, u[0] * U_SCALE, u[1] * U_SCALE, u[2] * U_SCALE], axis=-1)


def loss_and_grad(params, X0, rho, u):
    acts = forward(params, X0)
    T = targets(rho, u)
    Y = acts[-1]
    n = Y.size
    loss = float(((Y - T) ** 2).sum() / n)
    dY = 2.0 * (Y - T) / n
    grads = []
    layers = split(params)
    for l in range(NL - 1, -1, -1):
        W, b = layers[l]
        X = acts[l]
        shape = X.shape[:3]
        Xp = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
        dW = np.zeros_like(W)
        for tap, dx, dy, dz in taps():
            dW[:, :, tap] = np.einsum("zyxo,zyxc->oc", dY, shifted(Xp, dx, dy, dz, shape))
        db = dY.sum(axis=(0, 1, 2))
        grads.append(np.concatenate([dW.ravel(), db]))
        if l > 0:
            # dX[p] = sum_tap dY[p - off] W[:, :, tap]
            dYp = np.pad(dY, ((1, 1), (1, 1), (1, 1), (0, 0)))
            dX = np.zeros_like(X)
            for tap, dx, dy, dz in taps():
                dX += shifted(dYp, -dx, -dy, -dz, shape) @ W[:, :, tap]
            dY = dX * (acts[l] > 0)
    grads.reverse()
    return loss, np.concatenate(grads)


def features(shape, reynolds):
    """Input channels of the library, shape = (nx, ny, nz): r = (Re - 550)/450;
    node-centre coordinates x, y, z in [-1, 1]; lid flag on the top (+y)
    layer; cos(pi x/2), cos(pi y/2), cos(pi z/2); sin(pi x), sin(pi y),
    sin(pi z); cos(pi x), cos(pi y), cos(pi z); r^2; r (y + 1)/2."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xn = 2.0 * (x + 0.5) / nx - 1.0
    yn = 2.0 * (y + 0.5) / ny - 1.0
    zn = 2.0 * (z + 0.5) / nz - 1.0
    r = (reynolds - 550.0) / 450.0
    f = np.zeros((nz, ny, nx, 16))
    f[..., 0] = r
    f[..., 1], f[..., 2], f[..., 3] = xn, yn, zn
    f[..., 4] = (y == ny - 1).astype(np.float64)
    for k, v in enumerate((xn, yn, zn)):
        f[..., 5 + k] = np.cos(0.5 * np.pi * v)
        f[..., 8 + k] = np.sin(np.pi * v)
        f[..., 11 + k] = np.cos(np.pi * v)
    f[..., 14] = r * r
    f[..., 15] = r * 0.5 * (yn + 1.0)
    return f
