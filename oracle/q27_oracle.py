"""FP64 numpy oracle for the D3Q27 central-moment LBM of App. D (arXiv:2010.01628).

Test infrastructure only: the test-suite and the benchmark's CPU-baseline leg
call it; nothing in the CUDA library uses it.

Two collisions, agreeing to rounding:
  * dense (the definition): T(u) from the 27 central-moment rows printed in
    App. D, k = T f, k* = (I - K) k + K k_eq + (I - K/2) R, then T f* = k*;
  * factorised: the basis of App. D is spanned by the monomials
    cbar_x^a cbar_y^b cbar_z^c (a, b, c <= 2), and the D3Q27 lattice is the
    tensor product of three D1Q3 lattices, so central moments, their
    binomial shift to raw moments and M^-1 all act one axis at a time
    (1D transforms on three values).  This is the algorithm of the GPU kernel.

What App. D does not print is read from the rules that define the D3Q19 list
(Sec. II.B) and App. B:
  * equilibrium: only the zeroth central Hermite moment is nonzero, so the
    central moments are rho * prod(1, 0, c_s^2) per axis (the tensor-product
    D1Q3 equilibrium; velocity independent);
  * forcing: App. B states that only the first-order central Hermite moments of
    the force term are nonzero (F); expanded, the central moments are
    F_x a m_(a-1) m_b m_c + (y, z alike) with m = (1, 0, c_s^2): F at first,
    c_s^2 F at third (R_210 = c_s^2 F_y, ...) and c_s^4 F at fifth order
    (R_221 = c_s^4 F_z, ...);
  * relaxation: omega on the five deviatoric second-order rows (xy, xz, yz,
    x^2 - y^2, x^2 - z^2), 1 on every other row (bulk and higher orders
    equilibrated, as in Sec. II.B).
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0
Q27 = 27

# App. D lattice, in the printed order (opposite(i) = i +/- 13).
CX = np.array([0, -1, 0, 0, -1, -1, -1, -1, 0, 0, -1, -1, -1, -1, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 1, 1])
CY = np.array([0, 0, -1, 0, -1, 1, 0, 0, -1, -1, -1, -1, 1, 1, 0, 1, 0, 1, -1, 0, 0, 1, 1, 1, 1, -1, -1])
CZ = np.array([0, 0, 0, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1])
OPP = np.array([0] + [i + 13 for i in range(1, 14)] + [i - 13 for i in range(14, 27)])
_W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
W = np.array([_W1[a] * _W1[b] * _W1[c] for a, b, c in zip(CX, CY, CZ)])

# The 27 rows of App. D (T with cbar = c - u; M with c).
BASIS = [
    lambda x, y, z: np.ones_like(x),
    lambda x, y, z: x, lambda x, y, z: y, lambda x, y, z: z,
    lambda x, y, z: x * y, lambda x, y, z: x * z, lambda x, y, z: y * z,
    lambda x, y, z: x * x - y * y, lambda x, y, z: x * x - z * z, lambda x, y, z: x * x + y * y + z * z,
    lambda x, y, z: x * y * y + x * z * z, lambda x, y, z: x * x * y + y * z * z, lambda x, y, z: x * x * z + y * y * z,
    lambda x, y, z: x * y * y - x * z * z, lambda x, y, z: x * x * y - y * z * z, lambda x, y, z: x * x * z - y * y * z,
    lambda x, y, z: x * y * z,
    lambda x, y, z: x * x * y * y + x * x * z * z + y * y * z * z,
    lambda x, y, z: x * x * y * y + x * x * z * z - y * y * z * z,
    lambda x, y, z: x * x * y * y - x * x * z * z,
    lambda x, y, z: x * x * y * z, lambda x, y, z: x * y * y * z, lambda x, y, z: x * y * z * z,
    lambda x, y, z: x * y * y * z * z, lambda x, y, z: x * x * y * z * z, lambda x, y, z: x * x * y * y * z,
    lambda x, y, z: x * x * y * y * z * z,
]
RELAXED = (4, 5, 6, 7, 8)  # rows relaxed with omega; all others with 1


def T(u):
    """Central-moment matrix T(u), 27 x 27 (rows: App. D basis; columns: lattice)."""
    x, y, z = CX - u[0], CY - u[1], CZ - u[2]
    return np.array([b(x.astype(float), y.astype(float), z.astype(float)) for b in BASIS])


M = T((0.0, 0.0, 0.0))


def _monomial_rows():
    """Matrix P with basis = P @ monomials, monomials ordered (a, b, c) in 0..2, c fastest."""
    mono = [(a, b, c) for a in range(3) for b in range(3) for c in range(3)]
    # evaluate both on 27 generic points and solve: exact for these polynomial spans
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.3, 1.3, size=(3, 64))
    A = np.array([[p[0] ** a * p[1] ** b * p[2] ** c for (a, b, c) in mono] for p in pts.T])
    B = np.array([[bf(*p) for bf in BASIS] for p in pts.T])
    P = np.linalg.lstsq(A, B, rcond=None)[0].T
    return np.round(P, 12), mono


P_MONO, MONO = _monomial_rows()


def _m(a):
    return (1.0, 0.0, CS2)[a]


def central_eq(rho):
    """k_eq in the App. D basis: rho prod m_a with m = (1, 0, c_s^2)."""
    mu = np.array([_m(a) * _m(b) * _m(c) for (a, b, c) in MONO])
    return np.multiply.outer(np.asarray(rho, dtype=float), P_MONO @ mu)


def central_force(F):
    """Central moments of the force term in the App. D basis (F: [..., 3])."""
    F = np.asarray(F, dtype=float)
    cols = []
    for (a, b, c) in MONO:
        v = 0.0
        if a >= 1:
            v = v + F[..., 0] * a * _m(a - 1) * _m(b) * _m(c)
        if b >= 1:
            v = v + F[..., 1] * b * _m(a) * _m(b - 1) * _m(c)
        if c >= 1:
            v = v + F[..., 2] * c * _m(a) * _m(b) * _m(c - 1)
        cols.append(np.broadcast_to(v, F.shape[:-1]))
    mono = np.stack(cols, axis=-1)
    return mono @ P_MONO.T


def feq(rho, u):
    """Tensor-product D1Q3 equilibrium (central moments rho prod m)."""
    rho = np.asarray(rho, dtype=float)
    u = np.asarray(u, dtype=float)

    def phi(c, ua):
        if c == 0:
            return 1.0 - CS2 - ua * ua
        return 0.5 * (CS2 + ua * ua + c * ua)

    out = [rho * phi(cx, u[..., 0]) * phi(cy, u[..., 1]) * phi(cz, u[..., 2]) for cx, cy, cz in zip(CX, CY, CZ)]
    return np.stack(out, axis=-1)


def collide_dense(f, rho, u, F, omega):
    """The definition, batched over leading axes: f [..., 27]."""
    f = np.asarray(f, dtype=float)
    u = np.asarray(u, dtype=float)
    shp = f.shape[:-1]
    fb = f.reshape(-1, Q27)
    ub = np.broadcast_to(u, shp + (3,)).reshape(-1, 3)
    rb = np.broadcast_to(rho, shp).reshape(-1)
    Fb = np.broadcast_to(np.asarray(F, dtype=float), shp + (3,)).reshape(-1, 3)
    out = np.empty_like(fb)
    K = np.ones(Q27)
    K[list(RELAXED)] = omega
    for n in range(fb.shape[0]):
        Tn = T(ub[n])
        k = Tn @ fb[n]
        ks = (1 - K) * k + K * central_eq(rb[n]) + (1 - K / 2) * central_force(Fb[n])
        out[n] = np.linalg.solve(Tn, ks)
    return out.reshape(f.shape)


# --- factorised collision --------------------------------------------------
_IDX = np.array([(cx + 1) * 9 + (cy + 1) * 3 + (cz + 1) for cx, cy, cz in zip(CX, CY, CZ)])


def _to_cube(f):
    g = np.empty(f.shape[:-1] + (27,))
    g[..., _IDX] = f
    return g.reshape(f.shape[:-1] + (3, 3, 3))


def _from_cube(g):
    return g.reshape(g.shape[:-3] + (27,))[..., _IDX]


def _central_1d(g, u, axis):
    """Along one axis of a [..., 3, 3, 3] array: populations at c = -1, 0, 1 to
    central moments of order 0, 1, 2 about u (u broadcast over the cube)."""
    g = np.moveaxis(g, axis, -1)
    uu = u[..., None, None, None]
    cs = np.array([-1.0, 0.0, 1.0])
    out = np.stack([(g * (cs - uu) ** a).sum(axis=-1) for a in range(3)], axis=-1)
    return np.moveaxis(out, -1, axis)


def _populations_1d(k, u, axis):
    """Inverse of _central_1d: binomial shift to raw moments, then D1Q3."""
    k = np.moveaxis(k, axis, -1)
    uu = u[..., None, None]
    r0 = k[..., 0]
    r1 = k[..., 1] + uu * k[..., 0]
    r2 = k[..., 2] + 2 * uu * k[..., 1] + uu * uu * k[..., 0]
    out = np.stack([(r2 - r1) / 2, r0 - r2, (r2 + r1) / 2], axis=-1)
    return np.moveaxis(out, -1, axis)


def collide_factorised(f, rho, u, F, omega):
    f = np.asarray(f, dtype=float)
    u = np.asarray(u, dtype=float)
    ux, uy, uz = u[..., 0], u[..., 1], u[..., 2]
    g = _to_cube(f)
    axes = (g.ndim - 3, g.ndim - 2, g.ndim - 1)
    k = _central_1d(g, ux, axes[0])
    k = _central_1d(k, uy, axes[1])
    k = _central_1d(k, uz, axes[2])
    rho = np.asarray(rho, dtype=float)
    F = np.broadcast_to(np.asarray(F, dtype=float), u.shape)
    ks = np.empty_like(k)
    for (a, b, c) in MONO:
        v = rho * _m(a) * _m(b) * _m(c)
        half = 0.0
        if a >= 1:
            half = half + F[..., 0] * a * _m(a - 1) * _m(b) * _m(c)
        if b >= 1:
            half = half + F[..., 1] * b * _m(a) * _m(b - 1) * _m(c)
        if c >= 1:
            half = half + F[..., 2] * c * _m(a) * _m(b) * _m(c - 1)
        ks[..., a, b, c] = v + 0.5 * half
    # second order: trace at equilibrium, deviatoric parts relaxed with omega
    xx, yy, zz = k[..., 2, 0, 0], k[..., 0, 2, 0], k[..., 0, 0, 2]
    d1 = (1 - omega) * (xx - yy)
    d2 = (1 - omega) * (xx - zz)
    tr = 3 * rho * CS2
    ks[..., 2, 0, 0] = (tr + d1 + d2) / 3
    ks[..., 0, 2, 0] = (tr - 2 * d1 + d2) / 3
    ks[..., 0, 0, 2] = (tr + d1 - 2 * d2) / 3
    ks[..., 1, 1, 0] = (1 - omega) * k[..., 1, 1, 0]
    ks[..., 1, 0, 1] = (1 - omega) * k[..., 1, 0, 1]
    ks[..., 0, 1, 1] = (1 - omega) * k[..., 0, 1, 1]
    out = _populations_1d(ks, uz, axes[2])
    out = _populations_1d(out, uy, axes[1])
    out = _populations_1d(out, ux, axes[0])
    return _from_cube(out)


# --- a periodic / bounce-back box ------------------------------------------
class Domain27:
    """nx*ny*nz nodes, populations [27, nz, ny, nx]; a non-periodic axis has
    half-way bounce-back walls, the +y wall moving with lid_u (Ladd's term
    6 w_i c_i . u_lid).  Body force F = rho g; u = (Sum f c + F/2)/rho."""

    def __init__(self, shape, omega, *, periodic=(True, True, True), lid_u=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0),
                 collision="factorised"):
        self.shape = tuple(shape)
        self.omega = float(omega)
        self.periodic = tuple(bool(p) for p in periodic)
        self.lid = np.array(lid_u, dtype=float)
        self.g = np.array(g, dtype=float)
        self.collide = {"factorised": collide_factorised, "dense": collide_dense, "rm": collide_factorised_rm,
                        "dense_rm": collide_dense_rm}[collision]
        nx, ny, nz = self.shape
        self.f = np.zeros((Q27, nz, ny, nx))

    def init(self, rho, u):
        ug = np.moveaxis(np.asarray(u, dtype=float), 0, -1)
        self.f = np.moveaxis(feq(np.asarray(rho, dtype=float), ug), -1, 0).copy()

    def _pull(self):
        nx, ny, nz = self.shape
        out = np.empty_like(self.f)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        for i in range(Q27):
            sx, sy, sz = x - CX[i], y - CY[i], z - CZ[i]
            wall = np.zeros(x.shape, dtype=bool)
            for s, n, p in ((sx, nx, self.periodic[0]), (sy, ny, self.periodic[1]), (sz, nz, self.periodic[2])):
                if p:
                    s %= n
                else:
                    wall |= (s < 0) | (s >= n)
            sxc, syc, szc = np.clip(sx, 0, nx - 1), np.clip(sy, 0, ny - 1), np.clip(sz, 0, nz - 1)
            v = self.f[i][szc, syc, sxc]
            bb = self.f[OPP[i]].copy()
            if not self.periodic[1]:
                lid_hit = (y - CY[i]) >= ny
                bb = bb + lid_hit * 6.0 * W[i] * (CX[i] * self.lid[0] + CY[i] * self.lid[1] + CZ[i] * self.lid[2])
            out[i] = np.where(wall, bb, v)
        return out

    def _macro(self, fin):
        rho = fin.sum(axis=0)
        j = np.stack([np.tensordot(c, fin, axes=(0, 0)) for c in (CX, CY, CZ)])
        F = rho[None] * self.g[:, None, None, None]
        u = (j + 0.5 * F) / rho[None]
        return rho, u, F

    def step(self, n=1):
        for _ in range(n):
            fin = self._pull()
            rho, u, F = self._macro(fin)
            fl = np.moveaxis(fin, 0, -1)
            post = self.collide(fl, rho, np.moveaxis(u, 0, -1), np.moveaxis(F, 0, -1), self.omega)
            self.f = np.ascontiguousarray(np.moveaxis(post, -1, 0))

    def fields(self):
        fin = self._pull()
        rho, u, _ = self._macro(fin)
        return rho, u


# --- raw-moment variant (N = I) ---------------------------------------------
# The App. D timing table also runs D3Q27 with raw moments: the same basis,
# K and relaxation with T = M, equilibrium raw moments rho prod(1, u, u^2 + c_s^2)
# and the raw moments of the same force term (the central ones shifted by u).
def raw_eq(rho, u):
    rho = np.asarray(rho, dtype=float)
    u = np.asarray(u, dtype=float)
    mono = np.stack([rho * _mr(a, u[..., 0]) * _mr(b, u[..., 1]) * _mr(c, u[..., 2]) for (a, b, c) in MONO], axis=-1)
    return mono @ P_MONO.T


def _mr(a, ua):
    return (np.ones_like(ua), ua, ua * ua + CS2)[a]


def collide_dense_rm(f, rho, u, F, omega):
    f = np.asarray(f, dtype=float)
    shp = f.shape[:-1]
    fb = f.reshape(-1, Q27)
    ub = np.broadcast_to(np.asarray(u, dtype=float), shp + (3,)).reshape(-1, 3)
    rb = np.broadcast_to(rho, shp).reshape(-1)
    Fb = np.broadcast_to(np.asarray(F, dtype=float), shp + (3,)).reshape(-1, 3)
    K = np.ones(Q27)
    K[list(RELAXED)] = omega
    out = np.empty_like(fb)
    for n in range(fb.shape[0]):
        Fi = np.linalg.solve(T(ub[n]), central_force(Fb[n]))  # the force term's populations
        k = M @ fb[n]
        ks = (1 - K) * k + K * raw_eq(rb[n], ub[n]) + (1 - K / 2) * (M @ Fi)
        out[n] = np.linalg.solve(M, ks)
    return out.reshape(f.shape)


def collide_factorised_rm(f, rho, u, F, omega):
    """Raw moments by 1D transforms at zero shift; the force term's raw moments
    by the 1D binomial shift of its central moments."""
    f = np.asarray(f, dtype=float)
    u = np.asarray(u, dtype=float)
    ux, uy, uz = u[..., 0], u[..., 1], u[..., 2]
    zero = np.zeros_like(ux)
    g = _to_cube(f)
    axes = (g.ndim - 3, g.ndim - 2, g.ndim - 1)
    k = _central_1d(_central_1d(_central_1d(g, zero, axes[0]), zero, axes[1]), zero, axes[2])
    rho = np.asarray(rho, dtype=float)
    F = np.broadcast_to(np.asarray(F, dtype=float), u.shape)
    # central force moments -> raw (binomial shift per axis, as in _populations_1d's first half)
    Rc = np.zeros_like(k)
    for (a, b, c) in MONO:
        v = 0.0
        if a >= 1:
            v = v + F[..., 0] * a * _m(a - 1) * _m(b) * _m(c)
        if b >= 1:
            v = v + F[..., 1] * b * _m(a) * _m(b - 1) * _m(c)
        if c >= 1:
            v = v + F[..., 2] * c * _m(a) * _m(b) * _m(c - 1)
        Rc[..., a, b, c] = v

    def shift(x, ua, axis):
        x = np.moveaxis(x, axis, -1)
        uu = ua[..., None, None]
        out = np.stack([x[..., 0], x[..., 1] + uu * x[..., 0], x[..., 2] + 2 * uu * x[..., 1] + uu * uu * x[..., 0]],
                       axis=-1)
        return np.moveaxis(out, -1, axis)

    R = shift(shift(shift(Rc, ux, axes[0]), uy, axes[1]), uz, axes[2])
    ks = np.empty_like(k)
    for (a, b, c) in MONO:
        ks[..., a, b, c] = rho * _mr(a, ux) * _mr(b, uy) * _mr(c, uz) + 0.5 * R[..., a, b, c]
    xx, yy, zz = k[..., 2, 0, 0], k[..., 0, 2, 0], k[..., 0, 0, 2]
    exx, eyy, ezz = (rho * (ux * ux + CS2), rho * (uy * uy + CS2), rho * (uz * uz + CS2))
    Rxx, Ryy, Rzz = R[..., 2, 0, 0], R[..., 0, 2, 0], R[..., 0, 0, 2]
    d1 = (1 - omega) * (xx - yy) + omega * (exx - eyy) + (1 - omega / 2) * (Rxx - Ryy)
    d2 = (1 - omega) * (xx - zz) + omega * (exx - ezz) + (1 - omega / 2) * (Rxx - Rzz)
    tr = exx + eyy + ezz + 0.5 * (Rxx + Ryy + Rzz)
    ks[..., 2, 0, 0] = (tr + d1 + d2) / 3
    ks[..., 0, 2, 0] = (tr - 2 * d1 + d2) / 3
    ks[..., 0, 0, 2] = (tr + d1 - 2 * d2) / 3
    for (a, b, c), (p, q) in (((1, 1, 0), (ux, uy)), ((1, 0, 1), (ux, uz)), ((0, 1, 1), (uy, uz))):
        ks[..., a, b, c] = (1 - omega) * k[..., a, b, c] + omega * rho * p * q + (1 - omega / 2) * R[..., a, b, c]
    out = _populations_1d(ks, zero, axes[2])
    out = _populations_1d(out, zero, axes[1])
    out = _populations_1d(out, zero, axes[0])
    return _from_cube(out)
