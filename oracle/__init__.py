"""FP64 CPU oracle for the D3Q19 central-moment LBM (arXiv:2010.01628).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The arithmetic lives in
``cmlbm_oracle.c`` (plain C, binary64, built with ``-ffp-contract=off``); this
module compiles it with gcc on first use and marshals numpy arrays.  It shares
no code with the CUDA library.

Every parity claim rests on pins that tie this oracle to the paper and to
mathematics (``tests/test_oracle_pins.py``).  Functions whose only pin is
physical behaviour rather than a closed form say so in their docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
FLUID, MHD, CGM, SC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            P = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            lib.orc_feq.argtypes = [D, D, D, D, P]
            lib.orc_heq.argtypes = [D, D, D, D, D, P]
            lib.orc_T.argtypes = [D, D, D, P]
            lib.orc_solve19.argtypes = [P, P, P]
            lib.orc_forcing_rm.argtypes = [D, D, D, D, D, D, P]
            lib.orc_forcing_pop.argtypes = [D, D, D, D, D, D, P]
            lib.orc_collide_dense.argtypes = [P, D, D, D, D, D, D, D, D, D, D, D, I, D, P]
            lib.orc_collide_closed.argtypes = [P, D, D, D, D, D, D, D, D, I, D, P]
            lib.orc_kstar_fluid.argtypes = [P, D, D, D, D, D, D, D, D, P]
            lib.orc_kstar_cgm.argtypes = [P, D, D, D, D, D, D, D, D, D, P]
            lib.orc_back_transform.argtypes = [D, D, D, D, P, P]
            lib.orc_geq.argtypes = [D, D, D, D, D, D, P]
            lib.orc_current.argtypes = [P, D, D, D, D, P, P]
            lib.orc_cgm_perturb.argtypes = [P, D, P]
            lib.orc_cgm_recolour.argtypes = [P, P, D, D, D, D, P, P]
            lib.orc_lattice.argtypes = [ctypes.POINTER(I)] * 3 + [P]
            lib.orc_set_threads.argtypes = [I]
            lib.orc_max_threads.restype = I
            PP = ctypes.c_void_p
            lib.orc_init.argtypes = [PP, P, P, P, P, P, P, P, P]
            lib.orc_step.argtypes = [PP, P, P, P, P, P, P, P, P, P, ctypes.c_long]
            lib.orc_fields.argtypes = [PP, P, P, P, P, P, P, P, P]
            lib.orc_sc_force_field.argtypes = [PP, P, P]
            lib.orc_regularize.argtypes = [P, I, P, P, D]
            lib.orc_collide_rm.argtypes = [P, D, D, D, D, D, D, D, D, P]
            lib.orc_collide_rm.restype = None
            lib.orc_collide_dense_rm.argtypes = [P, D, D, D, D, D, D, D, D, P]
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(n=Q):
    return np.zeros(n, dtype=np.float64)


def lattice():
    """(c [19,3] int, w [19]) in the paper's direction order (Sec. II.A)."""
    lib = _load()
    cx = (ctypes.c_int * Q)()
    cy = (ctypes.c_int * Q)()
    cz = (ctypes.c_int * Q)()
    w = _vec()
    lib.orc_lattice(cx, cy, cz, _p(w))
    c = np.stack([np.array(cx[:]), np.array(cy[:]), np.array(cz[:])], axis=1)
    return c, w


def feq(rho, u):
    """Extended equilibrium of Eq. (eq:EqQ19RM)."""
    out = _vec()
    _load().orc_feq(float(rho), float(u[0]), float(u[1]), float(u[2]), _p(out))
    return out


def heq(rho, u, alpha):
    """Colour-gradient equilibrium, App. E Eq. (eq:feqCG)."""
    out = _vec()
    _load().orc_heq(float(rho), float(u[0]), float(u[1]), float(u[2]), float(alpha), _p(out))
    return out


def T(u):
    """Central-moment transformation matrix T(u), Eq. (eq:matrix), 19x19."""
    out = np.zeros((Q, Q))
    _load().orc_T(float(u[0]), float(u[1]), float(u[2]), _p(out))
    return out


def solve19(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = _vec()
    if _load().orc_solve19(_p(A), _p(b), _p(x)) != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def forcing_rm(u, F):
    """Raw forcing moments of Eq. (eq:RMQ19) placed on the rows of M."""
    out = _vec()
    _load().orc_forcing_rm(*map(float, u), *map(float, F), _p(out))
    return out


def forcing_pop(u, F):
    """Velocity-space forcing F_i = M^-1 R^RM (App. B moment matching)."""
    out = _vec()
    _load().orc_forcing_pop(*map(float, u), *map(float, F), _p(out))
    return out


def collide_dense(f, rho, u, F, omega, omega_b=1.0, omega_3=1.0, omega_4=1.0, cgm=False, alpha=1.0 / 3.0):
    """Oracle-A: Eq. (eq:posColl0) by dense matrices and a linear solve."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = _vec()
    rc = _load().orc_collide_dense(_p(f), float(rho), *map(float, u), *map(float, F), float(omega),
                                   float(omega_b), float(omega_3), float(omega_4), int(cgm), float(alpha), _p(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular T")
    return out


def collide_closed(f, rho, u, F, omega, cgm=False, alpha=1.0 / 3.0):
    """Oracle-B: printed post-collision CMs, then Eqs. (rawQ19), (pdfQ19)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = _vec()
    _load().orc_collide_closed(_p(f), float(rho), *map(float, u), *map(float, F), float(omega), int(cgm),
                               float(alpha), _p(out))
    return out


def kstar_fluid(f, rho, u, F, omega):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = _vec()
    _load().orc_kstar_fluid(_p(f), float(rho), *map(float, u), *map(float, F), float(omega), _p(out))
    return out


def kstar_cgm(f, rho, u, F, omega, alpha):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = _vec()
    _load().orc_kstar_cgm(_p(f), float(rho), *map(float, u), *map(float, F), float(omega), float(alpha), _p(out))
    return out


def back_transform(rho, u, kstar):
    k = np.ascontiguousarray(kstar, dtype=np.float64)
    out = _vec()
    _load().orc_back_transform(float(rho), *map(float, u), _p(k), _p(out))
    return out


def geq_magnetic(u, b):
    """D3Q7 vector-valued magnetic equilibrium (reading of Dellar's scheme); [7,3]."""
    out = _vec(21)
    _load().orc_geq(*map(float, u), *map(float, b), _p(out))
    return out.reshape(7, 3)


def current(g, u, tau_m):
    """(b, j) from the magnetic populations g [7,3] and velocity u."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(21))
    b = _vec(3)
    j = _vec(3)
    _load().orc_current(_p(g), *map(float, u), float(tau_m), _p(b), _p(j))
    return b, j


def cgm_perturb(f, grad, A):
    f = np.array(f, dtype=np.float64)
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    _load().orc_cgm_perturb(_p(grad), float(A), _p(f))
    return f


def cgm_recolour(f, grad, rho_r, rho_b, alpha, beta):
    f = np.ascontiguousarray(f, dtype=np.float64)
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    fr, fb = _vec(), _vec()
    _load().orc_cgm_recolour(_p(f), _p(grad), float(rho_r), float(rho_b), float(alpha), float(beta), _p(fr), _p(fb))
    return fr, fb


def collide_rm(f, rho, u, F, omega, dense=False):
    """Raw-moment variant of App. C: the printed list (closed) or the MRT
    definition with M = T(0) (dense)."""
    out = _vec()
    fn = _load().orc_collide_dense_rm if dense else _load().orc_collide_rm
    fn(_p(np.ascontiguousarray(f, dtype=np.float64)), float(rho), *map(float, u), *map(float, F), float(omega),
       _p(out))
    return out


def regularize(fin, sgn, u_w, g=(0.0, 0.0, 0.0), rho_ref=0.0):
    """Regularized on-node wall reconstruction of one node (orc_regularize)."""
    f = np.array(fin, dtype=np.float64)
    uw = np.array(u_w, dtype=np.float64)
    gg = np.array(g, dtype=np.float64)
    _load().orc_regularize(_p(f), int(sgn), _p(uw), _p(gg), float(rho_ref))
    return f


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("lid_u", ctypes.c_double * 3),
                ("omega", ctypes.c_double), ("omega_b", ctypes.c_double),
                ("omega_3", ctypes.c_double), ("omega_4", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("physics", ctypes.c_int), ("closed_form", ctypes.c_int),
                ("tau_m", ctypes.c_double), ("b_wall", ctypes.c_double * 3),
                ("alpha_r", ctypes.c_double), ("alpha_b", ctypes.c_double),
                ("A", ctypes.c_double), ("beta", ctypes.c_double), ("nthreads", ctypes.c_int),
                ("G", ctypes.c_double), ("rho_ref", ctypes.c_double), ("wall_model", ctypes.c_int),
                ("raw_moments", ctypes.c_int)]


class Domain:
    """A box of nx*ny*nz nodes advanced by the oracle.

    Fields use the layout [nz][ny][nx] (x fastest); u and B are [3, nz, ny, nx].
    ``periodic`` is a 3-tuple of booleans; a non-periodic axis has half-way
    bounce-back walls at both ends, the +y wall moving with ``lid_u``.
    """

    def __init__(self, shape, omega, *, periodic=(True, True, True), lid_u=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0),
                 physics=FLUID, closed_form=True, omega_b=1.0, omega_3=1.0, omega_4=1.0, tau_m=1.0,
                 b_wall=(0.0, 0.0, 0.0), alpha_r=1.0 / 3.0, alpha_b=1.0 / 3.0, A=0.0, beta=0.7, G=0.0, rho_ref=0.0,
                 wall_model="bounce_back", collision="cm"):
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        p = _Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for a in range(3):
            p.periodic[a] = int(bool(periodic[a]))
            p.lid_u[a] = float(lid_u[a])
            p.g[a] = float(g[a])
            p.b_wall[a] = float(b_wall[a])
        p.omega, p.omega_b, p.omega_3, p.omega_4 = map(float, (omega, omega_b, omega_3, omega_4))
        p.physics = int(physics)
        p.closed_form = int(bool(closed_form))
        p.tau_m = float(tau_m)
        p.alpha_r, p.alpha_b, p.A, p.beta = map(float, (alpha_r, alpha_b, A, beta))
        p.G = float(G)
        p.rho_ref = float(rho_ref)
        if wall_model not in ("bounce_back", "regularized"):
            raise ValueError(wall_model)
        if wall_model == "regularized":
            # on-node walls at y = 0 and y = ny - 1 only (straight channel walls)
            if periodic[1] or not (periodic[0] and periodic[2]) or ny < 3 or physics != FLUID:
                raise ValueError("regularized walls: single phase, walls on y only, ny >= 3")
        p.wall_model = 1 if wall_model == "regularized" else 0
        if collision not in ("cm", "rm"):
            raise ValueError(collision)
        p.raw_moments = int(collision == "rm")
        self.p = p
        self.physics = physics
        n = self.n
        z = lambda k: np.zeros(n * k, dtype=np.float64)
        self.f = z(Q)
        self.ftmp = z(Q) if physics != CGM else None
        self.psi = z(1) if physics == SC else None
        self.g = z(21) if physics == MHD else None
        self.gtmp = z(21) if physics == MHD else None
        if physics == CGM:
            self.fr, self.fb, self.frtmp, self.fbtmp, self.phi = z(Q), z(Q), z(Q), z(Q), z(1)
        else:
            self.fr = self.fb = self.frtmp = self.fbtmp = self.phi = None

    def _field(self, a, k=1):
        nx, ny, nz = self.shape
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.size == self.n * k
        return a.reshape(-1)

    def init(self, rho, u, phase=None, B=None):
        rho = self._field(rho)
        u = self._field(u, 3)
        phase = self._field(phase) if phase is not None else None
        B = self._field(B, 3) if B is not None else None
        _load().orc_init(ctypes.byref(self.p), _p(rho), _p(u), _p(phase), _p(B), _p(self.f), _p(self.g),
                         _p(self.fr), _p(self.fb))

    def step(self, n=1):
        rc = _load().orc_step(ctypes.byref(self.p), _p(self.f), _p(self.ftmp), _p(self.g), _p(self.gtmp),
                              _p(self.fr), _p(self.fb), _p(self.frtmp), _p(self.fbtmp),
                              _p(self.psi if self.physics == SC else self.phi), int(n))
        if rc != 0:
            raise RuntimeError("oracle: singular moment matrix")

    def fields(self):
        """(rho [nz,ny,nx], u [3,nz,ny,nx], phase or None, B or None)."""
        nx, ny, nz = self.shape
        rho = np.zeros(self.n)
        u = np.zeros(3 * self.n)
        phase = np.zeros(self.n) if self.physics in (CGM, SC) else None
        B = np.zeros(3 * self.n) if self.physics == MHD else None
        _load().orc_fields(ctypes.byref(self.p), _p(self.f), _p(self.g), _p(self.fr), _p(self.fb), _p(rho), _p(u),
                           _p(phase), _p(B))
        shp = (nz, ny, nx)
        return (rho.reshape(shp), u.reshape((3,) + shp), None if phase is None else phase.reshape(shp),
                None if B is None else B.reshape((3,) + shp))

    def sc_force(self, psi):
        """Shan-Chen force [3, nz, ny, nx] of a pseudopotential field psi [nz, ny, nx]
        on this machine (walls as configured)."""
        nx, ny, nz = self.shape
        psi = self._field(psi)
        F = np.zeros(3 * self.n)
        _load().orc_sc_force_field(ctypes.byref(self.p), _p(psi), _p(F))
        return F.reshape((3, nz, ny, nx))

    # populations in the oracle's cell-major layout [cell, 19]
    def populations(self):
        return self.f.reshape(self.n, Q)

    def set_populations(self, f):
        self.f[:] = np.asarray(f, dtype=np.float64).reshape(-1)
