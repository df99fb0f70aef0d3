"""ctypes binding of liblbm.so with the entry-point names of include/lbm.h.

Argument marshalling only: every step of the method runs in the CUDA library.
Device memory for the library comes from PyTorch's caching allocator (installed
through ``lbm_set_allocator`` on first use) and work is ordered on PyTorch's
current CUDA stream unless another stream is given.  If the library has not
been built, importing this module raises; there is no CPU fallback.

Field arrays are float64, layout [nz, ny, nx] (u, B: [3, nz, ny, nx]); they
may be numpy arrays (host) or torch tensors (host, pinned or CUDA).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED = range(7)
LBM_D3Q19 = 0
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
PHYSICS = {"fluid": 0, "mhd": 1, "cgm": 2, "sc": 3}
WALL_MODELS = {"bounce_back": 0, "regularized": 1}
MOMENT_SPACES = {"cm": 0, "rm": 1}

if not os.path.exists(_build.LIB):
    raise ImportError(f"liblbm.so is not built ({_build.LIB}); run paper_2010_01628_gb300.build.build() first")

_lib = ctypes.CDLL(_build.LIB)


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("periodic_mask", ctypes.c_uint),
                ("lid_u", ctypes.c_double * 3), ("wall_model", ctypes.c_int)]


class lbm_relax(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("omega_bulk", ctypes.c_double), ("omega_3", ctypes.c_double),
                ("omega_4", ctypes.c_double), ("moment_space", ctypes.c_int)]


class lbm_forcing(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double * 3), ("rho_ref", ctypes.c_double)]


class lbm_physparams(ctypes.Structure):
    _fields_ = [("tau_m", ctypes.c_double), ("b_wall", ctypes.c_double * 3), ("alpha_r", ctypes.c_double),
                ("alpha_b", ctypes.c_double), ("A", ctypes.c_double), ("beta", ctypes.c_double),
                ("G", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_V = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_lib.lbm_set_allocator.argtypes = [ALLOC_FN, FREE_FN, _V]
_lib.lbm_create.argtypes = [ctypes.POINTER(_V), ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.POINTER(lbm_relax),
                            ctypes.POINTER(lbm_forcing), ctypes.c_int, ctypes.POINTER(lbm_physparams), ctypes.c_int, _V]
_lib.lbm_init_fields.argtypes = [_V, _V, _V, _V, _V]
_lib.lbm_step.argtypes = [_V, ctypes.c_long]
_lib.lbm_fields.argtypes = [_V, _V, _V, _V, _V]
_lib.lbm_reduce.argtypes = [_V, _D, _D, _D]
_lib.lbm_run_to_steady.argtypes = [_V, ctypes.c_long, ctypes.c_long, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_long), _D]
_lib.lbm_sync.argtypes = [_V]
_lib.lbm_state_bytes.argtypes = [_V]
_lib.lbm_state_bytes.restype = ctypes.c_size_t
_lib.lbm_get_populations.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_set_populations.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_destroy.argtypes = [_V]
_lib.lbm_destroy.restype = None
_lib.lbm_last_error.argtypes = [_V]
_lib.lbm_last_error.restype = ctypes.c_char_p
_lib.lbm_status_string.argtypes = [ctypes.c_int]
_lib.lbm_status_string.restype = ctypes.c_char_p
for _name in ("lbm_set_allocator", "lbm_create", "lbm_init_fields", "lbm_step", "lbm_fields", "lbm_reduce",
              "lbm_run_to_steady", "lbm_sync", "lbm_get_populations", "lbm_set_populations"):
    getattr(_lib, _name).restype = ctypes.c_int


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.lbm_status_string(status).decode()}: {msg}")
        self.status = status


def _check(status, ctx=None):
    if status != LBM_OK:
        msg = _lib.lbm_last_error(ctx).decode() if ctx else ""
        raise LBMError(status, msg)


# --- device memory from PyTorch's caching allocator ------------------------------
_alloc_refs = None


def _torch():
    try:
        import torch
        return torch if torch.cuda.is_available() else None
    except ImportError:
        return None


def lbm_set_allocator(use_torch: bool = True) -> None:
    """Install torch's caching allocator as the library's device-memory provider
    (or restore cudaMalloc with use_torch=False)."""
    global _alloc_refs
    torch = _torch()
    if not use_torch or torch is None:
        _check(_lib.lbm_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _alloc_refs = None
        return

    def _alloc(size, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), int(stream or 0))
        except Exception:  # the library reports LBM_ERR_OOM for a NULL
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(_lib.lbm_set_allocator(_alloc_refs[0], _alloc_refs[1], None))


def _current_stream():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream if torch is not None else 0


def _ptr(a, n_expected=None, writable=False):
    """Raw pointer of a float64 C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("field arrays must be C-contiguous float64")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        if n_expected is not None and a.size != n_expected:
            raise ValueError(f"expected {n_expected} values, got {a.size}")
        return a.ctypes.data
    torch = __import__("torch")
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("field tensors must be contiguous float64")
        if n_expected is not None and a.numel() != n_expected:
            raise ValueError(f"expected {n_expected} values, got {a.numel()}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def lbm_create(shape, omega, *, periodic=(True, True, True), lid_u=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0),
               physics="fluid", precision="fp32", tau_m=1.0, b_wall=(0.0, 0.0, 0.0), alpha_r=1.0 / 3.0,
               alpha_b=1.0 / 3.0, A=0.0, beta=0.7, G=0.0, rho_ref=0.0, wall_model="bounce_back", collision="cm",
               lattice="d3q19", omega_bulk=1.0, omega_3=1.0, omega_4=1.0, stream=None):
    """Create a context; returns its handle (an int).  shape = (nx, ny, nz).
    physics: "fluid", "mhd" (tau_m, b_wall), "cgm" (alpha_r, alpha_b, A, beta)
    or "sc" (Shan-Chen, interaction strength G).  The body force is
    F = (rho - rho_ref) g (rho_ref != 0: two-phase modules only).  wall_model:
    "bounce_back" (half-way) or "regularized" (on-node walls on y, single phase).
    collision: "cm" (central moments) or "rm" (the raw-moment variant, single phase).
    lattice: "d3q19" or "d3q27" (single phase, FP32/FP64)."""
    if _alloc_refs is None and _torch() is not None:
        lbm_set_allocator(True)
    gr = lbm_grid()
    gr.nx, gr.ny, gr.nz = (int(v) for v in shape)
    gr.periodic_mask = sum((1 << a) for a in range(3) if periodic[a])
    for a in range(3):
        gr.lid_u[a] = float(lid_u[a])
    gr.wall_model = WALL_MODELS[wall_model]
    rl = lbm_relax(float(omega), float(omega_bulk), float(omega_3), float(omega_4), MOMENT_SPACES[collision])
    fo = lbm_forcing()
    for a in range(3):
        fo.g[a] = float(g[a])
    fo.rho_ref = float(rho_ref)
    ph = lbm_physparams()
    ph.tau_m = float(tau_m)
    for a in range(3):
        ph.b_wall[a] = float(b_wall[a])
    ph.alpha_r, ph.alpha_b, ph.A, ph.beta = float(alpha_r), float(alpha_b), float(A), float(beta)
    ph.G = float(G)
    ctx = _V()
    s = _current_stream() if stream is None else int(stream)
    _check(_lib.lbm_create(ctypes.byref(ctx), ctypes.byref(gr), {"d3q19": 0, "d3q27": 1}[lattice], ctypes.byref(rl),
                           ctypes.byref(fo),
                           PHYSICS[physics], ctypes.byref(ph), PRECISIONS[precision], _V(s)))
    return ctx.value


def _n(ctx_shape):
    nx, ny, nz = ctx_shape
    return nx * ny * nz


def lbm_init_fields(ctx, rho, u=None, phase=None, B=None):
    n = int(np.prod(rho.shape))
    _check(_lib.lbm_init_fields(ctx, _ptr(rho, n), _ptr(u, 3 * n), _ptr(phase, n), _ptr(B, 3 * n)), ctx)


def lbm_step(ctx, n=1):
    _check(_lib.lbm_step(ctx, int(n)), ctx)


def lbm_sync(ctx):
    _check(_lib.lbm_sync(ctx), ctx)


def lbm_fields(ctx, shape, rho=None, u=None, phase=None, B=None, want=("rho", "u")):
    """Fill (or allocate on the host) the requested fields; returns a dict."""
    nx, ny, nz = shape
    n = nx * ny * nz
    out = {}
    if rho is None and "rho" in want:
        rho = np.empty((nz, ny, nx))
    if u is None and "u" in want:
        u = np.empty((3, nz, ny, nx))
    if phase is None and "phase" in want:
        phase = np.empty((nz, ny, nx))
    if B is None and "B" in want:
        B = np.empty((3, nz, ny, nx))
    _check(_lib.lbm_fields(ctx, _ptr(rho, n, True), _ptr(u, 3 * n, True), _ptr(phase, n, True), _ptr(B, 3 * n, True)),
           ctx)
    for k, v in (("rho", rho), ("u", u), ("phase", phase), ("B", B)):
        if v is not None:
            out[k] = v
    return out


def lbm_reduce(ctx):
    """(mass, momentum[3], residual) with lbm_reduce's semantics."""
    m = ctypes.c_double()
    mom = (ctypes.c_double * 3)()
    r = ctypes.c_double()
    _check(_lib.lbm_reduce(ctx, ctypes.byref(m), mom, ctypes.byref(r)), ctx)
    return m.value, np.array(mom[:]), r.value


def lbm_run_to_steady(ctx, max_steps, check_every=100, tol=1e-6):
    steps = ctypes.c_long()
    r = ctypes.c_double()
    _check(_lib.lbm_run_to_steady(ctx, int(max_steps), int(check_every), float(tol), ctypes.byref(steps),
                                  ctypes.byref(r)), ctx)
    return steps.value, r.value


def lbm_state_bytes(ctx):
    return int(_lib.lbm_state_bytes(ctx))


def lbm_get_populations(ctx, dst=None):
    nb = lbm_state_bytes(ctx)
    if dst is None:
        dst = np.empty(nb, dtype=np.uint8)
    ptr = dst.ctypes.data if isinstance(dst, np.ndarray) else dst.data_ptr()
    _check(_lib.lbm_get_populations(ctx, _V(ptr), nb), ctx)
    return dst


def lbm_set_populations(ctx, src):
    nb = lbm_state_bytes(ctx)
    ptr = src.ctypes.data if isinstance(src, np.ndarray) else src.data_ptr()
    size = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    if size != nb:
        raise ValueError(f"state is {nb} bytes, got {size}")
    _check(_lib.lbm_set_populations(ctx, _V(ptr), nb), ctx)


_lib.lbm_reduce_state_noalloc.argtypes = [_V, ctypes.c_int, ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_forcing),
                                          _V, _V, ctypes.c_char_p, ctypes.c_size_t]
_lib.lbm_reduce_state_noalloc.restype = ctypes.c_int


_STORED_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


def _check_noalloc_tensors(populations, shape, out, precision):
    """Argument checks of lbm_reduce_state_noalloc, all made before any device
    work: the library writes 5 doubles through out and reads 19 planes of the
    grid through populations, so a host tensor, a wrong dtype or a short
    buffer would be an out-of-bounds device access."""
    import torch

    if precision not in _STORED_BYTES:
        raise ValueError(f"unknown precision {precision!r}")
    for name, t in (("populations", populations), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if out.dtype != torch.float64:
        raise ValueError("out must be float64")
    if out.numel() < 5:
        raise ValueError("out must hold at least 5 values")
    nx, ny, nz = (int(v) for v in shape)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid sizes must be >= 1")
    need = 19 * nx * ny * nz * _STORED_BYTES[precision]
    have = populations.numel() * populations.element_size()
    if have < need:
        raise ValueError(f"populations hold {have} bytes, the {precision} state of {shape} needs {need}")
    dev = torch.cuda.current_device()
    if populations.device.index != dev or out.device.index != dev:
        raise ValueError(f"populations and out must be on the current device cuda:{dev}")


def lbm_reduce_state_noalloc(populations, shape, out, *, precision="fp32", periodic=(True, True, True),
                             lid_u=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0), stream=None):
    """Allocation-free reduction of a caller-owned state.  populations: a
    contiguous CUDA tensor holding at least 19 * nx * ny * nz stored values of
    the precision; out: a contiguous CUDA float64 tensor of >= 5 values; both on
    the current device (checked before the call).  Enqueued on the stream, not
    synchronised."""
    _check_noalloc_tensors(populations, shape, out, precision)
    gr = lbm_grid()
    gr.nx, gr.ny, gr.nz = (int(v) for v in shape)
    gr.periodic_mask = sum((1 << a) for a in range(3) if periodic[a])
    for a in range(3):
        gr.lid_u[a] = float(lid_u[a])
    fo = lbm_forcing()
    for a in range(3):
        fo.g[a] = float(g[a])
    err = ctypes.create_string_buffer(256)
    s = _current_stream() if stream is None else int(stream)
    status = _lib.lbm_reduce_state_noalloc(_V(populations.data_ptr()), PRECISIONS[precision], ctypes.byref(gr),
                                           ctypes.byref(fo), _V(out.data_ptr()), _V(s), err, 256)
    if status != LBM_OK:
        raise LBMError(status, err.value.decode())


_lib.lbm_batch_create.argtypes = [ctypes.POINTER(_V), ctypes.c_int, ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_relax),
                                  ctypes.POINTER(lbm_forcing), ctypes.c_int, ctypes.POINTER(lbm_physparams),
                                  ctypes.c_int, _V]
_lib.lbm_batch_domain.argtypes = [_V, ctypes.c_int, ctypes.POINTER(_V)]
_lib.lbm_batch_step.argtypes = [_V, ctypes.c_long]
_lib.lbm_batch_info.argtypes = [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)]
_lib.lbm_barrier_selftest.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
_lib.lbm_autotune.argtypes = [_V, ctypes.c_char_p, ctypes.c_int, _D]
for _name in ("lbm_batch_create", "lbm_batch_domain", "lbm_batch_step", "lbm_batch_info", "lbm_barrier_selftest",
              "lbm_autotune"):
    getattr(_lib, _name).restype = ctypes.c_int


def _scalars(v, nd):
    """A scalar parameter given once (shared) or once per domain."""
    return [float(x) for x in v] if isinstance(v, (list, tuple, np.ndarray)) else [float(v)] * nd


def _vectors(v, nd):
    """A 3-vector parameter given once (shared) or once per domain."""
    if isinstance(v[0], (list, tuple, np.ndarray)):
        return [tuple(x) for x in v]
    return [tuple(v)] * nd


def lbm_batch_create(shapes, omegas, *, periodic=(True, True, True), lid_u=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0),
                     physics="fluid", precision="fp32", tau_m=1.0, b_wall=(0.0, 0.0, 0.0), alpha_r=1.0 / 3.0,
                     alpha_b=1.0 / 3.0, A=0.0, beta=0.7, G=0.0, rho_ref=0.0, stream=None):
    """Create a batch of len(shapes) domains; per-domain parameters may be
    given once (shared) or as lists of one entry per domain.  physics:
    "fluid", "mhd" (tau_m, b_wall), "cgm" (alpha_r, alpha_b, A, beta,
    rho_ref: colour-gradient sweeps over density ratio and surface tension)
    or "sc" (G, rho_ref: Shan-Chen sweeps over the interaction strength)."""
    if _alloc_refs is None and _torch() is not None:
        lbm_set_allocator(True)
    nd = len(shapes)
    omegas = _scalars(omegas, nd)
    tau_m = _scalars(tau_m, nd)
    alpha_r, alpha_b, A, beta, G, rho_ref = (_scalars(v, nd) for v in (alpha_r, alpha_b, A, beta, G, rho_ref))
    periodic = _vectors(periodic, nd)
    lid_u = _vectors(lid_u, nd)
    g = _vectors(g, nd)
    b_wall = _vectors(b_wall, nd)
    grids = (lbm_grid * nd)()
    relax = (lbm_relax * nd)()
    forc = (lbm_forcing * nd)()
    phys = (lbm_physparams * nd)()
    for d in range(nd):
        grids[d].nx, grids[d].ny, grids[d].nz = (int(v) for v in shapes[d])
        grids[d].periodic_mask = sum((1 << a) for a in range(3) if periodic[d][a])
        relax[d] = lbm_relax(float(omegas[d]), 1.0, 1.0, 1.0)
        phys[d].tau_m = float(tau_m[d])
        phys[d].alpha_r, phys[d].alpha_b = alpha_r[d], alpha_b[d]
        phys[d].A, phys[d].beta, phys[d].G = A[d], beta[d], G[d]
        forc[d].rho_ref = rho_ref[d]
        for a in range(3):
            grids[d].lid_u[a] = float(lid_u[d][a])
            forc[d].g[a] = float(g[d][a])
            phys[d].b_wall[a] = float(b_wall[d][a])
    ctx = _V()
    s = _current_stream() if stream is None else int(stream)
    _check(_lib.lbm_batch_create(ctypes.byref(ctx), nd, grids, relax, forc, PHYSICS[physics], phys,
                                 PRECISIONS[precision], _V(s)))
    return ctx.value


def lbm_batch_domain(ctx, d):
    v = _V()
    _check(_lib.lbm_batch_domain(ctx, int(d), ctypes.byref(v)), ctx)
    return v.value


def lbm_batch_step(ctx, n=1):
    _check(_lib.lbm_batch_step(ctx, int(n)), ctx)


def lbm_batch_info(ctx):
    t, g, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    tiles = ctypes.c_long()
    _check(_lib.lbm_batch_info(ctx, ctypes.byref(t), ctypes.byref(g), ctypes.byref(gr), ctypes.byref(tiles)), ctx)
    return {"threads": t.value, "grid": g.value, "graph": bool(gr.value), "tiles": tiles.value}


def lbm_barrier_selftest(timeout_s=0.2):
    obs = ctypes.c_int()
    _check(_lib.lbm_barrier_selftest(float(timeout_s), ctypes.byref(obs)))
    return obs.value


_lib.lbm_mbarrier_selftest.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
_lib.lbm_mbarrier_selftest.restype = ctypes.c_int


def lbm_mbarrier_selftest(timeout_s=0.2, arrive=False):
    obs = ctypes.c_int()
    _check(_lib.lbm_mbarrier_selftest(float(timeout_s), 1 if arrive else 0, ctypes.byref(obs)))
    return obs.value


_lib.lbm_set_launch_shape.argtypes = [_V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.lbm_set_launch_shape.restype = ctypes.c_int


def lbm_set_launch_shape(ctx, variant, threads=256, stages=4, ctas=1):
    _check(_lib.lbm_set_launch_shape(ctx, int(variant), int(threads), int(stages), int(ctas)), ctx)


_lib.lbm_get_launch_shape.argtypes = [_V] + [ctypes.POINTER(ctypes.c_int)] * 4
_lib.lbm_get_launch_shape.restype = ctypes.c_int


def lbm_get_launch_shape(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib.lbm_get_launch_shape(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return {"variant": ["direct", "tma", "pair", "fused", "zpair"][v[0].value], "threads": v[1].value, "stages": v[2].value,
            "ctas_per_sm": v[3].value}


def lbm_autotune(ctx, cache_path=None, force=False):
    m = ctypes.c_double()
    _check(_lib.lbm_autotune(ctx, cache_path.encode() if cache_path else None, int(bool(force)), ctypes.byref(m)), ctx)
    return m.value


# --- learned warm start ------------------------------------------------------------
_F = ctypes.POINTER(ctypes.c_float)
_lib.lbm_cnn_param_count.restype = ctypes.c_size_t
_lib.lbm_cnn_create.argtypes = [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_int, ctypes.c_int, _V, _V]
_lib.lbm_cnn_destroy.argtypes = [_V]
_lib.lbm_cnn_destroy.restype = None
_lib.lbm_cnn_last_error.argtypes = [_V]
_lib.lbm_cnn_last_error.restype = ctypes.c_char_p
_lib.lbm_cnn_set_weights.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_cnn_get_weights.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_cnn_set_input.argtypes = [_V, ctypes.c_double]
_lib.lbm_cnn_set_input_raw.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_cnn_forward.argtypes = [_V, _V, ctypes.c_size_t]
_lib.lbm_cnn_gradient.argtypes = [_V, _V, _V, _D, _V, ctypes.c_size_t]
_lib.lbm_cnn_train_step.argtypes = [_V, _V, _V, ctypes.c_float, _D]
_lib.lbm_cnn_warm_start.argtypes = [_V, _V, ctypes.c_double]
for _name in ("lbm_cnn_create", "lbm_cnn_set_weights", "lbm_cnn_get_weights", "lbm_cnn_set_input",
              "lbm_cnn_set_input_raw", "lbm_cnn_forward", "lbm_cnn_gradient", "lbm_cnn_train_step",
              "lbm_cnn_warm_start"):
    getattr(_lib, _name).restype = ctypes.c_int


def _check_cnn(status, net):
    if status != LBM_OK:
        raise LBMError(status, _lib.lbm_cnn_last_error(net).decode() if net else "")


def _fptr(a, dtype):
    if isinstance(a, np.ndarray):
        assert a.dtype == dtype and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def lbm_cnn_param_count():
    return int(_lib.lbm_cnn_param_count())


def lbm_cnn_create(shape, init_weights=None, stream=None):
    """Network for grids of shape (nx, ny, nz); init_weights: float32 array or None."""
    if _alloc_refs is None and _torch() is not None:
        lbm_set_allocator(True)
    net = _V()
    w = None
    if init_weights is not None:
        w = np.ascontiguousarray(init_weights, dtype=np.float32)
        assert w.size == lbm_cnn_param_count()
    s = _current_stream() if stream is None else int(stream)
    _check(_lib.lbm_cnn_create(ctypes.byref(net), *(int(v) for v in shape), _V(w.ctypes.data) if w is not None else None,
                               _V(s)))
    return net.value


def lbm_cnn_destroy(net):
    if net:
        _lib.lbm_cnn_destroy(net)


def lbm_cnn_set_weights(net, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check_cnn(_lib.lbm_cnn_set_weights(net, _V(w.ctypes.data), w.size), net)


def lbm_cnn_get_weights(net):
    w = np.empty(lbm_cnn_param_count(), dtype=np.float32)
    _check_cnn(_lib.lbm_cnn_get_weights(net, _V(w.ctypes.data), w.size), net)
    return w


def lbm_cnn_set_input(net, reynolds):
    _check_cnn(_lib.lbm_cnn_set_input(net, float(reynolds)), net)


def lbm_cnn_set_input_raw(net, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    _check_cnn(_lib.lbm_cnn_set_input_raw(net, _V(x.ctypes.data), x.size), net)


def lbm_cnn_forward(net, n_nodes=None):
    """Forward pass; with n_nodes, returns the [n_nodes, 4] FP32 outputs."""
    if n_nodes is None:
        _check_cnn(_lib.lbm_cnn_forward(net, None, 0), net)
        return None
    out = np.empty((n_nodes, 4), dtype=np.float32)
    _check_cnn(_lib.lbm_cnn_forward(net, _V(out.ctypes.data), out.size), net)
    return out


def lbm_cnn_gradient(net, rho, u):
    loss = ctypes.c_double()
    g = np.empty(lbm_cnn_param_count(), dtype=np.float32)
    _check_cnn(_lib.lbm_cnn_gradient(net, _V(_fptr(rho, np.float64)), _V(_fptr(u, np.float64)), ctypes.byref(loss),
                                     _V(g.ctypes.data), g.size), net)
    return loss.value, g


def lbm_cnn_train_step(net, rho, u, lr):
    loss = ctypes.c_double()
    _check_cnn(_lib.lbm_cnn_train_step(net, _V(_fptr(rho, np.float64)), _V(_fptr(u, np.float64)), float(lr),
                                       ctypes.byref(loss)), net)
    return loss.value


def lbm_cnn_warm_start(net, ctx, reynolds):
    _check_cnn(_lib.lbm_cnn_warm_start(net, ctx, float(reynolds)), net)


_lib.lbm_probe_fma_rate.argtypes = [_D, _D]
_lib.lbm_probe_fma_rate.restype = ctypes.c_int


def lbm_probe_fma_rate():
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.lbm_probe_fma_rate(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lbm_destroy(ctx):
    if ctx:
        _lib.lbm_destroy(ctx)


def lbm_last_error(ctx):
    return _lib.lbm_last_error(ctx).decode()


def lbm_status_string(status):
    return _lib.lbm_status_string(int(status)).decode()


def library_path() -> str:
    return _build.LIB
