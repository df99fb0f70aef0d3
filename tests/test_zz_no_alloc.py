"""The allocation-free reduction entry point (lbm_reduce_state_noalloc).

It serves callers that may not allocate device memory (applications owning
all device memory through their own pool, latency-critical loops, code inside
allocator callbacks).  Its output must match the context-based lbm_reduce on
the same state, call after call, although its scratch is a fixed device array
shared by every call, and the oracle's totals after the same steps.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2010_01628_gb300 import inputs
from helpers import oracle_run

# against lbm_reduce on the same stored state: the same per-node arithmetic,
# summed in another order
TOL_SAME_STATE = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-5, "bf16": 1e-5}
# against the FP64 oracle after the same steps: the storage precision's bound
TOL_ORACLE = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 4e-3}

CASES = {
    "walls_lid": dict(periodic=(True, False, True), lid_u=(0.05, 0.0, 0.0), g=(1e-4, 0.0, 2e-5)),
    "periodic": dict(periodic=(True, True, True), lid_u=(0.0, 0.0, 0.0), g=(0.0, 3e-5, 0.0)),
}


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_noalloc_reduction_matches_lbm_reduce_and_oracle(precision, case):
    import torch
    from paper_2010_01628_gb300 import binding as L

    shape = (70, 9, 6)
    kw = CASES[case]
    omega = 1.3
    rho, u = inputs.random_fields(shape, seed=91, u_amp=0.03)
    ctx = L.lbm_create(shape, omega, precision=precision, **kw)
    try:
        L.lbm_init_fields(ctx, rho, u)
        pops = torch.empty(L.lbm_state_bytes(ctx), dtype=torch.uint8, device="cuda")
        done = 0
        for call, steps in enumerate((5, 7)):  # two calls in a row on evolving states
            L.lbm_step(ctx, steps)
            done += steps
            mass, mom, _ = L.lbm_reduce(ctx)
            L.lbm_get_populations(ctx, pops)
            out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
            L.lbm_reduce_state_noalloc(pops, shape, out, precision=precision, **kw)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = mass * 0.03  # total mass x velocity scale of the flow
            tol = TOL_SAME_STATE[precision]
            assert got[4] == 0.0, (call, got)
            assert abs(got[0] - mass) <= tol * mass, (call, got[0], mass)
            np.testing.assert_allclose(got[1:4], mom, rtol=tol, atol=tol * scale)
            ref = oracle_run(shape, omega, done, rho, u, **kw)
            o_mass = ref["rho"].sum()
            o_mom = (ref["rho"][None] * ref["u"]).sum(axis=(1, 2, 3))
            tol = TOL_ORACLE[precision]
            assert abs(got[0] - o_mass) <= tol * o_mass, (call, got[0], o_mass)
            np.testing.assert_allclose(got[1:4], o_mom, rtol=0, atol=tol * scale)
    finally:
        L.lbm_destroy(ctx)


def _binding():
    from paper_2010_01628_gb300 import build

    build.build()
    from paper_2010_01628_gb300 import binding as L

    return L


def test_noalloc_rejects_oversized_grids():
    """Rejection happens before any device work (runs without a GPU too)."""
    L = _binding()
    err = ctypes.create_string_buffer(256)
    gr = L.lbm_grid(2048, 2048, 1024, 7)
    st = L._lib.lbm_reduce_state_noalloc(ctypes.c_void_p(1), 1, ctypes.byref(gr), None, ctypes.c_void_p(1), None,
                                         err, 256)
    assert st == L.LBM_ERR_ARG
    assert b"2^31" in err.value
    gr = L.lbm_grid(8, 70000, 8, 7)
    st = L._lib.lbm_reduce_state_noalloc(ctypes.c_void_p(1), 1, ctypes.byref(gr), None, ctypes.c_void_p(1), None,
                                         err, 256)
    assert st == L.LBM_ERR_ARG and b"65535" in err.value


def test_noalloc_binding_rejects_bad_buffers_before_any_launch():
    """The binding refuses host tensors, a non-float64 or short out, a short
    or non-contiguous population buffer and unknown precisions, raising before
    the library is called (runs without a GPU: every case fails a host check)."""
    torch = pytest.importorskip("torch")
    L = _binding()
    shape = (4, 3, 2)
    n = 4 * 3 * 2
    pops = torch.zeros(19 * n, dtype=torch.float32)
    out = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        L.lbm_reduce_state_noalloc(pops, shape, out, precision="fp32")
    with pytest.raises(ValueError, match="precision"):
        L.lbm_reduce_state_noalloc(pops, shape, out, precision="fp8")
    with pytest.raises(TypeError):
        L.lbm_reduce_state_noalloc(pops.numpy(), shape, out, precision="fp32")
    if torch.cuda.is_available():
        dev = torch.device("cuda", torch.cuda.current_device())
        good_p = torch.zeros(19 * n, dtype=torch.float32, device=dev)
        good_o = torch.zeros(5, dtype=torch.float64, device=dev)
        bad = [
            (good_p, torch.zeros(5, dtype=torch.float32, device=dev), "float64"),
            (good_p, torch.zeros(4, dtype=torch.float64, device=dev), "5 values"),
            (good_p[:-1], good_o, "needs"),
            (good_p.view(19, n)[:, ::2], good_o, "contiguous"),
            (good_p, out, "CUDA"),
        ]
        for p_, o_, msg in bad:
            with pytest.raises(ValueError, match=msg):
                L.lbm_reduce_state_noalloc(p_, shape, o_, precision="fp32")
