"""The allocation-free reduction entry point (lbm_reduce_state_noalloc).

It serves callers that may not allocate device memory (applications owning
all device memory through their own pool, latency-critical loops, code inside
allocator callbacks).  Its output must match the context-based lbm_reduce on
the same state, call after call, although its scratch is a fixed device array
shared by every call.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2010_01628_gb300 import inputs

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_reduction_matches_lbm_reduce(precision):
    import torch
    from paper_2010_01628_gb300 import binding as L

    shape = (70, 9, 6)
    kw = dict(periodic=(True, False, True), lid_u=(0.05, 0.0, 0.0), g=(1e-4, 0.0, 2e-5))
    rho, u = inputs.random_fields(shape, seed=91, u_amp=0.03)
    ctx = L.lbm_create(shape, 1.3, precision=precision, **kw)
    try:
        L.lbm_init_fields(ctx, rho, u)
        pops = torch.empty(L.lbm_state_bytes(ctx), dtype=torch.uint8, device="cuda")
        for call, steps in enumerate((5, 7)):  # two calls in a row on evolving states
            L.lbm_step(ctx, steps)
            mass, mom, _ = L.lbm_reduce(ctx)
            L.lbm_get_populations(ctx, pops)
            out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
            L.lbm_reduce_state_noalloc(pops, shape, out, precision=precision, **kw)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            tol = TOL[precision]
            assert got[4] == 0.0, (call, got)
            assert abs(got[0] - mass) <= tol * mass, (call, got[0], mass)
            scale = mass * 0.05  # total mass x velocity scale of the flow
            np.testing.assert_allclose(got[1:4], mom, rtol=tol, atol=tol * scale)
    finally:
        L.lbm_destroy(ctx)


def test_noalloc_rejects_oversized_grids():
    """Rejection happens before any device work (runs without a GPU too)."""
    from paper_2010_01628_gb300 import build

    build.build()
    from paper_2010_01628_gb300 import binding as L

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
