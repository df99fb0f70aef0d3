"""Shared helpers of the test-suite: run the same seeded workload through the
CUDA library (C ABI) and through the FP64 oracle, and compare."""
import numpy as np

import oracle as O

CS2 = 1.0 / 3.0


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_run(shape, omega, steps, rho, u, phase=None, B=None, closed_form=True, threads=None, **kw):
    if threads:
        O.set_threads(threads)
    phys = {"fluid": O.FLUID, "mhd": O.MHD, "cgm": O.CGM, "sc": O.SC}[kw.pop("physics", "fluid")]
    d = O.Domain(shape, omega, physics=phys, closed_form=closed_form, **kw)
    d.init(rho, u, phase=phase, B=B)
    if steps:
        d.step(steps)
    r, uu, ph, BB = d.fields()
    return {"rho": r, "u": uu, "phase": ph, "B": BB, "domain": d}


def gpu_run(shape, omega, steps, rho, u, phase=None, B=None, precision="fp64", physics="fluid", keep=False,
            launch=None, **kw):
    from paper_2010_01628_gb300 import binding as L

    ctx = L.lbm_create(shape, omega, physics=physics, precision=precision, **kw)
    try:
        if launch is not None:
            L.lbm_set_launch_shape(ctx, *launch)
        L.lbm_init_fields(ctx, np.ascontiguousarray(rho), np.ascontiguousarray(u),
                          None if phase is None else np.ascontiguousarray(phase),
                          None if B is None else np.ascontiguousarray(B))
        if steps:
            L.lbm_step(ctx, steps)
        want = ["rho", "u"] + (["phase"] if physics in ("cgm", "sc") else []) + (["B"] if physics == "mhd" else [])
        out = L.lbm_fields(ctx, shape, want=want)
        if keep:
            out["ctx"] = ctx
            ctx = None
        return out
    finally:
        if ctx:
            L.lbm_destroy(ctx)

