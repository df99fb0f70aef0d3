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



def round_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_fp16(x):
    """Round to the nearest FP16 value, returned as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def oracle_run_stored(shape, omega, steps, rho, u, storage, **kw):
    """The FP64 oracle with its populations rounded after initialisation and
    after every step as the 16-bit storage formats hold them, q = (f - w)/w
    rounded to BF16 or FP16 (through FP32): the error floor of the storage
    format itself, with exact arithmetic in between."""
    rnd = {"bf16": round_bf16, "fp16": round_fp16}[storage]
    _, w = O.lattice()
    d = O.Domain(shape, omega, **kw)
    d.init(rho, u)

    def store():
        f = d.populations()
        q = ((f - w) / w).astype(np.float32)
        d.set_populations(w * (1.0 + rnd(q)))

    store()
    for _ in range(steps):
        d.step(1)
        store()
    r, uu, _, _ = d.fields()
    return {"rho": r, "u": uu}
