"""The largest domains the library accepts, on the GPU: 2047 x 1024 x 1024 =
2,146,435,072 nodes (just under the 2^31 limit) in BF16 storage (163 GB of
populations), and 1024^3 in FP32 (163 GB).  From the rest state under a
uniform body force every node's reported velocity after n steps is exactly
(n + 1/2) g (rho u = Sum f c + F/2 with the momentum gain F per step) and the
mass stays N; the FP64 reductions check both over all nodes, so every index,
plane offset and block of the grid takes part."""
import gc

import pytest

pytestmark = pytest.mark.gpu


def run_uniform_acceleration(shape, precision, g, steps):
    import torch
    from paper_2010_01628_gb300 import binding as L
    ctx = L.lbm_create(shape, 1.2, g=(g, 0.0, 0.0), precision=precision)
    try:
        L.lbm_step(ctx, steps)
        mass, mom, _ = L.lbm_reduce(ctx)
    finally:
        L.lbm_destroy(ctx)
        gc.collect()
        torch.cuda.empty_cache()
    return mass, mom


# mass: every node holds the same state, so storage rounding is coherent; one
# rounding of the stored (f - w)/w moves rho by at most eps * Sum_i w_i |q_i|,
# about 2^-8 u ~ 4e-6 for BF16 at u ~ 1e-3 (measured 2.1e-6), 1e-9 for FP32.
@pytest.mark.parametrize("shape,precision,tol,tol_mass", [((2047, 1024, 1024), "bf16", 1e-2, 1e-5),
                                                          ((1024, 1024, 1024), "fp32", 1e-5, 1e-6)])
def test_largest_domains_uniform_acceleration(shape, precision, tol, tol_mass):
    n = shape[0] * shape[1] * shape[2]
    g, steps = 1e-4, 10
    mass, mom = run_uniform_acceleration(shape, precision, g, steps)
    assert abs(mass / n - 1.0) < tol_mass
    assert abs(mom[0] / (n * (steps + 0.5) * g) - 1.0) < tol
    assert abs(mom[1]) < 1e-9 * n and abs(mom[2]) < 1e-9 * n


def test_two_to_the_31_nodes_rejected():
    from paper_2010_01628_gb300 import binding as L
    with pytest.raises(Exception):
        L.lbm_create((2048, 1024, 1024), 1.2, precision="bf16")
