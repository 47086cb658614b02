"""The multigrid launch variants give the same bits.

The velocity multigrid of the Stokes blocks (W_j) and the pressure
multigrid (the corner-pinned K_p) have kernels whose level sizes are fixed
at compile time (iterates in shared memory, nodes stored per type or
colour) beside the general kernels (run-time level geometry, optional
staging of the iterates in shared memory); the pressure kernel keeps its
finest right-hand side in shared memory or in the workspace; all run 256,
512 or 1024 threads per CTA, chosen by the autotuner or fixed with
pint_mg_launch_config.  Every variant performs the same operations in the
same order on every value (each node's colour update, residual, transfer
and each coarse-grid output are computed by one thread with a fixed
summation order), so the results must agree bit for bit: the W_j and K_p
components (one field) and whole preconditioner applies (batches of fields
over all frequencies) are compared across the variants, in both
precisions, with the tuner off.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_pairs import make_pair, to_dev  # noqa: E402
from paper_2405_18964_gb300 import binding, inputs  # noqa: E402

# (threads per CTA, variant): 1 = the fastest that applies, staged (the
# compile-time-sized kernels), 2 = the same unstaged, 0 = the general
# kernels without staging
VARIANTS = [(512, 1), (256, 1), (1024, 1), (512, 2), (256, 2), (512, 0), (256, 0), (1024, 0)]


@pytest.fixture
def fixed_launches():
    binding.autotune(False)
    try:
        yield
    finally:
        binding.mg_launch_config(0, -1)
        binding.autotune(True)


def _runs(fn):
    out = []
    for threads, variant in VARIANTS:
        binding.mg_launch_config(threads, variant)
        out.append(fn())
        torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("which", ["mg_W", "mg_Kp"])
@pytest.mark.parametrize("level", [2, 4, 6, 7])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_component_same_bits(fixed_launches, which, level, prec):
    K = 4
    P, G = make_pair("stokes", level, K, beta=1e-4, prec=prec)
    n = G.sizes.n_q if which == "mg_Kp" else G.sizes.n_s
    x = to_dev(inputs.random_vector(n, 70 + level, np.complex128), "complex128")

    def run():
        y = torch.zeros(n, dtype=torch.complex128, device="cuda")
        G.component_apply(which, 1, x, y)
        return y

    ys = _runs(run)
    G.close()
    assert float(ys[0].abs().max()) > 0
    for v, y in zip(VARIANTS[1:], ys[1:]):
        assert torch.equal(y, ys[0]), (v, float((y - ys[0]).abs().max()))


@pytest.mark.parametrize("kind,level,K", [("stokes", 5, 16), ("stokes", 6, 8), ("oseen", 4, 8)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_preconditioner_apply_same_bits(fixed_launches, kind, level, K, prec):
    """Fixed inner counts, so every variant runs the same number of
    V-cycles on every frequency (Oseen: the general kernel for Q_j, Q_j^H
    and K_p under every variant, staged or not)."""
    P, G = make_pair(kind, level, K, beta=1e-4, prec=prec, fixed_inner_its=3)
    r = to_dev(inputs.random_vector(G.kkt_len, 80 + level))

    def run():
        z = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
        G.apply_preconditioner(r, z)
        return z

    zs = _runs(run)
    G.close()
    for v, z in zip(VARIANTS[1:], zs[1:]):
        assert torch.equal(z, zs[0]), (v, float((z - zs[0]).abs().max()))
