"""The allocation-free multigrid entry point agrees with the allocating one.

Some callers cannot allocate device memory while they run: an application
whose memory pool already holds the device's memory, or a latency-critical
loop where a cudaMalloc would synchronise the device.  For them the library
offers pint_mg_apply_noalloc, which takes its scratch from one fixed device
array.  These tests call it through the C ABI and compare it with the
ordinary entry point (pint_component_apply, same solve, handle workspace) on
two calls in a row, so the second call runs on the scratch the first one
left behind, and check that repeated calls allocate nothing (the device's
free memory does not move, and the multigrid autotuner, whose bookkeeping
allocates, is never consulted).  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_pairs import FP32_TOL, FP64_TOL, make_pair, relerr, to_dev  # noqa: E402
from paper_2405_18964_gb300 import binding, inputs  # noqa: E402

CASES = [("stokes", 3, 4, 0, "mg_W"), ("stokes", 6, 2, 0, "mg_W"), ("stokes", 6, 2, 1, "mg_Kp"),
         ("oseen", 4, 4, 0, "mg_Q"), ("oseen", 4, 4, 1, "mg_QH"), ("oseen", 3, 4, 0, "mg_Kp")]


@pytest.mark.parametrize("kind,level,K,prec,which", CASES,
                         ids=[f"{c[0]}-L{c[1]}-{'fp32' if c[3] else 'fp64'}-{c[4]}" for c in CASES])
def test_noalloc_matches_component_apply(kind, level, K, prec, which):
    P, G = make_pair(kind, level, K, beta=1e-3, prec=prec, inner_maxit=4)
    n = P.grid.nq if which == "mg_Kp" else P.grid.ns
    J = K // 2 + 1
    tol = FP32_TOL if prec else FP64_TOL
    for call, j in enumerate([J - 1, 0]):          # two calls in a row
        x = to_dev(inputs.random_vector(n, 100 + call, np.complex128), "complex128")
        ref = torch.zeros(n, dtype=torch.complex128, device="cuda")
        got = torch.full((n,), complex(7.0, -7.0), dtype=torch.complex128, device="cuda")
        G.component_apply(which, j, x, ref)
        G.mg_apply_noalloc(which, j, x, got)
        torch.cuda.synchronize()
        assert relerr(got.cpu().numpy(), ref.cpu().numpy()) <= tol, (call, j)
    G.close()


def test_noalloc_repeated_calls_allocate_nothing():
    """Twelve calls with the autotuner switched on (more than the tuner's
    three warm-up and six timed launches of a shape): the free device memory
    is the same after the last call as after the first, the tuner has no
    entry for a single-field launch, and the result stays the same."""
    binding.autotune(True)
    P, G = make_pair("stokes", 5, 4, prec=1, inner_maxit=4)
    n = P.grid.ns
    x = to_dev(inputs.random_vector(n, 7, np.complex128), "complex128")
    y = torch.zeros(n, dtype=torch.complex128, device="cuda")
    first = torch.zeros_like(y)
    G.mg_apply_noalloc("mg_W", 1, x, first)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(12):
        G.mg_apply_noalloc("mg_W", 1, x, y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(y, first)
    assert not [ln for ln in binding.autotune_report().splitlines() if " jobs=1 " in ln]
    G.close()


def test_noalloc_rejects_fields_beyond_its_scratch():
    P, G = make_pair("stokes", 7, 2, prec=0, inner_maxit=2)
    x = torch.zeros(P.grid.ns, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(binding.PintError) as err:
        G.mg_apply_noalloc("mg_W", 0, x, y)
    assert err.value.code == 1 and "bytes" in str(err.value)
    G.close()
