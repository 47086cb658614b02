"""Edge cases of the GPU path: degenerate sizes, zero data and error returns.

Degenerate sizes: one time step (K = 1, a single frequency with d_0 = 0), two
time steps (both frequencies real), and the coarsest grid (level 1, where the
multigrid is the dense coarse solve alone).  Error returns: every status the
header documents that a caller can provoke without a device fault.
"""
import ctypes

import numpy as np
import pytest

from gpu_pairs import FP32_TOL, FP64_TOL, make_pair, relerr, settings_of, to_dev
from oracle import inexact, layout
from paper_2405_18964_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SMALL = [("stokes", 2, 1), ("oseen", 2, 1), ("stokes", 1, 2), ("oseen", 1, 3), ("stokes", 2, 2)]
IDS = [f"{k}-L{l}-K{K}" for k, l, K in SMALL]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind,level,K", SMALL, ids=IDS)
def test_degenerate_sizes_apply(kind, level, K, prec):
    P, G = make_pair(kind, level, K, beta=1e-3, prec=prec, linear=1)
    pc = inexact.PinTPreconditioner(P, settings_of(G), linear=True)
    r = inputs.random_vector(G.kkt_len, 51)
    z = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    G.apply_preconditioner(to_dev(r), z)
    zo = pc(layout.to_oracle_time(P, r.reshape(K, -1)))
    assert relerr(layout.to_oracle_time(P, z.cpu().numpy().reshape(K, -1)), zo) <= (FP32_TOL if prec else FP64_TOL)
    G.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind,level,K", SMALL, ids=IDS)
def test_degenerate_sizes_solve(kind, level, K, prec):
    P, G = make_pair(kind, level, K, beta=1e-3, prec=prec)
    vd = inputs.desired_state(P.N, P.x0, P.x1, K, P.tau, 1.0, seed=2)
    v0 = inputs.random_vector((2, P.grid.ns), 3)
    G.set_data(vd, v0=v0)
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    A = P.kkt_matrix()
    b = P.rhs(vd, v0=v0)
    xs = layout.to_oracle_time(P, x.cpu().numpy().reshape(K, -1))
    assert info.relres <= 1e-8
    assert np.linalg.norm(b - A @ xs) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    xd, _ = P.reference_solution(b)
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) <= 1e-7
    G.close()


@pytest.mark.parametrize("kind", ["stokes", "oseen"])
def test_zero_data_gives_zero_solution(kind):
    P, G = make_pair(kind, 3, 4)
    G.set_data(np.zeros_like(inputs.desired_state(P.N, P.x0, P.x1, 4, P.tau, 1.0, seed=0)))
    x = torch.full((G.kkt_len,), 5.0, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    assert info.outer_iterations == 0 and info.relres == 0.0
    assert torch.count_nonzero(x).item() == 0
    G.close()


def test_solve_before_data_is_a_state_error():
    _, G = make_pair("stokes", 2, 2)
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PintError) as err:
        G.solve(x)
    assert err.value.code == 7
    G.close()


def test_nonfinite_data_is_rejected():
    P, G = make_pair("stokes", 2, 2)
    vd = inputs.desired_state(P.N, P.x0, P.x1, 2, P.tau, 1.0, seed=0)
    vd[1, 0, 7] = np.nan
    with pytest.raises(binding.PintError) as err:
        G.set_data(vd)
    assert err.value.code == 5
    G.close()


def test_outer_iteration_limit_reports_not_converged():
    P, G = make_pair("stokes", 3, 4, beta=1e-4, outer_maxit=1, outer_restart=1)
    G.set_data(inputs.desired_state(P.N, P.x0, P.x1, 4, P.tau, 1.0, seed=0))
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x, check=False)
    assert info.outer_iterations == 1 and info.relres > 1e-8
    code = binding.lib().pint_solve(G.h, ctypes.c_void_p(x.data_ptr()), ctypes.byref(binding.SolveInfo()))
    assert code == 4
    G.close()


def test_invalid_component_and_null_pointers():
    P, G = make_pair("stokes", 2, 4)
    J = G.sizes.J
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    lib = binding.lib()
    assert lib.pint_kkt_matvec(G.h, None, ctypes.c_void_p(x.data_ptr())) == 1
    assert lib.pint_apply_preconditioner(G.h, ctypes.c_void_p(x.data_ptr()), None) == 1
    assert lib.pint_kkt_matvec(None, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr())) == 1
    v = torch.zeros(P.grid.ns, dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.PintError) as err:
        G.component_apply(7, 0, v, v)
    assert err.value.code == 1
    with pytest.raises(binding.PintError) as err:
        G.component_apply("mg_W", J, v, v)
    assert err.value.code == 1 and "frequency" in str(err.value)
    with pytest.raises(binding.PintError) as err:
        G.component_apply("mg_Q", 0, v, v)          # Q_j exists for Oseen only
    assert err.value.code == 1
    G.close()


def test_dft_bounded_wait_reports_timeout_and_recovers():
    """The tensor-core DFT's pipeline waits are bounded: with a barrier that
    waits for bytes nobody sends, the call returns PINT_ERR_TIMEOUT within a
    few seconds, the handle stays usable, and the next call is correct."""
    P, G = make_pair("stokes", 3, 8, prec=1, dft_mode=2)
    x = inputs.random_vector((8, layout.block_len(P)), 3)
    x[:, ~layout.field_mask(P)] = 0.0
    xh = torch.zeros(G.freq_len, dtype=torch.complex128, device="cuda")
    G.debug_inject(1)
    with pytest.raises(binding.PintError) as err:
        G.dft_forward(to_dev(x.ravel()), xh)
    assert err.value.code == 6
    G.dft_forward(to_dev(x.ravel()), xh)
    ref = np.fft.fft(x, axis=0)[:5]
    assert relerr(xh.cpu().numpy().reshape(5, -1), ref) <= FP32_TOL
    # the injection needs a tensor-core DFT
    _, G64 = make_pair("stokes", 2, 2, prec=0)
    with pytest.raises(binding.PintError):
        G64.debug_inject(1)
    G.close()
    G64.close()
