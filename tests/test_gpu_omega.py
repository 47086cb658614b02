"""GPU: under-relaxed multicolour SOR (sor_omega < 1), the remedy for the
convection-dominated Q_j of the recirculating wind at beta >= 1e-2, where
Gauss-Seidel smoothing diverges.  The whole preconditioner apply against the
oracle at the same omega, and a solve that converges only with it."""
import numpy as np
import pytest

from gpu_pairs import FP64_TOL, make_pair, relerr, settings_of, to_dev
from oracle import inexact, layout
from paper_2405_18964_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("kind", ["stokes", "oseen"])
def test_apply_with_damped_sor_matches_oracle(kind):
    K = 8
    P, G = make_pair(kind, 3, K, beta=1e-2, sor_omega=0.7, fixed_inner_its=3)
    assert abs(G.params.sor_omega - 0.7) < 1e-15
    pc = inexact.PinTPreconditioner(P, settings_of(G), fixed_inner_its=3)
    r = inputs.random_vector(G.kkt_len, 41)
    z = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    G.apply_preconditioner(to_dev(r), z)
    zo = pc(layout.to_oracle_time(P, r.reshape(K, -1)))
    assert relerr(layout.to_oracle_time(P, z.cpu().numpy().reshape(K, -1)), zo) <= FP64_TOL
    G.close()


def test_recirculating_wind_at_beta_1e2_converges_with_damped_sor():
    """32x32, n_t = 8, nu = 1/100, beta = 1e-2, FP32 preconditioner,
    FGMRES(10): the oracle needs 16 iterations with omega = 0.7."""
    K = 8
    tau = 1.0 / (K + 1)
    p = binding.default_params(kind=1, level=5, n_t=K, tau=tau, beta=1e-2, nu=1e-2, x0=-1.0, x1=1.0, wind=1,
                               prec=1, sor_omega=0.7, outer_restart=10, outer_maxit=60)
    G = binding.Problem(p, stream=torch.cuda.current_stream().cuda_stream)
    G.set_data(inputs.desired_state(32, -1.0, 1.0, K, tau, 1.0, seed=0))
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    G.close()
    assert info.relres <= 1e-8 and info.outer_iterations <= 20, (info.outer_iterations, info.relres)
