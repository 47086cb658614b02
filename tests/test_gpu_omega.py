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


def test_damped_convection_multigrid_matches_oracle():
    """sor_omega_conv damps only the multigrids of Q_j and Q_j^H: on the GPU
    they match the oracle's (Settings.sor_omega_conv) to the FP64 bar, and
    the pressure multigrid keeps sor_omega = 1."""
    K = 8
    P, G = make_pair("oseen", 4, K, beta=1e-2, sor_omega_conv=0.5)
    s = settings_of(G)
    assert s.sor_omega_conv == 0.5 and s.sor_omega == 1.0
    for j in (0, 1, K // 2):
        blk = inexact.OseenBlockPreconditioner(P, j, s)
        for name, mg in (("mg_Q", blk.mgQ), ("mg_QH", blk.mgQH), ("mg_Kp", blk.mgKp)):
            q1 = name == "mg_Kp"
            n = P.grid.nq if q1 else P.grid.ns
            idx = P.pf if q1 else P.vi
            x = inputs.random_vector(n, 31 + j, np.complex128)
            y = torch.zeros(n, dtype=torch.complex128, device="cuda")
            G.component_apply(name, j, to_dev(x, "complex128"), y)
            ref = mg.solve(x[idx], s.mg_cycles)
            assert relerr(y.cpu().numpy()[idx], ref) <= FP64_TOL, (name, j)
    G.close()


def _golden_count():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "damped_oseen_count.txt")
    vals = dict(ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#"))
    return int(vals["outer_iterations"])


def test_recirculating_wind_at_beta_1e2_with_damped_convection_multigrids():
    """32x32, n_t = 16, nu = 1/100, beta = 1e-2, recirculating wind, FP32
    preconditioner, FGMRES(10), sor_omega_conv = 0.5 (K_p undamped): the
    solve converges and its outer count is within one of the oracle's
    (tests/golden/damped_oseen_count.txt, written by the oracle alone)."""
    K = 16
    tau = 1.0 / (K + 1)
    p = binding.default_params(kind=1, level=5, n_t=K, tau=tau, beta=1e-2, nu=1e-2, x0=-1.0, x1=1.0, wind=1,
                               prec=1, sor_omega_conv=0.5, outer_restart=10, outer_maxit=80)
    G = binding.Problem(p, stream=torch.cuda.current_stream().cuda_stream)
    G.set_data(inputs.desired_state(32, -1.0, 1.0, K, tau, 1.0, seed=0))
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    G.close()
    ref = _golden_count()
    print(f"damped convection multigrids: GPU {info.outer_iterations} its, oracle {ref}")
    assert info.relres <= 1e-8 and abs(info.outer_iterations - ref) <= 1, (info.outer_iterations, ref, info.relres)
