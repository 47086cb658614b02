"""GPU: a caller-given nodal wind (pint_create_wind).  The recirculating
wind's values at the Q2 nodes reproduce the built-in wind exactly in exact
arithmetic (a quadratic is its own Q2 interpolant, on every grid level), so
the two handles must agree to rounding: preconditioner applies and solves.
Parity of the nodal path against the oracle for a non-polynomial wind runs
in test_gpu_parity.py (kind "oseen-nodal")."""
import numpy as np
import pytest

from gpu_pairs import FP32_TOL, make_pair, relerr, to_dev
from oracle import fem
from paper_2405_18964_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_nodal_recirculating_wind_equals_builtin(prec):
    K, level = 8, 3
    P, Gr = make_pair("oseen", level, K, beta=1e-3, prec=prec, fixed_inner_its=3)
    X, Y = P.grid.q2_coords()
    W = np.stack(fem.recirculating_wind(X, Y))
    pn = binding.default_params(**{f: getattr(Gr.params, f) for f, _ in binding.Params._fields_})
    pn.wind = 3
    Gn = binding.Problem(pn, stream=torch.cuda.current_stream().cuda_stream, wind=W)
    r = to_dev(inputs.random_vector(Gr.kkt_len, 31))
    zr = torch.zeros_like(r)
    zn = torch.zeros_like(r)
    Gr.apply_preconditioner(r, zr)
    Gn.apply_preconditioner(r, zn)
    assert relerr(zn.cpu().numpy(), zr.cpu().numpy()) <= (1e-12 if prec == 0 else FP32_TOL)
    yr, yn = torch.zeros_like(r), torch.zeros_like(r)
    Gr.kkt_matvec(r, yr)
    Gn.kkt_matvec(r, yn)
    assert relerr(yn.cpu().numpy(), yr.cpu().numpy()) <= 1e-13
    Gr.close()
    Gn.close()
    # tolerance-driven solves: same outer count, solutions within the solve's accuracy
    pr = binding.default_params(kind=1, level=level, n_t=K, tau=P.tau, beta=1e-3, nu=1e-2, x0=-1.0, x1=1.0,
                                wind=1, prec=prec)
    pn = binding.default_params(kind=1, level=level, n_t=K, tau=P.tau, beta=1e-3, nu=1e-2, x0=-1.0, x1=1.0,
                                wind=3, prec=prec)
    vd = inputs.desired_state(P.N, -1.0, 1.0, K, P.tau, 1.0, seed=3)
    out = []
    for params, w in ((pr, None), (pn, W)):
        G = binding.Problem(params, stream=torch.cuda.current_stream().cuda_stream, wind=w)
        G.set_data(vd)
        x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
        info = G.solve(x)
        out.append((info.outer_iterations, x.cpu().numpy()))
        G.close()
    assert abs(out[0][0] - out[1][0]) <= 1
    assert relerr(out[1][1], out[0][1]) <= 1e-7
