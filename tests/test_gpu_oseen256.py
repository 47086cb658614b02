"""GPU parity at the large Oseen size: 256 x 256 Q2-Q1 on [-1,1]^2, n_t = 128,
nu = 1/500, recirculating wind, beta = 1e-6, FGMRES(20) with the FP64 basis
and the FP32 preconditioner (Algorithm 3 inside the inner GMRES).

The oracle solves sampled frequency blocks one at a time (about a minute
each at this size) and recomputes the true residual of a whole solve block
row by block row.  The FP32 block solves are held to max(1e-5, 3 x the
distance of the method executed in FP32, tests/fp32_emulation.py): at this
size two inner GMRES steps amplify FP32 rounding (6e-8) by ~1300x, the
emulation lands 8.0e-5 from the FP64 oracle at j = 1, and the GPU 1.7e-4
(2.2x): its block matvec evaluates the M, K and N terms separately from FP32
1-D bands and combines them, where the emulation rounds each combined matrix
entry once (at 128 x 128, nu = 1/100 the two agree within 1.3x).
"""
import numpy as np
import pytest

from gpu_pairs import FP32_TOL, fp32_emulated_solves, freq_blocks, make_pair, relerr, settings_of, to_dev
from oracle import inexact, layout
from paper_2405_18964_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

LEVEL, K, NU, BETA = 8, 128, 1.0 / 500.0, 1e-6
J = K // 2 + 1
EMU_FACTOR = 3.0


def test_oseen256_frequency_block_solves():
    """All 65 blocks in one call with two inner steps each; blocks j = 1 and
    j = K/2 against the oracle."""
    P, G = make_pair("oseen", LEVEL, K, beta=BETA, nu=NU, prec=1, fixed_inner_its=2, outer_restart=20)
    rh = inputs.random_vector((J, layout.block_len(P)), 45, np.complex128)
    yh = torch.zeros(G.freq_len, dtype=torch.complex128, device="cuda")
    its = G.freq_block_solve(to_dev(rh.ravel(), "complex128"), yh)
    assert all(i == 2 for i in its)
    got = freq_blocks(P, yh.cpu().numpy())
    G.close()
    rs = freq_blocks(P, rh)
    sample = [1, J - 1]
    s = settings_of(G)
    pc = inexact.PinTPreconditioner(P, s, fixed_inner_its=2)
    emu = fp32_emulated_solves(P, s, sample, rs, 2)
    for j in sample:
        ref = pc.solve_block(j, rs[j])
        e, e_emu = relerr(got[j], ref), relerr(emu[j], ref)
        bar = max(FP32_TOL, EMU_FACTOR * e_emu)
        print(f"Oseen 256 block solve j={j} FP32: GPU {e:.3e}, FP32 emulation {e_emu:.3e}, bar {bar:.3e}")
        assert e <= bar, (j, e, bar)


def test_oseen256_solve_fp32_fgmres20():
    """FP32-preconditioned FGMRES(20) to 1e-8 (inner GMRES capped at 40, the
    bench's setting for this size): the true residual recomputed by the
    oracle's block rows meets the tolerance."""
    P, G = make_pair("oseen", LEVEL, K, beta=BETA, nu=NU, prec=1, outer_restart=20, inner_maxit=40)
    vd = inputs.desired_state(P.N, P.x0, P.x1, K, P.tau, 1.0, seed=0)
    G.set_data(vd)
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    G.close()
    print(f"Oseen 256 solve: {info.outer_iterations} outer iterations, relres {info.relres:.2e}")
    assert info.relres <= 1e-8
    xs = layout.to_oracle_time(P, x.cpu().numpy().reshape(K, -1))
    b = P.rhs(vd)
    rows = P.kkt_rows(xs, range(2 * K))
    r = b.reshape(2 * K, P.nb).copy()
    for i, v in rows.items():
        r[i] -= v
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8 * (1 + 1e-6)
