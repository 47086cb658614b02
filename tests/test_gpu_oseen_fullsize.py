"""GPU parity at the Oseen workload size: 128 x 128 Q2-Q1 on [-1,1]^2,
n_t = 128, nu = 1/100, recirculating wind, beta = 1e-4 (the commutator-based
Schur approximation, Algorithm 3 inside the inner GMRES).

As for the Stokes benchmark size, the oracle evaluates only what it can one
piece at a time: every block row of the Eq. FinalA matvec, the DFT of every
column, sampled frequency-block solves, and the true residual of a full
solve recomputed row by row.
"""
import numpy as np
import pytest

from gpu_pairs import (FP32_TOL, FP64_TOL, KP_FP64_TOL, FP32_EMU_FACTOR, fp32_emulated_solves, freq_blocks, make_pair, part_errors,
                       relerr, settings_of, to_dev)
from oracle import inexact, layout
from paper_2405_18964_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

LEVEL, K, NU, BETA = 7, 128, 1e-2, 1e-4
J = K // 2 + 1


def _pair(prec, **kw):
    return make_pair("oseen", LEVEL, K, beta=BETA, nu=NU, prec=prec, **kw)


def test_oseen_kkt_matvec_full_size():
    P, G = _pair(0)
    x = inputs.random_vector(G.kkt_len, 21)
    y = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    G.kkt_matvec(to_dev(x), y)
    xo = layout.to_oracle_time(P, x.reshape(K, -1))
    yo = np.concatenate([v for _, v in sorted(P.kkt_rows(xo, range(2 * K)).items())])
    assert relerr(layout.to_oracle_time(P, y.cpu().numpy().reshape(K, -1)), yo) <= 1e-13
    G.close()


@pytest.mark.parametrize("prec,dft_mode", [(0, 0), (1, 2), (1, 3)], ids=["fp64", "fp32-bf16x6", "fp32-tf32x3"])
def test_oseen_dft_full_size(prec, dft_mode):
    P, G = _pair(prec, dft_mode=dft_mode)
    x = inputs.random_vector((K, layout.block_len(P)), 22)
    x[:, ~layout.field_mask(P)] = 0.0
    xh = torch.zeros(G.freq_len, dtype=torch.complex128, device="cuda")
    G.dft_forward(to_dev(x.ravel()), xh)
    ref = np.fft.fft(x, axis=0)[:J]
    tol = 1e-13 if prec == 0 else FP32_TOL
    assert relerr(xh.cpu().numpy().reshape(J, -1), ref) <= tol
    y = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    G.dft_inverse(to_dev(ref.ravel(), "complex128"), y)
    assert relerr(y.cpu().numpy().reshape(K, -1), x) <= tol
    G.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_oseen_frequency_block_solves_full_size(prec):
    """All J blocks in one call with two inner steps each (Algorithm 3 as the
    inner preconditioner); sampled blocks against the oracle."""
    P, G = _pair(prec, fixed_inner_its=2)
    rh = inputs.random_vector((J, layout.block_len(P)), 44, np.complex128)
    yh = torch.zeros(G.freq_len, dtype=torch.complex128, device="cuda")
    its = G.freq_block_solve(to_dev(rh.ravel(), "complex128"), yh)
    assert all(i == 2 for i in its)
    got = freq_blocks(P, yh.cpu().numpy())
    rs = freq_blocks(P, rh)
    sample = [1, J - 1]
    pc = inexact.PinTPreconditioner(P, settings_of(G), fixed_inner_its=2)
    emu = fp32_emulated_solves(P, settings_of(G), sample, rs, 2) if prec else {}
    for j in sample:
        ref = pc.solve_block(j, rs[j])
        if prec:
            e, e_emu = relerr(got[j], ref), relerr(emu[j], ref)
            bar = max(FP32_TOL, FP32_EMU_FACTOR * e_emu)
            print(f"Oseen block solve j={j} FP32: GPU {e:.3e}, FP32 emulation {e_emu:.3e}, bar {bar:.3e}")
            assert e <= bar, (j, e, bar)
        else:
            e = part_errors(P, got[j], ref)
            assert max(e["v"], e["lam"]) <= FP64_TOL and max(e["p"], e["mu"]) <= KP_FP64_TOL, (j, e)
    G.close()


def test_oseen_solve_full_size_fp32():
    """FP32-preconditioned solve to 1e-8: the true residual recomputed by the
    oracle's block rows meets the tolerance."""
    P, G = _pair(1)
    vd = inputs.desired_state(P.N, P.x0, P.x1, K, P.tau, 1.0, seed=0)
    G.set_data(vd)
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    assert info.relres <= 1e-8
    xs = layout.to_oracle_time(P, x.cpu().numpy().reshape(K, -1))
    b = P.rhs(vd)
    rows = P.kkt_rows(xs, range(2 * K))
    r = b.reshape(2 * K, P.nb).copy()
    for i, v in rows.items():
        r[i] -= v
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8 * (1 + 1e-6)
    G.close()
