"""The FP32 emulation of the nested preconditioner (tests/fp32_emulation.py)
is the oracle's method step for step: run in FP64 storage and arithmetic it
reproduces the oracle's frequency-block solves to rounding, and in FP32 it
moves them by an FP32-sized amount."""
import numpy as np
import pytest

import fp32_emulation as E
from oracle import inexact, kkt


def _max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("kind", ["stokes", "oseen"])
def test_emulation_in_fp64_is_the_oracle(kind, monkeypatch):
    monkeypatch.setattr(E, "C64", np.complex128)
    monkeypatch.setattr(E, "F32", np.float64)
    K = 8
    x0, wind = (0.0, None) if kind == "stokes" else (-1.0, "recirc")
    P = kkt.Problem(kind, 3, K, 1 / (K + 1), 1e-3, 1e-2, x0, 1.0, wind)
    pc = inexact.PinTPreconditioner(P, fixed_inner_its=3)
    em = E.PinT32(P, fixed_inner_its=3)
    rng = np.random.default_rng(3)
    nn = 2 * P.nv + 2 * P.np_
    for j in (0, 1, K // 2):
        g = rng.standard_normal(nn) + 1j * rng.standard_normal(nn)
        assert _max_rel(em.solve_block(j, g), pc.solve_block(j, g)) <= 1e-11, j


def test_emulation_in_fp32_differs_by_fp32_rounding():
    K = 8
    P = kkt.Problem("stokes", 3, K, 1 / (K + 1), 1e-3, 1e-2, 0.0, 1.0, None)
    pc = inexact.PinTPreconditioner(P, fixed_inner_its=3)
    em = E.PinT32(P, fixed_inner_its=3)
    g = np.random.default_rng(4).standard_normal(2 * P.nv + 2 * P.np_) + 0j
    err = _max_rel(em.solve_block(1, g), pc.solve_block(1, g))
    assert 1e-9 < err < 1e-4
