"""Pins of the oracle's non-homogeneous Dirichlet right-hand side against the
closed-form solution of the Sec. 5.1 Stokes control problem.

For nu = 1 the paper states the state velocity and pressure that its desired
state and forcing produce; the adjoint follows from them by the optimality
conditions (lambda = beta u, u = v_t - Lap v + grad p - f), which gives
lambda = beta (e^{T-t} - 1) curl psi with psi = (x^2-1)^2 (y^2-1)^2 / 2.  The
discrete solution of Eq. FinalA with `rhs_dirichlet` must approach all three
as h and tau shrink; a dropped lift, a wrong sign in a block or in a lift
term, or a transposed coupling stops that, which the planted cases show.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.kkt import Problem
from paper_2405_18964_gb300 import inputs as I

T = 1.0


def _exact(P, K, tau, beta):
    xs, ys = I.q2_nodes(P.N, -1.0, 1.0)
    ts = (np.arange(K) + 1) * tau
    v = np.stack([I.stokes_mms_velocity(xs, ys, t, T) for t in ts])
    a, b = xs ** 2 - 1.0, ys ** 2 - 1.0
    curl = np.stack([2 * ys * a * a * b, -2 * xs * a * b * b])
    lam = np.stack([beta * (np.exp(T - t) - 1.0) * curl for t in ts])
    qx, qy = P.grid.q1_coords()
    p = np.stack([I.stokes_mms_pressure(qx, qy, t, T) for t in ts])
    return v, lam, p - p[:, :1]            # pressure pinned at Q1 node 0


def _errors(level, K, beta, plant=None):
    N, tau = 2 ** level, T / (K + 1)
    P = Problem("stokes", level, K, tau, beta, 1.0, x0=-1.0, x1=1.0)
    vd, f, v0, g = I.stokes_mms_data(N, K, tau, T, beta)
    A = P.kkt_matrix()
    b = P.rhs_dirichlet(vd, f, v0, g)
    if plant == "no lift":
        b = P.rhs_dirichlet(vd, f, v0, None)
    elif plant == "divergence lift sign":
        b = b.reshape(2, K, P.nb).copy()
        b[1, :, P.nv:] *= -1.0
        b = b.ravel()
    elif plant == "control sign":
        A = Problem("stokes", level, K, tau, -beta, 1.0, x0=-1.0, x1=1.0).kkt_matrix()
    elif plant == "transposed time coupling":
        A = P.kkt_matrix()
        n = K * P.nb
        A = A.tolil()
        A[:n, n:], A[n:, :n] = A[n:, :n], A[:n, n:]        # E <-> E^T (S_L = S_LT for Stokes)
        A = A.tocsr()
    x = spla.spsolve(A.tocsc(), b)
    v, lam, p = _exact(P, K, tau, beta)
    X = x.reshape(2, K, P.nb)
    ev = np.abs(P.full_velocity(x, g) - v).max() / np.abs(v).max()
    el = np.abs(X[1][:, :P.nv] - lam[:, :, P.vi].reshape(K, -1)).max() / np.abs(lam).max()
    ep = np.abs(X[0][:, P.nv:] - p[:, 1:]).max() / np.abs(p).max()
    return ev, el, ep


def test_manufactured_solution_convergence():
    beta = 1e-2
    e = [_errors(level, K, beta) for level, K in ((1, 3), (2, 7), (3, 15))]
    for a, b in zip(e, e[1:]):
        assert all(x1 < x0 / 4.0 for x0, x1 in zip(a, b)), e        # each error falls by > 4x per refinement
    ev, el, ep = e[-1]
    assert ev < 1e-3 and el < 2e-2 and ep < 5e-3, e[-1]


@pytest.mark.parametrize("plant", ["no lift", "divergence lift sign", "control sign", "transposed time coupling"])
def test_planted_mistakes_break_convergence(plant):
    good = _errors(2, 7, 1e-2)
    bad = _errors(2, 7, 1e-2, plant)
    assert max(b / g for b, g in zip(bad, good)) > 5.0, (plant, good, bad)      # observed >= 10x


def test_homogeneous_data_reduce_to_rhs():
    rng = np.random.default_rng(3)
    P = Problem("oseen", 2, 4, 0.2, 1e-3, 0.05, x0=-1.0, x1=1.0, wind="recirc")
    ns = P.grid.ns
    bnd = np.setdiff1d(np.arange(ns), P.vi)
    vd, f = rng.standard_normal((2, 4, 2, ns))
    v0 = rng.standard_normal((2, ns))
    for a in (vd, f):
        a[:, :, bnd] = 0.0
    v0[:, bnd] = 0.0
    assert np.allclose(P.rhs_dirichlet(vd, f, v0, None), P.rhs(vd, f, v0), rtol=0, atol=1e-14)
