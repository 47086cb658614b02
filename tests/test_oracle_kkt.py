"""Pins for the oracle's KKT system and exact block-circulant preconditioner."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import inexact, kkt, layout
from oracle_golden import paper_bounds
from paper_2405_18964_gb300 import inputs


def stokes(level=1, K=3, beta=1e-2, tau=0.25):
    return kkt.Problem("stokes", level, K, tau, beta, 1e-2, 0.0, 1.0, None)


def oseen(level=1, K=3, beta=1e-3, tau=0.25, nu=1e-2, wind="recirc"):
    return kkt.Problem("oseen", level, K, tau, beta, nu, -1.0, 1.0, wind)


CASES = [stokes(1, 3), stokes(2, 4), oseen(1, 3), oseen(2, 4), oseen(2, 4, wind="two_vortex")]


@pytest.mark.parametrize("P", CASES, ids=lambda P: f"{P.kind}-{P.wind}-L{P.level}-K{P.K}")
def test_kkt_symmetric(P):
    A = P.kkt_matrix()
    assert abs(A - A.T).max() == 0.0


def _objective(P, v, u, vd):
    """J of Eq. OseenOptimization with the rectangle rule at t_k = k tau."""
    J = 0.0
    for k in range(P.K):
        e = v[k] - vd[k]
        J += 0.5 * P.tau * e @ (P.Mv @ e) + 0.5 * P.beta * P.tau * u[k] @ (P.Mv @ u[k])
    return J


def _forward(P, u, v0=None):
    """Backward-Euler state equation (Sec. 2.2) for a given control u."""
    S = sp.bmat([[P.Mv + P.tau * P.Lv, P.tau * P.Bv.T], [P.tau * P.Bv, None]], format="csc")
    lu = spla.splu(S)
    v = np.zeros((P.K, P.nv))
    prev = np.zeros(P.nv) if v0 is None else v0
    for k in range(P.K):
        rhs = np.concatenate([P.Mv @ prev + P.tau * (P.Mv @ u[k]), np.zeros(P.np_)])
        v[k] = lu.solve(rhs)[:P.nv]
        prev = v[k]
    return v


@pytest.mark.parametrize("P", [stokes(1, 3), stokes(2, 5), oseen(1, 4), oseen(2, 3),
                               oseen(2, 3, wind="two_vortex")],
                         ids=lambda P: f"{P.kind}-{P.wind}-L{P.level}-K{P.K}")
def test_kkt_solution_minimises_the_control_objective(P):
    """The solution of A x = b must be the minimiser of J subject to the
    discrete state equation, with u = lambda / beta (Sec. 2.1-2.2): this pins
    signs, tau scalings, E vs E^T and the right-hand side against the
    optimisation problem itself."""
    vd_full = inputs.desired_state(P.N, P.x0, P.x1, P.K, P.tau, P.tau * (P.K + 1), seed=3)
    b = P.rhs(vd_full)
    x = spla.spsolve(P.kkt_matrix().tocsc(), b)
    X = x.reshape(2, P.K, P.nb)
    v = X[0, :, :P.nv]
    lam = X[1, :, :P.nv]
    u = lam / P.beta
    vd = np.stack([np.concatenate([vd_full[k, 0, P.vi], vd_full[k, 1, P.vi]]) for k in range(P.K)])
    v_fw = _forward(P, u)
    np.testing.assert_allclose(v_fw, v, atol=1e-10 * np.abs(v).max())
    J0 = _objective(P, v, u, vd)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.standard_normal(u.shape) * np.abs(u).max()
        Jp = _objective(P, _forward(P, u + d), u + d, vd)
        Jm = _objective(P, _forward(P, u - d), u - d, vd)
        lin = 0.5 * (Jp - Jm)
        quad = 0.5 * (Jp + Jm) - J0
        assert quad > 0
        assert abs(lin) <= 1e-8 * (J0 + quad)
    # a sign error would be caught: the control lambda (not -lambda) is optimal
    Jw = _objective(P, _forward(P, -u), -u, vd)
    assert Jw > J0 * (1 + 1e-6)


@pytest.mark.parametrize("P", CASES, ids=lambda P: f"{P.kind}-{P.wind}-L{P.level}-K{P.K}")
def test_circulant_identity_and_real_output(P):
    r = np.random.default_rng(1).standard_normal(P.n)
    z, Y = P.pc_inverse(r)
    z_dense = spla.spsolve(P.kkt_matrix(circulant=True).tocsc(), r)
    assert np.linalg.norm(z - z_dense) <= 1e-12 * np.linalg.norm(z_dense)
    assert np.abs(Y.imag).max() <= 1e-12 * np.abs(Y).max()


@pytest.mark.parametrize("P", CASES, ids=lambda P: f"{P.kind}-{P.wind}-L{P.level}-K{P.K}")
def test_hermitian_pairing(P):
    r = np.random.default_rng(2).standard_normal(P.n).reshape(2, P.K, P.nb)
    Rh = np.fft.fft(r, axis=1)
    for j in range(1, P.K):
        np.testing.assert_allclose(Rh[:, P.K - j], np.conj(Rh[:, j]), atol=1e-12)
        assert abs(P.G(P.K - j) - P.G(j).conj()).max() < 1e-14
    assert abs(P.d(0)) == 0.0


@pytest.mark.parametrize("P", CASES, ids=lambda P: f"{P.kind}-{P.wind}-L{P.level}-K{P.K}")
def test_perturbation_rank(P):
    D = (P.kkt_matrix() - P.kkt_matrix(circulant=True)).toarray()
    assert np.linalg.matrix_rank(D) == 2 * P.nv


@pytest.mark.parametrize("P", [stokes(1, 3), oseen(1, 3), stokes(1, 4)], ids=lambda P: f"{P.kind}-K{P.K}")
def test_theorem1_eigenvalue_count(P):
    """Theorem 1: #{eig(P_C^{-1} A) = 1} >= 2 K (n_v + n_p) - 2 n_v (K blocks)."""
    A = P.kkt_matrix().toarray()
    PC = P.kkt_matrix(circulant=True).toarray()
    ev = np.linalg.eigvals(np.linalg.solve(PC, A))
    n_one = int(np.sum(np.abs(ev - 1.0) < 1e-6))
    assert n_one >= 2 * P.K * (P.nv + P.np_) - 2 * P.nv


@pytest.mark.parametrize("P", [stokes(1, 3), stokes(2, 4), oseen(1, 4), oseen(2, 3)],
                         ids=lambda P: f"{P.kind}-L{P.level}-K{P.K}")
def test_fgmres_exact_pc_matches_dense_solve(P):
    r = np.random.default_rng(4).standard_normal(P.n)
    A = P.kkt_matrix()
    x, info = kkt.fgmres(A, r, lambda v: P.pc_inverse(v)[0], tol=1e-12, restart=30)
    xd = np.linalg.solve(A.toarray(), r)
    assert info["relres"] <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    # Theorem 1 bounds the Krylov dimension by 2 n_v + 1
    assert info["its"] <= 2 * P.nv + 1


@pytest.mark.parametrize("K", [3, 4, 8])
def test_stokes_transform_identity(K):
    """G_j = T_j^l Z_j T_j^r with c_{j,1} read as d_r / sqrt(tau^2/beta + d_c^2)."""
    P = stokes(1, K, beta=1e-2, tau=0.3)
    for j in range(K):
        Tl, Tr = inexact.T_matrices(P, j)
        Gt = (Tl @ inexact.Z_matrix(P, j) @ Tr).toarray()
        G = P.G(j).toarray()
        assert np.abs(Gt - G).max() <= 1e-13 * np.abs(G).max()
        # the inverse transforms undo T^l and T^r
        u = np.random.default_rng(j).standard_normal(G.shape[0]) + 0j
        np.testing.assert_allclose(inexact.Tl_inverse(P, j, Tl @ u), u, atol=1e-12)
        np.testing.assert_allclose(inexact.Tr_inverse(P, j, Tr @ u), u, atol=1e-12)


def test_printed_c1_fails_the_identity():
    """The c_{j,1} printed without the square does not reproduce G_j: this
    documents reading R4 (the test fails if the reading were unnecessary)."""
    P = stokes(1, 8, beta=1e-2, tau=0.3)
    bad = 0
    for j in range(1, 8):
        d = P.d(j)
        c1_printed = d.real / np.sqrt(P.tau ** 2 / P.beta + d.imag)
        _, _, _, c1, c2 = inexact.stokes_constants(P, j)
        if abs(d.imag) > 1e-12 and abs(c1 - c1_printed) > 1e-6:
            bad += 1
    assert bad > 0


@pytest.mark.parametrize("j", [0, 1, 2])
def test_hat_Pj_eigenvalue_bounds(j):
    """Eq. SchurComplementHatBounds: |lambda(P^_j^{-1} Z_j)| in [1/sqrt(12), (1+sqrt(5))/2]."""
    g = paper_bounds()
    P = stokes(2, 4, beta=1e-2, tau=0.2)
    _, _, _, c1, c2 = inexact.stokes_constants(P, j)
    W = ((1 + c1) * P.Mv + c2 * P.Lv).toarray()
    B = P.Bv.toarray()
    S = B @ np.linalg.solve(W, B.T)
    Ph = np.zeros((2 * P.nv + 2 * P.np_,) * 2)
    nv, npp = P.nv, P.np_
    Ph[:nv, :nv] = W
    Ph[nv:2 * nv, nv:2 * nv] = W
    Ph[2 * nv:2 * nv + npp, 2 * nv:2 * nv + npp] = S
    Ph[2 * nv + npp:, 2 * nv + npp:] = S
    ev = np.abs(np.linalg.eigvals(np.linalg.solve(Ph, inexact.Z_matrix(P, j).toarray())))
    assert ev.min() >= g["hat_P_j_abs_lower"] - 1e-10
    assert ev.max() <= g["hat_P_j_abs_upper"] + 1e-10


@pytest.mark.parametrize("wind", ["recirc", "two_vortex"])
@pytest.mark.parametrize("j", [0, 1, 3])
def test_pearson_wathen_bounds_complex(j, wind):
    """lambda(S^^{-1} S) in [1/2, 1] for the Oseen (1,1) block (Sec. 2.3, Sec. 4);
    the bound needs L + L^T = 2 nu K (skew N), which the skew-symmetric form
    of the two-vortex wind keeps."""
    g = paper_bounds()
    P = oseen(2, 6, beta=1e-3, tau=0.2, wind=wind)
    t, b = P.tau, P.beta
    d = P.d(j)
    M = P.Mv.toarray()
    L = P.Lv.toarray()
    Psi = d * M + t * L
    S = (t / b) * M + Psi @ np.linalg.solve(t * M, Psi.conj().T)
    Q = Psi + (t / np.sqrt(b)) * M
    Sh = Q @ np.linalg.solve(M, Q.conj().T) / t
    ev = np.linalg.eigvals(np.linalg.solve(Sh, S))
    assert np.abs(ev.imag).max() < 1e-8
    assert ev.real.min() >= g["pearson_wathen_lower"] - 1e-10
    assert ev.real.max() <= g["pearson_wathen_upper"] + 1e-10


def test_layout_roundtrip():
    P = stokes(2, 3)
    x = np.random.default_rng(5).standard_normal(P.n)
    X = layout.from_oracle_time(P, x)
    assert X.shape == (P.K, layout.block_len(P))
    np.testing.assert_array_equal(layout.to_oracle_time(P, X), x)
    g = np.random.default_rng(6).standard_normal(P.nb * 2) + 0j
    np.testing.assert_array_equal(layout.to_oracle_freq(P, layout.from_oracle_freq(P, g)), g)
    assert layout.field_mask(P).sum() == P.nb * 2


@pytest.mark.parametrize("P", [stokes(2, 5), oseen(2, 4)], ids=lambda P: f"{P.kind}")
def test_kkt_rows_match_assembled_matrix(P):
    """The row-wise evaluation used for full-size sampled checks agrees with
    the assembled Eq. FinalA."""
    x = np.random.default_rng(8).standard_normal(P.n)
    y = P.kkt_matrix() @ x
    rows = [0, 1, P.K - 1, P.K, 2 * P.K - 1]
    got = P.kkt_rows(x, rows)
    for r in rows:
        np.testing.assert_allclose(got[r], y[r * P.nb:(r + 1) * P.nb], rtol=1e-13, atol=1e-13 * np.abs(y).max())
