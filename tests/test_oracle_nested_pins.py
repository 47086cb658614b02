"""Pins of the oracle's nested iterations against their definitions written
as explicit matrix iterations (dense, tiny grids).

* Multigrid (Sec. 3.4; reading R13): one V-cycle from a zero initial guess
  is x = (I - E) A^{-1} b with the error propagation
      E_l = S_post (I - P B_{l+1} P^T A_l) S_pre,   B_{l+1} = (I - E_{l+1}) A_{l+1}^{-1},
  B = A^{-1} on the coarsest grid, S_pre = (S_last ... S_1 S_0)^pre and
  S_post = (S_0 S_1 ... S_last)^post with the colour updates
  S_c = I - omega Pi_c D^{-1} A (Pi_c selects the nodes of colour c, D the
  diagonal), so c cycles give (I - E^c) A^{-1} b.  The matrices are formed
  here from the assembled operators, the colours of the node coordinates and
  the nested interpolation; the oracle's Multigrid.solve must reproduce them
  column by column.  A reversed sweep order, a wrong omega, a wrong transfer
  or a dropped coarse correction changes them.
* Chebyshev semi-iteration (Sec. 3.4, Jacobi-Chebyshev on the mass
  matrices): from x = 0 the error after k steps is
      x* - x_k = T_k(sigma I - D^{-1} A / delta) / T_k(sigma) x*,
  sigma = theta / delta, T_k the Chebyshev polynomial; the matrix polynomial
  is built here by its three-term recurrence on dense matrices and must
  reproduce the oracle's vector recurrence for every k.
* Uzawa (Eq. Uzawa11): the two-line update is the block iteration
  x <- x + Pc^{-1} (b - G^(1,1) x) with Pc = [[tau Mhat, 0], [d_j M + tau L,
  -mu Shat]], G^(1,1) = [[tau M, (d_j M + tau L)^H], [d_j M + tau L,
  -(tau/beta) M]], from x = 0; Mhat^{-1} and Shat^{-1} are substituted by the
  dense matrices of the oracle's Chebyshev and tau Q^{-H} M Q^{-1} pieces.
"""
import numpy as np
import pytest

from oracle import fem, inexact, kkt


def _colour_masks(free, n1, ncol):
    ix, iy = free % n1, free // n1
    col = (ix % ncol) + ncol * (iy % ncol)
    return [np.diag((col == c).astype(float)) for c in range(ncol * ncol)]


def _levels(space, level, x0, x1, wind, aM, aK, aN, transpose_n=False):
    """Dense A_l, colour masks and prolongations (fine l <- coarse l+1)."""
    out = []
    for lv in range(level, 0, -1):
        N = 2 ** lv
        wf, skew = fem.wind_by_name(wind, N, x0, x1)
        o = fem.assemble(N, x0, x1, wf, skew=skew)
        if space == "q2":
            Nc = o.N.T if transpose_n else o.N
            A = aM * o.M + aK * o.K + aN * Nc
            free, n1, ncol = o.grid.velocity_interior(), o.grid.n2, 3
        else:
            A = aM * o.Mp + aK * o.Kp + aN * o.Np
            free, n1, ncol = o.grid.pressure_free(), o.grid.n1, 2
        out.append({"N": N, "A": A.toarray()[np.ix_(free, free)], "free": free,
                    "Pi": _colour_masks(free, n1, ncol)})
    for l in range(len(out) - 1):
        Pf = fem.prolongation_2d(out[l + 1]["N"], 2 if space == "q2" else 1).toarray()
        out[l]["P"] = Pf[np.ix_(out[l]["free"], out[l + 1]["free"])]
    return out


def _vcycle_operator(lev, l, omega, pre, post, post_forward=False):
    """B_l with x = B_l b for one V-cycle from x = 0 (post_forward: the
    post-sweeps in colour order 0..last, a mistake the pin must catch)."""
    A = lev[l]["A"]
    n = A.shape[0]
    if l == len(lev) - 1:
        return np.linalg.inv(A)
    Dinv = np.diag(1.0 / np.diag(A))
    S = [np.eye(n) - omega * Pi @ Dinv @ A for Pi in lev[l]["Pi"]]
    sweep_fwd = np.eye(n)
    for Sc in S:                      # colour 0 first
        sweep_fwd = Sc @ sweep_fwd
    sweep_bwd = np.eye(n)
    for Sc in reversed(S):            # last colour first
        sweep_bwd = Sc @ sweep_bwd
    Spre = np.linalg.matrix_power(sweep_fwd, pre)
    Spost = np.linalg.matrix_power(sweep_fwd if post_forward else sweep_bwd, post)
    P = lev[l]["P"]
    Bc = _vcycle_operator(lev, l + 1, omega, pre, post, post_forward)
    E = Spost @ (np.eye(n) - P @ Bc @ P.T @ A) @ Spre
    return (np.eye(n) - E) @ np.linalg.inv(A)


def _mg_matrix(mg, n, cycles):
    return np.column_stack([mg.solve(np.eye(n)[:, k].astype(complex), cycles) for k in range(n)])


CASES = [
    # space, wind, aM, aK, aN, omega, pre, post
    ("q2", None, 1.3, 0.02, 0.0, 1.0, 2, 2),                       # W_j (Stokes)
    ("q1", None, 0.0, 1.0, 0.0, 1.0, 2, 2),                        # K_p (pinned corner)
    ("q2", "recirc", 0.2 + 0.7j, 1e-3, 0.05, 0.7, 2, 2),           # Q_j, damped
    ("q2", "recirc", 0.4 - 0.3j, 1e-2, 0.1, 1.0, 1, 3),            # Q_j, uneven sweeps
]


@pytest.mark.parametrize("space,wind,aM,aK,aN,omega,pre,post", CASES,
                         ids=["W", "Kp", "Q-damped", "Q-1-3"])
def test_multigrid_is_its_error_propagation_operator(space, wind, aM, aK, aN, omega, pre, post):
    level = 3                                                      # grids 8, 4, 2
    x0 = -1.0 if wind else 0.0
    mg = inexact.Multigrid(space, level, x0, 1.0, wind, aM, aK, aN, pre, post, omega)
    lev = _levels(space, level, x0, 1.0, wind, aM, aK, aN)
    n = lev[0]["A"].shape[0]
    B = _vcycle_operator(lev, 0, omega, pre, post)
    A = lev[0]["A"]
    E = np.eye(n) - B @ A
    for cycles in (1, 3):
        ref = (np.eye(n) - np.linalg.matrix_power(E, cycles)) @ np.linalg.inv(A)
        got = _mg_matrix(mg, n, cycles)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), cycles


def test_multigrid_of_q_hermitian_uses_the_transposed_convection():
    """The Q_j^H multigrid of the Oseen block (N^T, conjugate mass shift)
    against its error propagation built from N^T."""
    K = 4
    P = kkt.Problem("oseen", 3, K, 0.2, 1e-3, 1e-2, -1.0, 1.0, "recirc")
    s = inexact.Settings(sor_omega_conv=0.8)
    blk = inexact.OseenBlockPreconditioner(P, 1, s)
    aQ = P.d(1) + P.tau / np.sqrt(P.beta)
    lev = _levels("q2", 3, -1.0, 1.0, "recirc", np.conj(aQ), P.tau * P.nu, P.tau, transpose_n=True)
    n = lev[0]["A"].shape[0]
    B = _vcycle_operator(lev, 0, 0.8, s.mg_pre, s.mg_post)
    E = np.eye(n) - B @ lev[0]["A"]
    ref = (np.eye(n) - np.linalg.matrix_power(E, s.mg_cycles)) @ np.linalg.inv(lev[0]["A"])
    got = _mg_matrix(blk.mgQH, n, s.mg_cycles)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("j", [0, 1, 2])
def test_uzawa_is_the_block_iteration_of_eq_uzawa11(j):
    K = 4
    P = kkt.Problem("oseen", 2, K, 0.2, 1e-3, 1e-2, -1.0, 1.0, "recirc")
    nv, t, be = P.nv, P.tau, P.beta
    I = np.eye(nv)
    M = P.Mv.toarray()
    Psi = P.d(j) * M + t * P.Lv.toarray()
    G11 = np.block([[t * M, Psi.conj().T], [Psi, -(t / be) * M]])
    rng = np.random.default_rng(j)
    b = rng.standard_normal(2 * nv) + 1j * rng.standard_normal(2 * nv)
    for steps in (1, 5):
        s = inexact.Settings(uzawa_steps=steps)
        blk = inexact.OseenBlockPreconditioner(P, j, s)
        mu = s.uzawa_mu
        Mhat_inv = np.column_stack([blk.M_hat_inv(I[:, k].astype(complex)) for k in range(nv)])
        Shat_inv = np.column_stack([blk.S11_inv(I[:, k].astype(complex)) for k in range(nv)])

        def iterate(mu_eff):
            Pc = np.block([[t * np.linalg.inv(Mhat_inv), np.zeros((nv, nv))],
                           [Psi, -mu_eff * np.linalg.inv(Shat_inv)]])
            x = np.zeros(2 * nv, dtype=complex)
            for _ in range(steps):
                x = x + np.linalg.solve(Pc, b - G11 @ x)
            return x

        x = iterate(mu)
        y1, y2 = blk.uzawa(b[:nv], b[nv:])
        got = np.concatenate([y1, y2])
        assert np.abs(got - x).max() <= 1e-10 * np.abs(x).max(), steps
        # a plausible mistake (mu in the numerator) changes the second block
        if steps == 1:
            bad = iterate(1.0 / mu)
            assert np.abs(got[nv:] - bad[nv:]).max() > 0.1 * np.abs(x[nv:]).max()


def test_multigrid_pin_sees_plausible_mistakes():
    """The explicit operator distinguishes the oracle's V-cycle from one with
    the post-sweeps in forward colour order and from one with another omega."""
    level, aM, aK = 3, 1.3, 0.02
    mg = inexact.Multigrid("q2", level, 0.0, 1.0, None, aM, aK, 0.0, 2, 2, 1.0)
    lev = _levels("q2", level, 0.0, 1.0, None, aM, aK, 0.0)
    n = lev[0]["A"].shape[0]
    got = _mg_matrix(mg, n, 1)
    for wrong in (_vcycle_operator(lev, 0, 1.0, 2, 2, post_forward=True), _vcycle_operator(lev, 0, 0.9, 2, 2)):
        assert np.abs(got - wrong).max() > 1e-6 * np.abs(got).max()


def _cheb_matrix(A, steps, bounds):
    """x_k = (I - T_k(sigma I - E / delta) / T_k(sigma)) A^{-1}, E = D^{-1} A."""
    lmin, lmax = bounds
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    n = A.shape[0]
    Z = sigma * np.eye(n) - np.diag(1.0 / np.diag(A)) @ A / delta
    Tm, T = np.eye(n), Z.copy()          # T_0, T_1 of the matrix
    tm, t = 1.0, sigma                   # T_0, T_1 at sigma
    for _ in range(steps - 1):
        Tm, T = T, 2.0 * Z @ T - Tm
        tm, t = t, 2.0 * sigma * t - tm
    return (np.eye(n) - T / t) @ np.linalg.inv(A)


@pytest.mark.parametrize("space", ["q2", "q1"])
def test_chebyshev_is_its_error_polynomial(space):
    P = kkt.Problem("stokes", 2, 4, 0.2, 1e-2, 1e-2, 0.0, 1.0, None)
    A = (P.Ms if space == "q2" else P.Mpr).toarray()
    bounds = inexact.element_jacobi_bounds(2 if space == "q2" else 1)
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    for steps in (1, 2, 5, 10):
        ref = _cheb_matrix(A, steps, bounds) @ b
        got = inexact.chebyshev(P.Ms if space == "q2" else P.Mpr, b, steps, bounds)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), steps
    # a plausible mistake (bounds taken for the other element) changes the iterate
    wrong = _cheb_matrix(A, 5, inexact.element_jacobi_bounds(1 if space == "q2" else 2)) @ b
    assert np.abs(inexact.chebyshev(P.Ms if space == "q2" else P.Mpr, b, 5, bounds) - wrong).max() > 1e-6 * np.abs(wrong).max()

