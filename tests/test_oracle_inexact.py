"""Pins for the oracle's inexact nested solvers (Chebyshev, MG, Uzawa, GMRES)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import inexact, kkt
from oracle_golden import paper_bounds


def stokes(level=2, K=4, beta=1e-2, tau=0.2):
    return kkt.Problem("stokes", level, K, tau, beta, 1e-2, 0.0, 1.0, None)


def oseen(level=2, K=4, beta=1e-3, tau=0.2, nu=1e-2, wind="recirc"):
    return kkt.Problem("oseen", level, K, tau, beta, nu, -1.0, 1.0, wind)


def problem(kind, level, K):
    """kind: "stokes", "oseen" (recirculating wind) or "oseen-2v" (Sec. 5.2 wind)."""
    if kind == "stokes":
        return stokes(level, K)
    return oseen(level, K, wind="two_vortex" if kind == "oseen-2v" else "recirc")


KINDS = ["stokes", "oseen", "oseen-2v"]


@pytest.mark.parametrize("space", ["q2", "q1"])
@pytest.mark.parametrize("steps", [1, 3, 10])
def test_chebyshev_energy_error_bound(space, steps):
    P = stokes(3)
    A = (P.Ms if space == "q2" else P.Mpr).toarray()
    bounds = inexact.element_jacobi_bounds(2 if space == "q2" else 1)
    b = np.random.default_rng(steps).standard_normal(A.shape[0])
    xt = np.linalg.solve(A, b)
    x = inexact.chebyshev(P.Ms if space == "q2" else P.Mpr, b, steps, bounds)
    en = lambda e: np.sqrt(e @ A @ e)
    kappa = bounds[1] / bounds[0]
    rho = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    bound = 2 * rho ** steps / (1 + rho ** (2 * steps))
    assert en(x - xt) <= bound * en(xt) * (1 + 1e-12)
    if steps == 10:
        assert en(x - xt) <= 3e-3 * en(xt)


def test_chebyshev_converges_to_exact():
    P = stokes(3)
    b = np.random.default_rng(0).standard_normal(P.Ms.shape[0])
    x = inexact.chebyshev(P.Ms, b, 60, inexact.element_jacobi_bounds(2))
    np.testing.assert_allclose(x, spla.spsolve(P.Ms.tocsc(), b), rtol=1e-11, atol=1e-11 * np.abs(x).max())


def _mgs():
    P = stokes(3)
    d, dr, dc, c1, c2 = inexact.stokes_constants(P, 1)
    Po = oseen(3)
    B = inexact.OseenBlockPreconditioner(Po, 1, inexact.Settings())
    return {
        "W": inexact.Multigrid("q2", 3, 0, 1, None, 1 + c1, c2 * P.nu),
        "Kp": inexact.Multigrid("q1", 3, 0, 1, None, 0.0, 1.0),
        "Q": B.mgQ,
        "QH": B.mgQH,
    }


MGS = _mgs()


@pytest.mark.parametrize("name", list(MGS))
def test_mg_is_linear_and_contracts(name):
    mg = MGS[name]
    A = mg.levels[0].A
    n = A.shape[0]
    rng = np.random.default_rng(3)
    b1 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b2 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a, c = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = mg.solve(a * b1 + c * b2, 2)
    rhs = a * mg.solve(b1, 2) + c * mg.solve(b2, 2)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
    xt = spla.spsolve(A.tocsc().astype(complex), b1)
    errs = [np.linalg.norm(mg.solve(b1, k) - xt) / np.linalg.norm(xt) for k in (1, 2, 3)]
    assert errs[0] < 1 and errs[1] < errs[0] and errs[2] < errs[1]
    assert np.linalg.norm(mg.solve(b1, 40) - xt) <= 1e-9 * np.linalg.norm(xt)


@pytest.mark.parametrize("name", list(MGS))
def test_multicolour_sets_are_independent(name):
    """Nodes of one colour never couple, so the colour-wise update equals a
    sequential Gauss-Seidel sweep over that colour."""
    for L in MGS[name].levels:
        for idx in L.colours:
            sub = L.A[idx][:, idx].toarray()
            assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0


def test_gmres_minimal_residual_property():
    """k-step GMRES returns the minimiser of ||s - A P^{-1} u|| over the
    Krylov space K_k(A P^{-1}, s): brute force with an explicit basis."""
    P = stokes(1, 3)
    j = 1
    Z = inexact.Z_matrix(P, j).toarray().astype(complex)
    prec = inexact.StokesBlockPreconditioner(P, j, inexact.Settings())
    n = Z.shape[0]
    Pinv = np.column_stack([prec(e) for e in np.eye(n, dtype=complex)])   # linear operator
    s = np.random.default_rng(9).standard_normal(n) + 1j * np.random.default_rng(10).standard_normal(n)
    AP = Z @ Pinv
    for k in (1, 3, 6):
        x, its = inexact.gmres(Z, prec, s, 1e-30, 100, fixed_its=k)
        assert its == k
        Kb = np.column_stack([np.linalg.matrix_power(AP, i) @ s for i in range(k)])
        Qb, _ = np.linalg.qr(Kb)
        c, *_ = np.linalg.lstsq(AP @ Qb, s, rcond=None)
        best = np.linalg.norm(s - AP @ Qb @ c)
        got = np.linalg.norm(s - Z @ x)
        assert abs(got - best) <= 1e-9 * np.linalg.norm(s)
        # x lies in P^{-1} K_k
        u = np.linalg.solve(Pinv, x)
        proj = Qb @ (Qb.conj().T @ u)
        assert np.linalg.norm(u - proj) <= 1e-8 * np.linalg.norm(u)


def test_gmres_tolerance_stop():
    P = stokes(2, 4)
    j = 2
    Z = inexact.Z_matrix(P, j).astype(complex)
    prec = inexact.StokesBlockPreconditioner(P, j, inexact.Settings())
    s = np.random.default_rng(1).standard_normal(Z.shape[0]) + 0j
    x, its = inexact.gmres(Z, prec, s, 1e-2, 100)
    res = np.linalg.norm(s - Z @ x) / np.linalg.norm(s)
    assert res <= 1e-2 * (1 + 1e-8)
    _, its_prev = inexact.gmres(Z, prec, s, 1e-30, 100, fixed_its=its - 1)
    x_prev, _ = inexact.gmres(Z, prec, s, 1e-30, 100, fixed_its=its - 1)
    assert np.linalg.norm(s - Z @ x_prev) / np.linalg.norm(s) > 1e-2


@pytest.mark.parametrize("wind", ["recirc", "two_vortex"])
def test_uzawa_with_exact_inner_solves_converges(wind):
    """Eq. Uzawa11 with M^ = M and S^^{-1} exact is a contraction with factor
    max |1 - lambda/mu| = 1/3 for lambda in [1/2, 1], mu = 3/4 (Sec. 4):
    it converges to the solution of G_j^(1,1) x = b."""
    g = paper_bounds()
    P = oseen(2, 4, wind=wind)
    j = 1
    s = inexact.Settings(uzawa_steps=40, uzawa_mu=g["uzawa_mu"])
    B = inexact.OseenBlockPreconditioner(P, j, s)
    M = P.Mv.toarray().astype(complex)
    t, be = P.tau, P.beta
    Q = (B.d * P.Mv + t * P.Lv + (t / np.sqrt(be)) * P.Mv).toarray()
    B.M_hat_inv = lambda u: np.linalg.solve(M, u)
    B.S11_inv = lambda u: t * np.linalg.solve(Q.conj().T, M @ np.linalg.solve(Q, u))
    G11 = np.block([[t * M, (np.conj(B.d) * P.Mv + t * P.Lv.T).toarray()],
                    [(B.d * P.Mv + t * P.Lv).toarray(), -(t / be) * M]])
    rng = np.random.default_rng(2)
    b = rng.standard_normal(2 * P.nv) + 1j * rng.standard_normal(2 * P.nv)
    x1, x2 = B.uzawa(b[:P.nv], b[P.nv:])
    xt = np.linalg.solve(G11, b)
    assert np.linalg.norm(np.concatenate([x1, x2]) - xt) <= 1e-10 * np.linalg.norm(xt)
    # the 6-step inexact version is a good approximation (relative error < 1)
    B6 = inexact.OseenBlockPreconditioner(P, j, inexact.Settings())
    y1, y2 = B6.uzawa(b[:P.nv], b[P.nv:])
    assert np.linalg.norm(np.concatenate([y1, y2]) - xt) < 0.5 * np.linalg.norm(xt)


@pytest.mark.parametrize("wind", ["recirc", "two_vortex"])
def test_algorithm3_with_exact_pieces_is_block_triangular_solve(wind):
    """With exact (1,1) and exact commutator Schur pieces, Algorithm 3 solves
    [[G11, 0], [G21, -S^]] y = r (reading R6)."""
    P = oseen(1 if wind == "recirc" else 2, 4, wind=wind)
    j = 1
    s = inexact.Settings(uzawa_steps=60, mg_cycles=60, cheb_steps=80)
    B = inexact.OseenBlockPreconditioner(P, j, s)
    r = np.random.default_rng(4).standard_normal(P.nb * 2) + 0j
    y = B(r)
    t, be, d = P.tau, P.beta, B.d
    G = P.G(j).toarray()
    nv, npp = P.nv, P.np_
    Mp, Kp, Lp = P.Mpr.toarray(), P.Kpr.toarray(), P.Lpr.toarray()
    Xp = np.block([[t * Mp, np.conj(d) * Mp + t * Lp.T], [d * Mp + t * Lp, -(t / be) * Mp]])
    O = np.zeros_like(Mp)
    Sh = np.block([[O, t * Mp], [t * Mp, O]]) @ np.linalg.solve(Xp, np.block([[O, t * Kp], [t * Kp, O]]))
    T = np.zeros_like(G)
    T[:2 * nv, :2 * nv] = G[:2 * nv, :2 * nv]
    T[2 * nv:, :2 * nv] = G[2 * nv:, :2 * nv]
    T[2 * nv:, 2 * nv:] = -Sh
    yt = np.linalg.solve(T, r)
    assert np.linalg.norm(y - yt) <= 1e-7 * np.linalg.norm(yt)


@pytest.mark.parametrize("kind", KINDS)
def test_algorithm2_with_tight_inner_tolerance_is_exact_pc(kind):
    P = problem(kind, 1 if kind != "oseen-2v" else 2, 4)
    s = inexact.Settings(inner_tol=1e-13, inner_maxit=200)
    pc = inexact.PinTPreconditioner(P, s)
    r = np.random.default_rng(5).standard_normal(P.n)
    z = pc(r)
    z_exact = P.pc_inverse(r)[0]
    assert np.linalg.norm(z - z_exact) <= 1e-9 * np.linalg.norm(z_exact)


@pytest.mark.parametrize("kind", KINDS)
def test_hermitian_half_suffices(kind):
    """The frequency-j solve of the conjugate right-hand side is the conjugate
    solution (G_{K-j} = conj(G_j)); the inexact nested solvers preserve this."""
    P = problem(kind, 2, 4)
    pc = inexact.PinTPreconditioner(P)
    g = np.random.default_rng(6).standard_normal(P.nb * 2) + 1j * np.random.default_rng(7).standard_normal(P.nb * 2)
    y1 = pc.solve_block(1, g)
    y3 = pc.solve_block(3, np.conj(g))
    assert np.linalg.norm(y3 - np.conj(y1)) <= 1e-12 * np.linalg.norm(y1)


@pytest.mark.parametrize("kind", KINDS)
def test_full_solve_alg2_fgmres(kind):
    from paper_2405_18964_gb300 import inputs
    P = problem(kind, 2, 4)
    vd = inputs.desired_state(P.N, P.x0, P.x1, P.K, P.tau, P.tau * (P.K + 1), seed=0)
    b = P.rhs(vd)
    A = P.kkt_matrix()
    pc = inexact.PinTPreconditioner(P)
    x, info = kkt.fgmres(A, b, pc, tol=1e-8, restart=30)
    assert info["relres"] <= 1e-8
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    X = x.reshape(2, P.K, P.nb)
    for k in range(P.K):
        v, lam = X[0, k, :P.nv], X[1, k, :P.nv]
        assert np.linalg.norm(P.Bv @ v) <= 1e-7 * np.linalg.norm(v)
        assert np.linalg.norm(P.Bv @ lam) <= 1e-7 * np.linalg.norm(lam)


def test_pressure_multigrid_rounding_spread():
    """The corner-pinned pressure Laplacian K_p is nearly singular (its
    near-null constant mode is held only by the pin), so 4 V-cycles amplify
    rounding in the residuals.  Evaluating the same operator in band form,
    K_p X = M1 X K1^T + K1 X M1^T (1-D Q1 mass / stiffness bands), instead of
    through the assembled rows changes the 64 x 64 result by ~1e-12: FP64
    comparisons of values that pass through this multigrid cannot be held
    tighter than this spread."""
    import scipy.linalg as sla
    from oracle import fem
    from paper_2405_18964_gb300 import inputs

    mg = inexact.Multigrid("q1", 6, 0.0, 1.0, None, 0.0, 1.0, 0.0)
    b = inputs.random_vector(65 * 65, 18, np.complex128)[mg.levels[0].free]
    x_rows = mg.solve(b, 4)

    def band_apply(L, xf):
        N = L.N
        m, k = fem.element_matrices_1d(1, 1.0 / N)
        M1, K1 = np.zeros((N + 1, N + 1)), np.zeros((N + 1, N + 1))
        for e in range(N):
            M1[e:e + 2, e:e + 2] += m
            K1[e:e + 2, e:e + 2] += k
        X = np.zeros((N + 1) ** 2, complex)
        X[L.free] = xf
        X = X.reshape(N + 1, N + 1)
        return (M1 @ (X @ K1.T) + K1 @ (X @ M1.T)).ravel()[L.free]

    def sweep(L, x, b, order):
        for c in order:
            idx = L.colours[c]
            x[idx] = x[idx] + mg.omega * (b[idx] - band_apply(L, x)[idx]) / L.diag[idx]
        return x

    def vcycle(l, x, b):
        L = mg.levels[l]
        if l == len(mg.levels) - 1:
            return sla.lu_solve(mg.coarse_lu, b)
        for _ in range(mg.pre):
            x = sweep(L, x, b, range(4))
        xc = vcycle(l + 1, np.zeros(L.P.shape[1], complex), L.P.T @ (b - band_apply(L, x)))
        x = x + L.P @ xc
        for _ in range(mg.post):
            x = sweep(L, x, b, range(3, -1, -1))
        return x

    x_band = np.zeros_like(x_rows)
    for _ in range(4):
        x_band = vcycle(0, x_band, b)
    spread = np.abs(x_band - x_rows).max() / np.abs(x_rows).max()
    # the two evaluations are the same operator: they agree far beyond FP32,
    # and differ by more than the generic FP64 bar of 1e-12
    assert 5e-13 < spread < 4e-12, spread


def test_fp32_krylov_emulation_is_fp32_level():
    """The FP32-Krylov emulation that sets the full-size FP32 bars changes a
    frequency-block solve at FP32 level: above FP64 rounding,
    far below the inner tolerance."""
    from gpu_pairs import fp32_arnoldi_solves
    from oracle import layout
    P = kkt.Problem("stokes", 3, 8, 1 / 9, 1e-3, 1e-2, 0.0, 1.0, None)
    s = inexact.Settings()
    g = {1: layout.to_oracle_freq(P, np.random.default_rng(4).standard_normal(layout.block_len(P)) + 0j)}
    exact = inexact.PinTPreconditioner(P, s, fixed_inner_its=3).solve_block(1, g[1])
    emu = fp32_arnoldi_solves(P, s, [1], g, 3)[1]
    d = np.abs(emu - exact).max() / np.abs(exact).max()
    assert 1e-10 < d < 1e-5, d


def _hat_preconditioned_operator(P, schur):
    """Dense matrix of P_C^{-1} A for the block preconditioner diag(W_j, W_j,
    S_j, S_j) of Z_j (Sec. 3.2) inside the FFT diagonalisation:
    schur='exact' uses S_j = B W_j^{-1} B^T (P^_C, Theorem 2), schur='commutator'
    the approximation S^_j (P~_C, Theorem 3)."""
    import scipy.linalg as sla
    blocks = {}
    for j in range(P.K):
        _, _, _, c1, c2 = inexact.stokes_constants(P, j)
        W = ((1 + c1) * P.Ms + c2 * P.Ls).toarray()
        Wv = sla.block_diag(W, W)
        B = P.Bv.toarray()
        if schur == "exact":
            S = B @ np.linalg.solve(Wv, B.T)
        else:
            Kp, Mp = P.Kpr.toarray(), P.Mpr.toarray()
            S = np.linalg.inv((1 + c1) * np.linalg.inv(Kp) + P.nu * c2 * np.linalg.inv(Mp))
        Pj = sla.block_diag(Wv, Wv, S, S)
        Tl, Tr = inexact.T_matrices(P, j)
        blocks[j] = np.linalg.inv(Tl.toarray() @ Pj @ Tr.toarray())

    def solver(j, rhs):
        return P.g_to_ylam(blocks[j] @ P.ylam_to_g(rhs))

    A = P.kkt_matrix().toarray()
    return np.column_stack([P.pc_inverse(A[:, k], solver)[0] for k in range(A.shape[1])])


@pytest.mark.parametrize("schur", ["exact", "commutator"])
def test_theorems_2_3_eigenvalue_clusters(schur):
    """Theorems 2 and 3: at most 4 n_v eigenvalues of P^_C^{-1} A (P~_C^{-1} A)
    lie outside |mu| in [a, b], with [a, b] = [1/sqrt(12), (1+sqrt(5))/2] for
    the exact Schur complement (Eq. SchurComplementHatBounds) and [a c, b d]
    for the commutator one, [c, d] bounding |lambda(S^_j^{-1} B W_j^{-1} B^T)|
    over the frequencies (the lemma before Theorem 3)."""
    P = kkt.Problem("stokes", 2, 4, 1 / 5, 1e-2, 1e-2, 0.0, 1.0, None)
    a, b = 1 / np.sqrt(12), (1 + np.sqrt(5)) / 2
    if schur == "commutator":
        cs, ds = [], []
        for j in range(P.K):
            _, _, _, c1, c2 = inexact.stokes_constants(P, j)
            W = ((1 + c1) * P.Ms + c2 * P.Ls).toarray()
            import scipy.linalg as sla
            B = P.Bv.toarray()
            S = B @ np.linalg.solve(sla.block_diag(W, W), B.T)
            Shat_inv = (1 + c1) * np.linalg.inv(P.Kpr.toarray()) + P.nu * c2 * np.linalg.inv(P.Mpr.toarray())
            ev = np.abs(np.linalg.eigvals(Shat_inv @ S))
            cs.append(ev.min())
            ds.append(ev.max())
        a, b = a * min(cs), b * max(ds)
    mu = np.abs(np.linalg.eigvals(_hat_preconditioned_operator(P, schur)))
    inside = np.count_nonzero((mu >= a * (1 - 1e-9)) & (mu <= b * (1 + 1e-9)))
    assert inside >= len(mu) - 4 * P.nv, (inside, len(mu), P.nv)


def test_damped_sor_rescues_the_convection_dominated_Q0():
    """The limitation of the recirculating wind at beta >= 1e-2: the Q_0
    multigrid with Gauss-Seidel smoothing (omega = 1) diverges, more sweeps
    make it worse (the smoother itself amplifies), and under-relaxed SOR
    (omega = 0.7) converges.  Q_0 = (tau / sqrt(beta)) M + tau (nu K + N)."""
    K, beta, nu = 8, 1e-2, 1e-2
    tau = 1.0 / (K + 1)
    aM, aK, aN = tau / np.sqrt(beta), tau * nu, tau

    def err(**kw):
        mg = inexact.Multigrid("q2", 3, -1.0, 1.0, "recirc", aM, aK, aN, **kw)
        A = mg.levels[0].A
        rng = np.random.default_rng(0)
        b = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
        xt = spla.spsolve(A.tocsc().astype(complex), b)
        with np.errstate(all="ignore"):
            return np.linalg.norm(mg.solve(b, 4) - xt) / np.linalg.norm(xt)

    e1, e_more, e07 = err(), err(pre=4, post=4), err(omega=0.7)
    assert e1 > 1.0 and e_more > e1
    assert e07 < 0.1


def test_convection_only_damping_converges_the_recirculating_wind():
    """Damping only the SOR of Q_j and Q_j^H (sor_omega_conv), with K_p keeping
    Gauss-Seidel, is enough: the beta = 1e-2 recirculating-wind problem whose
    Q_0 multigrid diverges at omega = 1 converges in FGMRES(10)."""
    P = kkt.Problem("oseen", 3, 4, 0.2, 1e-2, 1e-2, -1.0, 1.0, "recirc")
    s = inexact.Settings(sor_omega_conv=0.5, inner_maxit=60)
    pc = inexact.PinTPreconditioner(P, s)
    blk = pc.block_prec(0)
    assert blk.mgQ.omega == 0.5 and blk.mgQH.omega == 0.5 and blk.mgKp.omega == 1.0
    from paper_2405_18964_gb300 import inputs
    b = P.rhs(inputs.desired_state(P.N, -1.0, 1.0, P.K, P.tau, 1.0, seed=0))
    x, info = kkt.fgmres(P.kkt_matrix(), b, pc, restart=10, tol=1e-8, maxit=30)
    assert info["relres"] <= 1e-8 and info["its"] <= 15, info["its"]
