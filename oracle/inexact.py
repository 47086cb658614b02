"""Inexact per-frequency preconditioners and the nested solvers (FP64/complex128).

TEST INFRASTRUCTURE (oracle): see the package header.

What it follows
  * Chebyshev semi-iteration for mass matrices (Sec. 3.4, Golub & Varga):
    Jacobi-preconditioned, zero initial guess, `steps` updates of x, written
    from the three-term recurrence of the scaled Chebyshev polynomials.
  * Geometric multigrid with SOR smoothing (Sec. 3.4).
  * Stokes: G_j = T_j^l Z_j T_j^r (Eq. GJTransformation) and the commutator
    preconditioner P~_j = diag(W_j, W_j, S^_j, S^_j), W_j = M + c1 M + c2 L,
    S^_j^{-1} = (1 + c1) K_p^{-1} + nu c2 M_p^{-1} (Sec. 3.2).
  * Oseen: inexact preconditioned Uzawa (Eq. Uzawa11) on G_j^(1,1) with the
    Pearson-Wathen Schur approximation S^ = (1/tau) Q_j M^{-1} Q_j^H,
    Q_j = d_j M + tau L + tau/sqrt(beta) M, and the commutator approximation
    of the outer Schur complement (Sec. 4); together Algorithm 3.
  * Inner GMRES (Sec. 3.4) and Algorithms 1 (linear) and 2 (nonlinear).

Readings where the paper is silent, ambiguous or garbled
  R4  c_{j,1} = d_{j,r} / sqrt(tau^2/beta + d_{j,c}^2)  (the printed formula
      lacks the square; only the squared form makes T^l Z T^r = G_j).
  R5  the inner preconditioner of Algorithm 2 is P~_j (commutator), as in
      the text and the solver-overview figure.
  R6  Algorithm 3's sign: y34 = -S^_j^{-1}(r34 - tau (B y2; B y1)).
  R13 MG: nested grids N, N/2, ..., 2 (N = 2^level), rediscretised coarse
      operators (equal to Galerkin: nested spaces, exact quadrature),
      exact nested interpolation for P and R = P^T, multicolour SOR with
      9 colours (ix mod 3) + 3 (iy mod 3) for Q2 and 4 colours
      (ix mod 2) + 2 (iy mod 2) for Q1, omega = 1, `pre` sweeps in colour
      order 0..last and `post` sweeps in reverse order, dense solve on the
      coarsest grid, zero initial guess, `cycles` V-cycles.
  R14 Chebyshev eigenvalue bounds of D^{-1} M: the extreme eigenvalues of
      D_e^{-1} M_e of the element mass matrix (computed here).
  R15 inner GMRES: right preconditioned, complex, MGS, x0 = 0, no restart,
      stop when the Arnoldi residual estimate <= eps ||s||, or after
      `fixed_its` iterations when that is given.
  R17 Uzawa: M^ = Chebyshev(M); Q_j^{-1}, Q_j^{-H} each by MG; x^(0) = 0.

Parity unpinned: the paper prints no intermediate values for these nested
iterations.  They are pinned by convergence to the exact inverses as the
iteration counts grow, by the Chebyshev error bound, by the brute-force
Krylov minimal-residual property of GMRES, and by the eigenvalue bounds the
paper prints (Eqs. SchurComplementHatBounds, SchurComplementPearsonWathen).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem


# --------------------------------------------------------------------------
# Chebyshev semi-iteration
# --------------------------------------------------------------------------
def element_jacobi_bounds(degree):
    """Extreme eigenvalues of D_e^{-1} M_e for the 2-D Lagrange element of
    `degree` (tensor product of the 1-D element mass matrices)."""
    m1, _ = fem.element_matrices_1d(degree, 1.0)
    me = np.kron(m1, m1)
    ev = np.linalg.eigvals(np.diag(1.0 / np.diag(me)) @ me).real
    return float(ev.min()), float(ev.max())


def chebyshev(A, b, steps, bounds):
    """Jacobi-Chebyshev semi-iteration for A x = b, x0 = 0.

    With theta = (l_max + l_min)/2 and delta = (l_max - l_min)/2 the iterate
    after k steps is x_k = p_{k-1}(D^{-1} A) D^{-1} b where the error
    polynomial is the Chebyshev polynomial T_k scaled to [l_min, l_max].
    Recurrence: x_{k+1} = x_k + d_k, r_{k+1} = r_k - A d_k,
    rho_{k+1} = 1 / (2 sigma - rho_k), d_{k+1} = rho_{k+1} rho_k d_k
    + (2 rho_{k+1} / delta) D^{-1} r_{k+1}, sigma = theta / delta.
    """
    lmin, lmax = bounds
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    dinv = 1.0 / A.diagonal()
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = b.copy()
    d = (dinv * r) / theta
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (rho_new * rho) * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x


# --------------------------------------------------------------------------
# Geometric multigrid
# --------------------------------------------------------------------------
class _Level:
    pass


class Multigrid:
    """V-cycle multigrid for  aM M + aK K + aN N  on one scalar field.

    space "q2": a velocity component (Dirichlet nodes eliminated);
    space "q1": the pressure (corner node pinned).  Coefficients may be
    complex.  Reading R13 (see module header).
    """

    def __init__(self, space, level, x0, x1, wind, aM, aK, aN=0.0, pre=2, post=2, omega=1.0):
        self.space = space
        self.pre, self.post, self.omega = pre, post, omega
        self.levels = []
        for lv in range(level, 0, -1):
            N = 2 ** lv
            wf, skew = fem.wind_by_name(wind, N, x0, x1)
            ops = fem.assemble(N, x0, x1, wf, skew=skew)
            g = ops.grid
            if space == "q2":
                M, K, Nc = ops.M, ops.K, ops.N
                free = g.velocity_interior()
                n1 = g.n2
                ncol = 3
            else:
                M, K, Nc = ops.Mp, ops.Kp, ops.Np
                free = g.pressure_free()
                n1 = g.n1
                ncol = 2
            A = (aM * M + aK * K + aN * Nc)[free][:, free].tocsr()
            L = _Level()
            L.N, L.free, L.A = N, free, A
            L.diag = A.diagonal()
            ix, iy = free % n1, free // n1
            col = (ix % ncol) + ncol * (iy % ncol)
            L.colours = [np.flatnonzero(col == c) for c in range(ncol * ncol)]
            L.rows = [A[idx] for idx in L.colours]
            self.levels.append(L)
        # prolongations between consecutive levels (coarse l+1 -> fine l)
        deg = 2 if space == "q2" else 1
        for l in range(len(self.levels) - 1):
            fine, coarse = self.levels[l], self.levels[l + 1]
            Pf = fem.prolongation_2d(coarse.N, deg)
            fine.P = Pf[fine.free][:, coarse.free].tocsr()
        self.coarse_lu = sla.lu_factor(self.levels[-1].A.toarray())

    def _sweep(self, L, x, b, order):
        for c in order:
            idx = L.colours[c]
            r = b[idx] - L.rows[c] @ x
            x[idx] = x[idx] + self.omega * r / L.diag[idx]
        return x

    def vcycle(self, l, x, b):
        L = self.levels[l]
        if l == len(self.levels) - 1:
            return sla.lu_solve(self.coarse_lu, b)
        nc = len(L.colours)
        for _ in range(self.pre):
            x = self._sweep(L, x, b, range(nc))
        r = b - L.A @ x
        bc = L.P.T @ r
        xc = self.vcycle(l + 1, np.zeros_like(bc), bc)
        x = x + L.P @ xc
        for _ in range(self.post):
            x = self._sweep(L, x, b, range(nc - 1, -1, -1))
        return x

    def solve(self, b, cycles):
        dt = np.result_type(b.dtype, self.levels[0].A.dtype)
        x = np.zeros(len(b), dtype=dt)
        b = b.astype(dt)
        for _ in range(cycles):
            x = self.vcycle(0, x, b)
        return x


# --------------------------------------------------------------------------
# Stokes: transform, commutator preconditioner
# --------------------------------------------------------------------------
def stokes_constants(P, j):
    """d_j, d_{j,r}, d_{j,c}, c_{j,1} (reading R4), c_{j,2} (Sec. 3.2)."""
    d = P.d(j)
    dr, dc = d.real, d.imag
    t, b = P.tau, P.beta
    c1 = dr / np.sqrt(t * t / b + dc * dc)
    c2 = 1.0 / np.sqrt(1.0 / b + dc * dc / (t * t))
    return d, dr, dc, c1, c2


def Z_matrix(P, j):
    """Z_j of Eq. GJTransformation, (v, lambda, p, mu) ordering."""
    _, _, _, c1, c2 = stokes_constants(P, j)
    M, L, B = P.Mv, P.Lv, P.Bv
    X = c1 * M + c2 * L
    Zp = sp.csr_matrix((P.np_, P.np_))
    return sp.bmat([[M, X, None, B.T], [X, -M, B.T, None], [None, B, Zp, None], [B, None, None, Zp]],
                   format="csr")


def T_matrices(P, j):
    """T_j^l and T_j^r of Eq. GJTransformation as sparse matrices."""
    _, _, dc, _, c2 = stokes_constants(P, j)
    s = np.sqrt(P.tau)
    Iv = sp.eye(P.nv, format="csr")
    Ip = sp.eye(P.np_, format="csr")
    Tl = sp.bmat([[s * Iv, None, None, None],
                  [(1j * dc / s) * Iv, (s / c2) * Iv, None, None],
                  [None, None, (s * c2) * Ip, None],
                  [None, None, (1j * dc * c2 / s) * Ip, s * Ip]], format="csr")
    Tr = sp.bmat([[s * Iv, (-1j * dc / s) * Iv, None, None],
                  [None, (s / c2) * Iv, None, None],
                  [None, None, (s * c2) * Ip, (-1j * dc * c2 / s) * Ip],
                  [None, None, None, s * Ip]], format="csr")
    return Tl, Tr


def split4(P, u):
    nv, npp = P.nv, P.np_
    return u[:nv], u[nv:2 * nv], u[2 * nv:2 * nv + npp], u[2 * nv + npp:]


def Tl_inverse(P, j, r):
    """(T_j^l)^{-1} r by forward substitution of the block rows."""
    _, _, dc, _, c2 = stokes_constants(P, j)
    s = np.sqrt(P.tau)
    r1, r2, r3, r4 = split4(P, r)
    s1 = r1 / s
    s2 = (r2 - (1j * dc / s) * s1) * (c2 / s)
    s3 = r3 / (s * c2)
    s4 = (r4 - (1j * dc * c2 / s) * s3) / s
    return np.concatenate([s1, s2, s3, s4])


def Tr_inverse(P, j, x):
    """(T_j^r)^{-1} x by back substitution of the block rows."""
    _, _, dc, _, c2 = stokes_constants(P, j)
    s = np.sqrt(P.tau)
    x1, x2, x3, x4 = split4(P, x)
    y2 = x2 * (c2 / s)
    y1 = (x1 + (1j * dc / s) * y2) / s
    y4 = x4 / s
    y3 = (x3 + (1j * dc * c2 / s) * y4) / (s * c2)
    return np.concatenate([y1, y2, y3, y4])


class Settings:
    """Inner-solver parameters (defaults from Sec. 5: 4 V-cycles, 10
    Chebyshev steps, 6 Uzawa steps, mu = 3/4, inner tolerance 1e-2)."""

    def __init__(self, mg_cycles=4, mg_pre=2, mg_post=2, sor_omega=1.0, cheb_steps=10,
                 uzawa_steps=6, uzawa_mu=0.75, inner_tol=1e-2, inner_maxit=100, sor_omega_conv=None):
        self.mg_cycles, self.mg_pre, self.mg_post = mg_cycles, mg_pre, mg_post
        self.sor_omega = sor_omega
        # SOR relaxation of the convection operators Q_j, Q_j^H (default: sor_omega)
        self.sor_omega_conv = sor_omega if sor_omega_conv is None else sor_omega_conv
        self.cheb_steps = cheb_steps
        self.uzawa_steps, self.uzawa_mu = uzawa_steps, uzawa_mu
        self.inner_tol, self.inner_maxit = inner_tol, inner_maxit


Q2_BOUNDS = None
Q1_BOUNDS = None


def mass_bounds():
    global Q2_BOUNDS, Q1_BOUNDS
    if Q2_BOUNDS is None:
        Q2_BOUNDS = element_jacobi_bounds(2)
        Q1_BOUNDS = element_jacobi_bounds(1)
    return Q2_BOUNDS, Q1_BOUNDS


class StokesBlockPreconditioner:
    """P~_j^{-1} for Z_j (Sec. 3.2): W_j^{-1} by MG on each velocity
    component of the v and lambda blocks; S^_j^{-1} = (1 + c1) MG(K_p) +
    nu c2 Cheb(M_p) on the p and mu blocks."""

    def __init__(self, P, j, s: Settings, kp_mg=None):
        self.P, self.j, self.s = P, j, s
        _, _, _, c1, c2 = stokes_constants(P, j)
        self.c1, self.c2 = c1, c2
        self.mgW = Multigrid("q2", P.level, P.x0, P.x1, None, 1.0 + c1, c2 * P.nu, 0.0,
                             s.mg_pre, s.mg_post, s.sor_omega)
        self.mgKp = kp_mg if kp_mg is not None else Multigrid(
            "q1", P.level, P.x0, P.x1, None, 0.0, 1.0, 0.0, s.mg_pre, s.mg_post, s.sor_omega)

    def W_inv(self, u):
        n = self.P.nvc
        return np.concatenate([self.mgW.solve(u[:n], self.s.mg_cycles),
                               self.mgW.solve(u[n:], self.s.mg_cycles)])

    def S_inv(self, u):
        _, q1b = mass_bounds()
        return (1.0 + self.c1) * self.mgKp.solve(u, self.s.mg_cycles) + \
            self.P.nu * self.c2 * chebyshev(self.P.Mpr.astype(complex), u.astype(complex), self.s.cheb_steps, q1b)

    def __call__(self, u):
        u1, u2, u3, u4 = split4(self.P, u)
        return np.concatenate([self.W_inv(u1), self.W_inv(u2), self.S_inv(u3), self.S_inv(u4)])


class OseenBlockPreconditioner:
    """(P~_j^(UZ))^{-1} of Algorithm 3 (Sec. 4)."""

    def __init__(self, P, j, s: Settings, kp_mg=None):
        self.P, self.j, self.s = P, j, s
        t, b = P.tau, P.beta
        d = P.d(j)
        self.d = d
        aQ = d + t / np.sqrt(b)
        # Q_j = d M + tau (nu K + N) + tau/sqrt(beta) M ; Q_j^H = conj(.) M + tau (nu K + N^T)
        self.mgQ = Multigrid("q2", P.level, P.x0, P.x1, P.wind, aQ, t * P.nu, t,
                             s.mg_pre, s.mg_post, s.sor_omega_conv)
        self.mgQH = _TransposedMG(P, np.conj(aQ), t * P.nu, t, s)
        self.mgKp = kp_mg if kp_mg is not None else Multigrid(
            "q1", P.level, P.x0, P.x1, None, 0.0, 1.0, 0.0, s.mg_pre, s.mg_post, s.sor_omega)
        self.Mv = P.Mv.astype(complex)
        self.Lv = P.Lv.astype(complex)
        self.Mpr = P.Mpr.astype(complex)

    def _percomp(self, f, u):
        n = self.P.nvc
        return np.concatenate([f(u[:n]), f(u[n:])])

    def M_hat_inv(self, u):
        q2b, _ = mass_bounds()
        Ms = self.P.Ms.astype(complex)
        return self._percomp(lambda x: chebyshev(Ms, x, self.s.cheb_steps, q2b), u)

    def S11_inv(self, u):
        """S^^{-1} = tau Q^{-H} M Q^{-1} (Pearson-Wathen, Sec. 4)."""
        c = self.s.mg_cycles
        a = self._percomp(lambda x: self.mgQ.solve(x, c), u)
        a = self.Mv @ a
        a = self._percomp(lambda x: self.mgQH.solve(x, c), a)
        return self.P.tau * a

    def uzawa(self, b1, b2):
        """Eq. Uzawa11 from x^(0) = 0, `uzawa_steps` steps."""
        P, t, be, mu = self.P, self.P.tau, self.P.beta, self.s.uzawa_mu
        Psi = self.d * self.Mv + t * self.Lv                     # d_j M + tau L
        PsiH = np.conj(self.d) * self.Mv + t * self.Lv.T        # (d_j M + tau L)^H
        x1 = np.zeros(P.nv, dtype=complex)
        x2 = np.zeros(P.nv, dtype=complex)
        for _ in range(self.s.uzawa_steps):
            x1 = x1 + (1.0 / t) * self.M_hat_inv(b1 - t * (self.Mv @ x1) - PsiH @ x2)
            x2 = x2 - (1.0 / mu) * self.S11_inv(b2 - Psi @ x1 + (t / be) * (self.Mv @ x2))
        return x1, x2

    def schur_inv(self, a, b):
        """S^_j^{-1} (a; b) of the commutator approximation (Sec. 4):
        [[0, (tau K_p)^{-1}], [(tau K_p)^{-1}, 0]] X_p [[0, (tau M_p)^{-1}], [(tau M_p)^{-1}, 0]]."""
        P, t, be = self.P, self.P.tau, self.P.beta
        _, q1b = mass_bounds()
        a1 = chebyshev(self.Mpr, b.astype(complex), self.s.cheb_steps, q1b) / t
        b1 = chebyshev(self.Mpr, a.astype(complex), self.s.cheb_steps, q1b) / t
        Mp, Lp = self.Mpr, P.Lpr.astype(complex)
        a2 = t * (Mp @ a1) + (np.conj(self.d) * Mp + t * Lp.T) @ b1
        b2 = (self.d * Mp + t * Lp) @ a1 - (t / be) * (Mp @ b1)
        c = self.s.mg_cycles
        y3 = self.mgKp.solve(b2, c) / t
        y4 = self.mgKp.solve(a2, c) / t
        return y3, y4

    def __call__(self, r):
        P = self.P
        r1, r2, r3, r4 = split4(P, r)
        y1, y2 = self.uzawa(r1, r2)
        t = P.tau
        a = r3 - t * (P.Bv @ y2)
        b = r4 - t * (P.Bv @ y1)
        z3, z4 = self.schur_inv(a, b)
        return np.concatenate([y1, y2, -z3, -z4])


class _TransposedMG(Multigrid):
    """MG for Q_j^H = conj(aQ) M + tau nu K + tau N^T (assembled transpose)."""

    def __init__(self, P, aM, aK, aNT, s):
        self.space = "q2"
        self.pre, self.post, self.omega = s.mg_pre, s.mg_post, s.sor_omega_conv
        self.levels = []
        for lv in range(P.level, 0, -1):
            N = 2 ** lv
            wf, skew = fem.wind_by_name(P.wind, N, P.x0, P.x1)
            ops = fem.assemble(N, P.x0, P.x1, wf, skew=skew)
            g = ops.grid
            free = g.velocity_interior()
            A = (aM * ops.M + aK * ops.K + aNT * ops.N.T)[free][:, free].tocsr()
            L = _Level()
            L.N, L.free, L.A, L.diag = N, free, A, A.diagonal()
            ix, iy = free % g.n2, free // g.n2
            col = (ix % 3) + 3 * (iy % 3)
            L.colours = [np.flatnonzero(col == c) for c in range(9)]
            L.rows = [A[idx] for idx in L.colours]
            self.levels.append(L)
        for l in range(len(self.levels) - 1):
            fine, coarse = self.levels[l], self.levels[l + 1]
            Pf = fem.prolongation_2d(coarse.N, 2)
            fine.P = Pf[fine.free][:, coarse.free].tocsr()
        self.coarse_lu = sla.lu_factor(self.levels[-1].A.toarray())


# --------------------------------------------------------------------------
# Inner GMRES (complex, right preconditioned)
# --------------------------------------------------------------------------
def givens(a, b):
    """Complex Givens rotation (c real, s complex) with
    [c, s; -conj(s), c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b) + 0.0j
    t = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    ph = a / abs(a)
    return abs(a) / t, ph * np.conj(b) / t, ph * t


def gmres(A, Pinv, s, tol, maxit, fixed_its=0):
    """Right-preconditioned GMRES from x0 = 0 (reading R15).

    Stores Z_i = Pinv(V_i) and returns x = sum y_i Z_i (identical to
    x = Pinv(V y) for a linear Pinv).  Stops when |g_{i+1}| <= tol ||s|| or,
    with fixed_its > 0, after exactly fixed_its iterations.
    Returns (x, iterations).
    """
    Amul = (lambda v: A @ v) if not callable(A) else A
    n = len(s)
    s = s.astype(complex)
    beta0 = np.linalg.norm(s)
    if beta0 == 0:
        return np.zeros(n, dtype=complex), 0
    m = fixed_its if fixed_its > 0 else maxit
    V = np.zeros((m + 1, n), dtype=complex)
    Zs = np.zeros((m, n), dtype=complex)
    H = np.zeros((m + 1, m), dtype=complex)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=complex)
    g = np.zeros(m + 1, dtype=complex)
    g[0] = beta0
    V[0] = s / beta0
    k = 0
    for i in range(m):
        Zs[i] = Pinv(V[i])
        w = Amul(Zs[i])
        for l in range(i + 1):
            H[l, i] = np.vdot(V[l], w)
            w = w - H[l, i] * V[l]
        hn = np.linalg.norm(w)
        H[i + 1, i] = hn
        if hn != 0:
            V[i + 1] = w / hn
        for l in range(i):
            t = cs[l] * H[l, i] + sn[l] * H[l + 1, i]
            H[l + 1, i] = -np.conj(sn[l]) * H[l, i] + cs[l] * H[l + 1, i]
            H[l, i] = t
        cs[i], sn[i], H[i, i] = givens(H[i, i], H[i + 1, i])
        H[i + 1, i] = 0.0
        g[i + 1] = -np.conj(sn[i]) * g[i]
        g[i] = cs[i] * g[i]
        k = i + 1
        if fixed_its == 0 and abs(g[i + 1]) <= tol * beta0:
            break
        if hn == 0:
            break
    y = sla.solve_triangular(H[:k, :k], g[:k])
    return Zs[:k].T @ y, k


# --------------------------------------------------------------------------
# Algorithms 1 and 2 over all frequencies
# --------------------------------------------------------------------------
class PinTPreconditioner:
    """The parallel-in-time preconditioner for the whole KKT system.

    linear=True: Algorithm 1 (P~_C: one application of the block
    preconditioner per frequency).  linear=False: Algorithm 2 for Stokes /
    the Uzawa variant for Oseen (inner GMRES per frequency with the block
    preconditioner, tolerance inner_tol).  All K frequencies are processed.
    """

    def __init__(self, P, s: Settings = None, linear=False, fixed_inner_its=0):
        self.P = P
        self.s = s or Settings()
        self.linear = linear
        self.fixed = fixed_inner_its
        self._kp = Multigrid("q1", P.level, P.x0, P.x1, None, 0.0, 1.0, 0.0,
                             self.s.mg_pre, self.s.mg_post, self.s.sor_omega)
        self._blocks = {}
        self.inner_its = {}

    def block_prec(self, j):
        if j not in self._blocks:
            cls = StokesBlockPreconditioner if self.P.kind == "stokes" else OseenBlockPreconditioner
            self._blocks[j] = cls(self.P, j, self.s, self._kp)
        return self._blocks[j]

    def solve_block(self, j, rhat_g):
        """One frequency: input and output in the (v, lambda, p, mu) ordering
        of Eq. SubBlockG (the input holds the residual rows in the same slot
        order, i.e. row blocks 1..4 of G_j)."""
        P = self.P
        B = self.block_prec(j)
        if P.kind == "stokes":
            s = Tl_inverse(P, j, rhat_g)
            if self.linear:
                x = B(s)
                its = 0
            else:
                x, its = gmres(Z_matrix(P, j).astype(complex), B, s, self.s.inner_tol,
                               self.s.inner_maxit, self.fixed)
            y = Tr_inverse(P, j, x)
        else:
            if self.linear:
                y, its = B(rhat_g.astype(complex)), 0
            else:
                y, its = gmres(P.G(j).astype(complex), B, rhat_g, self.s.inner_tol,
                               self.s.inner_maxit, self.fixed)
        self.inner_its[j] = its
        return y

    def __call__(self, r, js=None):
        """Apply to a real all-at-once residual r (length P.n)."""
        P = self.P

        def block_solver(j, rhs_ylam):
            g = P.ylam_to_g(rhs_ylam)
            return P.g_to_ylam(self.solve_block(j, g))

        return P.pc_inverse(r, block_solver)[0]
