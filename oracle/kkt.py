"""All-at-once KKT system and the exact block-circulant preconditioner (FP64).

TEST INFRASTRUCTURE (oracle): see the package header.

What it follows
  * Eq. FinalA (Sec. 2.2): the permuted Kronecker form
        A = [[tau I, E^T], [E, -tau/beta I]] (x) [[M, 0], [0, 0]]
          + tau [[0, 0], [I, 0]] (x) [[L, B^T], [B, 0]]
          + tau [[0, I], [0, 0]] (x) [[L^T, B^T], [B, 0]]
    with E the lower-bidiagonal backward-Euler matrix.  Unknown ordering is
    [Y_1..Y_K, Lambda_1..Lambda_K], Y_k = (v_k, p_k), Lambda_k = (lambda_k, mu_k).
  * Sec. 2.2 backward-Euler equations for the right-hand side: the adjoint
    rows carry tau M v_d(t_k), the first state row carries M v_0, state rows
    carry tau M f_k.
  * Sec. 3.1: P_C replaces E by the circulant C; C = F^{-1} D F with
    D = diag(F c_1), so d_j = 1 - exp(-2 pi i j / K); P_C^{-1} r is the
    forward FFT along time, one solve with the frequency block per j, the
    inverse FFT.  The frequency block is Eq. SubBlockG.
  * Sec. 3.4: flexible GMRES (Saad 1993) as the outer solver.

  * Sec. 5 problems (`rhs_dirichlet`): the prescribed boundary velocity is
    a known part of the state, moved to the right-hand side; the data are
    nodal interpolants on the whole grid, loaded with the full mass rows.

Readings (the paper is ambiguous here):
  R1  K = n_t time blocks, block k <-> t_k = k tau for state and adjoint;
      lambda_{K+1} = 0, v_0 enters the right-hand side.  tau is an input.
  R2  F_{jk} = exp(-2 pi i j k / K), unnormalised; the inverse carries 1/K.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


class Problem:
    """Discrete Stokes / Oseen control problem (Sec. 2).

    kind: "stokes" or "oseen"; level: N = 2**level elements per side;
    K: number of time blocks; tau, beta, nu as in the paper; wind: None,
    "recirc" (w = (2y(1-x^2), -2x(1-y^2))), "two_vortex" (the Sec. 5.2
    wind, `fem.two_vortex_wind`) or ("nodal", W), W the wind's values at the
    Q2 nodes, shape (2, (2N+1)^2) (`fem.wind_by_name`).
    """

    def __init__(self, kind, level, K, tau, beta, nu, x0=0.0, x1=1.0, wind=None):
        self.kind = kind
        self.level = level
        self.N = 2 ** level
        self.K = K
        self.tau = float(tau)
        self.beta = float(beta)
        self.nu = float(nu)
        self.x0, self.x1 = float(x0), float(x1)
        self.wind = wind
        wf, skew = fem.wind_by_name(wind, self.N, x0, x1)
        self.ops = fem.assemble(self.N, x0, x1, wf, skew=skew)
        g = self.ops.grid
        self.grid = g
        self.vi = g.velocity_interior()
        self.pf = g.pressure_free()
        self.nvc = len(self.vi)          # velocity unknowns per component
        self.nv = 2 * self.nvc           # n_v (both components)
        self.np_ = len(self.pf)          # n_p (pinned)
        self.nb = self.nv + self.np_     # unknowns of one (v, p) block
        o = self.ops
        r = lambda A, rows, cols: A[rows][:, cols].tocsr()
        self.Ms = r(o.M, self.vi, self.vi)
        self.Ks = r(o.K, self.vi, self.vi)
        self.Ns = r(o.N, self.vi, self.vi)
        self.Ls = (self.nu * self.Ks + self.Ns).tocsr()          # L = nu K + N(w)
        self.Bxr = r(o.Bx, self.pf, self.vi)
        self.Byr = r(o.By, self.pf, self.vi)
        self.Mpr = r(o.Mp, self.pf, self.pf)
        self.Kpr = r(o.Kp, self.pf, self.pf)
        self.Npr = r(o.Np, self.pf, self.pf)
        self.Lpr = (self.nu * self.Kpr + self.Npr).tocsr()
        # vector (two-component) velocity operators
        self.Mv = sp.block_diag([self.Ms, self.Ms], format="csr")
        self.Lv = sp.block_diag([self.Ls, self.Ls], format="csr")
        self.Bv = sp.hstack([self.Bxr, self.Byr], format="csr")      # n_p x n_v
        Z = lambda a, b: sp.csr_matrix((a, b))
        self.S_M = sp.bmat([[self.Mv, None], [None, Z(self.np_, self.np_)]], format="csr")
        self.S_L = sp.bmat([[self.Lv, self.Bv.T], [self.Bv, None]], format="csr")
        self.S_LT = sp.bmat([[self.Lv.T, self.Bv.T], [self.Bv, None]], format="csr")

    # ------------------------------------------------------------------ sizes
    @property
    def n(self):
        """Total unknowns 2 K (n_v + n_p)."""
        return 2 * self.K * self.nb

    # --------------------------------------------------------------- matrices
    def time_matrix(self, circulant=False):
        """E (backward Euler) or its circulant perturbation C (Sec. 3.1)."""
        K = self.K
        E = np.eye(K) - np.eye(K, k=-1)
        if circulant:
            E[0, K - 1] -= 1.0
        return sp.csr_matrix(E)

    def kkt_matrix(self, circulant=False):
        """Eq. FinalA (circulant=False) or P_C (circulant=True)."""
        K = self.K
        E = self.time_matrix(circulant)
        I = sp.eye(K, format="csr")
        T1 = sp.bmat([[self.tau * I, E.T], [E, -(self.tau / self.beta) * I]], format="csr")
        O = sp.csr_matrix((K, K))
        T2 = sp.bmat([[O, None], [I, O]], format="csr")      # [[0, 0], [I, 0]]
        T3 = sp.bmat([[O, I], [None, O]], format="csr")      # [[0, I], [0, 0]]
        A = sp.kron(T1, self.S_M) + self.tau * sp.kron(T2, self.S_L) + self.tau * sp.kron(T3, self.S_LT)
        return A.tocsr()

    def kkt_rows(self, x, block_rows):
        """Selected block rows of A x (Eq. FinalA) without assembling A.

        The Kronecker form is sum_t T_t (x) S_t with 2K x 2K time matrices
        T_1 = [[tau I, E^T], [E, -tau/beta I]], T_2 = tau [[0, 0], [I, 0]],
        T_3 = tau [[0, I], [0, 0]] and spatial blocks S_M, S_L, S_LT; block row
        r of A x is sum_t sum_c T_t[r, c] S_t x_c.  block_rows: indices r in
        [0, 2K) (r < K: adjoint-equation rows of time block r; r >= K: state
        rows of block r - K).  Returns {r: vector of length nb}.
        """
        K, nb = self.K, self.nb
        X = x.reshape(2 * K, nb)
        E = self.time_matrix()
        I = sp.eye(K, format="csr")
        O = sp.csr_matrix((K, K))
        T1 = sp.bmat([[self.tau * I, E.T], [E, -(self.tau / self.beta) * I]], format="csr")
        T2 = self.tau * sp.bmat([[O, None], [I, O]], format="csr")
        T3 = self.tau * sp.bmat([[O, I], [None, O]], format="csr")
        out = {}
        for r in block_rows:
            y = np.zeros(nb)
            for T, S in ((T1, self.S_M), (T2, self.S_L), (T3, self.S_LT)):
                row = T.getrow(r)
                for c, v in zip(row.indices, row.data):
                    y += v * (S @ X[c])
            out[r] = y
        return out

    # -------------------------------------------------------- right-hand side
    def rhs(self, vd, f=None, v0=None):
        """Right-hand side from the backward-Euler equations (Sec. 2.2).

        vd: (K, 2, ns) desired velocity at t_k = k tau on the full Q2 grid;
        f:  (K, 2, ns) forcing or None; v0: (2, ns) initial velocity or None.
        """
        K, nb, nvc = self.K, self.nb, self.nvc
        b = np.zeros((2, K, nb))
        for k in range(K):
            for c in range(2):
                vdc = vd[k, c, self.vi]
                b[0, k, c * nvc:(c + 1) * nvc] = self.tau * (self.Ms @ vdc)
                if f is not None:
                    b[1, k, c * nvc:(c + 1) * nvc] += self.tau * (self.Ms @ f[k, c, self.vi])
        if v0 is not None:
            for c in range(2):
                b[1, 0, c * nvc:(c + 1) * nvc] += self.Ms @ v0[c, self.vi]
        return b.ravel()

    def rhs_dirichlet(self, vd, f=None, v0=None, g=None):
        """Right-hand side with non-zero Dirichlet velocity data (the Sec. 5 problems).

        The state velocity on the full Q2 grid is v_k = (interior unknowns) +
        (boundary values g_k); the adjoint velocity is zero on the boundary.
        The data vd, f, v0 are nodal interpolants on the full grid, so each
        load is the full-grid mass row M_{I,:} times the nodal vector.  Write
        kn_k for the known part of the state at t_k: g_k on the boundary and 0
        inside for k >= 1, the whole of v0 for k = 0.  Moving the known
        columns of the Sec. 2.2 backward-Euler equations to the right gives
          adjoint velocity rows  tau M_{I,:} vd_k - tau M_{I,:} kn_k
          state velocity rows    tau M_{I,:} f_k - M_{I,:} (kn_k - kn_{k-1}) - tau L_{I,:} kn_k
          state pressure rows    -tau B_{free,:} kn_k
        and zero adjoint pressure rows.  With g = None and v0, vd, f zero on
        the boundary this equals `rhs`.  Shapes as in `rhs`; g: (K, 2, ns)
        (interior entries ignored) or None.
        """
        K, nb, nvc, nv = self.K, self.nb, self.nvc, self.nv
        o, vi, pf, tau = self.ops, self.vi, self.pf, self.tau
        ns = o.grid.ns
        bnd = np.setdiff1d(np.arange(ns), vi)
        MI = o.M[vi]                                     # M_{I,:}
        LI = (self.nu * o.K + o.N)[vi]                   # L_{I,:}
        Bf = (o.Bx[pf], o.By[pf])                        # B_{free,:} per component

        def known(k):
            kn = np.zeros((2, ns))
            if k == 0:
                if v0 is not None:
                    kn[:] = v0
            elif g is not None:
                kn[:, bnd] = g[k - 1][:, bnd]
            return kn

        b = np.zeros((2, K, nb))
        for k in range(1, K + 1):
            kn, kp = known(k), known(k - 1)
            for c in range(2):
                s = slice(c * nvc, (c + 1) * nvc)
                b[0, k - 1, s] = tau * (MI @ vd[k - 1, c]) - tau * (MI @ kn[c])
                load = tau * (MI @ f[k - 1, c]) if f is not None else 0.0
                b[1, k - 1, s] = load - MI @ (kn[c] - kp[c]) - tau * (LI @ kn[c])
            b[1, k - 1, nv:] = -tau * (Bf[0] @ kn[0] + Bf[1] @ kn[1])
        return b.ravel()

    def full_velocity(self, x, g=None):
        """State velocity of a KKT solution x on the full Q2 grid, (K, 2, ns):
        the interior unknowns plus the boundary values of g (Sec. 5 data)."""
        K, nb, nvc = self.K, self.nb, self.nvc
        ns = self.ops.grid.ns
        X = x.reshape(2, K, nb)[0]
        out = np.zeros((K, 2, ns))
        if g is not None:
            bnd = np.setdiff1d(np.arange(ns), self.vi)
            out[:, :, bnd] = g[:, :, bnd]
        for c in range(2):
            out[:, c, self.vi] = X[:, c * nvc:(c + 1) * nvc]
        return out

    # ----------------------------------------------------- frequency blocks
    def d(self, j):
        """j-th eigenvalue of C: d_j = 1 - exp(-2 pi i j / K)  (Sec. 3.1)."""
        return 1.0 - np.exp(-2j * np.pi * j / self.K)

    def G_bar(self, j):
        """Frequency block in (Y, Lambda) ordering:
        [[tau S_M, conj(d) S_M + tau S_LT], [d S_M + tau S_L, -tau/beta S_M]]."""
        dj = self.d(j)
        t, b = self.tau, self.beta
        return sp.bmat([[t * self.S_M, np.conj(dj) * self.S_M + t * self.S_LT],
                        [dj * self.S_M + t * self.S_L, -(t / b) * self.S_M]], format="csc")

    def G(self, j):
        """Eq. SubBlockG in the (v, lambda, p, mu) ordering."""
        dj = self.d(j)
        t, b = self.tau, self.beta
        M, L, B = self.Mv, self.Lv, self.Bv
        nv, npp = self.nv, self.np_
        Zp = sp.csr_matrix((npp, npp))
        return sp.bmat([[t * M, np.conj(dj) * M + t * L.T, None, t * B.T],
                        [dj * M + t * L, -(t / b) * M, t * B.T, None],
                        [None, t * B, Zp, None],
                        [t * B, None, None, Zp]], format="csr")

    # ------------------------------------------------ orderings (per block)
    def ylam_to_g(self, yl):
        """(Y, Lambda) frequency vector -> (v, lambda, p, mu) ordering."""
        nv, nb = self.nv, self.nb
        y, l = yl[:nb], yl[nb:]
        return np.concatenate([y[:nv], l[:nv], y[nv:], l[nv:]])

    def g_to_ylam(self, g):
        nv, npp = self.nv, self.np_
        v, lam, p, mu = g[:nv], g[nv:2 * nv], g[2 * nv:2 * nv + npp], g[2 * nv + npp:]
        return np.concatenate([v, p, lam, mu])

    # ------------------------------------------ exact P_C^{-1} via the FFT
    def pc_inverse(self, r, block_solver=None):
        """P_C^{-1} r by diagonalisation (Sec. 3.1):  r^ = F r along time,
        one block solve per frequency, then F^{-1}.  `block_solver(j, rhs)`
        defaults to a sparse LU solve with G_bar(j) (factorisations cached);
        all K frequencies are solved (no Hermitian shortcut), and the real
        part is returned."""

        K, nb = self.K, self.nb
        R = r.reshape(2, K, nb)
        Rh = np.fft.fft(R, axis=1)                     # F along time, per group
        Yh = np.empty_like(Rh)
        if block_solver is None and not hasattr(self, "_lu"):
            self._lu = {}
        for j in range(K):
            rhs = np.concatenate([Rh[0, j], Rh[1, j]])
            if block_solver is None:
                if j not in self._lu:
                    self._lu[j] = spla.splu(self.G_bar(j))
                sol = self._lu[j].solve(rhs)
            else:
                sol = block_solver(j, rhs)
            Yh[0, j], Yh[1, j] = sol[:nb], sol[nb:]
        Y = np.fft.ifft(Yh, axis=1)
        return Y.real.ravel(), Y

    def reference_solution(self, b, tol=1e-12):
        """Reference solution of A x = b: FP64 FGMRES preconditioned by the
        exact P_C^{-1} (Theorem 1 bounds its iterations by 2 n_v + 1)."""
        x, info = fgmres(self.kkt_matrix(), b, lambda v: self.pc_inverse(v)[0], tol=tol,
                         restart=min(200, 2 * self.nv + 2), maxit=4 * self.nv + 10)
        return x, info


def fgmres(A, b, Pinv, x0=None, restart=30, tol=1e-8, maxit=1000):
    """Flexible GMRES (Saad 1993) with right preconditioning, modified
    Gram-Schmidt and Givens rotations, FP64.

    Pinv(v) may change from call to call.  Stops when the TRUE relative
    residual ||b - A x|| / ||b|| <= tol (checked at each restart and when the
    Arnoldi estimate reaches tol).  Returns (x, info) with info holding the
    total iteration count and the residual history.
    """
    Amul = (lambda v: A @ v) if not callable(A) else A
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    hist = []
    its = 0
    if bnorm == 0:
        return x, {"its": 0, "relres": 0.0, "hist": hist}
    r = b - Amul(x)
    relres = np.linalg.norm(r) / bnorm
    while its < maxit and relres > tol:
        beta0 = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n))
        Zs = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta0
        V[0] = r / beta0
        k_done = 0
        for i in range(m):
            Zs[i] = Pinv(V[i])
            w = Amul(Zs[i])
            for k in range(i + 1):
                H[k, i] = np.dot(V[k], w)
                w = w - H[k, i] * V[k]
            H[i + 1, i] = np.linalg.norm(w)
            if H[i + 1, i] != 0:
                V[i + 1] = w / H[i + 1, i]
            for k in range(i):
                t = cs[k] * H[k, i] + sn[k] * H[k + 1, i]
                H[k + 1, i] = -sn[k] * H[k, i] + cs[k] * H[k + 1, i]
                H[k, i] = t
            den = np.hypot(H[i, i], H[i + 1, i])
            cs[i], sn[i] = H[i, i] / den, H[i + 1, i] / den
            H[i, i] = den
            H[i + 1, i] = 0.0
            g[i + 1] = -sn[i] * g[i]
            g[i] = cs[i] * g[i]
            its += 1
            k_done = i + 1
            hist.append(abs(g[i + 1]) / bnorm)
            if abs(g[i + 1]) <= tol * bnorm or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + Zs[:k_done].T @ y
        r = b - Amul(x)
        relres = np.linalg.norm(r) / bnorm
    return x, {"its": its, "relres": relres, "hist": hist}
