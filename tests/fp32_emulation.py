"""FP32 execution of the oracle's nested preconditioner (test helper).

The oracle (oracle/inexact.py) states the method in FP64.  An FP32
preconditioner cannot match it to FP64 accuracy: the inner GMRES of the
frequency blocks (Sec. 3.4, Algorithm 2) amplifies any perturbation of its
preconditioned vectors (at 64 x 64, n_t = 256 a relative change of 6e-8 in
the stored vectors moves a three-step block solve at j = K/4 by up to 4e-5).
This module runs the oracle's own operators and steps with the storage and
arithmetic of an FP32 preconditioner, so that a test can state how far FP32
execution of the method itself lands from its FP64 result, and hold the GPU
to a multiple of that:

  * multigrid sweeps, residuals and transfers in complex64 on the oracle's
    level matrices rounded once to FP32; inverse diagonals rounded from FP64;
    the corner-pinned pressure Laplacian in difference form
    (sum_k a_ik (x_k - x_i) + row sum x_i, the pinned value 0), coarsest
    solve in FP64 rounded to FP32;
  * Chebyshev semi-iteration in complex64 (coefficients formed in FP64);
  * block preconditioners, Uzawa steps and the Stokes transforms in
    complex64 with coefficients rounded to FP32;
  * inner GMRES with complex64 Krylov vectors, Gram-Schmidt coefficients
    formed in FP64 from the stored vectors and applied in FP32 (two passes),
    FP64 Givens and least squares, the update sum_l y_l Z_l accumulated in
    FP64 and rounded once.

It imports the oracle and numpy/scipy only.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem, inexact

# storage and arithmetic types (a test sets them to complex128 / float64 to
# check that the emulation is the oracle's method step for step)
C64 = np.complex64
F32 = np.float32


def r32(v):
    return np.asarray(v).astype(C64)



class Multigrid32:
    """The V-cycles of an oracle Multigrid (same levels, colours, sweep
    order, transfers and coarse solve) in FP32.  diff_form: evaluate rows in
    difference form (the pinned pressure Laplacian)."""

    def __init__(self, mg, diff_form=False, full_rows=None):
        self.mg = mg
        self.omega = F32(mg.omega)
        self.diff = diff_form
        self.lev = []
        for li, L in enumerate(mg.levels):
            e = {}
            e["A"] = L.A.astype(C64).tocsr()
            e["rows"] = [r.astype(C64).tocsr() for r in L.rows]
            e["col"] = L.colours
            e["dinv"] = (1.0 / L.diag).astype(C64)
            if hasattr(L, "P"):
                e["P"] = L.P.astype(F32).tocsr()
            if diff_form:
                # full rows including the pinned column (x there is 0), FP32 entries;
                # row sums formed in FP64 and rounded once
                Af, free = full_rows[li]
                Af = Af.tocsr()
                e["full"] = Af[free].astype(C64).tocsr()
                e["free"] = free
                e["n"] = Af.shape[0]
                e["rs"] = np.asarray(Af[free].sum(axis=1)).ravel().astype(C64)
            self.lev.append(e)

    def _diff_rows(self, e, idx):
        """Cached CSR pieces of the full rows idx for the difference form."""
        key = ("d", id(idx))
        if key not in e:
            F = e["full"][idx].tocsr()
            rep = np.repeat(np.arange(len(idx)), np.diff(F.indptr))
            offd = F.indices != e["free"][idx][rep]
            e[key] = (F.indices, F.data * offd, rep, F.indptr[:-1].copy(), e["rs"][idx])
        return e[key]

    def _ax(self, e, x, rows=None):
        """(A x) at the given rows (all if None), FP32."""
        if not self.diff:
            A = e["A"] if rows is None else e["rows"][rows]
            return A @ x
        idx = e.setdefault("all", np.arange(len(e["free"]))) if rows is None else e["col"][rows]
        cols, vals, rep, starts, rs = self._diff_rows(e, idx)
        xf = np.zeros(e["n"], dtype=C64)
        xf[e["free"]] = x
        xi = x[idx]
        prods = (vals * (xf[cols] - xi[rep])).astype(C64)
        return (rs * xi + np.add.reduceat(prods, starts)).astype(C64)

    def _sweep(self, e, x, b, order):
        for c in order:
            idx = e["col"][c]
            r = b[idx] - self._ax(e, x, c)
            x[idx] = x[idx] + self.omega * (e["dinv"][idx] * r)
        return x

    def vcycle(self, l, x, b):
        e = self.lev[l]
        if l == len(self.lev) - 1:
            return r32(sla.lu_solve(self.mg.coarse_lu, b.astype(complex)))
        nc = len(e["col"])
        for _ in range(self.mg.pre):
            x = self._sweep(e, x, b, range(nc))
        r = b - self._ax(e, x)
        bc = (e["P"].T @ r).astype(C64)
        xc = self.vcycle(l + 1, np.zeros_like(bc), bc)
        x = x + (e["P"] @ xc).astype(C64)
        for _ in range(self.mg.post):
            x = self._sweep(e, x, b, range(nc - 1, -1, -1))
        return x

    def solve(self, b, cycles):
        b = r32(b)
        x = np.zeros(len(b), dtype=C64)
        for _ in range(cycles):
            x = self.vcycle(0, x, b)
        return x


def pressure_full_rows(level, x0, x1, aM, aK):
    """Per multigrid level: the full Q1 matrix aM M_p + aK K_p (pinned node
    included) and the free (unpinned) node indices."""
    out = []
    for lv in range(level, 0, -1):
        ops = fem.assemble(2 ** lv, x0, x1, None)
        out.append(((aM * ops.Mp + aK * ops.Kp).tocsr(), ops.grid.pressure_free()))
    return out


def chebyshev32(A, b, steps, bounds):
    """inexact.chebyshev in FP32 (recurrence coefficients formed in FP64)."""
    lmin, lmax = bounds
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    A32 = A.astype(C64).tocsr()
    dinv = (1.0 / A.diagonal().real).astype(F32)
    rho = 1.0 / sigma
    b = r32(b)
    x = np.zeros_like(b)
    r = b.copy()
    d = ((dinv / F32(theta)) * r).astype(C64)
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        r = r - A32 @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        c1, c2 = F32(rho_new * rho), F32(2.0 * rho_new / delta)
        d = (c1 * d + (c2 * dinv) * r).astype(C64)
        rho = rho_new
    return x


class StokesBlock32:
    """P~_j^{-1} of the Stokes block (Sec. 3.2) in FP32."""

    def __init__(self, P, blk, kp32):
        self.P, self.blk = P, blk
        self.mgW = Multigrid32(blk.mgW)
        self.mgKp = kp32
        self.c1, self.c2 = blk.c1, blk.c2

    def __call__(self, u):
        P, s = self.P, self.blk.s
        n = P.nvc
        u1, u2, u3, u4 = inexact.split4(P, r32(u))
        W = lambda v: np.concatenate([self.mgW.solve(v[:n], s.mg_cycles), self.mgW.solve(v[n:], s.mg_cycles)])
        _, q1b = inexact.mass_bounds()
        sa, sb = C64(1.0 + self.c1), C64(P.nu * self.c2)
        S = lambda v: (sa * self.mgKp.solve(v, s.mg_cycles) + sb * chebyshev32(P.Mpr, v, s.cheb_steps, q1b))
        return np.concatenate([W(u1), W(u2), S(u3), S(u4)]).astype(C64)


class OseenBlock32:
    """(P~_j^(UZ))^{-1} of Algorithm 3 (Sec. 4) in FP32."""

    def __init__(self, P, blk, kp32):
        self.P, self.blk = P, blk
        self.mgQ = Multigrid32(blk.mgQ)
        self.mgQH = Multigrid32(blk.mgQH)
        self.mgKp = kp32
        t, d = P.tau, blk.d
        self.Mv = P.Mv.astype(C64).tocsr()
        self.Psi = (d * P.Mv + t * P.Lv).astype(C64).tocsr()
        self.PsiH = (np.conj(d) * P.Mv + t * P.Lv.T).astype(C64).tocsr()
        self.Mp = P.Mpr.astype(C64).tocsr()
        Lp = P.Lpr.astype(complex)
        self.Xa = (np.conj(d) * P.Mpr + t * Lp.T).astype(C64).tocsr()
        self.Xb = (d * P.Mpr + t * Lp).astype(C64).tocsr()
        self.Bv = P.Bv.astype(C64).tocsr()

    def _percomp(self, f, u):
        n = self.P.nvc
        return np.concatenate([f(u[:n]), f(u[n:])]).astype(C64)

    def __call__(self, r):
        P, s = self.P, self.blk.s
        t, be, mu = C64(P.tau), C64(P.beta), C64(s.uzawa_mu)
        q2b, q1b = inexact.mass_bounds()
        r1, r2, r3, r4 = inexact.split4(P, r32(r))
        c = s.mg_cycles
        x1 = np.zeros(P.nv, dtype=C64)
        x2 = np.zeros(P.nv, dtype=C64)
        Ms = P.Ms.astype(complex)
        for _ in range(s.uzawa_steps):
            g = r1 - t * (self.Mv @ x1) - self.PsiH @ x2
            x1 = x1 + C64(1.0 / P.tau) * self._percomp(lambda v: chebyshev32(Ms, v, s.cheb_steps, q2b), g)
            h = r2 - self.Psi @ x1 + C64(P.tau / P.beta) * (self.Mv @ x2)
            a = self._percomp(lambda v: self.mgQ.solve(v, c), h)
            a = self.Mv @ a
            a = self._percomp(lambda v: self.mgQH.solve(v, c), a)
            x2 = x2 - C64(P.tau / s.uzawa_mu) * a
        a3 = r3 - t * (self.Bv @ x2)
        b4 = r4 - t * (self.Bv @ x1)
        a1 = chebyshev32(P.Mpr, b4, s.cheb_steps, q1b) * C64(1.0 / P.tau)
        b1 = chebyshev32(P.Mpr, a3, s.cheb_steps, q1b) * C64(1.0 / P.tau)
        a2 = t * (self.Mp @ a1) + self.Xa @ b1
        b2 = self.Xb @ a1 - C64(P.tau / P.beta) * (self.Mp @ b1)
        y3 = self.mgKp.solve(b2, c) * C64(1.0 / P.tau)
        y4 = self.mgKp.solve(a2, c) * C64(1.0 / P.tau)
        return np.concatenate([x1, x2, -y3, -y4]).astype(C64)


def gmres32(A, Pinv, s, tol, maxit, fixed_its=0):
    """inexact.gmres with FP32 Krylov vectors: operator and preconditioner
    applied in FP32, classical Gram-Schmidt with one reorthogonalisation
    (coefficients formed in FP64 from the stored vectors, applied in FP32),
    FP64 Hessenberg, Givens rotations and least squares, the update
    accumulated in FP64 and rounded once."""
    A32 = A.astype(C64).tocsr()
    s = r32(s)
    beta0 = np.linalg.norm(s.astype(complex))
    if beta0 == 0:
        return np.zeros(len(s), dtype=C64), 0
    m = fixed_its if fixed_its > 0 else maxit
    V = np.zeros((m + 1, len(s)), dtype=C64)
    Zs = np.zeros((m, len(s)), dtype=C64)
    H = np.zeros((m + 1, m), dtype=complex)
    cs, sn = np.zeros(m), np.zeros(m, dtype=complex)
    g = np.zeros(m + 1, dtype=complex)
    g[0] = beta0
    V[0] = (s / F32(beta0)).astype(C64)
    k = 0
    for i in range(m):
        Zs[i] = r32(Pinv(V[i]))
        w = (A32 @ Zs[i]).astype(C64)
        Vd = V[:i + 1].astype(complex)
        h1 = Vd.conj() @ w.astype(complex)
        for l in range(i + 1):
            w = (w - C64(h1[l]) * V[l]).astype(C64)
        h2 = Vd.conj() @ w.astype(complex)
        for l in range(i + 1):
            w = (w - C64(h2[l]) * V[l]).astype(C64)
        H[:i + 1, i] = h1 + h2
        hn = np.linalg.norm(w.astype(complex))
        H[i + 1, i] = hn
        if hn != 0:
            V[i + 1] = (w / F32(hn)).astype(C64)
        for l in range(i):
            t = cs[l] * H[l, i] + sn[l] * H[l + 1, i]
            H[l + 1, i] = -np.conj(sn[l]) * H[l, i] + cs[l] * H[l + 1, i]
            H[l, i] = t
        cs[i], sn[i], H[i, i] = inexact.givens(H[i, i], H[i + 1, i])
        H[i + 1, i] = 0.0
        g[i + 1] = -np.conj(sn[i]) * g[i]
        g[i] = cs[i] * g[i]
        k = i + 1
        if fixed_its == 0 and abs(g[i + 1]) <= tol * beta0:
            break
        if hn == 0:
            break
    y = sla.solve_triangular(H[:k, :k], g[:k])
    return r32(Zs[:k].astype(complex).T @ y), k


def _tl_inv32(P, j, r):
    _, _, dc, _, c2 = inexact.stokes_constants(P, j)
    sq = np.sqrt(P.tau)
    r1, r2, r3, r4 = inexact.split4(P, r32(r))
    s1 = r1 * C64(1.0 / sq)
    s2 = (r2 - C64(1j * dc / sq) * s1) * C64(c2 / sq)
    s3 = r3 * C64(1.0 / (sq * c2))
    s4 = (r4 - C64(1j * dc * c2 / sq) * s3) * C64(1.0 / sq)
    return np.concatenate([s1, s2, s3, s4]).astype(C64)


def _tr_inv32(P, j, x):
    _, _, dc, _, c2 = inexact.stokes_constants(P, j)
    sq = np.sqrt(P.tau)
    x1, x2, x3, x4 = inexact.split4(P, r32(x))
    y2 = x2 * C64(c2 / sq)
    y1 = (x1 + C64(1j * dc / sq) * y2) * C64(1.0 / sq)
    y4 = x4 * C64(1.0 / sq)
    y3 = (x3 + C64(1j * dc * c2 / sq) * y4) * C64(1.0 / (sq * c2))
    return np.concatenate([y1, y2, y3, y4]).astype(C64)


class PinT32:
    """Frequency-block solves of inexact.PinTPreconditioner (Algorithm 2 /
    the Uzawa variant) executed in FP32."""

    def __init__(self, P, s=None, fixed_inner_its=0, linear=False):
        self.P = P
        self.s = s or inexact.Settings()
        self.ref = inexact.PinTPreconditioner(P, self.s, fixed_inner_its=fixed_inner_its)
        self.fixed = fixed_inner_its
        self.linear = linear
        rows = pressure_full_rows(P.level, P.x0, P.x1, 0.0, 1.0)
        self.kp32 = Multigrid32(self.ref._kp, diff_form=True, full_rows=rows)
        self._blocks = {}

    def block(self, j):
        if j not in self._blocks:
            b = self.ref.block_prec(j)
            cls = StokesBlock32 if self.P.kind == "stokes" else OseenBlock32
            self._blocks[j] = cls(self.P, b, self.kp32)
        return self._blocks[j]

    def solve_block(self, j, rhat_g):
        """Input and output as inexact.PinTPreconditioner.solve_block; the
        result is FP32 (returned as complex128)."""
        P, B, s = self.P, self.block(j), self.s
        if self.linear:  # Algorithm 1: one application of the block preconditioner
            if P.kind == "stokes":
                return _tr_inv32(P, j, B(_tl_inv32(P, j, rhat_g))).astype(complex)
            return B(r32(rhat_g)).astype(complex)
        if P.kind == "stokes":
            x, _ = gmres32(inexact.Z_matrix(P, j).astype(complex), B, _tl_inv32(P, j, rhat_g), s.inner_tol,
                           s.inner_maxit, self.fixed)
            return _tr_inv32(P, j, x).astype(complex)
        y, _ = gmres32(P.G(j).astype(complex), B, r32(rhat_g), s.inner_tol, s.inner_maxit, self.fixed)
        return y.astype(complex)
