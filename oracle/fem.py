"""Q2-Q1 Taylor-Hood finite-element operators on a uniform square grid (FP64).

TEST INFRASTRUCTURE (oracle): see the package header.  Nothing here is used
by the CUDA library.

The paper discretises the optimality system with Taylor-Hood elements in
space (Sec. 2.2, "P2-P1 ... and Q2-Q1"); the matrices named there are

  M   velocity mass matrix                  (Sec. 2.2)
  L   weak form of -nu Laplace + w . grad   (Sec. 2.2), L = nu K + N(w)
  B   discretised *negative* divergence     (Sec. 2.2)
  M_p, K_p, L_p = nu K_p + N_p(w)           pressure-space mass, stiffness,
                                            convection-diffusion (Sec. 2.3,
                                            commutator argument)

Everything is assembled by a plain element loop with a generic Lagrange
basis evaluated at 4x4 Gauss points (exact for every integrand of the
polynomial recirculating wind).  Readings where the paper is silent:
velocity boundary nodes carry Dirichlet conditions and are eliminated (their
values, when not zero, enter the right-hand side: `kkt.Problem.rhs_dirichlet`);
the pressure is pinned at the lower-left Q1 node (index 0), "one
pre-defined point" (Sec. 2.2); K_p and N_p use natural boundary conditions.
Winds: the recirculating wind; the Sec. 5.2 two-vortex wind, whose printed
second branch is read as the divergence-free vortex about (-1/2, 0); a
caller-given nodal wind (its Q2 interpolant, injected to coarser grids).
The last two are not polynomials, so their convection matrices are taken in
the skew-symmetric form (N - N^T)/2 (`wind_by_name`).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# 1-D Lagrange bases and Gauss quadrature
# --------------------------------------------------------------------------
def lagrange(nodes, x):
    """Values and first derivatives of the Lagrange basis on `nodes` at `x`.

    Returns (val, der) with shapes (len(nodes), len(x)).  Written from the
    product formula phi_a(x) = prod_{b != a} (x - n_b) / (n_a - n_b).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    val = np.ones((n, len(x)))
    der = np.zeros((n, len(x)))
    for a in range(n):
        for b in range(n):
            if b != a:
                val[a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            der[a] += term
    return val, der


Q2_REF_NODES = np.array([0.0, 0.5, 1.0])
Q1_REF_NODES = np.array([0.0, 1.0])


def gauss01(npts=4):
    """Gauss-Legendre points and weights mapped to [0, 1]."""
    g, w = np.polynomial.legendre.leggauss(npts)
    return (g + 1.0) / 2.0, w / 2.0


def element_matrices_1d(degree, h, npts=4):
    """1-D element mass and stiffness matrices of the Lagrange element of
    `degree` (1 or 2) on an interval of length h, by quadrature."""
    nodes = Q2_REF_NODES if degree == 2 else Q1_REF_NODES
    xi, w = gauss01(npts)
    val, der = lagrange(nodes, xi)
    mass = h * np.einsum("aq,bq,q->ab", val, val, w)
    stiff = (1.0 / h) * np.einsum("aq,bq,q->ab", der, der, w)
    return mass, stiff


# --------------------------------------------------------------------------
# Wind
# --------------------------------------------------------------------------
def recirculating_wind(x, y):
    """w = (2y(1-x^2), -2x(1-y^2)): divergence free, tangential on the
    boundary of [-1,1]^2."""
    return 2.0 * y * (1.0 - x * x), -2.0 * x * (1.0 - y * y)


TWO_VORTEX_A = 100.0 / 99.0     # 1 / semi-axis in y of both vortices
TWO_VORTEX_B = 100.0 / 49.0     # 1 / semi-axis in x


def two_vortex_wind(x, y):
    """Sec. 5.2 wind: two elliptic vortices centred at (1/2, 0) and (-1/2, 0).

    c1 = 1 - sqrt((B (x - 1/2))^2 + (A y)^2), c2 likewise about x = -1/2;
    w = c1 (A^2 y, -B^2 (x - 1/2)) where c1 >= 0, w = c2 (-A^2 y, B^2 (x + 1/2))
    where c2 >= 0, else 0.  The printed second branch is garbled; this
    reading is the one that makes it a divergence-free vortex about its own
    centre, turning the other way.  w is Lipschitz, zero outside the two
    ellipses (so on the boundary of [-1,1]^2) and divergence free.
    """
    A, B = TWO_VORTEX_A, TWO_VORTEX_B
    c1 = 1.0 - np.sqrt((B * (x - 0.5)) ** 2 + (A * y) ** 2)
    c2 = 1.0 - np.sqrt((B * (x + 0.5)) ** 2 + (A * y) ** 2)
    wx = np.where(c1 >= 0, c1 * A * A * y, np.where(c2 >= 0, -c2 * A * A * y, 0.0))
    wy = np.where(c1 >= 0, -c1 * B * B * (x - 0.5), np.where(c2 >= 0, c2 * B * B * (x + 0.5), 0.0))
    return wx, wy


def q2_interpolant(W, N, x0, x1):
    """(x, y) -> (wx, wy): the Q2 interpolant of nodal values W, shape
    (2, (2N+1)^2) with node index iy*(2N+1)+ix, on the N x N grid of
    [x0, x1]^2 (a caller-given nodal wind)."""
    W = np.asarray(W, dtype=np.float64).reshape(2, 2 * N + 1, 2 * N + 1)
    h = (x1 - x0) / N

    def wind(x, y):
        shape = np.shape(x)
        x, y = np.ravel(x), np.ravel(y)
        ex = np.clip(np.floor((x - x0) / h).astype(int), 0, N - 1)
        ey = np.clip(np.floor((y - x0) / h).astype(int), 0, N - 1)
        vx, _ = lagrange(Q2_REF_NODES, (x - x0) / h - ex)        # (3, n)
        vy, _ = lagrange(Q2_REF_NODES, (y - x0) / h - ey)
        out = []
        for c in range(2):
            acc = np.zeros_like(x)
            for b in range(3):
                for a in range(3):
                    acc += vx[a] * vy[b] * W[c, 2 * ey + b, 2 * ex + a]
            out.append(acc.reshape(shape))
        return out[0], out[1]
    return wind


def inject_q2(W, N, Nc):
    """Nodal values on the nested coarse grid with Nc elements per side: the
    coarse Q2 nodes are fine nodes (every (N/Nc)-th), so this is a copy."""
    r = N // Nc
    W = np.asarray(W, dtype=np.float64).reshape(2, 2 * N + 1, 2 * N + 1)
    return W[:, ::r, ::r].reshape(2, -1).copy()


def wind_by_name(name, N=None, x0=None, x1=None):
    """(callable or None, skew): the wind on the grid with N elements per side
    of [x0, x1]^2 and whether its convection matrices are taken in
    skew-symmetric form.  The recirculating wind is a polynomial that the
    quadrature integrates exactly, so its N is already skew (w . n = 0 on the
    boundary, div w = 0); for the two-vortex wind and for a caller-given
    nodal wind it is not, and N is replaced by (N - N^T)/2, the discrete form
    of the skew-symmetric convection (u, w . grad v) - (v, w . grad u) / 2
    terms, which equals N for exact integration of a divergence-free wind.
    name: None, "recirc", "two_vortex" or ("nodal", W) with W the nodal
    values (2, (2Nf+1)^2) on the finest grid; coarser grids use the Q2
    interpolant of the injected nodal values."""
    if name is None:
        return None, False
    if isinstance(name, tuple) and name[0] == "nodal":
        W = np.asarray(name[1], dtype=np.float64).reshape(2, -1)
        Nf = (int(round(np.sqrt(W.shape[1]))) - 1) // 2
        return q2_interpolant(inject_q2(W, Nf, N), N, x0, x1), True
    if name == "recirc":
        return recirculating_wind, False
    if name == "two_vortex":
        return two_vortex_wind, True
    raise ValueError(f"unknown wind {name!r}")


# --------------------------------------------------------------------------
# Grid and assembled operators
# --------------------------------------------------------------------------
@dataclass
class Grid:
    N: int          # elements per side
    x0: float
    x1: float

    @property
    def h(self):
        return (self.x1 - self.x0) / self.N

    @property
    def n2(self):   # Q2 nodes per side
        return 2 * self.N + 1

    @property
    def n1(self):   # Q1 nodes per side
        return self.N + 1

    @property
    def ns(self):   # Q2 nodes (one velocity component), full grid
        return self.n2 ** 2

    @property
    def nq(self):   # Q1 nodes, full grid
        return self.n1 ** 2

    def q2_coords(self):
        """Node coordinates, node index = iy * n2 + ix."""
        s = self.x0 + np.arange(self.n2) * (self.h / 2.0)
        X, Y = np.meshgrid(s, s, indexing="xy")
        return X.ravel(), Y.ravel()

    def q1_coords(self):
        s = self.x0 + np.arange(self.n1) * self.h
        X, Y = np.meshgrid(s, s, indexing="xy")
        return X.ravel(), Y.ravel()

    def velocity_interior(self):
        """Indices of Q2 nodes off the boundary (the velocity unknowns)."""
        i = np.arange(self.n2)
        IX, IY = np.meshgrid(i, i, indexing="xy")
        m = (IX > 0) & (IX < self.n2 - 1) & (IY > 0) & (IY < self.n2 - 1)
        return np.flatnonzero(m.ravel())

    def pressure_free(self):
        """Indices of Q1 nodes except the pinned corner node 0."""
        return np.arange(1, self.nq)


@dataclass
class Operators:
    grid: Grid
    M: sp.csr_matrix     # Q2 scalar mass            (ns x ns), full grid
    K: sp.csr_matrix     # Q2 scalar stiffness
    N: sp.csr_matrix     # Q2 scalar convection  int phi_i w.grad phi_j
    Bx: sp.csr_matrix    # -int psi_k d/dx phi_j     (nq x ns)
    By: sp.csr_matrix    # -int psi_k d/dy phi_j
    Mp: sp.csr_matrix    # Q1 mass                   (nq x nq)
    Kp: sp.csr_matrix    # Q1 stiffness
    Np: sp.csr_matrix    # Q1 convection


def assemble(N, x0=0.0, x1=1.0, wind=None, npts=4, skew=False):
    """Element-loop assembly of all operators on the full (unrestricted) grid.

    `wind` is None (Stokes, w = 0) or a callable (x, y) -> (wx, wy), evaluated
    at the npts x npts Gauss points of each element; skew: return the
    skew-symmetric parts (N - N^T)/2, (Np - Np^T)/2 of the convection matrices.
    """
    g = Grid(N, x0, x1)
    h = g.h
    xi, wq = gauss01(npts)
    v2, d2 = lagrange(Q2_REF_NODES, xi)   # (3, nq1)
    v1, d1 = lagrange(Q1_REF_NODES, xi)   # (2, nq1)
    nq1 = len(xi)
    # tensor quadrature: q = qa + nq1 * qb ; local node l = a + 3 b (Q2), a + 2 b (Q1)
    W = (np.outer(wq, wq).T.ravel()) * h * h          # index [qb, qa] -> q
    qa = np.tile(np.arange(nq1), nq1)
    qb = np.repeat(np.arange(nq1), nq1)
    la2 = np.tile(np.arange(3), 3)
    lb2 = np.repeat(np.arange(3), 3)
    la1 = np.tile(np.arange(2), 2)
    lb1 = np.repeat(np.arange(2), 2)
    phi = v2[la2][:, qa] * v2[lb2][:, qb]                  # (9, Q)
    phix = d2[la2][:, qa] * v2[lb2][:, qb] / h
    phiy = v2[la2][:, qa] * d2[lb2][:, qb] / h
    psi = v1[la1][:, qa] * v1[lb1][:, qb]                  # (4, Q)
    psix = d1[la1][:, qa] * v1[lb1][:, qb] / h
    psiy = v1[la1][:, qa] * d1[lb1][:, qb] / h

    Me = np.einsum("iq,jq,q->ij", phi, phi, W)
    Ke = np.einsum("iq,jq,q->ij", phix, phix, W) + np.einsum("iq,jq,q->ij", phiy, phiy, W)
    Bxe = -np.einsum("kq,jq,q->kj", psi, phix, W)
    Bye = -np.einsum("kq,jq,q->kj", psi, phiy, W)
    Mpe = np.einsum("iq,jq,q->ij", psi, psi, W)
    Kpe = np.einsum("iq,jq,q->ij", psix, psix, W) + np.einsum("iq,jq,q->ij", psiy, psiy, W)

    ex = np.tile(np.arange(N), N)
    ey = np.repeat(np.arange(N), N)
    E = N * N
    glob2 = (2 * ex[:, None] + la2[None, :]) + (2 * ey[:, None] + lb2[None, :]) * g.n2  # (E, 9)
    glob1 = (ex[:, None] + la1[None, :]) + (ey[:, None] + lb1[None, :]) * g.n1          # (E, 4)

    if wind is not None:
        X = x0 + (ex[:, None] + xi[qa][None, :]) * h    # (E, Q)
        Y = x0 + (ey[:, None] + xi[qb][None, :]) * h
        wx, wy = wind(X, Y)
        Ne = np.einsum("iq,eq,jq,q->eij", phi, wx, phix, W) + np.einsum("iq,eq,jq,q->eij", phi, wy, phiy, W)
        Npe = np.einsum("iq,eq,jq,q->eij", psi, wx, psix, W) + np.einsum("iq,eq,jq,q->eij", psi, wy, psiy, W)
    else:
        Ne = np.zeros((E, 9, 9))
        Npe = np.zeros((E, 4, 4))

    def scatter(rows_idx, cols_idx, local, shape):
        # local: (ni, nj) shared by all elements or (E, ni, nj)
        ni, nj = rows_idx.shape[1], cols_idx.shape[1]
        r = np.repeat(rows_idx[:, :, None], nj, axis=2).ravel()
        c = np.repeat(cols_idx[:, None, :], ni, axis=1).ravel()
        if local.ndim == 2:
            v = np.broadcast_to(local, (E, ni, nj)).ravel()
        else:
            v = local.ravel()
        return sp.coo_matrix((v, (r, c)), shape=shape).tocsr()

    ns, nq = g.ns, g.nq
    Nm = scatter(glob2, glob2, Ne, (ns, ns))
    Npm = scatter(glob1, glob1, Npe, (nq, nq))
    if skew:
        Nm = (0.5 * (Nm - Nm.T)).tocsr()
        Npm = (0.5 * (Npm - Npm.T)).tocsr()
    return Operators(
        grid=g,
        M=scatter(glob2, glob2, Me, (ns, ns)),
        K=scatter(glob2, glob2, Ke, (ns, ns)),
        N=Nm,
        Bx=scatter(glob1, glob2, Bxe, (nq, ns)),
        By=scatter(glob1, glob2, Bye, (nq, ns)),
        Mp=scatter(glob1, glob1, Mpe, (nq, nq)),
        Kp=scatter(glob1, glob1, Kpe, (nq, nq)),
        Np=Npm,
    )


# --------------------------------------------------------------------------
# Nested-grid prolongation (exact interpolation of the coarse FE space)
# --------------------------------------------------------------------------
def prolongation_1d(Nc, degree):
    """Fine-node values of each coarse basis function: P[f, c] = phi_c(x_f)
    for the 1-D grid with Nc coarse elements refined once (unit length)."""
    nodes = Q2_REF_NODES if degree == 2 else Q1_REF_NODES
    per = degree                     # nodes per element minus one
    nc = per * Nc + 1
    nf = per * 2 * Nc + 1
    xf = np.arange(nf) / (per * 2 * Nc)
    P = np.zeros((nf, nc))
    for f, x in enumerate(xf):
        e = min(int(np.floor(x * Nc)), Nc - 1)
        xi = x * Nc - e
        val, _ = lagrange(nodes, [xi])
        for a in range(per + 1):
            P[f, per * e + a] = val[a, 0]
    P[np.abs(P) < 1e-15] = 0.0
    return sp.csr_matrix(P)


def prolongation_2d(Nc, degree):
    """2-D tensor-product prolongation from the Nc grid to the 2Nc grid on
    the full node sets (node index = iy * n + ix)."""
    P1 = prolongation_1d(Nc, degree)
    return sp.kron(P1, P1, format="csr")
