"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the solver: it only draws random numbers
and evaluates the synthetic desired velocity at grid nodes.

Desired state (the workload recipe): a stream function made of four seeded
sine modes on the mapped unit square (xi, eta) in [0, 1]^2,

    psi(xi, eta, t) = sum_k a_k sin(m_k pi xi) sin(n_k pi eta) cos(2 pi q_k t / T),

with a_k ~ N(0, 1), m_k, n_k ~ U{1..4}, q_k ~ U{0, 1, 2}, drawn in that order
from numpy.random.default_rng(seed); the desired velocity is its curl
v_d = (d psi / dy, -d psi / dx), evaluated at the Q2 nodes at t_k = k tau,
k = 1..K.  It is divergence free, and zero-flux through the boundary.
"""
import numpy as np


def q2_axis(N, x0, x1):
    """Coordinates of the 2N+1 Q2 nodes along one axis."""
    return x0 + np.arange(2 * N + 1) * ((x1 - x0) / (2 * N))


def desired_state(N, x0, x1, K, tau, T, seed):
    """v_d as a (K, 2, (2N+1)^2) float64 array, node index iy*(2N+1)+ix."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(4)
    m = rng.integers(1, 5, size=4)
    n = rng.integers(1, 5, size=4)
    q = rng.integers(0, 3, size=4)
    s = q2_axis(N, x0, x1)
    ell = x1 - x0
    xi = (s - x0) / ell
    X, Y = np.meshgrid(xi, xi, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    out = np.zeros((K, 2, X.size))
    for k in range(K):
        t = (k + 1) * tau
        for i in range(4):
            amp = a[i] * np.cos(2.0 * np.pi * q[i] * t / T)
            sx, cx = np.sin(m[i] * np.pi * X), np.cos(m[i] * np.pi * X)
            sy, cy = np.sin(n[i] * np.pi * Y), np.cos(n[i] * np.pi * Y)
            out[k, 0] += amp * sx * (n[i] * np.pi / ell) * cy      # d psi / dy
            out[k, 1] -= amp * (m[i] * np.pi / ell) * cx * sy      # -d psi / dx
    return out


def random_vector(shape, seed, dtype=np.float64):
    """Standard-normal test vector (real or complex)."""
    rng = np.random.default_rng(seed)
    if np.dtype(dtype).kind == "c":
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
    return rng.standard_normal(shape).astype(dtype)


# ---------------------------------------------------------------------------
# The problems of the paper's experiments (Sec. 5), on [-1, 1]^2.  These are
# data, not method: nodal values of closed-form fields at the Q2 nodes.
# ---------------------------------------------------------------------------
def q2_nodes(N, x0, x1):
    """(x, y) of the (2N+1)^2 Q2 nodes, node index iy*(2N+1)+ix."""
    s = q2_axis(N, x0, x1)
    X, Y = np.meshgrid(s, s, indexing="xy")
    return X.ravel(), Y.ravel()


def q2_boundary_mask(N):
    """True at the Q2 nodes on the boundary of the square."""
    n2 = 2 * N + 1
    i = np.arange(n2)
    IX, IY = np.meshgrid(i, i, indexing="xy")
    return ((IX == 0) | (IX == n2 - 1) | (IY == 0) | (IY == n2 - 1)).ravel()


def stokes_mms_velocity(x, y, t, T):
    """Velocity of the Sec. 5.1 Stokes problem: e^{T-t} (20 x y^3, 5 x^4 - 5 y^4)."""
    e = np.exp(T - t)
    return np.stack([20.0 * x * y ** 3 * e, (5.0 * x ** 4 - 5.0 * y ** 4) * e])


def stokes_mms_pressure(x, y, t, T):
    """Pressure of the Sec. 5.1 Stokes problem, up to a constant: e^{T-t} (60 x^2 y - 20 y^3)."""
    return np.exp(T - t) * (60.0 * x * x * y - 20.0 * y ** 3)


def stokes_mms_desired(x, y, t, T, beta):
    """Desired velocity v_d of the Sec. 5.1 Stokes problem."""
    e = np.exp(T - t)
    a, b = x * x - 1.0, y * y - 1.0
    c0 = 4.0 * beta * y * (2.0 * (3.0 * x * x - 1.0) * b + 3.0 * a * a)
    c1 = -4.0 * beta * x * (3.0 * b * b + 2.0 * a * (3.0 * y * y - 1.0))
    d0 = 20.0 * x * y ** 3 + 2.0 * beta * y * (a * a * (y * y - 7.0) - 4.0 * (3.0 * x * x - 1.0) * b + 2.0)
    d1 = 5.0 * (x ** 4 - y ** 4) - 2.0 * beta * x * (b * b * (x * x - 7.0) - 4.0 * a * (3.0 * y * y - 1.0) - 2.0)
    return np.stack([c0 + e * d0, c1 + e * d1])


def stokes_mms_forcing(x, y, t, T):
    """Forcing f of the Sec. 5.1 Stokes problem."""
    e = np.exp(T - t)
    a, b = x * x - 1.0, y * y - 1.0
    s0 = 2.0 * y * a * a * b
    s1 = 2.0 * x * a * b * b
    return np.stack([e * (-20.0 * x * y ** 3 - s0) + s0, e * (5.0 * (y ** 4 - x ** 4) + s1) - s1])


def stokes_mms_data(N, K, tau, T, beta):
    """Sec. 5.1 data on the Q2 grid of [-1, 1]^2 at t_k = k tau, k = 1..K.

    Returns (vd, f, v0, g): vd, f, g of shape (K, 2, (2N+1)^2), v0 of shape
    (2, (2N+1)^2).  The initial and boundary velocities are those of the
    closed-form solution: v0 = v(., 0) and g_k = v(., t_k), whose boundary
    nodal values are the Dirichlet data (interior entries of g are unused).
    """
    x, y = q2_nodes(N, -1.0, 1.0)
    ts = (np.arange(K) + 1) * tau
    vd = np.stack([stokes_mms_desired(x, y, t, T, beta) for t in ts])
    f = np.stack([stokes_mms_forcing(x, y, t, T) for t in ts])
    g = np.stack([stokes_mms_velocity(x, y, t, T) for t in ts])
    v0 = stokes_mms_velocity(x, y, 0.0, T)
    return vd, f, v0, g


def cavity_data(N, K):
    """Sec. 5.2 lid-driven cavity data on the Q2 grid of [-1, 1]^2 (time independent).

    Returns (vd, f, v0, g) like `stokes_mms_data`: desired state with one
    vortex plus a jet below the lid, the same forcing shape as Sec. 5.1
    without its time factor, an initial velocity (1, 0) on the wedge
    |x| < y, and the lid velocity (1, 0) on y = 1 (zero on the other sides).
    """
    x, y = q2_nodes(N, -1.0, 1.0)
    q = (1.0 - x ** 4) * (1.0 - y ** 4)
    vd = np.stack([2.0 * y * q + np.where(y >= 0.8, 5.0 * y - 4.0, 0.0), -2.0 * x * q])
    a, b = x * x - 1.0, y * y - 1.0
    f = np.stack([-20.0 * x * y ** 3 - 2.0 * y * a * a * b, 5.0 * (y ** 4 - x ** 4) + 2.0 * x * a * b * b])
    wedge = (x > -y) & (x < y)
    v0 = np.stack([np.where(wedge, 1.0, 0.0), np.zeros_like(x)])
    lid = np.stack([np.where(y == 1.0, 1.0, 0.0), np.zeros_like(x)])
    rep = lambda a: np.repeat(a[None], K, axis=0)
    return rep(vd), rep(f), v0, rep(lid)
