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
