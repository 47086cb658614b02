"""Maps between the library's full-grid storage and the oracle's reduced vectors.

TEST INFRASTRUCTURE (oracle): see the package header.

Library storage (time domain, real): X[k, :] for block k = 0..K-1 holds six
fields back to back: v_x, v_y (Q2 full grid, ns = (2N+1)^2 nodes each), p
(Q1 full grid, nq = (N+1)^2), lambda_x, lambda_y, mu.  Dirichlet velocity
nodes and the pinned pressure node are stored as 0.  Residuals use the same
slots: the adjoint-equation rows (first block row of Eq. FinalA) sit in the
(v, p) slots, the state-equation rows in the (lambda, mu) slots.  The
frequency-domain storage is the same per frequency, complex.

Oracle ordering: [Y_1..Y_K, Lambda_1..Lambda_K], Y_k = (v_x, v_y, p) and
Lambda_k = (lambda_x, lambda_y, mu) restricted to the unknowns; per
frequency, Eq. SubBlockG's (v, lambda, p, mu) ordering.
"""
import numpy as np


def block_len(P):
    return 4 * P.grid.ns + 2 * P.grid.nq


def slots(P):
    ns, nq = P.grid.ns, P.grid.nq
    o = np.cumsum([0, ns, ns, nq, ns, ns, nq])
    return {"vx": (o[0], o[1]), "vy": (o[1], o[2]), "p": (o[2], o[3]),
            "lx": (o[3], o[4]), "ly": (o[4], o[5]), "mu": (o[5], o[6])}


def _take(P, blk, names):
    s = slots(P)
    out = []
    for nm in names:
        a, b = s[nm]
        f = blk[a:b]
        out.append(f[P.pf] if nm in ("p", "mu") else f[P.vi])
    return np.concatenate(out)


def _put(P, vec, names, dtype):
    s = slots(P)
    blk = np.zeros(block_len(P), dtype=dtype)
    pos = 0
    for nm in names:
        a, b = s[nm]
        idx = P.pf if nm in ("p", "mu") else P.vi
        blk[a + idx] = vec[pos:pos + len(idx)]
        pos += len(idx)
    return blk


def to_oracle_time(P, X):
    X = np.asarray(X).reshape(P.K, block_len(P))
    Y = [_take(P, X[k], ("vx", "vy", "p")) for k in range(P.K)]
    L = [_take(P, X[k], ("lx", "ly", "mu")) for k in range(P.K)]
    return np.concatenate(Y + L)


def from_oracle_time(P, x):
    nb, K = P.nb, P.K
    X = np.zeros((K, block_len(P)), dtype=x.dtype)
    for k in range(K):
        y = x[k * nb:(k + 1) * nb]
        l = x[(K + k) * nb:(K + k + 1) * nb]
        X[k] = _put(P, np.concatenate([y, l]), ("vx", "vy", "p", "lx", "ly", "mu"), x.dtype)
    return X


def to_oracle_freq(P, blk):
    """One frequency block (library slots) -> (v, lambda, p, mu) ordering."""
    return _take(P, np.asarray(blk), ("vx", "vy", "lx", "ly", "p", "mu"))


def from_oracle_freq(P, g):
    return _put(P, g, ("vx", "vy", "lx", "ly", "p", "mu"), np.complex128)


def field_mask(P):
    """Boolean mask over one library block: True at stored unknowns."""
    m = np.zeros(block_len(P), dtype=bool)
    s = slots(P)
    for nm, (a, b) in s.items():
        idx = P.pf if nm in ("p", "mu") else P.vi
        m[a + idx] = True
    return m
