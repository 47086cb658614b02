"""Pin of reading R1 (the number of time blocks) against the paper's printed
degree-of-freedom counts.

The discretised formulas leave the block count ambiguous (n_t - 1 blocks by
the size of I_t and E, n_t by the tables).  Table 1 prints the size of the
all-at-once system for seven values of n_t on two meshes, to three
significant digits.  Only "K = n_t blocks of 2 (n_v + n_p) unknowns" makes
#DOFs / K constant within that rounding; K = n_t - 1 or n_t + 1 leave a
spread of several percent.  The oracle's system has 2 K (n_v + n_p)
unknowns with K = n_t."""
import os

import numpy as np

from oracle import kkt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_dofs.txt")


def _table():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    a = np.array([[float(v) for v in r] for r in rows])
    return a[:, 0], a[:, 1], a[:, 2]


def _spread(dofs, blocks):
    per = dofs / blocks
    return per.max() / per.min() - 1.0


def test_dofs_are_proportional_to_nt():
    nt, hc, hf = _table()
    for dofs in (hc, hf):
        assert _spread(dofs, nt) < 0.01                 # 3-digit rounding: +-0.5% per entry
        assert _spread(dofs, nt - 1) > 0.05
        assert _spread(dofs, nt + 1) > 0.05
    # halving h about quadruples the unknowns per block (a 2-D mesh)
    assert 3.8 < np.median(hf / hc) < 4.1


def test_oracle_unknowns_are_2K_blocks():
    for K in (3, 4, 8):
        P = kkt.Problem("stokes", 2, K, 0.1, 1e-2, 1e-2, 0.0, 1.0, None)
        assert P.n == 2 * K * (P.nv + P.np_)
        assert P.kkt_matrix().shape == (P.n, P.n)
