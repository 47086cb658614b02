"""Build the same discrete problem on the oracle side and on the GPU side."""
import numpy as np

from oracle import inexact, kkt, layout
from paper_2405_18964_gb300 import binding

FP64_TOL = 1e-12   # FP64 preconditioner / component parity (relative, max-norm)
FP32_TOL = 1e-5    # FP32 preconditioner / component parity
# FP64 bar for pressure values that pass through the multigrid on the
# corner-pinned pressure Laplacian K_p at 64 x 64: evaluating the same K_p in
# band form (M1 X K1^T + K1 X M1^T) instead of assembled rows moves the
# oracle's own 4-V-cycle result by 2.7e-12 (tests/test_oracle_inexact.py::
# test_pressure_multigrid_rounding_spread), so differences of that size are
# evaluation order, not error.  Velocity and multiplier parts keep FP64_TOL.
KP_FP64_TOL = 4e-12


def make_pair(kind, level, K, beta=1e-2, nu=1e-2, prec=0, T=1.0, **kw):
    import torch
    tau = T / (K + 1)
    if kind == "stokes":
        x0, x1, wind, wcode = 0.0, 1.0, None, 0
    else:
        x0, x1, wind, wcode = -1.0, 1.0, "recirc", 1
    P = kkt.Problem(kind, level, K, tau, beta, nu, x0, x1, wind)
    params = binding.default_params(kind=0 if kind == "stokes" else 1, level=level, n_t=K, tau=tau, beta=beta,
                                    nu=nu, x0=x0, x1=x1, wind=wcode, prec=prec, **kw)
    G = binding.Problem(params, stream=torch.cuda.current_stream().cuda_stream)
    return P, G


def settings_of(G):
    p = G.params
    return inexact.Settings(mg_cycles=p.mg_cycles, mg_pre=p.mg_pre, mg_post=p.mg_post, sor_omega=p.sor_omega,
                            cheb_steps=p.cheb_steps, uzawa_steps=p.uzawa_steps, uzawa_mu=p.uzawa_mu,
                            inner_tol=p.inner_tol, inner_maxit=p.inner_maxit)


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def to_dev(a, dtype="float64"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=getattr(torch, dtype))


def part_slices(P):
    """Slices of the oracle's frequency-block vector (v, lambda, p, mu)."""
    nv, npf = 2 * len(P.vi), len(P.pf)
    return {"v": slice(0, nv), "lam": slice(nv, 2 * nv), "p": slice(2 * nv, 2 * nv + npf),
            "mu": slice(2 * nv + npf, None)}


def part_errors(P, got, ref):
    """Max-norm error of each part relative to the largest entry of ref."""
    den = np.abs(ref).max()
    den = den if den > 0 else 1.0
    return {k: float(np.abs(got[sl] - ref[sl]).max() / den) for k, sl in part_slices(P).items()}


def freq_blocks(P, Xh):
    """GPU frequency vector [J][nblk] -> list of oracle (v, lam, p, mu) vectors."""
    Xh = np.asarray(Xh).reshape(-1, layout.block_len(P))
    return [layout.to_oracle_freq(P, Xh[j]) for j in range(Xh.shape[0])]
