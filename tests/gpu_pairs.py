"""Build the same discrete problem on the oracle side and on the GPU side."""
import numpy as np

from oracle import inexact, kkt, layout
from paper_2405_18964_gb300 import binding

FP64_TOL = 1e-12   # FP64 preconditioner / component parity (relative, max-norm)
FP32_TOL = 1e-5    # FP32 preconditioner / component parity


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


def freq_blocks(P, Xh):
    """GPU frequency vector [J][nblk] -> list of oracle (v, lam, p, mu) vectors."""
    Xh = np.asarray(Xh).reshape(-1, layout.block_len(P))
    return [layout.to_oracle_freq(P, Xh[j]) for j in range(Xh.shape[0])]
