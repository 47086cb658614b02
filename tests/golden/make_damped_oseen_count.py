"""Writes damped_oseen_count.txt: the oracle's FGMRES(10) iteration count for
the recirculating-wind Oseen problem at beta = 1e-2 that converges only with
damped SOR on the convection multigrids (sor_omega_conv = 0.5).

Runs the oracle alone (no GPU code): 32 x 32 elements on [-1,1]^2, n_t = 16,
T = 1 (tau = 1/17), nu = 1/100, seeded desired state (seed 0), outer
tolerance 1e-8, inner GMRES to 1e-2 (cap 100), 4 V-cycles, 10 Chebyshev and
6 Uzawa steps (Sec. 5 defaults)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import inexact, kkt  # noqa: E402
from paper_2405_18964_gb300 import inputs  # noqa: E402

LEVEL, K, BETA, NU, OMEGA_CONV = 5, 16, 1e-2, 1e-2, 0.5


def main():
    tau = 1.0 / (K + 1)
    P = kkt.Problem("oseen", LEVEL, K, tau, BETA, NU, -1.0, 1.0, "recirc")
    pc = inexact.PinTPreconditioner(P, inexact.Settings(sor_omega_conv=OMEGA_CONV))
    b = P.rhs(inputs.desired_state(P.N, -1.0, 1.0, K, tau, 1.0, seed=0))
    _, info = kkt.fgmres(P.kkt_matrix(), b, pc, restart=10, tol=1e-8, maxit=80)
    with open(os.path.join(HERE, "damped_oseen_count.txt"), "w") as f:
        f.write("# oracle FGMRES(10) iterations, recirculating wind, 32x32, n_t = 16, beta = 1e-2, nu = 1e-2,\n")
        f.write("# sor_omega_conv = 0.5, seed 0, tol 1e-8 (written by make_damped_oseen_count.py)\n")
        f.write(f"outer_iterations {info['its']}\nrelres {info['relres']:.3e}\n")


if __name__ == "__main__":
    main()
