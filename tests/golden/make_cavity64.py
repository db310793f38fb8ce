"""Write the oracle's 64 x 64 lid cavity after 2000 RK3 steps (the parity size
of the 256 x 256 cavity workload: walls on all four sides, FC(Gram) d = 5,
C = 25 in x and y, G8 with h = 1.3 dx, Re = 1000, dt = 1e-3, fluid at rest).

Calls only the oracle (oracle.step with the oracle-written FC(Gram) table) and
stores u, v and phi, and the same three after a start perturbed by one ulp of
the lid speed on every node (seeded signs), from which the tests take the
problem's own FP64 rounding floor.  Run from the repo root (a few minutes):

    python tests/golden/make_cavity64.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import step as ostep  # noqa: E402

N, NSTEPS = 64, 2000
PATH = os.path.join(HERE, "cavity64_rk3_2000.npz")


def problem():
    E = np.loadtxt(os.path.join(HERE, "fc_gram_d5_c25.txt"))
    return ostep.Problem(nx=N, ny=N, Lx=1.0, Ly=1.0, x_walls=True, family="G8", h_over_dx=1.3, E_dir=E, E_neu=E,
                         nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3").build_symbols()


def main():
    p = problem()
    z = np.zeros((N, N))
    u, v, phi = ostep.isph_steps(p, z, z, NSTEPS)
    rng = np.random.default_rng(0)
    du = 2.0 ** -52 * rng.choice([-1.0, 1.0], size=(N, N))
    dv = 2.0 ** -52 * rng.choice([-1.0, 1.0], size=(N, N))
    up, vp, phip = ostep.isph_steps(p, z + du, z + dv, NSTEPS)
    np.savez_compressed(PATH, u=u, v=v, phi=phi, u_ulp=up, v_ulp=vp, phi_ulp=phip, nsteps=NSTEPS)


if __name__ == "__main__":
    main()
