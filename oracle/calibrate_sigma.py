"""Calibrates the Li forcing parameter sigma (Eq. 8; the paper calls it
tunable and gives no value) on the CPU oracle: an isothermal flat liquid slab
at 0.86 T_c is run to steady state for each sigma, and the sigma whose bulk
densities best match the Maxwell coexistence densities is printed.

TEST INFRASTRUCTURE: runs the oracle only.

    python oracle/calibrate_sigma.py 1.20 1.25 1.30
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2205_00686_gb300 import workloads as W  # noqa: E402


def slab(sigma, Tr=0.86, ny=200, steps=20000):
    rg, rl = W.COEXISTENCE[Tr]
    nx = 2
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    rho = rg + (rl - rg) * 0.5 * (np.tanh((y - ny / 4) / 2) - np.tanh((y - 3 * ny / 4) / 2))
    z = np.zeros((ny, nx))
    s = oracle.Sim(nx, ny, W.params(sigma=sigma, frozen_thermal=1), W.periodic_bc())
    s.init(rho, z, z, np.full((ny, nx), Tr * W.TC))
    s.step(steps)
    r = s.fields()[0][:, 0]
    return r[ny // 2], r[0]


def main(argv):
    rg, rl = W.COEXISTENCE[0.86]
    best = None
    for sigma in [float(a) for a in argv] or [1.2, 1.25, 1.3]:
        l, g = slab(sigma)
        err = abs(l - rl) / rl + abs(g - rg) / rg
        print("sigma %.4f  rho_l %.6f (%+.2e)  rho_g %.6f (%+.2e)" %
              (sigma, l, (l - rl) / rl, g, (g - rg) / rg))
        if best is None or err < best[0]:
            best = (err, sigma)
    print("best sigma", best[1])


if __name__ == "__main__":
    main(sys.argv[1:])
