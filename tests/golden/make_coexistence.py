"""Writes tests/golden/coexistence.txt: flat-interface coexistence densities
(rho_g, rho_l) of the Peng-Robinson EOS of Section 2 (a = 3/49, b = 2/21,
R = 1, omega = 0.344) by Maxwell's equal-area construction, computed by the
CPU oracle only.  The same numbers are the COEXISTENCE input table of
paper_2205_00686_gb300/workloads.py.

    python tests/golden/make_coexistence.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

PARAMS = dict(a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344)


def main():
    Tc = oracle.Tc(PARAMS)
    lines = ["# T/Tc rho_g rho_l  (Maxwell construction, oracle/lbm_oracle.c)"]
    for Tr in (0.80, 0.86, 0.90, 0.95):
        rg, rl = oracle.maxwell(PARAMS, Tr * Tc)
        lines.append("%.2f %.14f %.14f" % (Tr, rg, rl))
    with open(os.path.join(HERE, "coexistence.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
