"""Writes oracle_config1.txt: the FP64 oracle's permeability and stop step
for the 32^3 simple-cubic cell (centred sphere r = 12, Set E with Lambda =
3/16, tau = 1, F = 1e-6 along x, stopping rule 1e-9 checked every step).
Calls only the oracle and the voxel-image generator."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1902_11193_gb300 import geometry  # noqa: E402


def main():
    mask = geometry.sphere_array(32, "sc", r=12)
    O = oracle.Solver(mask, oracle.rates("E", 1.0, 3 / 16), [1e-6, 0, 0])
    rc, steps, U = O.run_to_convergence(1e-9, K=1, max_steps=100000)
    assert rc == 0
    k = O.permeability(1.0)[0]
    with open(os.path.join(HERE, "oracle_config1.txt"), "w") as fh:
        fh.write("# FP64 oracle, 32^3 SC r=12, Set E(3/16), tau=1, F=1e-6 x, tol 1e-9 (K=1)\n")
        fh.write("# written by tests/golden/make_oracle_values.py\n")
        fh.write("# steps  k_lu  Ux\n")
        fh.write(f"{steps} {k:.17g} {U[0]:.17g}\n")


if __name__ == "__main__":
    main()
