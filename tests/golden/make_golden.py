"""Writes tests/golden/app_c_xy_chain.txt from the oracle's App. C closed form only.

Rows: N  beta  p1 p2 p3 p4 (ascending eigenvalues of rho*)  ln Z*  ln Z_N
for the open isotropic XY chain with J = 1, h = 0.3, system = first two sites
(the setting of the paper's Sec. 5.1 / Fig. 1, App. C). Run from the repo root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import closed_form  # noqa: E402


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "app_c_xy_chain.txt")
    with open(out, "w") as f:
        f.write("# App. C closed form, open XY chain (J/2)(XX+YY) + (h/2)Z, J=1, h=0.3, N_s=2\n")
        f.write("# N beta p1 p2 p3 p4 lnZstar lnZ_N\n")
        for n in (8, 10, 12, 14, 18):
            for beta in np.geomspace(0.1, 10.0, 7):
                p = closed_form.rho_eigenvalues(n, beta, 1.0, 0.3)
                f.write(f"{n} {beta:.17g} " + " ".join(f"{x:.17g}" for x in p)
                        + f" {closed_form.log_z_star(n, beta, 1.0, 0.3):.17g}"
                        + f" {closed_form.log_partition_chain(n, beta, 1.0, 0.3):.17g}\n")


if __name__ == "__main__":
    main()
