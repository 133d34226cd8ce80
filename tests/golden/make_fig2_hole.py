"""Writes fig2_hole_densities.txt: the exact curves of Sec. III.A, Fig. 2, from App. A's closed form.

Test infrastructure: calls only `oracle/` (closed_forms.hole_x, closed_forms.ground_density and the
hopping matrices of oracle.ed).  The systems are those of Fig. 2: (b) the 16-site open chain and (a) the
8 x 2 two-leg ladder (rung-first labels, t_leg = 1, t_rung = 0.5: the figure does not give the rung
hopping, and the isotropic ladder's U=0 ground state is degenerate), U = 0, half filling, the hole
c_{8 up} on the ground state.  Stored: the normalised density <n_{j up}>(t) = X_{8j}(t) / R_8 of every
site j at t = 0, 0.1, ..., 1.2 (App. A, Eq. xij: X_ij(t) = R_i R_j - |T_ij(t)|^2, R_8 = <phi|phi>).

Run from the repository root:  python tests/golden/make_fig2_hole.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import closed_forms, ed  # noqa: E402

NSITES, I_SITE, T_RUNG = 16, 8, 0.5
TIMES = [round(0.1 * k, 10) for k in range(13)]
LATTICES = {"chain": ed.chain_hopping(NSITES), "ladder": ed.ladder_hopping(NSITES // 2, 1.0, T_RUNG)}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fig2_hole_densities.txt")


def rows():
    for name, hop in LATTICES.items():
        r8 = closed_forms.ground_density(hop, NSITES // 2)[I_SITE]
        for t in TIMES:
            dens = [closed_forms.hole_x(hop, NSITES // 2, I_SITE, j, t) / r8 for j in range(NSITES)]
            yield name, t, dens


def main():
    with open(OUT, "w") as f:
        f.write("# Sec. III.A, Fig. 2 (a: ladder, b: chain) from App. A, Eq. xij: <n_{j up}>(t) after c_{8 up} on the\n")
        f.write("# U=0 half-filled ground state; 16-site open chain, 8 x 2 ladder (rung-first labels, t_rung = 0.5).\n")
        f.write("# Written by tests/golden/make_fig2_hole.py (oracle.closed_forms only).\n")
        f.write("# lattice t n_0 ... n_15\n")
        for name, t, dens in rows():
            f.write(name + " " + repr(t) + " " + " ".join("%.17e" % x for x in dens) + "\n")


if __name__ == "__main__":
    main()
