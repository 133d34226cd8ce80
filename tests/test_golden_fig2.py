"""Golden values of Sec. III.A, Fig. 2 (tests/golden/fig2_hole_densities.txt, written from App. A's closed
form by tests/golden/make_fig2_hole.py) pinned at the figure's own sizes by exact time evolution.

At U = 0 the two spin species do not interact, so after c_{8 up} the up electrons evolve as 8 spinless
fermions on the 16 sites whatever the down electrons do: the spinless sector (8 up, 0 down) has 12,870
states, small enough for ED (sparse H, ARPACK ground state, expm_multiply) at the paper's 16-site chain
and 8 x 2 ladder.  This checks App. A's X_ij (oracle.closed_forms.hole_x) at the figure's system and
site, beyond the 8-site chain of the oracle's other pins; and the stored file against the oracle as it
stands (a change to either shows here)."""
import os

import numpy as np
import pytest

from oracle import closed_forms, ed

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fig2_hole_densities.txt")
NSITES, I_SITE, T_RUNG = 16, 8, 0.5


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, t, *dens = line.split()
            out.setdefault(name, {})[float(t)] = np.array([float(x) for x in dens])
    return out


def _hop(name):
    return ed.chain_hopping(NSITES) if name == "chain" else ed.ladder_hopping(NSITES // 2, 1.0, T_RUNG)


def test_golden_file_equals_the_closed_form():
    g = _golden()
    assert set(g) == {"chain", "ladder"} and all(len(v) == 13 for v in g.values())
    for name, curves in g.items():
        hop = _hop(name)
        r8 = closed_forms.ground_density(hop, NSITES // 2)[I_SITE]
        for t, dens in curves.items():
            want = [closed_forms.hole_x(hop, NSITES // 2, I_SITE, j, t) / r8 for j in range(NSITES)]
            assert np.abs(dens - want).max() < 1e-14


@pytest.mark.parametrize("name", ["chain", "ladder"])
def test_golden_fig2_against_spinless_ed(name):
    curves = _golden()[name]
    hop = _hop(name)
    s8, s7 = ed.Sector(NSITES, NSITES // 2, 0), ed.Sector(NSITES, NSITES // 2 - 1, 0)
    e0, psi = ed.ground_state(ed.hamiltonian(s8, hop, 0.0))
    assert abs(e0 - np.linalg.eigvalsh(hop)[: NSITES // 2].sum()) < 1e-10    # non-degenerate filled Fermi sea
    phi = ed.apply_site_op(psi, s8, s7, [("c", ed.mode(I_SITE, 0))])
    H7 = ed.hamiltonian(s7, hop, 0.0)
    times = sorted(curves)
    worst = 0.0
    for t, v in zip(times, ed.evolve(H7, phi, times)):
        got = np.array([ed.density(v, s7, j, 0) for j in range(NSITES)])
        worst = max(worst, np.abs(got - curves[t]).max())
    assert worst < 1e-9, worst
    assert np.abs(curves[0.0][I_SITE]) < 1e-14 and np.abs(curves[1.2] - curves[0.0]).max() > 0.05   # the hole moves
