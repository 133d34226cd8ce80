"""Host logic of the device sweep's lattice (paper_1103_5391_gb300.sweep.Lattice) against the oracle's bond
rule (oracle.dmrg.Geometry, itself pinned to the ED hopping matrices): for chains and two-leg ladders of
4 to 24 sites, every enlargement's bonds (left and right blocks of every size) and every cut's bonds
agree, and the bonds a full set of enlargements and cuts produces are exactly the lattice's bonds, each
once."""
import numpy as np
import pytest

from oracle import dmrg, ed


@pytest.mark.parametrize("legs,t_leg,t_rung", [(1, 1.0, 1.0), (1, 0.7, 1.0), (2, 1.0, 1.0), (2, 1.0, 0.5)])
def test_lattice_rules_match_the_oracle(legs, t_leg, t_rung):
    from paper_1103_5391_gb300 import sweep as S
    lat, geo = S.Lattice(legs, t_leg, t_rung), dmrg.Geometry(legs, t_leg, t_rung)
    for k in range(1, 24):
        assert lat.new_site_bonds(k) == geo.new_site_bonds(k)
    for l in range(1, 22):
        assert lat.cut_bonds(l) == geo.cut_bonds(l)
    for n in range(4, 25, 2):
        # the left block grown site by site (site k bonds to k-1 and k-2), then the cut after site l:
        # every lattice bond (i < j) is made once by an enlargement (j <= l) or crosses the cut
        l = n // 2 - 1
        h = np.zeros((n, n))
        for j in range(1, l + 1):
            for d, tb in zip((1, 2), lat.new_site_bonds(j)):
                if tb != 0.0:
                    assert h[j - d, j] == 0.0
                    h[j - d, j] = h[j, j - d] = -tb
        for j in range(l + 1, n):   # the right block, mirrored: site n - 1 - m grows with m sites after it
            m = n - 1 - j
            for d, tb in zip((1, 2), lat.new_site_bonds(m)):
                if tb != 0.0 and j + d < n:
                    assert h[j, j + d] == 0.0
                    h[j, j + d] = h[j + d, j] = -tb
        for eL, eR, tb in lat.cut_bonds(l):
            i, j = l - eL, l + 1 + eR
            if tb != 0.0:
                assert h[i, j] == 0.0
                h[i, j] = h[j, i] = -tb
        want = ed.chain_hopping(n, t_leg) if legs == 1 else ed.ladder_hopping(n // 2, t_leg, t_rung)
        assert np.array_equal(h, want), n
