"""The seeded synthetic superblocks the bench times (Gaussian sector model of a truncated DMRG superblock
at the central cut): their sizes are the ones quoted for them and used by the bench's roofline, their
operators have the structure the model states, and a seed gives the same arrays every time."""
import numpy as np
import pytest

from workloads import sectors as S

# (left sectors, D_L, largest left sector, sector pairs in the excited sector, D of the excited sector)
SIZES = {"C2": (144, 1732, 60, 110, 46940), "C3": (144, 3252, 120, 110, 183952),
         "C4": (144, 4052, 152, 110, 292472)}


def _make(key):
    import bench
    wl = bench.CONFIGS[key]
    return wl, S.make_synthetic(wl["L"], wl["m"], wl["U"], t=wl["t"], nbonds=wl["nbonds"],
                                seed=S.SEED_BASE + wl["seed_index"])


@pytest.mark.parametrize("key", sorted(SIZES))
def test_bench_workload_sizes(key):
    wl, ss = _make(key)
    nsec, dl, dmax, npairs, d1 = SIZES[key]
    rid = {q: k for k, q in enumerate(ss.rsec)}
    pairs = [(k, rid[(ss.Q1[0] - q[0], ss.Q1[1] - q[1])]) for k, q in enumerate(ss.lsec)
             if (ss.Q1[0] - q[0], ss.Q1[1] - q[1]) in rid]
    assert (len(ss.lsec), sum(ss.ldim), max(ss.ldim), len(pairs)) == (nsec, dl, dmax, npairs)
    assert sum(ss.ldim[a] * ss.rdim[b] for a, b in pairs) == d1 == len(ss.phi)
    assert ss.Q0 == (wl["L"] // 2, wl["L"] // 2) and ss.Q1 == (wl["L"] // 2 + 1, wl["L"] // 2)
    assert len(ss.cdagL) == len(ss.cR) == wl["nbonds"]


def test_model_structure_and_seeding():
    wl, ss = _make("C2")
    # block Hamiltonians: block diagonal, Hermitian, spectrum within about l (2t + U/4) of the block
    lb = wl["L"] // 2
    radius = lb * (2 * wl["t"] + wl["U"] / 4)
    for Hb in (ss.HL, ss.HR):
        assert all(a == b for a, b in Hb)
        top = 0.0
        for blk in Hb.values():
            assert np.abs(blk - blk.conj().T).max() < 1e-12
            top = max(top, np.abs(np.linalg.eigvalsh(blk)).max())
        assert 0.3 * radius < top < 1.5 * radius
    # connection operators change one spin's count by one on each side, blocks sized by their sectors
    for b in range(wl["nbonds"]):
        for s in range(2):
            e = [0, 0]
            e[s] = 1
            for (qo, qi), blk in ss.cdagL[b][s].items():
                assert tuple(np.subtract(ss.lsec[qo], ss.lsec[qi])) == tuple(e)
                assert blk.shape == (ss.ldim[qo], ss.ldim[qi])
            for (ro, ri), blk in ss.cR[b][s].items():
                assert tuple(np.subtract(ss.rsec[ri], ss.rsec[ro])) == tuple(e)
                assert blk.shape == (ss.rdim[ro], ss.rdim[ri])
    assert abs(np.linalg.norm(ss.phi) - 1.0) < 1e-12 and abs(np.linalg.norm(ss.psi_gs) - 1.0) < 1e-12
    # the same seed gives the same arrays
    _, again = _make("C2")
    assert np.array_equal(again.phi, ss.phi) and np.array_equal(again.psi_gs, ss.psi_gs)
    assert all(np.array_equal(again.HL[k], ss.HL[k]) for k in ss.HL)
