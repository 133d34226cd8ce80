"""Pins of the oracle's finite sweep with time-step targeting (Sec. II.B-II.D).

Without truncation (L=6, m=256: no block of the sweep has more than 4^4 states) the superblock of every
step spans the whole Hilbert space and its Hamiltonian is the chain's, so the sweep's targets must be the
exact time evolution of phi = c^dag_{3 up} psi whatever the wave-function transformations (both
directions), the density matrices and the schedule did: at every step the densities of the two central
sites and the bond between them, for each target time t + t_x, against exact diagonalisation in the Fock
basis (1e-11; Krylov and ground-state errors are below 1e-12), the ground-state energy against ED, and
zero discarded weight.  (At L=8 the five-site blocks are cut to m states; the targets then leave the kept
space as they advance, so L=8 is not an exact case.)  With truncation (L=10,
m=24) the invariants: Tr rho = 1 (the weights sum to one), the discarded weight is the sum of the dropped
eigenvalues, no more than m states are kept, and the targets' norms never grow."""
import copy

import numpy as np
import pytest

from oracle import dmrg, ed, tst

U, T_HOP = 4.0, 1.0


@pytest.fixture(scope="module", params=[1, 2])
def exact_sweep(request):
    d = dmrg.ChainDMRG(6, T_HOP, U, 256)
    d.run(sweeps=1)
    s = tst.TSTSweep(d, 256, n_v=4, tau=0.1, nk=12, advance_every=request.param)
    return s, s.run()


def _ed_trajectory(L, times):
    sec0 = ed.Sector(L, L // 2, L // 2)
    sec1 = ed.Sector(L, L // 2 + 1, L // 2)
    hop = ed.chain_hopping(L, T_HOP)
    e0, gs = ed.ground_state(ed.hamiltonian(sec0, hop, U))
    phi = ed.apply_site_op(gs, sec0, sec1, [("cdag", ed.mode(L // 2, 0))])
    H1 = ed.hamiltonian(sec1, hop, U)
    return e0, sec1, dict(zip(times, ed.evolve(H1, phi, times)))


def test_exact_sweep_is_exact_time_evolution(exact_sweep):
    s, recs = exact_sweep
    times = sorted({round(r["t"] + tx, 12) for r in recs for tx in s.times})
    e0, sec1, traj = _ed_trajectory(6, times)
    assert [(r["l"], r["move"]) for r in recs] == tst.sweep_path(6)
    assert [r["action"] for r in recs][0] == "excite"
    assert sum(r["action"] == "advance" for r in recs) == (len(recs) - 1) // s.advance_every
    for r in recs:
        assert abs(r["energy"] - e0) < 1e-12
        if r["move"] is not None:
            assert r["discarded"] == 0.0
        for tx, o in zip(s.times, r["targets"]):
            v = traj[round(r["t"] + tx, 12)]
            l = r["l"]
            assert abs(o["n_left"] - ed.density(v, sec1, l, 0)) < 1e-11
            assert abs(o["n_right"] - ed.density(v, sec1, l + 1, 0)) < 1e-11
            w = ed.apply_site_op(v, sec1, sec1, [("cdag", ed.mode(l, 0)), ("c", ed.mode(l + 1, 0))])
            assert abs(o["bond"] - np.vdot(v, w) / np.vdot(v, v)) < 1e-11
            assert abs(o["norm2"] - np.vdot(v, v).real) < 1e-11


def test_truncated_sweep_invariants():
    d = dmrg.ChainDMRG(10, T_HOP, U, 24)
    d.run(sweeps=1)
    s = tst.TSTSweep(copy.deepcopy(d), 24, n_v=4, tau=0.1, nk=10, advance_every=2)
    recs = s.run()
    prev = None
    for r in recs:
        if r["move"] is None:
            continue
        lam = np.concatenate(r["evals"])
        assert abs(lam.sum() - 1.0) < 1e-12
        assert sum(r["kept"]) <= 24
        dropped = sum(float(np.sum(ev[k:])) for ev, k in zip(r["evals"], r["kept"]))
        assert abs(r["discarded"] - dropped) < 1e-14
        n2 = [o["norm2"] for o in r["targets"]]
        if prev is not None and r["action"] == "keep":
            assert all(a <= b + 1e-12 for a, b in zip(n2, prev))
        prev = n2
