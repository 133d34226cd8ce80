"""Pins of the oracle's finite sweep with time-step targeting (Sec. II.B-II.D).

Without truncation (L=6, m=256: no block of the sweep has more than 4^4 states) the superblock of every
step spans the whole Hilbert space and its Hamiltonian is the chain's, so the sweep's targets must be the
exact time evolution of phi (Eq. b: c^dag_{3 up} psi, and products with a second operator reached later in
the sweep) whatever the wave-function transformations (both directions), the density matrices and the
schedule did; while the product is partial, the targets are the partial state: at every step the densities of the two central
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


CASES = [
    (1, [(3, "cdag", 0)]),
    (2, [(3, "cdag", 0)]),
    (1, [(3, "cdag", 0), (4, "c", 1)]),    # completed at the second step (centre sites 3, 4)
    (1, [(3, "cdag", 0), (1, "c", 0)]),    # completed at the left end of the sweep
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def exact_sweep(request):
    every, exc = CASES[request.param]
    d = dmrg.ChainDMRG(6, T_HOP, U, 256)
    d.run(sweeps=1)
    s = tst.TSTSweep(d, 256, n_v=4, tau=0.1, nk=12, advance_every=every, excitations=exc)
    return s, s.run()


def _ed_states(L, exc, times):
    """Ground state, the partial products B_k ... B_0 psi (Eq. b) and exp(-i H t) phi (Fock basis)."""
    hop = ed.chain_hopping(L, T_HOP)
    sec = ed.Sector(L, L // 2, L // 2)
    e0, v = ed.ground_state(ed.hamiltonian(sec, hop, U))
    partial = []
    for site, kind, sigma in exc:
        dq = [0, 0]
        dq[sigma] = 1 if kind == "cdag" else -1
        nsec = ed.Sector(L, sec.nup + dq[0], sec.ndn + dq[1])
        v = ed.apply_site_op(v, sec, nsec, [(kind, ed.mode(site, sigma))])
        sec = nsec
        partial.append((sec, v))
    H1 = ed.hamiltonian(sec, hop, U)
    return e0, partial, sec, dict(zip(times, ed.evolve(H1, v, times)))


def _check_target(o, v, sec, l):
    assert abs(o["n_left"] - ed.density(v, sec, l, 0)) < 1e-11
    assert abs(o["n_right"] - ed.density(v, sec, l + 1, 0)) < 1e-11
    w = ed.apply_site_op(v, sec, sec, [("cdag", ed.mode(l, 0)), ("c", ed.mode(l + 1, 0))])
    assert abs(o["bond"] - np.vdot(v, w) / np.vdot(v, v)) < 1e-11
    assert abs(o["norm2"] - np.vdot(v, v).real) < 1e-11


def test_exact_sweep_is_exact_time_evolution(exact_sweep):
    s, recs = exact_sweep
    times = sorted({round(r["t"] + tx, 12) for r in recs for tx in s.times})
    e0, partial, sec1, traj = _ed_states(6, s.excitations, times)
    assert [(r["l"], r["move"]) for r in recs] == tst.sweep_path(6)
    acts = [r["action"] for r in recs]
    k = acts.index("excite")
    assert all(a in ("ground", "partial") for a in acts[:k])
    assert sum(a == "advance" for a in acts) == (len(recs) - 1 - k) // s.advance_every
    for r in recs:
        assert abs(r["energy"] - e0) < 1e-12
        if r["move"] is not None:
            assert r["discarded"] == 0.0
        if r["action"] in ("ground", "partial"):
            assert len(r["targets"]) == (0 if r["action"] == "ground" else s.n_v)
            for o in r["targets"]:
                psec, pv = partial[r["applied"] - 1]
                _check_target(o, pv, psec, r["l"])
            continue
        for tx, o in zip(s.times, r["targets"]):
            _check_target(o, traj[round(r["t"] + tx, 12)], sec1, r["l"])


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
