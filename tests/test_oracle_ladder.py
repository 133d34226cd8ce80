"""Pins of the oracle's two-leg ladder DMRG and sweep (Sec. III: the 8 x 2 ladder of Fig. 2, the 2 x 4
ladders of Figs. 3-4), against exact diagonalisation with the lattice built independently (ed.py).

  - the bond rule of dmrg.Geometry (a new site bonds to the block's edge across a rung when it has an
    odd number of sites before it, and to the second site from the edge along a leg) gives exactly the
    hopping matrix of ed.ladder_hopping, and the chain rule that of ed.chain_hopping;
  - 2 x 4 ladder (t_leg = 1, t_rung = 0.5, U = 4) with m = 256: every block is exact, so the DMRG energy,
    the densities of the two central sites and the Krylov dynamics of c^dag_{4 up} psi equal ED;
  - 2 x 5 ladder with m = 16, 32, 64: the energy is variational and decreases with m (the error 0.33,
    0.046, 0.0074: a ladder needs more states than a chain of the same length);
  - 2 x 3 ladder with m = 256: the sweep with time-step targeting is the exact time evolution of
    c^dag_{3 up} psi (every target's central densities, bond and norm against ED, 1e-11)."""
import numpy as np
import pytest

from oracle import dmrg, ed, krylov, superblock, tst

T_LEG, T_RUNG, U = 1.0, 0.5, 4.0


def _geom():
    return dmrg.Geometry(2, T_LEG, T_RUNG)


@pytest.mark.parametrize("lx", range(1, 7))
def test_geometry_is_the_lattice(lx):
    for tl, tr in ((1.0, 1.0), (1.0, 0.5), (0.7, 1.3)):
        assert np.array_equal(dmrg.Geometry(2, tl, tr).hopping(2 * lx), ed.ladder_hopping(lx, tl, tr))
    assert np.array_equal(dmrg.Geometry(1, 0.8).hopping(2 * lx), ed.chain_hopping(2 * lx, 0.8))


@pytest.fixture(scope="module")
def exact_ladder():
    d = dmrg.ChainDMRG(8, T_LEG, U, 256, geom=_geom())
    return d, d.run(sweeps=1)


def test_ladder_exact_blocks_match_ed(exact_ladder):
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = exact_ladder
    sec = ed.Sector(8, 4, 4)
    e_ed, v_ed = ed.ground_state(ed.hamiltonian(sec, ed.ladder_hopping(4, T_LEG, T_RUNG), U))
    assert abs(e - e_ed) < 1e-10
    assert sb.size((4, 4)) == sec.dim
    assert len(conns) == 2 * 2 * 2   # the central cut (sites 3 | 4) crosses two legs and no rung
    for blk, side, site in ((Lenl, 0, 3), (Renl, 1, 4)):
        for sig in range(2):
            n_op = blk.blockop(blk.cdag[sig] @ blk.cdag[sig].conj().T, False)
            A, B = (n_op, None) if side == 0 else (None, n_op)
            assert abs(superblock.expect(sb, A, B, (4, 4), psi).real - ed.density(v_ed, sec, site, sig)) < 1e-10


def test_ladder_superblock_dynamics_match_ed(exact_ladder):
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = exact_ladder
    Q0, Q1 = (4, 4), (5, 4)
    phi = superblock.apply_op(sb, None, Renl.blockop(Renl.cdag[0], True), Q0, psi, Q1)
    hop = ed.ladder_hopping(4, T_LEG, T_RUNG)
    sec0, sec1 = ed.Sector(8, 4, 4), ed.Sector(8, 5, 4)
    _, v_ed = ed.ground_state(ed.hamiltonian(sec0, hop, U))
    phi_ed = ed.apply_site_op(v_ed, sec0, sec1, [("cdag", ed.mode(4, 0))])
    H1 = ed.hamiltonian(sec1, hop, U)
    traj = krylov.time_steps(lambda v: superblock.apply_h(sb, HL, HR, conns, Q1, v), phi, 0.1, 5, 4, 12)
    n4 = Renl.blockop(Renl.cdag[0] @ Renl.cdag[0].conj().T, False)
    n3 = Lenl.blockop(Lenl.cdag[0] @ Lenl.cdag[0].conj().T, False)
    for s, (tg, _, _) in enumerate(traj):
        ex = ed.evolve(H1, phi_ed, [(s + 1) * 0.1])[0]
        assert abs(superblock.expect(sb, None, n4, Q1, tg[-1]).real - ed.density(ex, sec1, 4, 0)) < 1e-9
        assert abs(superblock.expect(sb, n3, None, Q1, tg[-1]).real - ed.density(ex, sec1, 3, 0)) < 1e-9


def test_ladder_energy_variational_in_m():
    e_ed, _ = ed.ground_state(ed.hamiltonian(ed.Sector(10, 5, 5), ed.ladder_hopping(5, T_LEG, T_RUNG), U))
    es = [dmrg.ChainDMRG(10, T_LEG, U, m, geom=_geom()).run(sweeps=1)[6] for m in (16, 32, 64)]
    assert all(x >= e_ed - 1e-10 for x in es), (es, e_ed)
    assert es[0] >= es[1] - 1e-10 >= es[2] - 2e-10, es
    assert es[2] - e_ed < 0.05 * (es[0] - e_ed) and es[2] - e_ed < 1e-2, (es, e_ed)   # 3.4e-1, 7.4e-3


def test_ladder_exact_sweep_is_exact_time_evolution():
    d = dmrg.ChainDMRG(6, T_LEG, U, 256, geom=_geom())
    d.run(sweeps=1)
    s = tst.TSTSweep(d, 256, n_v=4, tau=0.1, nk=12, advance_every=1, excitations=[(3, "cdag", 0)])
    recs = s.run()
    hop = ed.ladder_hopping(3, T_LEG, T_RUNG)
    sec0, sec1 = ed.Sector(6, 3, 3), ed.Sector(6, 4, 3)
    e0, v = ed.ground_state(ed.hamiltonian(sec0, hop, U))
    phi = ed.apply_site_op(v, sec0, sec1, [("cdag", ed.mode(3, 0))])
    times = sorted({round(r["t"] + tx, 12) for r in recs for tx in s.times})
    traj = dict(zip(times, ed.evolve(ed.hamiltonian(sec1, hop, U), phi, times)))
    assert recs[0]["action"] == "excite" and sum(r["action"] == "advance" for r in recs) == len(recs) - 1
    for r in recs:
        assert abs(r["energy"] - e0) < 1e-12
        if r["move"] is not None:
            assert r["discarded"] == 0.0
        l = r["l"]
        for tx, o in zip(s.times, r["targets"]):
            x = traj[round(r["t"] + tx, 12)]
            assert abs(o["n_left"] - ed.density(x, sec1, l, 0)) < 1e-11
            assert abs(o["n_right"] - ed.density(x, sec1, l + 1, 0)) < 1e-11
            w = ed.apply_site_op(x, sec1, sec1, [("cdag", ed.mode(l, 0)), ("c", ed.mode(l + 1, 0))])
            assert abs(o["bond"] - np.vdot(x, w) / np.vdot(x, x)) < 1e-11
            assert abs(o["norm2"] - np.vdot(x, x).real) < 1e-11
