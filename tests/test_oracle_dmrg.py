"""Pins of the oracle's two-site DMRG (Sec. I) against exact diagonalisation and against the
definition of the truncation rule.

  - L = 8 with m = 256: every block is exact, so the DMRG ground-state energy, the densities of the two
    central sites and the Krylov dynamics of c^dag_{4 up} psi on the DMRG superblock equal ED;
  - L = 10 with m = 8, 16, 32: the energy is variational (above ED) and decreases with m;
  - kept_counts: on random spectra with planted ties across sectors, the kept set is the unique one
    with (a) min(m, total) states, (b) no dropped state above a kept one beyond the tie tolerance,
    (c) among tied states, kept ones before dropped ones in (sector, index) order."""
import itertools

import numpy as np
import pytest

from oracle import density, dmrg, ed, krylov, superblock


@pytest.fixture(scope="module")
def exact8():
    d = dmrg.ChainDMRG(8, 1.0, 4.0, 256)
    return d, d.run(sweeps=1)


def test_dmrg_exact_blocks_match_ed(exact8):
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = exact8
    sec = ed.Sector(8, 4, 4)
    H = ed.hamiltonian(sec, ed.chain_hopping(8), 4.0)
    e_ed, v_ed = ed.ground_state(H)
    assert abs(e - e_ed) < 1e-10
    assert sb.size((4, 4)) == sec.dim
    # densities of the central sites 3 (left edge) and 4 (right edge) from the edge operators
    for blk, side, site in ((Lenl, 0, 3), (Renl, 1, 4)):
        for sig in range(2):
            n_op = blk.blockop(blk.cdag[sig] @ blk.cdag[sig].conj().T, False)
            A, B = (n_op, None) if side == 0 else (None, n_op)
            got = superblock.expect(sb, A, B, (4, 4), psi).real
            assert abs(got - ed.density(v_ed, sec, site, sig)) < 1e-10


def test_dmrg_superblock_dynamics_match_ed(exact8):
    """phi = c^dag_{4 up} psi (the right edge operator with the left parity) evolved by the oracle's
    Krylov steps on the DMRG superblock: n_{4 up}(t) and n_{3 up}(t) equal ED's."""
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = exact8
    Q0, Q1 = (4, 4), (5, 4)
    cd4 = Renl.blockop(Renl.cdag[0], True)
    phi = superblock.apply_op(sb, None, cd4, Q0, psi, Q1)
    sec0, sec1 = ed.Sector(8, 4, 4), ed.Sector(8, 5, 4)
    e_ed, v_ed = ed.ground_state(ed.hamiltonian(sec0, ed.chain_hopping(8), 4.0))
    phi_ed = ed.apply_site_op(v_ed, sec0, sec1, [("cdag", ed.mode(4, 0))])
    H1 = ed.hamiltonian(sec1, ed.chain_hopping(8), 4.0)
    hf = lambda v: superblock.apply_h(sb, HL, HR, conns, Q1, v)
    traj = krylov.time_steps(hf, phi, 0.1, 5, 4, 12)
    n4 = Renl.blockop(Renl.cdag[0] @ Renl.cdag[0].conj().T, False)
    n3 = Lenl.blockop(Lenl.cdag[0] @ Lenl.cdag[0].conj().T, False)
    for s, (tg, _, _) in enumerate(traj):
        ex = ed.evolve(H1, phi_ed, [(s + 1) * 0.1])[0]
        assert abs(superblock.expect(sb, None, n4, Q1, tg[-1]).real - ed.density(ex, sec1, 4, 0)) < 1e-9
        assert abs(superblock.expect(sb, n3, None, Q1, tg[-1]).real - ed.density(ex, sec1, 3, 0)) < 1e-9


def test_dmrg_energy_variational_in_m():
    sec = ed.Sector(10, 5, 5)
    e_ed, _ = ed.ground_state(ed.hamiltonian(sec, ed.chain_hopping(10), 4.0))
    es = []
    for m in (8, 16, 32):
        es.append(dmrg.ChainDMRG(10, 1.0, 4.0, m).run(sweeps=1)[6])
    assert all(e >= e_ed - 1e-10 for e in es), (es, e_ed)
    assert es[0] >= es[1] - 1e-10 >= es[2] - 2e-10, es
    assert es[2] - e_ed < 1e-3


def _check_kept(evals, m, counts, tie_rel=dmrg.TIE_REL):
    total = sum(len(e) for e in evals)
    assert sum(counts) == min(m, total)
    kept = [(lam, s, k) for s, ev in enumerate(evals) for k, lam in enumerate(ev) if k < counts[s]]
    drop = [(lam, s, k) for s, ev in enumerate(evals) for k, lam in enumerate(ev) if k >= counts[s]]
    if not drop or not kept:
        return
    lam_max = max(max(ev) for ev in evals if len(ev))
    tol = tie_rel * lam_max
    assert min(x[0] for x in kept) >= max(x[0] for x in drop) - tol
    lam_m = sorted((x[0] for x in kept + drop), reverse=True)[m - 1]
    tied = sorted([x for x in kept + drop if abs(x[0] - lam_m) <= tol], key=lambda x: (x[1], x[2]))
    flags = [x in kept for x in tied]
    assert flags == sorted(flags, reverse=True)        # kept ties first in (sector, index) order


@pytest.mark.parametrize("seed", range(6))
def test_kept_counts_rule(seed):
    rng = np.random.default_rng(seed)
    nsec = 7
    base = [np.sort(rng.exponential(1.0, rng.integers(1, 6)) * 10.0 ** -rng.integers(0, 4))[::-1] for _ in range(nsec)]
    evals = [b.copy() for b in base]
    evals[3] = evals[1].copy()                        # two sectors with identical spectra (spin flip)
    evals[5] = np.concatenate([evals[5], [evals[0][0]] * 2])[::-1]
    evals = [np.sort(e)[::-1] for e in evals]
    total = sum(len(e) for e in evals)
    for m in range(1, total + 2):
        _check_kept(evals, m, dmrg.kept_counts(evals, m))


def test_kept_counts_brute_force_small():
    """On tiny spectra with exact ties the rule's choice is the only prefix choice with properties (a)-(c)."""
    evals = [np.array([0.5, 0.25]), np.array([0.25, 0.1]), np.array([0.25])]
    for m in range(1, 6):
        counts = dmrg.kept_counts(evals, m)
        valid = []
        for c in itertools.product(*[range(len(e) + 1) for e in evals]):
            try:
                _check_kept(evals, m, list(c))
                valid.append(list(c))
            except AssertionError:
                pass
        assert valid == [counts], (m, valid, counts)
    assert dmrg.kept_counts(evals, 2) == [2, 0, 0]        # the 0.25 tie goes to the lowest sector first
    assert dmrg.kept_counts(evals, 3) == [2, 1, 0]


def _position(d, l):
    """Superblock pieces at left-block size l of a finished run: (Lenl, Renl, r) with r = L - 2 - l."""
    r = d.L - 2 - l
    return dmrg.enlarge(d.left[l], "L", d.t, d.U), dmrg.enlarge(d.right[r], "R", d.t, d.U), r


def test_wft_exact_without_truncation():
    """L=8 with m=256: no state is dropped, so the wave-function transformation is a change of basis --
    the ground state at the centre, moved one site to the right, is the ground state of the next
    superblock (H psi' = E psi' to 1e-10) with the same norm and central densities."""
    d = dmrg.ChainDMRG(8, 1.0, 4.0, 256)
    Lenl, Renl, sb, HL, HR, conns, e, psi = d.run(sweeps=1)
    Q = (4, 4)
    l = 3
    Lc, Rc, r = _position(d, l)
    assert Lc.dim == Lenl.dim and Rc.dim == Renl.dim
    rho = density.rho_left(sb, [(Q, psi)], [1.0])
    Lb, counts, lam, disc, U = dmrg.truncate(Lenl, rho, 256)
    Ln = dmrg.enlarge(Lb, "L", 1.0, 4.0)
    Rn = dmrg.enlarge(d.right[r - 1], "R", 1.0, 4.0)
    psi2 = dmrg.wft_right(Lenl, Renl, Q, psi, U, d.right[r], d.right_U[r], Ln, Rn)
    sb2, HL2, HR2, conns2 = dmrg.superblock_of(Ln, Rn, 1.0)
    assert abs(np.linalg.norm(psi2) - 1.0) < 1e-12
    res = superblock.apply_h(sb2, HL2, HR2, conns2, Q, psi2) - e * psi2
    assert np.abs(res).max() < 1e-10
    # the density of site 4 (right edge before, left edge after the move)
    n_before = Renl.blockop(Renl.cdag[0] @ Renl.cdag[0].conj().T, False)
    n_after = Ln.blockop(Ln.cdag[0] @ Ln.cdag[0].conj().T, False)
    assert abs(superblock.expect(sb, None, n_before, Q, psi) - superblock.expect(sb2, n_after, None, Q, psi2)) < 1e-12
