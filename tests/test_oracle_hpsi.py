"""Pins of the oracle's sector-pair H psi (Sec. IV, Hamiltonian connections) against
brute force and exact diagonalisation."""
import numpy as np
import pytest

from oracle import blocks, ed, models, superblock
from workloads import sectors as S


def _oracle_ops(ss):
    HL = blocks.BlockOp(ss.HL, False)
    HR = blocks.BlockOp(ss.HR, False)
    conns = []
    for b in range(ss.nbonds):
        for s in range(2):
            A = blocks.BlockOp(ss.cdagL[b][s], True)
            B = blocks.BlockOp(ss.cR[b][s], True)
            conns.append((ss.coeff_t, A, B))
            conns.append((-ss.coeff_t, A.dagger(), B.dagger()))
    return HL, HR, conns


def test_sector_hpsi_matches_dense_kron():
    """Sector-pair H psi equals the dense np.kron superblock matrix on random blocks."""
    ss = S.make_synthetic(8, 10, 4.0, nbonds=2, seed=5)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    HL, HR, conns = _oracle_ops(ss)
    terms = superblock.hamiltonian_terms(HL, HR, conns)
    for Q in (ss.Q0, ss.Q1):
        M = superblock.dense_terms(sb, terms, Q, Q)
        rng = np.random.default_rng(1)
        x = rng.standard_normal(sb.size(Q)) + 1j * rng.standard_normal(sb.size(Q))
        y = superblock.apply_h(sb, HL, HR, conns, Q, x)
        assert np.abs(y - M @ x).max() < 1e-12 * max(1.0, np.abs(y).max())
        assert np.abs(M - M.conj().T).max() < 1e-12          # the term list is Hermitian


def test_excitation_matches_dense_kron_across_sectors():
    ss = S.make_synthetic(8, 10, 4.0, seed=6)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    B = blocks.BlockOp(ss.cdag_exc, True)
    A = blocks.BlockOp(ss.cdagL[0][1], True)
    for (a, b, Qo) in ((None, B, (ss.Q0[0] + 1, ss.Q0[1])), (A, None, (ss.Q0[0], ss.Q0[1] + 1)),
                       (A, B, (ss.Q0[0] + 1, ss.Q0[1] + 1))):
        M = superblock.dense_terms(sb, [(1.0, a, b)], ss.Q0, Qo)
        y = superblock.apply_op(sb, a, b, ss.Q0, ss.psi_gs, Qo)
        assert np.abs(y - M @ ss.psi_gs).max() < 1e-13


def _fock_perm(p, sector):
    return superblock.fock_to_psi(p.cut, sector, np.arange(sector.dim) + 0j).real.astype(int)


@pytest.mark.parametrize("geom", ["chain", "ladder"])
def test_exact_cut_hpsi_equals_ed(geom):
    """At a fixed cut with exact blocks the sector H psi is the ED Hamiltonian (pins P_L signs)."""
    if geom == "chain":
        p = models.chain(8, U=4.0)
        hop = ed.chain_hopping(8)
    else:
        p = models.ladder(4, t_leg=1.0, t_rung=0.5, U=10.0)
        hop = ed.ladder_hopping(4, 1.0, 0.5)
    for Q in ((4, 4), (5, 4), (3, 4)):
        sec = ed.Sector(8, *Q)
        H = ed.hamiltonian(sec, hop, p.U)
        perm = _fock_perm(p, sec)
        rng = np.random.default_rng(2)
        x = rng.standard_normal(sec.dim) + 1j * rng.standard_normal(sec.dim)
        y = superblock.apply_h(p.sb, p.HL, p.HR, p.conns, Q, x)
        xf = np.zeros(sec.dim, complex); xf[perm] = x
        assert np.abs((H @ xf)[perm] - y).max() < 1e-12


def test_local_operators_equal_ed():
    """c^dag, c, n on both blocks agree with the ED mode operators (Jordan-Wigner strings)."""
    p = models.chain(8, U=4.0)
    s44, s54, s34 = ed.Sector(8, 4, 4), ed.Sector(8, 5, 4), ed.Sector(8, 3, 4)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s44.dim) + 1j * rng.standard_normal(s44.dim)
    perm44 = _fock_perm(p, s44)
    xf = np.zeros(s44.dim, complex); xf[perm44] = x
    for site in (1, 3, 4, 6):
        for sig in (0, 1):
            Qo = (5, 4) if sig == 0 else (4, 5)
            so = ed.Sector(8, *Qo)
            y = p.apply_local("cdag", site, sig, (4, 4), x, Qo)
            yf = ed.apply_site_op(xf, s44, so, [("cdag", ed.mode(site, sig))])
            assert np.abs(yf[_fock_perm(p, so)] - y).max() < 1e-13
    y = p.apply_local("c", 5, 0, (4, 4), x, (3, 4))
    yf = ed.apply_site_op(xf, s44, s34, [("c", ed.mode(5, 0))])
    assert np.abs(yf[_fock_perm(p, s34)] - y).max() < 1e-13


def test_hermiticity_and_ground_state(c1_problem, c1_ground):
    p = c1_problem
    rng = np.random.default_rng(4)
    n = p.sb.size(p.Q)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Hx, Hz = p.apply_h(p.Q)(x), p.apply_h(p.Q)(z)
    assert abs(np.vdot(x, Hz) - np.vdot(Hx, z)) < 1e-10
    e_blk, v = c1_ground
    sec = ed.Sector(8, 4, 4)
    e_ed, _ = ed.ground_state(ed.hamiltonian(sec, ed.chain_hopping(8), 4.0))
    assert abs(e_blk - e_ed) < 1e-11
    assert np.linalg.norm(p.apply_h(p.Q)(v) - e_blk * v) < 1e-9
