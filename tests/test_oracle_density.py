"""Pins of the oracle's weighted reduced density matrix (Eq. rdensitymatrix) and
target weights (Sec. II.C)."""
import numpy as np
import pytest

from oracle import density, superblock
from workloads import sectors as S


def test_weights():
    wgs, w = density.tst_weights(4)
    assert wgs == pytest.approx(2 / 8) and w == pytest.approx([2 / 8, 1 / 8, 1 / 8, 2 / 8])
    for nv in range(2, 9):
        wgs, w = density.tst_weights(nv)
        assert wgs + sum(w) == pytest.approx(1.0, abs=1e-15)
        assert min(w) > 0
    with pytest.raises(ValueError):
        density.tst_weights(1)


def _full_matrix(sb, Q, psi):
    """Psi as a dense DL x DR matrix over the whole block bases."""
    DL, DR = sum(sb.ldim), sum(sb.rdim)
    M = np.zeros(DL * DR, dtype=complex)
    M[superblock.superblock_index(sb, Q)] = psi
    return M.reshape(DL, DR)


def test_single_target_spectrum_is_schmidt():
    """One target, weight 1: eigenvalues of rho_L are the squared singular values of Psi."""
    ss = S.make_synthetic(8, 12, 4.0, seed=7)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    rho = density.rho_left(sb, [(ss.Q0, 3.0 * ss.psi_gs)], [1.0])
    lam = np.sort(np.concatenate([e for e, U in density.rho_eig(rho)]))[::-1]
    sv = np.linalg.svd(_full_matrix(sb, ss.Q0, ss.psi_gs), compute_uv=False)
    sv2 = np.concatenate([sv ** 2, np.zeros(len(lam) - len(sv))])
    assert np.abs(lam - sv2).max() < 1e-13


def test_mixed_sector_rho_properties():
    """Targets in two sectors: rho_L is Hermitian, PSD, trace = sum of weights; equals the dense sum."""
    ss = S.make_synthetic(8, 12, 4.0, seed=8)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    rng = np.random.default_rng(0)
    states = [(ss.Q0, ss.psi_gs), (ss.Q1, ss.phi), (ss.Q1, ss.phi * 1j + 0.1)]
    wgs, w = density.tst_weights(2)
    weights = [wgs] + w
    rho = density.rho_left(sb, states, weights)
    tr = sum(np.trace(r).real for r in rho)
    assert abs(tr - 1.0) < 1e-13
    dense = sum(wt * (lambda M: M @ M.conj().T)(_full_matrix(sb, Q, v)) / np.vdot(v, v).real
                for (Q, v), wt in zip(states, weights))
    offs = np.concatenate([[0], np.cumsum(sb.ldim)])
    for qi, r in enumerate(rho):
        assert np.abs(r - r.conj().T).max() < 1e-15
        assert np.linalg.eigvalsh(r).min() > -1e-14
        assert np.abs(r - dense[offs[qi]:offs[qi + 1], offs[qi]:offs[qi + 1]]).max() < 1e-14
    for (lam, U), r in zip(density.rho_eig(rho), rho):
        assert np.all(np.diff(lam) <= 1e-15)
        assert np.abs(U @ np.diag(lam) @ U.conj().T - r).max() < 1e-13


def test_real_basis_rho_is_real_part():
    """Targeting the real and imaginary parts apart gives Re rho_L (the real part of the Hermitian
    rho_L): checked against np.real of the complex rho_L, which is computed by a different formula;
    for real targets the two coincide; trace = sum of weights, positive semidefinite."""
    from oracle import density, superblock
    from workloads import sectors as S
    ss = S.make_synthetic(10, 40, 4.0, nbonds=1, seed=S.SEED_BASE + 21)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    states = [(ss.Q0, ss.psi_gs), (ss.Q1, ss.phi)]
    w = [0.75, 0.25]
    rc = density.rho_left(sb, states, w)
    rr = density.rho_left(sb, states, w, real_basis=True)
    for a, b in zip(rc, rr):
        assert np.abs(b.imag).max() == 0.0
        assert np.abs(b - a.real).max() < 1e-15
        assert np.linalg.eigvalsh(b).min() > -1e-14
    assert abs(sum(np.trace(b).real for b in rr) - 1.0) < 1e-13
    real_states = [(Q, v.real + 0j) for Q, v in states]
    for a, b in zip(density.rho_left(sb, real_states, w), density.rho_left(sb, real_states, w, real_basis=True)):
        assert np.abs(a - b).max() < 1e-15


def test_rho_right_is_the_partial_trace():
    """rho_R (Eq. rdensitymatrix for the right block, Sec. II.B) against the definition of the reduced
    density matrix: the partial trace over the left block of the full density matrix |psi><psi| (einsum on
    the DL x DR x DL x DR tensor), for the weighted rho_R of the sweep and the one-state rho_R of the DMRG;
    and against an independent route: Tr(rho_R O_R) = <psi| 1 x O_R |psi> / <psi|psi> (and the same for
    rho_L) with the complex Hermitian block Hamiltonians as O, through the sector-pair product.  A complex
    conjugated (transposed) rho_R fails the trace against a complex O."""
    from oracle import dmrg
    ss = S.make_synthetic(6, 8, 4.0, seed=S.SEED_BASE + 31)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    states = [(ss.Q0, ss.psi_gs), (ss.Q1, ss.phi * (0.3 - 0.8j))]
    weights = [0.6, 0.4]
    roffs = np.concatenate([[0], np.cumsum(sb.rdim)])
    loffs = np.concatenate([[0], np.cumsum(sb.ldim)])
    full_r = 0
    for (Q, v), w in zip(states, weights):
        M = _full_matrix(sb, Q, v)
        D = np.einsum("ab,cd->abcd", M, M.conj()) / np.vdot(v, v).real    # <a b|psi><psi|c d>
        full_r = full_r + w * np.einsum("abad->bd", D)
    rr = density.rho_right(sb, states, weights)
    for ri, r in enumerate(rr):
        blk = full_r[roffs[ri]:roffs[ri + 1], roffs[ri]:roffs[ri + 1]]
        assert np.abs(r - blk).max() < 1e-14
    # nothing outside the sector blocks (rho_R commutes with the right block's quantum numbers)
    mask = np.zeros_like(full_r, dtype=bool)
    for ri in range(len(rr)):
        mask[roffs[ri]:roffs[ri + 1], roffs[ri]:roffs[ri + 1]] = True
    assert np.abs(full_r[~mask]).max() < 1e-14
    # the DMRG's one-state rho_R (unnormalised psi, weight 1)
    v = 1.7 * ss.psi_gs
    M = _full_matrix(sb, ss.Q0, v)
    pt = np.einsum("ab,ad->bd", M, M.conj())
    for ri, r in enumerate(dmrg.rho_right(sb, ss.Q0, v)):
        assert np.abs(r - pt[roffs[ri]:roffs[ri + 1], roffs[ri]:roffs[ri + 1]]).max() < 1e-13
    # expectation values of complex Hermitian block operators through H psi's product route
    from oracle import blocks
    OL, OR = blocks.BlockOp(ss.HL, False), blocks.BlockOp(ss.HR, False)
    rl = density.rho_left(sb, states, weights)
    want_l = sum(w * superblock.expect(sb, OL, None, Q, x).real for (Q, x), w in zip(states, weights))
    want_r = sum(w * superblock.expect(sb, None, OR, Q, x).real for (Q, x), w in zip(states, weights))
    got_l = sum(np.trace(rl[k] @ ss.HL[(k, k)]).real for k in range(len(rl)) if (k, k) in ss.HL)
    got_r = sum(np.trace(rr[k] @ ss.HR[(k, k)]).real for k in range(len(rr)) if (k, k) in ss.HR)
    assert abs(got_l - want_l) < 1e-12 and abs(got_r - want_r) < 1e-12
    # the check is not vacuous: the conjugated matrix gives a different trace against the complex O
    bad_r = sum(np.trace(rr[k].conj() @ ss.HR[(k, k)]).real for k in range(len(rr)) if (k, k) in ss.HR)
    assert abs(bad_r - want_r) > 1e-3
