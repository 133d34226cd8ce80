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
