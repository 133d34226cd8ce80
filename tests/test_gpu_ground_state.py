"""Device ground-state solver (ground-state targeting of Sec. II.B): restarted Lanczos with the lowest
eigenvector of the tridiagonal combined in place, FP64 throughout.

  - L=8 exact chain (half filling): the energy against the oracle's exact-cut ground state (1e-11), the
    state against it up to a global phase (1 - |<a|b>| < 1e-10) and its residual ||H psi - E psi||;
  - one electron on the open L=8 chain (sector (1, 0), dimension 8, Lanczos breaks down inside the
    first restart): the closed form E = -2 t cos(pi / (L + 1));
  - L=10 m=32 DMRG superblock: the energy against the oracle DMRG's ground state (1e-10) and the
    overlap with it."""
import numpy as np
import pytest

from oracle import dmrg, superblock
from tests.gpu_util import DmrgLoader, ExactLoader, dev, host, new_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _start(n, seed=7):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def test_ground_state_exact_chain(lib, c1_problem, c1_ground):
    p = c1_problem
    e_ref, psi_ref = c1_ground
    ctx = new_ctx(nk_max=32)
    try:
        ExactLoader(ctx, p)
        psi = dev(_start(len(psi_ref)))
        e = lib.tdmrg_ground_state(ctx, p.Q, psi, nk=32, restarts=40)
        v = host(psi)
        assert abs(e - e_ref) < 1e-11
        assert abs(np.linalg.norm(v) - 1.0) < 1e-13
        assert 1.0 - abs(np.vdot(v, psi_ref)) < 1e-10
        assert np.linalg.norm(p.apply_h(p.Q)(v) - e * v) < 1e-6
    finally:
        lib.tdmrg_destroy(ctx)


def test_ground_state_one_electron_closed_form(lib, c1_problem):
    """A single up electron on the open chain: H is the hopping matrix, lowest level -2 t cos(pi/(L+1))."""
    p = c1_problem
    Q = (1, 0)
    ctx = new_ctx(nk_max=32)
    try:
        ExactLoader(ctx, p)
        n = lib.tdmrg_sector_size(ctx, Q)
        assert n == 8
        psi = dev(_start(n, seed=3))
        e = lib.tdmrg_ground_state(ctx, Q, psi, nk=16, restarts=3)
        assert abs(e - (-2.0 * np.cos(np.pi / 9.0))) < 1e-13
        v = host(psi)
        assert np.linalg.norm(p.apply_h(Q)(v) - e * v) < 1e-12
    finally:
        lib.tdmrg_destroy(ctx)


def test_ground_state_dmrg_superblock(lib):
    Lsites, U, t, m = 10, 4.0, 1.0, 32
    Lenl, Renl, sb, HL, HR, conns, e_ref, psi_ref = dmrg.ChainDMRG(Lsites, t, U, m).run(sweeps=1)
    Q = (Lsites // 2, Lsites // 2)
    ctx = new_ctx(nk_max=32)
    try:
        DmrgLoader(ctx, Lenl, Renl, t)
        psi = dev(_start(len(psi_ref), seed=11))
        e = lib.tdmrg_ground_state(ctx, Q, psi, nk=32, restarts=40)
        v = host(psi)
        assert abs(e - e_ref) < 1e-10
        assert 1.0 - abs(np.vdot(v, psi_ref)) < 1e-9
        r = superblock.apply_h(sb, HL, HR, conns, Q, v) - e * v
        assert np.linalg.norm(r) < 1e-6
    finally:
        lib.tdmrg_destroy(ctx)
