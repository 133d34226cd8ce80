"""Correlation grid <phi1| A_i B_j |phi2> (Eq. generalcorrelation, one local operator per block; the
Green's function G_ij(t) of Sec. I) on the exact L=8 chain: the whole grid of c_{i up} (left sites
0..3) times c^dag_{j up} (right sites 4..7) against the oracle's product-by-product loop and against
exact diagonalisation in the Fock basis (which fixes the fermion signs), and a time series
G_ij(t) = <psi(t)| c_i c^dag_j |psi(t)> over Krylov steps of the excited state, reusing the grid's
plan.  FP64 throughout: bound 1e-13 absolute on entries of order one."""
import numpy as np
import pytest

from oracle import ed, krylov, superblock
from tests.gpu_util import ExactLoader, dev, host, new_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _fock(p, Q, v):
    sec = ed.Sector(8, *Q)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    out = np.zeros(sec.dim, complex)
    out[perm] = v
    return sec, out


def test_correlation_grid_against_oracle_and_ed(lib, c1_problem, c1_ground):
    p = c1_problem
    e, psi = c1_ground
    Q = p.Q
    rng = np.random.default_rng(5)
    phi1 = rng.standard_normal(len(psi)) + 1j * rng.standard_normal(len(psi))
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        left = [ld.local("c", i, 0)[0] for i in range(4)]
        right = [ld.local("cdag", j, 0)[1] for j in range(4, 8)]
        out = dev(np.zeros(16))
        lib.tdmrg_correlation(ctx, left, right, Q, dev(phi1), Q, dev(psi), out)
        got = host(out).reshape(4, 4)
        sec, psi_f = _fock(p, Q, psi)
        _, phi1_f = _fock(p, Q, phi1)
        for i in range(4):
            for j in range(4):
                A, B = p.op("c", i, 0)[1], p.op("cdag", 4 + j, 0)[1]
                ref = np.vdot(phi1, superblock.apply_op(p.sb, A, B, Q, psi, Q))
                x = ed.apply_site_op(psi_f, sec, sec, [("c", ed.mode(i, 0)), ("cdag", ed.mode(4 + j, 0))])
                assert abs(got[i, j] - ref) < 1e-13
                assert abs(got[i, j] - np.vdot(phi1_f, x)) < 1e-12
    finally:
        lib.tdmrg_destroy(ctx)


def test_correlation_time_series(lib, c1_problem, c1_ground):
    """G_ij(t) = <phi(t)| c_i c^dag_j |phi(t)> for phi = c^dag_{4 up} psi evolved by 3 Krylov steps, one
    grid per step (the plan built at the first step is reused)."""
    p = c1_problem
    e, psi = c1_ground
    Q1 = (5, 4)
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        oL, oR = ld.local("cdag", 4, 0)
        left = [ld.local("c", i, 0)[0] for i in range(4)]
        right = [ld.local("cdag", j, 0)[1] for j in (5, 6)]
        n = lib.tdmrg_sector_size(ctx, Q1)
        phi = dev(np.zeros(n))
        lib.tdmrg_apply_op(ctx, oL, oR, p.Q, dev(psi), Q1, phi)
        times = krylov.target_times(0.1, 3)
        tg = [dev(np.zeros(n)) for _ in range(2)] + [phi]
        ref_phi = superblock.apply_op(p.sb, None, p.op("cdag", 4, 0)[1], p.Q, psi, Q1)
        traj = krylov.time_steps(p.apply_h(Q1), ref_phi, 0.1, 3, 3, 12)
        out = dev(np.zeros(8))
        for s in range(3):
            lib.tdmrg_evolve(ctx, Q1, phi, times, 12, tg)
            lib.tdmrg_correlation(ctx, left, right, Q1, phi, Q1, phi, out)
            got = host(out).reshape(4, 2)
            v = traj[s][0][-1]
            for i in range(4):
                for jj, j in enumerate((5, 6)):
                    A, B = p.op("c", i, 0)[1], p.op("cdag", j, 0)[1]
                    ref = np.vdot(v, superblock.apply_op(p.sb, A, B, Q1, v, Q1))
                    assert abs(got[i, jj] - ref) < 1e-12
        lib.tdmrg_evolve_info(ctx)
    finally:
        lib.tdmrg_destroy(ctx)
