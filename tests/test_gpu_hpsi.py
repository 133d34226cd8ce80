"""GPU parity of the superblock product H psi and the excitation operators against the oracle
(Sec. IV Hamiltonian connections; Eq. b).  FP64 path tolerance: max |GPU - oracle| <= 1e-12 of
max |oracle| (K <= ~750 FP64 products per entry: K * 2^-53 ~ 1e-13)."""
import numpy as np
import pytest

from oracle import blocks as oblocks
from oracle import models, superblock
from tests.gpu_util import ExactLoader, dev, host, new_ctx, oracle_ops_of_synthetic, rel_err
from workloads import sectors as S

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("geom", ["chain", "ladder"])
def test_exact_cut_hpsi(lib, geom):
    p = models.chain(8, U=4.0) if geom == "chain" else models.ladder(4, 1.0, 0.5, U=10.0)
    ctx = new_ctx()
    try:
        ExactLoader(ctx, p)
        for Q in ((4, 4), (5, 4), (3, 4), (0, 0), (8, 8)):
            n = lib.tdmrg_sector_size(ctx, Q)
            assert n == p.sb.size(Q)
            x = _rand(n, 1)
            out = dev(np.zeros(n))
            lib.tdmrg_apply_h(ctx, Q, dev(x), out)
            ref = superblock.apply_h(p.sb, p.HL, p.HR, p.conns, Q, x)
            assert rel_err(host(out), ref) < TOL
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("L,m,nb,seed", [(8, 24, 2, 3), (12, 37, 1, 4), (32, 400, 1, S.SEED_BASE + 1),
                                         (32, 800, 2, S.SEED_BASE + 2)])
def test_synthetic_hpsi(lib, L, m, nb, seed):
    """Ragged Gaussian-sector superblocks, up to the L=32 m=400 chain and the 2x16 m=800 ladder."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(L, m, 4.0, nbonds=nb, seed=seed)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        for Q in (ss.Q0, ss.Q1, (ss.Q0[0] - 3, ss.Q0[1] + 2)):
            n = lib.tdmrg_sector_size(ctx, Q)
            assert n == sb.size(Q)
            x = _rand(n, 2)
            out = dev(np.full(n, np.nan + 0j))        # every entry must be written
            lib.tdmrg_apply_h(ctx, Q, dev(x), out)
            ref = superblock.apply_h(sb, HL, HR, conns, Q, x)
            assert rel_err(host(out), ref) < TOL
    finally:
        lib.tdmrg_destroy(ctx)


def test_excitations_and_sign(lib):
    """Cross-sector local operators: right-odd ops carry (-1)^{N_L}; left-only, right-only and both."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(10, 30, 4.0, nbonds=1, seed=9)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    B = oblocks.BlockOp(ss.cdag_exc, True)
    A = oblocks.BlockOp(ss.cdagL[0][1], True)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        for a_id, b_id, a, b, Qo in ((-1, problem.OP_EXC, None, B, (ss.Q0[0] + 1, ss.Q0[1])),
                                     (problem.OP_CDAG + 1, -1, A, None, (ss.Q0[0], ss.Q0[1] + 1)),
                                     (problem.OP_CDAG + 1, problem.OP_EXC, A, B, (ss.Q0[0] + 1, ss.Q0[1] + 1))):
            out = dev(np.zeros(sb.size(Qo)))
            lib.tdmrg_apply_op(ctx, a_id, b_id, ss.Q0, dev(ss.psi_gs), Qo, out)
            ref = superblock.apply_op(sb, a, b, ss.Q0, ss.psi_gs, Qo)
            assert rel_err(host(out), ref) < TOL
    finally:
        lib.tdmrg_destroy(ctx)


def test_exact_local_ops_match_oracle(lib):
    p = models.chain(8, U=4.0)
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        x = _rand(p.sb.size((4, 4)), 5)
        for site in (2, 3, 4, 7):
            for sig in (0, 1):
                oL, oR = ld.local("cdag", site, sig)
                Qo = (5, 4) if sig == 0 else (4, 5)
                out = dev(np.zeros(p.sb.size(Qo)))
                lib.tdmrg_apply_op(ctx, oL, oR, (4, 4), dev(x), Qo, out)
                ref = p.apply_local("cdag", site, sig, (4, 4), x, Qo)
                assert rel_err(host(out), ref) < TOL
    finally:
        lib.tdmrg_destroy(ctx)


def test_hermiticity_on_device(lib):
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 120, 4.0, nbonds=2, seed=12)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        x, y = _rand(n, 6), _rand(n, 7)
        hx, hy = dev(np.zeros(n)), dev(np.zeros(n))
        lib.tdmrg_apply_h(ctx, ss.Q1, dev(x), hx)
        lib.tdmrg_apply_h(ctx, ss.Q1, dev(y), hy)
        a, b = np.vdot(x, host(hy)), np.vdot(host(hx), y)
        assert abs(a - b) < 1e-11 * abs(a)
    finally:
        lib.tdmrg_destroy(ctx)
