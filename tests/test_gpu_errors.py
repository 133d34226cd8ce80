"""Error behaviour of the C ABI on a GPU: negative codes, never an abort."""
import numpy as np
import pytest

from tests.gpu_util import dev, new_ctx
from workloads import sectors as S

pytestmark = pytest.mark.gpu


def test_error_codes():
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ctx = new_ctx()
    try:
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_set_block(ctx, 0, [(1, 0), (0, 0)], [1, 1])
        assert e.value.code == T.TDMRG_ESECTOR
        ss = S.make_synthetic(8, 20, 4.0, seed=2)
        T.tdmrg_set_block(ctx, 0, ss.lsec, ss.ldim)
        T.tdmrg_set_block(ctx, 1, ss.rsec, ss.rdim)
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_apply_h(ctx, ss.Q0, dev(np.zeros(4)), dev(np.zeros(4)))
        assert e.value.code == T.TDMRG_ESTATE
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_set_op(ctx, 0, 1, 0, [((99, 0), (0, 0), np.zeros((1, 1)))])
        assert e.value.code == T.TDMRG_ESECTOR
        with pytest.raises(T.TdmrgError) as e:      # parity flag contradicts the blocks
            T.tdmrg_set_op(ctx, 0, 1, 0, [(ss.lsec[1], ss.lsec[0], np.zeros((ss.ldim[1], ss.ldim[0])))])
        assert e.value.code == T.TDMRG_ESECTOR
        problem.load_synthetic(ctx, ss)
        n = T.tdmrg_sector_size(ctx, ss.Q1)
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_evolve(ctx, ss.Q1, dev(np.zeros(n)), [0.0, 0.1], 40, [dev(np.zeros(n))] * 2)
        assert e.value.code == T.TDMRG_EINVAL
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_apply_op(ctx, 77, -1, ss.Q0, dev(np.zeros(4)), ss.Q0, dev(np.zeros(4)))
        assert e.value.code == T.TDMRG_EINVAL
        assert "77" in T.tdmrg_last_error(ctx)
    finally:
        T.tdmrg_destroy(ctx)
    with pytest.raises(T.TdmrgError) as e:          # the context's own workspace exceeds 1 KB
        new_ctx(hbm_budget=1024)
    assert e.value.code == T.TDMRG_ENOMEM
    small = new_ctx(hbm_budget=1 << 20)              # workspace fits, the L=32 m=400 operators do not
    try:
        with pytest.raises(T.TdmrgError) as e:
            problem.load_synthetic(small, S.make_synthetic(32, 400, 4.0, seed=2))
        assert e.value.code == T.TDMRG_ENOMEM
    finally:
        T.tdmrg_destroy(small)


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a word that nothing sets gives up after its bound and reports TDMRG_ETIMEOUT
    through the context's status word; the context keeps working and its results are unchanged."""
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ss = S.make_synthetic(12, 60, 4.0, nbonds=1, seed=5)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = T.tdmrg_sector_size(ctx, ss.Q1)
        x = dev(np.random.default_rng(4).standard_normal(n) + 0j)
        y0, y1 = dev(np.zeros(n)), dev(np.zeros(n))
        T.tdmrg_apply_h(ctx, ss.Q1, x, y0)
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_probe_wait(ctx, 100000)
        assert e.value.code == T.TDMRG_ETIMEOUT
        assert "bounded device wait" in T.tdmrg_last_error(ctx)
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_probe_wait(ctx, 0)
        assert e.value.code == T.TDMRG_EINVAL
        T.tdmrg_apply_h(ctx, ss.Q1, x, y1)
        assert np.array_equal(y0.cpu().numpy(), y1.cpu().numpy())
        T.tdmrg_evolve(ctx, ss.Q1, dev(ss.phi), [0.0, 0.05], 8, [dev(np.zeros(n)), dev(np.zeros(n))])
        T.tdmrg_evolve_info(ctx)   # the status word was consumed: no stale timeout
    finally:
        T.tdmrg_destroy(ctx)
