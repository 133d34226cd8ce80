"""The allocation-free H psi entry point (tdmrg_apply_h_static) against tdmrg_apply_h.

It serves callers that may not allocate device memory while running (allocation-free real-time
loops, frameworks whose pool owns the device memory, plugins limited to the buffers they are
handed).  Its scratch is the library's static 32 MiB device array, shared by all calls, so this
checks two calls in a row with different inputs: the second must not be disturbed by what the first
left in the array.  Tolerance as for the FP64 H psi parity tests (1e-12 relative).  The entry point
always computes in FP64, so on a mixed-precision context its result is compared with the FP64 path's
H psi, and with the tensor path's within that path's slicing error.  The primary no-allocation check
is the library's own allocation counter; the device-wide free memory is a secondary check.  This
file is collected last on purpose."""
import numpy as np
import pytest

from tests.gpu_util import dev, host, new_ctx, rel_err
from workloads import sectors as S

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def test_static_scratch_matches_apply_h_twice():
    torch = pytest.importorskip("torch")
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ss = S.make_synthetic(32, 400, 4.0, nbonds=1, seed=S.SEED_BASE + 1)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = T.tdmrg_sector_size(ctx, ss.Q1)
        with pytest.raises(T.TdmrgError) as e:           # not prepared yet: refuses rather than allocates
            T.tdmrg_apply_h_static(ctx, ss.Q1, dev(np.zeros(n)), dev(np.zeros(n)))
        assert e.value.code == T.TDMRG_ESTATE
        xs = [dev(_rand(n, 1)), dev(_rand(n, 2))]
        refs = []
        for x in xs:                                      # prepares the sector (may allocate)
            r = dev(np.zeros(n))
            T.tdmrg_apply_h(ctx, ss.Q1, x, r)
            refs.append(host(r))
        outs = [dev(np.full(n, np.nan + 0j)) for _ in range(3)]
        # the first call on a device loads the module that holds the static array and looks up its
        # address; the calls after it must not take any device memory
        alloc0 = T.tdmrg_alloc_count(ctx)
        T.tdmrg_apply_h_static(ctx, ss.Q1, xs[1], outs[0])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        T.tdmrg_apply_h_static(ctx, ss.Q1, xs[0], outs[1])   # two calls in a row, different inputs
        T.tdmrg_apply_h_static(ctx, ss.Q1, xs[1], outs[2])
        torch.cuda.synchronize()
        assert T.tdmrg_alloc_count(ctx) == alloc0             # the library allocated nothing
        assert torch.cuda.mem_get_info()[0] == free0
        for o, r in zip(outs, (refs[1], refs[0], refs[1])):
            assert rel_err(host(o), r) < TOL
    finally:
        T.tdmrg_destroy(ctx)


def test_static_scratch_on_mixed_context_is_fp64():
    """On a tensor-core (Ozaki, 4 slices) context the entry point still computes the FP64 product:
    equal to an FP64 context's tdmrg_apply_h bit for bit, and to the context's own tensor-core
    tdmrg_apply_h within the slicing error bound of the tensor-path tests (140 2^-28 relative at 4
    slices)."""
    torch = pytest.importorskip("torch")
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ss = S.make_synthetic(32, 400, 4.0, nbonds=1, seed=S.SEED_BASE + 1)
    ctx64, ctxm = new_ctx(), new_ctx(prec=T.TDMRG_OZAKI_BF16, ozaki_slices=4)
    try:
        problem.load_synthetic(ctx64, ss)
        problem.load_synthetic(ctxm, ss)
        n = T.tdmrg_sector_size(ctxm, ss.Q1)
        xs = [dev(_rand(n, 3)), dev(_rand(n, 4))]
        for x in xs:
            r64, rm = dev(np.zeros(n)), dev(np.zeros(n))
            T.tdmrg_apply_h(ctx64, ss.Q1, x, r64)
            T.tdmrg_apply_h(ctxm, ss.Q1, x, rm)              # prepares the sector (may allocate)
            a0 = T.tdmrg_alloc_count(ctxm)
            outs = [dev(np.full(n, np.nan + 0j)) for _ in range(2)]
            for o in outs:                                    # two calls in a row
                T.tdmrg_apply_h_static(ctxm, ss.Q1, x, o)
            torch.cuda.synchronize()
            assert T.tdmrg_alloc_count(ctxm) == a0
            for o in outs:
                assert np.array_equal(host(o).view(np.float64), host(r64).view(np.float64))
                assert rel_err(host(o), host(rm)) < 140.0 * 2.0 ** -28
    finally:
        T.tdmrg_destroy(ctx64)
        T.tdmrg_destroy(ctxm)


def test_static_scratch_rejects_oversized_sector():
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ss = S.make_synthetic(32, 1600, 8.0, nbonds=2, seed=S.SEED_BASE + 5)   # 8 intermediates of ~0.7M entries
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = T.tdmrg_sector_size(ctx, ss.Q1)
        T.tdmrg_hpsi_flops(ctx, ss.Q1)                    # prepares the sector
        with pytest.raises(T.TdmrgError) as e:
            T.tdmrg_apply_h_static(ctx, ss.Q1, dev(np.zeros(n)), dev(np.zeros(n)))
        assert e.value.code == T.TDMRG_ENOMEM
        assert "32 MiB" in T.tdmrg_last_error(ctx)
    finally:
        T.tdmrg_destroy(ctx)
