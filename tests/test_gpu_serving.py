"""Serving (continuous batching of time-evolution jobs): every job's observables in the mix equal
the same job run alone (bit for bit: deterministic kernels, no shared memory between jobs); jobs
arriving while others run are admitted as slots and budget free up; cancellation frees a slot."""
import time

import numpy as np
import pytest

from tests.gpu_util import new_ctx, torch_cuda
from workloads import sectors as S

pytestmark = pytest.mark.gpu


def _job(T, problem, torch, L, m, nb, seed, prec):
    ss = S.make_synthetic(L, m, 4.0, nbonds=nb, seed=seed)
    ctx = new_ctx(prec=prec, ozaki_slices=4)
    problem.load_synthetic(ctx, ss)
    psi = torch.as_tensor(ss.psi_gs).cuda()
    phi = torch.zeros(T.tdmrg_sector_size(ctx, ss.Q1), dtype=torch.complex128, device="cuda")
    T.tdmrg_apply_op(ctx, -1, problem.OP_EXC, ss.Q0, psi, ss.Q1, phi)
    torch.cuda.synchronize()
    return ss, ctx, psi, phi


def _run(T, srv, jobs, steps, arrivals, problem):
    ids = []
    t0 = time.time()
    for (ss, ctx, psi, phi), at in zip(jobs, arrivals):
        while time.time() - t0 < at:
            time.sleep(0.001)
        ids.append(T.tdmrg_server_submit(srv, ctx, ss.Q0, psi, ss.Q1, phi, 0.05, 4, 8, steps,
                                         [(problem.OP_N, -1), (-1, problem.OP_N)]))
    out = {}
    deadline = time.time() + 300
    while len(out) < len(ids) and time.time() < deadline:
        for jid in ids:
            if jid in out:
                continue
            st, n, obs, ms = T.tdmrg_server_poll(srv, jid, steps, 2)
            if st >= T.TDMRG_JOB_DONE:
                assert st == T.TDMRG_JOB_DONE, T.tdmrg_server_last_error(srv, jid)
                out[jid] = (st, obs, ms)
        time.sleep(0.005)
    return [out[j] for j in ids]


@pytest.mark.parametrize("prec", [0, 1])
def test_mix_equals_alone(prec):
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    specs = [(16, 128, 1, 101), (20, 200, 2, 102), (24, 300, 1, 103), (16, 160, 2, 104), (28, 256, 1, 105)]
    steps = 6
    jobs = [_job(T, problem, torch, *sp, prec) for sp in specs]
    try:
        alone = []
        for jb in jobs:   # one at a time
            srv = T.tdmrg_server_create(0, 0, 1)
            try:
                alone.append(_run(T, srv, [jb], steps, [0.0], problem)[0])
            finally:
                T.tdmrg_server_destroy(srv)
        srv = T.tdmrg_server_create(0, 0, 3)   # three slots: later arrivals wait for a free slot
        try:
            mixed = _run(T, srv, jobs, steps, [0.0, 0.0, 0.01, 0.02, 0.03], problem)
            q, r, f, b = T.tdmrg_server_stats(srv)
            assert (q, r, f) == (0, 0, len(jobs))
        finally:
            T.tdmrg_server_destroy(srv)
        for (sa, oa, ma), (sm, om, mm) in zip(alone, mixed):
            assert sa == sm == T.TDMRG_JOB_DONE
            assert oa.shape == (steps, 2) and np.isfinite(oa).all()
            assert np.array_equal(oa, om)
            assert len(mm) == steps and (mm > 0).all()
    finally:
        for ss, ctx, psi, phi in jobs:
            T.tdmrg_destroy(ctx)


def test_budget_cancel_and_errors():
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    jobs = [_job(T, problem, torch, 20, 200, 1, 200 + k, 0) for k in range(3)]
    try:
        srv = T.tdmrg_server_create(0, 1, 4)   # 1-byte budget: one job at a time, in arrival order
        try:
            ids = [T.tdmrg_server_submit(srv, ctx, ss.Q0, psi, ss.Q1, phi, 0.05, 4, 8, 40, [(problem.OP_N, -1)])
                   for ss, ctx, psi, phi in jobs]
            seen_running = 0
            for _ in range(2000):
                q, r, f, b = T.tdmrg_server_stats(srv)
                seen_running = max(seen_running, r)
                if r == 1 and q == 2:
                    break
                time.sleep(0.001)
            assert seen_running <= 1
            T.tdmrg_server_cancel(srv, ids[0])
            T.tdmrg_server_cancel(srv, ids[2])
            for _ in range(20000):
                st = [T.tdmrg_server_poll(srv, j, 40, 1)[0] for j in ids]
                if all(x >= T.TDMRG_JOB_DONE for x in st):
                    break
                time.sleep(0.002)
            assert st[0] == T.TDMRG_JOB_CANCELLED and st[2] == T.TDMRG_JOB_CANCELLED
            assert st[1] == T.TDMRG_JOB_DONE
            assert T.tdmrg_server_poll(srv, ids[1], 40, 1)[1] == 40
            with pytest.raises(T.TdmrgError):
                T.tdmrg_server_poll(srv, 999, 1, 1)
            ss, ctx, psi, phi = jobs[0]
            with pytest.raises(T.TdmrgError):   # n_v = 1 is not time-step targeting
                T.tdmrg_server_submit(srv, ctx, ss.Q0, psi, ss.Q1, phi, 0.05, 1, 8, 4)
            with pytest.raises(T.TdmrgError):   # rho_L would take 13 states
                T.tdmrg_server_submit(srv, ctx, ss.Q0, psi, ss.Q1, phi, 0.05, 12, 8, 4)
        finally:
            T.tdmrg_server_destroy(srv)
    finally:
        for ss, ctx, psi, phi in jobs:
            T.tdmrg_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_server_job_against_oracle(prec):
    """A server job's observables after every time step against the oracle's trajectory of the same job
    (Krylov advance with 4 targets, n_K = 8, tau = 0.05), while a second job runs beside it.  Bounds:
    FP64 path 1e-12; tensor path (4 slices) 1e-8, the observable accuracy target."""
    torch = torch_cuda()
    from oracle import krylov, superblock
    from oracle import blocks as oblocks
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    from tests.gpu_util import oracle_ops_of_synthetic
    steps = 5
    jobs = [_job(T, problem, torch, 16, 128, 1, 111, prec), _job(T, problem, torch, 20, 200, 2, 112, prec)]
    ss = jobs[0][0]
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    phi0 = superblock.apply_op(sb, None, oblocks.BlockOp(ss.cdag_exc, True), ss.Q0, ss.psi_gs, ss.Q1)
    traj = krylov.time_steps(lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v), phi0, 0.05, steps, 4, 8)
    nL, nR = oblocks.BlockOp(ss.nL, False), oblocks.BlockOp(ss.nR, False)
    want = np.array([[superblock.expect(sb, nL, None, ss.Q1, tg[-1]), superblock.expect(sb, None, nR, ss.Q1, tg[-1])]
                     for tg, _, _ in traj])
    srv = T.tdmrg_server_create(0, 0, 2)
    try:
        res = _run(T, srv, jobs, steps, [0.0, 0.0], problem)
    finally:
        T.tdmrg_server_destroy(srv)
        for jb in jobs:
            T.tdmrg_destroy(jb[1])
    got = res[0][1].reshape(steps, 2)
    assert np.abs(got - want).max() < (1e-12 if prec == 0 else 1e-8)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_mix_equals_alone(prec):
    """Batching on (groups of up to 4): jobs queued together run as groups on the direct sum of their
    superblocks; every job's observables equal the job alone up to the order of the FP64 reductions
    (1e-12 on the FP64 path, 1e-10 on the tensor path, both far below the 1e-8 target)."""
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    specs = [(16, 128, 1, 101), (20, 200, 2, 102), (24, 300, 1, 103), (16, 160, 2, 104), (28, 256, 1, 105)]
    steps = 6
    jobs = [_job(T, problem, torch, *sp, prec) for sp in specs]
    try:
        alone = []
        for jb in jobs:
            srv = T.tdmrg_server_create(0, 0, 1)
            try:
                alone.append(_run(T, srv, [jb], steps, [0.0], problem)[0])
            finally:
                T.tdmrg_server_destroy(srv)
        srv = T.tdmrg_server_create(0, 0, 8)
        T.tdmrg_server_set_batching(srv, 4, 200000)   # the front waits up to 0.2 s for partners
        try:
            mixed = _run(T, srv, jobs, steps, [0.0] * len(jobs), problem)
            q, r, f, b = T.tdmrg_server_stats(srv)
            assert (q, r, f) == (0, 0, len(jobs))
            groups, grouped = T.tdmrg_server_batch_stats(srv)
            assert groups >= 1 and grouped >= 2
        finally:
            T.tdmrg_server_destroy(srv)
        tol = 1e-12 if prec == 0 else 1e-10
        for (sa, oa, ma), (sm, om, mm) in zip(alone, mixed):
            assert sa == sm == T.TDMRG_JOB_DONE
            assert np.abs(oa - om).max() < tol
            assert len(mm) == steps and (mm > 0).all()
    finally:
        for ss, ctx, psi, phi in jobs:
            T.tdmrg_destroy(ctx)
