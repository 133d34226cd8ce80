"""Batching of independent jobs (grouped products over many superblocks, Sec. IV): the direct sum of
several synthetic superblocks (chains and a ladder, different L, m and U) loaded into one context, and
independent Krylov advances side by side in its vector.

  - one H psi of the direct sum = the concatenation of every job's own H psi (FP64 path: bit-equal,
    the same sector-pair tasks; tensor path S = 4: the same slicing, within the slicing bound);
  - the segmented advance (each job its own Lanczos recursion, one product per step for all) against
    every job's tdmrg_evolve alone: FP64 1e-13 relative per target, tensor path 1e-9 (both runs on the
    tensor path differ only in reduction order); Krylov dimensions and error estimates per job;
  - a segment with a zero start vector (stopped before its first step) next to ones that run all steps."""
import numpy as np
import pytest

from tests.gpu_util import new_ctx, rel_err, torch_cuda
from workloads import sectors as S

pytestmark = pytest.mark.gpu
JOBS = [(16, 96, 4.0, 1, 101), (24, 128, 2.0, 1, 102), (12, 64, 8.0, 2, 103)]   # (L, m, U, bonds, seed)


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _jobs(lib, prec):
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    out = []
    for L, m, U, nb, seed in JOBS:
        ss = S.make_synthetic(L, m, U, nbonds=nb, seed=seed)
        ctx = new_ctx(prec=prec, ozaki_slices=4)
        problem.load_synthetic(ctx, ss)
        psi = torch.as_tensor(ss.psi_gs).cuda()
        phi = torch.zeros(lib.tdmrg_sector_size(ctx, ss.Q1), dtype=torch.complex128, device="cuda")
        lib.tdmrg_apply_op(ctx, -1, problem.OP_EXC, ss.Q0, psi, ss.Q1, phi)
        out.append((ss, ctx, phi))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("tensor", [False, True])
def test_direct_sum_hpsi_and_segmented_evolve(lib, tensor):
    torch = torch_cuda()
    prec = lib.TDMRG_OZAKI_BF16 if tensor else lib.TDMRG_FP64
    jobs = _jobs(lib, prec)
    big = new_ctx(prec=prec, ozaki_slices=4)
    try:
        Qsum, off = lib.tdmrg_direct_sum(big, [c for _, c, _ in jobs], [ss.Q1 for ss, _, _ in jobs])
        n = lib.tdmrg_sector_size(big, Qsum)
        assert n == off[-1] == sum(int(p.numel()) for _, _, p in jobs)
        phi = torch.cat([p for _, _, p in jobs])
        # one product over all jobs = each job's own product
        y = torch.zeros_like(phi)
        lib.tdmrg_apply_h(big, Qsum, phi, y)
        for k, (ss, ctx, p) in enumerate(jobs):
            yk = torch.zeros_like(p)
            lib.tdmrg_apply_h(ctx, ss.Q1, p, yk)
            got = y[off[k]: off[k + 1]]
            if tensor:
                assert rel_err(got.cpu().numpy(), yk.cpu().numpy()) < 140.0 * 2.0 ** -28
            else:
                assert torch.equal(got, yk)
        # the segmented advance against each job alone
        times = [0.0, 0.05 / 3, 0.1 / 3, 0.05]
        seg = [off[k + 1] - off[k] for k in range(len(jobs))]
        tg = [torch.zeros_like(phi) for _ in times]
        lib.tdmrg_evolve_segments(big, Qsum, phi, seg, times, 10, tg)
        nk_used, err = lib.tdmrg_evolve_segments_info(big, Qsum, 10, len(jobs))
        for k, (ss, ctx, p) in enumerate(jobs):
            alone = [torch.zeros_like(p) for _ in times]
            lib.tdmrg_evolve(ctx, ss.Q1, p, times, 10, alone)
            nu, e_alone, _, _ = lib.tdmrg_evolve_info(ctx)
            assert nk_used[k] == nu
            assert abs(err[k] - e_alone) <= 1e-6 * max(e_alone, 1e-30) + 1e-30
            for x in range(len(times)):
                d = rel_err(tg[x][off[k]: off[k + 1]].cpu().numpy(), alone[x].cpu().numpy())
                assert d < (1e-9 if tensor else 1e-13), (k, x, d)
    finally:
        lib.tdmrg_destroy(big)
        for _, c, _ in jobs:
            lib.tdmrg_destroy(c)


def test_inactive_segment(lib):
    """A segment whose start vector is zero stops before its first step (n_K used 0, targets zero) while
    the others run all 24 steps beside it; every segment equals its job alone."""
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    tiny = S.make_synthetic(6, 16, 4.0, nbonds=1, seed=7)
    ctx0 = new_ctx(nk_max=32)
    problem.load_synthetic(ctx0, tiny)
    p0 = torch.zeros(lib.tdmrg_sector_size(ctx0, tiny.Q1), dtype=torch.complex128, device="cuda")
    all_jobs = [(tiny, ctx0, p0)]
    for L, m, U, nb, seed in JOBS:
        ss = S.make_synthetic(L, m, U, nbonds=nb, seed=seed)
        ctx = new_ctx(nk_max=32)
        problem.load_synthetic(ctx, ss)
        psi = torch.as_tensor(ss.psi_gs).cuda()
        p = torch.zeros(lib.tdmrg_sector_size(ctx, ss.Q1), dtype=torch.complex128, device="cuda")
        lib.tdmrg_apply_op(ctx, -1, problem.OP_EXC, ss.Q0, psi, ss.Q1, p)
        all_jobs.append((ss, ctx, p))
    big = new_ctx(nk_max=32)
    try:
        Qsum, off = lib.tdmrg_direct_sum(big, [c for _, c, _ in all_jobs], [ss.Q1 for ss, _, _ in all_jobs])
        phi = torch.cat([p for _, _, p in all_jobs])
        times = [0.0, 0.2]
        tg = [torch.full_like(phi, 7.0) for _ in times]
        lib.tdmrg_evolve_segments(big, Qsum, phi, [off[k + 1] - off[k] for k in range(len(all_jobs))], times, 24, tg)
        nk_used, _ = lib.tdmrg_evolve_segments_info(big, Qsum, 24, len(all_jobs))
        assert nk_used[0] == 0 and all(v == 24 for v in nk_used[1:])
        for x in range(len(times)):
            assert not torch.any(tg[x][off[0]: off[1]])
        for k, (ss, ctx, p) in enumerate(all_jobs[1:], start=1):
            alone = [torch.zeros_like(p) for _ in times]
            lib.tdmrg_evolve(ctx, ss.Q1, p, times, 24, alone)
            for x in range(len(times)):
                assert rel_err(tg[x][off[k]: off[k + 1]].cpu().numpy(), alone[x].cpu().numpy()) < 1e-12
    finally:
        lib.tdmrg_destroy(big)
        for _, c, _ in all_jobs:
            lib.tdmrg_destroy(c)


def test_direct_sum_rho_and_eig(lib):
    """rho_L of the direct sum (ground states in the sum's sector Q0, targets in Q1, weights of Sec. II.C,
    every target normalised per job) = every job's own rho_L, packed in job order (1e-14); the
    eigendecomposition over all jobs' sectors in one call = each job's (eigenvalues 1e-13)."""
    torch = torch_cuda()
    jobs = _jobs(lib, lib.TDMRG_FP64)
    big = new_ctx()
    try:
        Qsum, off = lib.tdmrg_direct_sum(big, [c for _, c, _ in jobs], [ss.Q1 for ss, _, _ in jobs])
        Q0sum = (Qsum[0] - 1, Qsum[1])
        rng = np.random.default_rng(4)
        psis, tgts = [], []
        for ss, ctx, p in jobs:
            psis.append(torch.as_tensor(ss.psi_gs).cuda())
            tgts.append([p] + [p * complex(rng.standard_normal(), rng.standard_normal()) +
                               torch.roll(p, x + 1) for x in range(3)])
        wgs, w = lib.tdmrg_tst_weights(4)
        big_states = [(Q0sum, torch.cat(psis))] + [(Qsum, torch.cat([t[x] for t in tgts])) for x in range(4)]
        assert lib.tdmrg_sector_size(big, Q0sum) == sum(int(q.numel()) for q in psis)
        nr, ne = lib.tdmrg_rho_size(big)
        rho = torch.zeros(nr, dtype=torch.complex128, device="cuda")
        lib.tdmrg_density_matrix(big, big_states, [wgs] + w, rho)
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U = torch.zeros_like(rho)
        lib.tdmrg_rho_eig(big, rho, ev, U)
        ro = eo = 0
        for (ss, ctx, p), q, t in zip(jobs, psis, tgts):
            nrk, nek = lib.tdmrg_rho_size(ctx)
            rk = torch.zeros(nrk, dtype=torch.complex128, device="cuda")
            lib.tdmrg_density_matrix(ctx, [(ss.Q0, q)] + [(ss.Q1, x) for x in t], [wgs] + w, rk)
            assert float((rho[ro: ro + nrk] - rk).abs().max()) < 1e-14
            evk = torch.zeros(nek, dtype=torch.float64, device="cuda")
            lib.tdmrg_rho_eig(ctx, rk, evk, torch.zeros_like(rk))
            assert float((ev[eo: eo + nek] - evk).abs().max()) < 1e-13
            ro += nrk
            eo += nek
        assert ro == nr and eo == ne
    finally:
        lib.tdmrg_destroy(big)
        for _, c, _ in jobs:
            lib.tdmrg_destroy(c)
