"""The benchmark's own time step (bench.Runner: Krylov advance with 4 time targets, weighted rho_L of the
ground state and the targets, its eigendecomposition, two observables on a second stream) on the
L=32 m=400 chain workload, 20 time steps from the c^dag excitation, against the oracle's 20-step
trajectory (Sec. II.A Eq. lanczosevolution, Sec. II.C Eq. lanczosevolution2, Eq. rdensitymatrix).

Checked every step: both observables; at the last step: every target and the rho_L spectrum.
Bounds:
  - FP64 path: observables 1e-12, targets 1e-10 relative (the per-step bound of the FP64 path, here
    over 20 steps; measured 1.7e-14), eigenvalues 1e-12;
  - tensor path, 4 slices (the bench's setting): observables 1e-8 (the accuracy target; measured
    3.5e-10), last target 1.1e-6 relative (10x the measured 1.09e-7), eigenvalues by Weyl's
    inequality: |d lambda| <= ||d rho||_2 <= sum_l w_l 2 ||d psi_l|| / ||psi_l|| for the normalised
    targets, evaluated with the measured target differences."""
import numpy as np
import pytest

from oracle import density, krylov, superblock
from oracle import blocks as oblocks
from tests.gpu_util import dev, host, new_ctx, oracle_ops_of_synthetic, torch_cuda

pytestmark = pytest.mark.gpu
STEPS = 20


@pytest.fixture(scope="module")
def oracle_trajectory():
    import bench
    wl = bench.CONFIGS["C2"]
    ss = bench.workload(wl)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    exc = oblocks.BlockOp(ss.cdag_exc, True)
    nL, nR = oblocks.BlockOp(ss.nL, False), oblocks.BlockOp(ss.nR, False)
    phi = superblock.apply_op(sb, None, exc, ss.Q0, ss.psi_gs, ss.Q1)
    hf = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
    traj = krylov.time_steps(hf, phi, wl["tau"], STEPS, wl["n_v"], wl["nk"])
    obs = np.array([[superblock.expect(sb, nL, None, ss.Q1, tg[-1]), superblock.expect(sb, None, nR, ss.Q1, tg[-1])]
                    for tg, _, _ in traj])
    wgs, w = density.tst_weights(wl["n_v"])
    last = traj[-1][0]
    rho = density.rho_left(sb, [(ss.Q0, ss.psi_gs)] + [(ss.Q1, t) for t in last], [wgs] + w)
    lam = np.concatenate([e for e, _ in density.rho_eig(rho)])
    return ss, obs, last, lam, w


@pytest.mark.parametrize("slices", [0, 4])
def test_bench_step_trajectory_against_oracle(oracle_trajectory, slices):
    torch = torch_cuda()
    import bench
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    ss, obs_ref, last_ref, lam_ref, w = oracle_trajectory
    kw = dict(prec=T.TDMRG_OZAKI_BF16, ozaki_slices=slices) if slices else {}
    ctx = new_ctx(**kw)
    stream = torch.cuda.current_stream()
    try:
        problem.load_synthetic(ctx, ss)
        run = bench.Runner(T, problem, ctx, ss, torch.device("cuda", torch.cuda.current_device()), stream,
                           bench.CONFIGS["C2"])
        obs = []
        for _ in range(STEPS):
            run.step()
            obs.append(host(run.obs).copy())
        torch.cuda.synchronize()
        T.tdmrg_evolve_info(ctx)          # raises if a bounded device wait ran out
        obs = np.array(obs)
        got = [host(t) for t in run.targets]
        d_rel = [np.linalg.norm(g - r) / np.linalg.norm(r) for g, r in zip(got, last_ref)]
        max_rel = [np.abs(g - r).max() / np.abs(r).max() for g, r in zip(got, last_ref)]
        lam = run.evals.cpu().numpy()
        d_lam = np.abs(lam - lam_ref).max()
        if slices == 0:
            assert np.abs(obs - obs_ref).max() < 1e-12
            assert max(max_rel) < 1e-10
            assert d_lam < 1e-12
        else:
            assert np.abs(obs - obs_ref).max() < 1e-8
            assert max_rel[-1] < 1.1e-6
            weyl = sum(wx * 2.0 * e for wx, e in zip(w, d_rel))
            assert d_lam <= weyl + 1e-13, (d_lam, weyl)
    finally:
        T.tdmrg_destroy(ctx)
