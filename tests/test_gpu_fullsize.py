"""GPU parity at the full sizes of the paper-scale workloads, through the C ABI: the L=48 U=10 chain
twin with m=1000 (D = 292,472 in the excited sector, left sectors up to dL = 152, so the
eigendecomposition runs its global-memory Jacobi path) and the 2x16 ladder twin with m=800 and two
boundary bonds.  The oracle finishes one H psi at these sizes in a fraction of a second, so the checks
are element by element: H psi on both paths, one time step of the Krylov advance, rho_L of the
resulting targets and its eigendecomposition, and an observable.

Bounds: FP64 path 1e-12 (H psi) and 1e-10 (targets, the per-step bound for the FP64 path); tensor
path with S = 4 slices 140 2^{-28} = 5.2e-7 relative for H psi (10x the largest error measured over
the tensor-path tests, see test_gpu_ozaki) and 6e-7 relative for the targets of one step (10x the
measured 3.0e-8 on the chain and 5.7e-8 on the ladder)."""
import numpy as np
import pytest

from oracle import density, krylov, superblock
from oracle import blocks as oblocks
from tests.gpu_util import dev, host, new_ctx, oracle_ops_of_synthetic
from workloads import sectors as S

pytestmark = pytest.mark.gpu

# (L, m, U, bonds, tau): the L=48 m=1000 chain (tau = 0.02) and the 2x16 m=800 ladder (tau = 0.05)
CASES = [(48, 1000, 10.0, 1, 0.02), (32, 800, 8.0, 2, 0.05)]


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L,m,U,nb,tau", CASES)
def test_fullsize_hpsi(lib, L, m, U, nb, tau):
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(L, m, U, nbonds=nb, seed=S.SEED_BASE + 4)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    n = ss.sector_size(ss.Q1)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = superblock.apply_h(sb, HL, HR, conns, ss.Q1, x)
    for prec, bound in (("fp64", 1e-12), ("ozaki", 140.0 * 2.0 ** -28)):
        kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=4) if prec == "ozaki" else {}
        ctx = new_ctx(**kw)
        try:
            problem.load_synthetic(ctx, ss)
            assert lib.tdmrg_sector_size(ctx, ss.Q1) == n
            y = dev(np.full(n, np.nan + 0j))
            lib.tdmrg_apply_h(ctx, ss.Q1, dev(x), y)
            assert _rel(host(y), ref) < bound, prec
        finally:
            lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("L,m,U,nb,tau", CASES)
def test_fullsize_time_step(lib, L, m, U, nb, tau, mixed):
    """One time step as the bench runs it: Krylov advance with n_K = 10 and 4 targets, rho_L of the
    ground state and the targets, its eigendecomposition, and <n_L> on the last target."""
    from paper_1103_5391_gb300 import problem
    torch = pytest.importorskip("torch")
    ss = S.make_synthetic(L, m, U, nbonds=nb, seed=S.SEED_BASE + 4)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    nk, nv = 10, 4
    times = krylov.target_times(tau, nv)
    hf = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
    ref, n_used, err = krylov.evolve(hf, ss.phi, times, nk)
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=4) if mixed else {}
    ctx = new_ctx(**kw)
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        tg = [dev(np.zeros(n)) for _ in range(nv)]
        lib.tdmrg_evolve(ctx, ss.Q1, dev(ss.phi), times, nk, tg)
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == n_used
        bound = 6e-7 if mixed else 1e-10
        got = [host(t) for t in tg]
        for x in range(nv):
            assert _rel(got[x], ref[x]) < bound, x
        # rho_L of the device targets against the oracle's rho_L of the same vectors
        wgs, w = density.tst_weights(nv)
        sts = [(ss.Q0, ss.psi_gs)] + [(ss.Q1, g) for g in got]
        rho_ref = density.rho_left(sb, sts, [wgs] + w)
        nr, ne = lib.tdmrg_rho_size(ctx)
        rho = dev(np.zeros(nr))
        lib.tdmrg_density_matrix(ctx, [(ss.Q0, dev(ss.psi_gs))] + [(ss.Q1, t) for t in tg], [wgs] + w, rho)
        rho_h = host(rho)
        off = 0
        for qi, d in enumerate(ss.ldim):
            assert np.abs(rho_h[off: off + d * d].reshape(d, d) - rho_ref[qi]).max() < 1e-14
            off += d * d
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U_d = dev(np.zeros(nr))
        lib.tdmrg_rho_eig(ctx, rho, ev, U_d)
        ev, U_h = ev.cpu().numpy(), host(U_d)
        off = eo = 0
        for (lam, _), d, r in zip(density.rho_eig(rho_ref), ss.ldim, rho_ref):
            g_l = ev[eo: eo + d]
            g_U = U_h[off: off + d * d].reshape(d, d)
            assert np.abs(g_l - lam).max() < 1e-13
            assert np.abs(g_U @ np.diag(g_l) @ g_U.conj().T - r).max() < 1e-13
            assert np.abs(g_U.conj().T @ g_U - np.eye(d)).max() < 1e-11
            off += d * d
            eo += d
        # an observable of the last target
        nL = oblocks.BlockOp(ss.nL, False)
        want = superblock.expect(sb, nL, None, ss.Q1, got[-1])
        out = dev(np.zeros(1))
        lib.tdmrg_expect(ctx, problem.OP_N, -1, ss.Q1, tg[-1], out)
        assert abs(host(out)[0] - want) < 1e-12 * max(1.0, abs(want))
    finally:
        lib.tdmrg_destroy(ctx)
