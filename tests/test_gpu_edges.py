"""Edge cases of the hot path at the limits of the C ABI: the largest Krylov dimension (n_K = 32, the
full warp of the tridiagonal exponential) with the most targets (n_v = 16), a zero state (Lanczos
breakdown before the first vector), the largest eigendecomposition sector (dL = 512, the global-memory
Jacobi path) and the rejection of a larger one."""
import numpy as np
import pytest

from oracle import density, krylov, superblock
from tests.gpu_util import dev, host, new_ctx, oracle_ops_of_synthetic
from workloads import sectors as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("mixed", [False, True])
def test_max_krylov_dim_and_targets(lib, mixed):
    """n_K = 32 and 16 targets (unequally spaced) on a ragged ladder twin against the oracle."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 150, 4.0, nbonds=2, seed=S.SEED_BASE + 6)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    nk, nv = 32, 16
    times = list(np.linspace(0.0, 0.3, nv) ** 1.5)
    hf = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
    ref, n_used, err = krylov.evolve(hf, ss.phi, times, nk)
    assert n_used == nk
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=5) if mixed else {}
    ctx = new_ctx(nk_max=32, **kw)
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        tg = [dev(np.zeros(n)) for _ in range(nv)]
        lib.tdmrg_evolve(ctx, ss.Q1, dev(ss.phi), times, nk, tg)
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == nk
        for x in range(nv):
            assert _rel(host(tg[x]), ref[x]) < (1e-8 if mixed else 1e-10), x
        # rho_L of the ground state and the first 11 targets: the 12 states rho_L takes at most
        # (weights of Sec. II.C for n_v = 11)
        nrho = 11
        wgs, w = density.tst_weights(nrho)
        got = [host(t) for t in tg[:nrho]]
        rho_ref = density.rho_left(sb, [(ss.Q0, ss.psi_gs)] + [(ss.Q1, g) for g in got], [wgs] + w)
        nr, ne = lib.tdmrg_rho_size(ctx)
        rho = dev(np.zeros(nr))
        lib.tdmrg_density_matrix(ctx, [(ss.Q0, dev(ss.psi_gs))] + [(ss.Q1, t) for t in tg[:nrho]], [wgs] + w, rho)
        with pytest.raises(lib.TdmrgError):   # 13 states
            lib.tdmrg_density_matrix(ctx, [(ss.Q0, dev(ss.psi_gs))] + [(ss.Q1, t) for t in tg[:12]],
                                     [1.0 / 13] * 13, rho)
        rho_h = host(rho)
        off = 0
        for qi, d in enumerate(ss.ldim):
            assert np.abs(rho_h[off: off + d * d].reshape(d, d) - rho_ref[qi]).max() < 1e-14
            off += d * d
    finally:
        lib.tdmrg_destroy(ctx)


def test_zero_state(lib):
    """phi = 0: the Krylov space is empty, every target is exactly zero and n_used = 0."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(12, 60, 4.0, nbonds=1, seed=S.SEED_BASE + 7)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        tg = [dev(np.full(n, np.nan + 0j)) for _ in range(3)]
        lib.tdmrg_evolve(ctx, ss.Q1, dev(np.zeros(n)), [0.0, 0.1, 0.2], 10, tg)
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == 0 and err_gpu == 0.0
        for t in tg:
            assert np.array_equal(host(t), np.zeros(n, dtype=np.complex128))
    finally:
        lib.tdmrg_destroy(ctx)


def test_max_eig_sector(lib):
    """Left sectors up to dL = 512 (the eigensolver's limit): rho blocks U diag(lambda) U^dag with
    lambda_k = 0.99^k, decomposed to FP64 accuracy."""
    from paper_1103_5391_gb300 import problem
    torch = pytest.importorskip("torch")
    ss = S.make_synthetic(32, 3370, 4.0, nbonds=1, seed=S.SEED_BASE + 5)
    assert max(ss.ldim) == 512
    rng = np.random.default_rng(13)
    lams = [0.99 ** np.arange(d) for d in ss.ldim]
    tr = sum(l.sum() for l in lams)
    blocks = []
    for d, lam in zip(ss.ldim, lams):
        lam /= tr
        q, _ = np.linalg.qr(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
        blocks.append((q * lam) @ q.conj().T)
    scale = max(l.max() for l in lams)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        nr, ne = lib.tdmrg_rho_size(ctx)
        rho = dev(np.concatenate([b.ravel() for b in blocks]))
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U = dev(np.zeros(nr))
        lib.tdmrg_rho_eig(ctx, rho, ev, U)
        ev, U = ev.cpu().numpy(), host(U)
        off = eo = 0
        for d, lam, r in zip(ss.ldim, lams, blocks):
            g_l = ev[eo: eo + d]
            g_U = U[off: off + d * d].reshape(d, d)
            assert np.all(np.diff(g_l) <= 0)
            assert np.abs(g_l - lam).max() < 1e-12 * scale, d
            assert np.abs(g_U @ np.diag(g_l) @ g_U.conj().T - r).max() < 1e-12 * scale, d
            assert np.abs(g_U.conj().T @ g_U - np.eye(d)).max() < 1e-10, d
            off += d * d
            eo += d
    finally:
        lib.tdmrg_destroy(ctx)


def test_eig_sector_above_limit_rejected(lib):
    from paper_1103_5391_gb300 import problem
    torch = pytest.importorskip("torch")
    ss = S.make_synthetic(32, 3400, 4.0, nbonds=1, seed=S.SEED_BASE + 5)
    assert max(ss.ldim) > 512
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        nr, ne = lib.tdmrg_rho_size(ctx)
        rho = dev(np.zeros(nr))
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        with pytest.raises(lib.TdmrgError):
            lib.tdmrg_rho_eig(ctx, rho, ev, dev(np.zeros(nr)))
    finally:
        lib.tdmrg_destroy(ctx)
