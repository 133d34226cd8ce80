"""GPU parity of the weighted reduced density matrix (Eq. rdensitymatrix, weights of Sec. II.C) and
of its FP64 Jacobi eigendecomposition against the oracle."""
import numpy as np
import pytest

from oracle import density, superblock
from tests.gpu_util import dev, host, new_ctx
from workloads import sectors as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _states(ss, nv, seed):
    rng = np.random.default_rng(seed)
    sts = [(ss.Q0, ss.psi_gs)]
    for x in range(nv):
        n = ss.sector_size(ss.Q1)
        sts.append((ss.Q1, (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * (x + 1)))
    return sts


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("L,m,nb", [(8, 24, 1), (32, 400, 1), (32, 800, 2)])
def test_rho_and_eig(lib, L, m, nb, mixed):
    """rho_L (an FP64 HERK in either precision of the context) within 1e-14 of the oracle's, and its
    eigendecomposition to FP64 accuracy."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(L, m, 4.0, nbonds=nb, seed=S.SEED_BASE + 7)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    wgs, w = density.tst_weights(4)
    sts = _states(ss, 4, 1)
    weights = [wgs] + w
    ref = density.rho_left(sb, sts, weights)
    ctx = new_ctx(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=4) if mixed else new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        nr, ne = lib.tdmrg_rho_size(ctx)
        assert nr == sum(d * d for d in ss.ldim) and ne == sum(ss.ldim)
        rho = dev(np.full(nr, np.nan + 0j))
        dsts = [(Q, dev(v)) for Q, v in sts]
        lib.tdmrg_density_matrix(ctx, dsts, weights, rho)
        got = host(rho)
        off = 0
        tr = 0.0
        for qi, d in enumerate(ss.ldim):
            blk = got[off: off + d * d].reshape(d, d)
            assert np.abs(blk - ref[qi]).max() < 1e-14
            tr += np.trace(blk).real
            off += d * d
        assert abs(tr - 1.0) < 1e-13
        torch = pytest.importorskip("torch")
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U = dev(np.zeros(nr))
        lib.tdmrg_rho_eig(ctx, rho, ev, U)
        ev, U = ev.cpu().numpy(), host(U)
        off = eo = 0
        for (lam, V), d, r in zip(density.rho_eig(ref), ss.ldim, ref):
            g_l = ev[eo: eo + d]
            g_U = U[off: off + d * d].reshape(d, d)
            assert np.abs(g_l - lam).max() < 1e-13
            assert np.abs(g_U @ np.diag(g_l) @ g_U.conj().T - r).max() < 1e-13
            assert np.abs(g_U.conj().T @ g_U - np.eye(d)).max() < 1e-12
            off += d * d
            eo += d
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("kind,orth_tol", [("mixed", 1e-11), ("graded", 1e-10)])
def test_rho_eig_hard_spectra(lib, kind, orth_tol):
    """rho blocks U diag(lambda) U^dag with prescribed spectra on the L=32 m=400 sector layout:
    'mixed' has exactly degenerate pairs, pairs 1e-4 apart and a rank-deficient tail of zeros (lambda_k
    = 0.9^k otherwise); 'graded' decays as 0.8^k, so that the smallest eigenvalues and their gaps lie
    below FP32's resolution of rho and are found by the re-seed in the refined basis.  Eigenvalues and
    U diag(lambda) U^dag to 1e-12 of the largest eigenvalue, U^dag U to orth_tol."""
    from paper_1103_5391_gb300 import problem
    torch = pytest.importorskip("torch")
    ss = S.make_synthetic(32, 400, 4.0, nbonds=1, seed=S.SEED_BASE + 9)
    rng = np.random.default_rng(12)
    blocks, lams = [], []
    for d in ss.ldim:
        lam = (0.9 if kind == "mixed" else 0.8) ** np.arange(d)
        if kind == "mixed":
            lam[1::4] = lam[0::4][: len(lam[1::4])]                   # exact pairs
            lam[3::4] = lam[2::4][: len(lam[3::4])] * (1 - 1e-4)      # pairs 1e-4 apart
            lam[(d + 1) // 2:] = 0.0                                  # rank deficient
        lams.append(np.sort(lam)[::-1])
    tr = sum(l.sum() for l in lams)
    for d, lam in zip(ss.ldim, lams):
        lam /= tr                                                     # trace 1 over all sectors
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
            assert np.abs(g_U.conj().T @ g_U - np.eye(d)).max() < orth_tol, d
            off += d * d
            eo += d
    finally:
        lib.tdmrg_destroy(ctx)


def test_expect(lib):
    from paper_1103_5391_gb300 import problem
    from oracle import blocks as oblocks
    ss = S.make_synthetic(16, 100, 4.0, nbonds=1, seed=31)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        out = dev(np.zeros(1))
        for a, b, A, B in ((problem.OP_N, -1, oblocks.BlockOp(ss.nL, False), None),
                           (-1, problem.OP_N, None, oblocks.BlockOp(ss.nR, False)),
                           (problem.OP_N, problem.OP_N, oblocks.BlockOp(ss.nL, False), oblocks.BlockOp(ss.nR, False))):
            lib.tdmrg_expect(ctx, a, b, ss.Q0, dev(ss.psi_gs * 3.0), out)
            want = superblock.expect(sb, A, B, ss.Q0, ss.psi_gs)
            assert abs(host(out)[0] - want) < 1e-14
    finally:
        lib.tdmrg_destroy(ctx)


def test_overlap_op(lib):
    """<phi1| A (x) B |phi2> between different states and sectors (the two-state form of
    Eq. generalcorrelation): a left creation operator, the right excitation operator and a hopping
    across the cut, against the oracle's operator application and inner product."""
    from paper_1103_5391_gb300 import problem
    from oracle import blocks as oblocks
    ss = S.make_synthetic(16, 120, 4.0, nbonds=1, seed=37)
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    assert tuple(ss.Q1) == (ss.Q0[0] + 1, ss.Q0[1])   # the excited sector has one more up electron
    rng = np.random.default_rng(9)
    n0, n1 = ss.sector_size(ss.Q0), ss.sector_size(ss.Q1)
    phi_q1 = rng.standard_normal(n1) + 1j * rng.standard_normal(n1)
    phi_q0 = rng.standard_normal(n0) + 1j * rng.standard_normal(n0)
    cdagL = oblocks.BlockOp(ss.cdagL[0][0], True)
    cR = oblocks.BlockOp(ss.cR[0][0], True)
    exc = oblocks.BlockOp(ss.cdag_exc, True)
    cases = [  # (opL, opR, oracle A, oracle B, Q of phi1, phi1)
        (problem.OP_CDAG, -1, cdagL, None, ss.Q1, phi_q1),
        (-1, problem.OP_EXC, None, exc, ss.Q1, phi_q1),
        (problem.OP_CDAG, problem.OP_CDAG, cdagL, cR, ss.Q0, phi_q0),   # c^dag_L c_R: hop across the cut
    ]
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        out = dev(np.zeros(1))
        for opL, opR, A, B, Qo, phi1 in cases:
            lib.tdmrg_overlap_op(ctx, opL, opR, Qo, dev(phi1), ss.Q0, dev(ss.psi_gs), out)
            want = np.vdot(phi1, superblock.apply_op(sb, A, B, ss.Q0, ss.psi_gs, Qo))
            assert abs(host(out)[0] - want) < 1e-12 * np.linalg.norm(phi1), (opL, opR)
        with pytest.raises(lib.TdmrgError):   # phi1 sector does not match where the operator leads
            lib.tdmrg_overlap_op(ctx, 123, -1, ss.Q1, dev(phi_q1), ss.Q0, dev(ss.psi_gs), out)
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("L,m,side", [(8, 24, 0), (32, 400, 0), (32, 400, 1), (48, 1000, 0)])
def test_density_eig_equals_the_two_calls(lib, L, m, side):
    """tdmrg_density_eig (rho of the first eigensolver group formed on that group's stream) = the two calls:
    rho, eigenvalues and eigenvectors bit-equal, on layouts with one group (L=8) and two (L=32, 48)."""
    torch = pytest.importorskip("torch")
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(L, m, 4.0, nbonds=1, seed=S.SEED_BASE + 21)
    sts = [(Q, dev(v)) for Q, v in _states(ss, 4, 5)]
    wgs, w = lib.tdmrg_tst_weights(4)
    out = []
    for fused in (False, True):
        ctx = new_ctx()
        try:
            problem.load_synthetic(ctx, ss)
            nr, ne = lib.tdmrg_rho_size(ctx, side=side)
            rho = torch.zeros(nr, dtype=torch.complex128, device="cuda")
            ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
            U = torch.zeros_like(rho)
            for _ in range(2):   # the second call reuses the compiled plans and workspaces
                if fused:
                    lib.tdmrg_density_eig(ctx, sts, [wgs] + w, rho, ev, U, side=side)
                else:
                    lib.tdmrg_density_matrix(ctx, sts, [wgs] + w, rho, side=side)
                    lib.tdmrg_rho_eig(ctx, rho, ev, U, side=side)
            torch.cuda.synchronize()
            out.append((rho.clone(), ev.clone(), U.clone()))
        finally:
            lib.tdmrg_destroy(ctx)
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)
