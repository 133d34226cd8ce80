"""GPU parity on a physical truncated superblock: the central cut of the oracle's two-site DMRG of the
L=10 Hubbard chain (U=4, half filling, m=32; the oracle DMRG is pinned against ED in
test_oracle_dmrg), loaded through the C ABI.

  - H psi and a 10-step Krylov trajectory of phi = c^dag_{5 up} psi (the right block's edge site, with
    the left parity) against the oracle on the same blocks: FP64 path 1e-12 (H psi) and observables
    1e-12; tensor path (4 slices) the slicing bound for H psi and 1e-8 for the observables;
  - truncation (Sec. I): rho_L of the ground state, its eigendecomposition and tdmrg_truncate against
    the oracle's kept set for every m from 1 to the block size (the spin-flip symmetric sectors have
    equal spectra, so many cuts fall inside tied pairs), and the discarded weight to 1e-12;
  - renormalisation U^dag O U of H_L and c^dag_L with the device's eigenvectors against the same
    products in the oracle (1e-12), and the spectrum of the renormalised H_L per sector against the
    oracle's own truncation (equal kept subspaces where no tied cluster is cut)."""
import numpy as np
import pytest

from oracle import density, dmrg, krylov, superblock
from tests.gpu_util import DmrgLoader, dev, host, new_ctx, rel_err, torch_cuda

pytestmark = pytest.mark.gpu
L, U, T_HOP, M = 10, 4.0, 1.0, 32


@pytest.fixture(scope="module")
def chain():
    return dmrg.ChainDMRG(L, T_HOP, U, M).run(sweeps=1)


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


@pytest.mark.parametrize("slices", [0, 4])
def test_dmrg_superblock_hpsi_and_trajectory(lib, chain, slices):
    Lenl, Renl, sb, HL, HR, conns, e, psi = chain
    Q0, Q1 = (L // 2, L // 2), (L // 2 + 1, L // 2)
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=slices) if slices else {}
    ctx = new_ctx(**kw)
    try:
        ld = DmrgLoader(ctx, Lenl, Renl, T_HOP)
        n0 = lib.tdmrg_sector_size(ctx, Q0)
        assert n0 == sb.size(Q0)
        y = dev(np.zeros(n0))
        lib.tdmrg_apply_h(ctx, Q0, dev(psi), y)
        ref = superblock.apply_h(sb, HL, HR, conns, Q0, psi)
        assert rel_err(host(y), ref) < (1e-12 if not slices else 140.0 * 2.0 ** -28)
        # the ground state is an eigenvector: H psi = E psi
        assert np.abs(ref - e * psi).max() < 1e-8
        n1 = lib.tdmrg_sector_size(ctx, Q1)
        phi = dev(np.zeros(n1))
        lib.tdmrg_apply_op(ctx, -1, 10, Q0, dev(psi), Q1, phi)            # c^dag_{5 up} psi (Eq. b)
        cd = Renl.blockop(Renl.cdag[0], True)
        phi_ref = superblock.apply_op(sb, None, cd, Q0, psi, Q1)
        assert rel_err(host(phi), phi_ref) < 1e-14
        times = krylov.target_times(0.1, 4)
        tg = [dev(np.zeros(n1)) for _ in range(3)] + [phi]
        traj = krylov.time_steps(lambda v: superblock.apply_h(sb, HL, HR, conns, Q1, v), phi_ref, 0.1, 10, 4, 10)
        nR = Renl.blockop(Renl.cdag[0] @ Renl.cdag[0].conj().T, False)
        nL = Lenl.blockop(Lenl.cdag[0] @ Lenl.cdag[0].conj().T, False)
        out = dev(np.zeros(2))
        worst = 0.0
        for s in range(10):
            lib.tdmrg_evolve(ctx, Q1, phi, times, 10, tg)
            lib.tdmrg_expect(ctx, -1, 50, Q1, phi, out[0:1])
            lib.tdmrg_expect(ctx, 50, -1, Q1, phi, out[1:2])
            o = host(out)
            want = (superblock.expect(sb, None, nR, Q1, traj[s][0][-1]), superblock.expect(sb, nL, None, Q1, traj[s][0][-1]))
            worst = max(worst, abs(o[0] - want[0]), abs(o[1] - want[1]))
        lib.tdmrg_evolve_info(ctx)
        assert worst < (1e-12 if not slices else 1e-8), worst
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.fixture(scope="module")
def device_rho(lib, chain):
    """rho_L of the DMRG ground state, its device eigendecomposition, and the oracle's."""
    torch = torch_cuda()
    Lenl, Renl, sb, HL, HR, conns, e, psi = chain
    Q0 = (L // 2, L // 2)
    ctx = new_ctx()
    ld = DmrgLoader(ctx, Lenl, Renl, T_HOP)
    nr, ne = lib.tdmrg_rho_size(ctx)
    rho = dev(np.zeros(nr))
    lib.tdmrg_density_matrix(ctx, [(Q0, dev(psi))], [1.0], rho)
    ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
    Ud = dev(np.zeros(nr))
    lib.tdmrg_rho_eig(ctx, rho, ev, Ud)
    rho_ref = density.rho_left(sb, [(Q0, psi)], [1.0])
    yield ctx, ld, ev, Ud, rho_ref
    lib.tdmrg_destroy(ctx)


def test_truncation_matches_oracle(lib, chain, device_rho):
    torch = torch_cuda()
    ctx, ld, ev, Ud, rho_ref = device_rho
    Lenl = chain[0]
    secs, dims, _ = Lenl.sectors()
    lam_ref = [lam for lam, _ in density.rho_eig(rho_ref)]
    kept = torch.zeros(len(dims), dtype=torch.int32, device="cuda")
    disc = torch.zeros(1, dtype=torch.float64, device="cuda")
    ties = 0
    for m in range(1, sum(dims) + 2):
        lib.tdmrg_truncate(ctx, ev, m, kept, disc)
        want = dmrg.kept_counts(lam_ref, m)
        got = kept.cpu().numpy().tolist()
        assert got == want, m
        w_ref = sum(float(np.sum(l[k:])) for l, k in zip(lam_ref, want))
        assert abs(disc.item() - w_ref) < 1e-12
        srt = sorted(np.concatenate(lam_ref), reverse=True)
        if m < len(srt) and abs(srt[m - 1] - srt[m]) <= 1e-12 * srt[0]:
            ties += 1
    assert ties > 0                                   # cuts inside tied clusters were exercised


def test_renormalization_matches_oracle(lib, chain, device_rho):
    torch = torch_cuda()
    ctx, ld, ev, Ud, rho_ref = device_rho
    Lenl = chain[0]
    secs, dims, starts = Lenl.sectors()
    lam_ref = [lam for lam, _ in density.rho_eig(rho_ref)]
    kept = dmrg.kept_counts(lam_ref, M)
    U_h = host(Ud)
    Us, off = [], 0
    for d in dims:
        Us.append(U_h[off: off + d * d].reshape(d, d))
        off += d * d
    for op_id, dense, odd in ((0, Lenl.H, False), (10, Lenl.cdag[0], True), (11, Lenl.cdag[1], True)):
        bo = Lenl.blockop(dense, odd)
        want = []
        for (qo, qi), blk in bo.blocks.items():
            if kept[qo] and kept[qi]:
                want.append(Us[qo][:, :kept[qo]].conj().T @ blk @ Us[qi][:, :kept[qi]])
        n = sum(w.size for w in want)
        out = dev(np.full(max(n, 1), np.nan + 0j))
        nb = lib.tdmrg_renormalize_op(ctx, 0, op_id, Ud, kept, out)
        assert nb == len(want)
        got = host(out)[:n]
        ref = np.concatenate([w.ravel() for w in want])
        assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max()), op_id
    # spectrum of the renormalised H_L per sector against the oracle's own truncation
    blk_new, counts, lam, disc, _ = dmrg.truncate(Lenl, rho_ref, M)
    assert counts == kept
    hb = Lenl.blockop(Lenl.H, False)
    want = [np.linalg.eigvalsh(Us[q][:, :k].conj().T @ hb.blocks[(q, q)] @ Us[q][:, :k]) for q, k in enumerate(kept) if k]
    new_secs, new_dims, new_starts = blk_new.sectors()
    mine = [np.linalg.eigvalsh(blk_new.H[s0: s0 + d, s0: s0 + d]) for s0, d in zip(new_starts, new_dims)]
    for a, b in zip(want, mine):
        assert np.abs(a - b).max() < 1e-10


@pytest.fixture(scope="module")
def run_object():
    d = dmrg.ChainDMRG(L, T_HOP, U, M)
    return d, d.run(sweeps=1)


def _eig_layout_of_V(V, Rn, Rb):
    """Rb's states (columns of V over Rn, grouped by Rb's sectors) in the layout of tdmrg_rho_eig: per
    sector of Rn a dim x dim matrix whose first columns are Rb's states; with the counts per sector."""
    rn_secs, rn_dims, rn_starts = Rn.sectors()
    rb_secs, rb_dims, rb_starts = Rb.sectors()
    parts, kept = [], []
    for q, dq, s0 in zip(rn_secs, rn_dims, rn_starts):
        M_ = np.zeros((dq, dq), complex)
        k = 0
        if q in rb_secs:
            j = rb_secs.index(q)
            k = rb_dims[j]
            M_[:, :k] = V[s0: s0 + dq, rb_starts[j]: rb_starts[j] + k]
        parts.append(M_.ravel())
        kept.append(k)
    return np.concatenate(parts), kept


def test_wft_right_matches_oracle(lib, run_object):
    """The ground state at the centre of the L=10 m=32 chain moved one site to the right (truncation to
    m = 32 on the left, the right block expanded in the next right enlarged block) against the oracle's
    wave-function transformation: 1e-13; its squared norm is 1 minus the discarded weight."""
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = run_object
    Q = (L // 2, L // 2)
    r = L // 2 - 1
    rho = density.rho_left(sb, [(Q, psi)], [1.0])
    Lb, counts, lam, disc, Uf = dmrg.truncate(Lenl, rho, M)
    Ln = dmrg.enlarge(Lb, "L", T_HOP, U)
    Rn = dmrg.enlarge(d.right[r - 1], "R", T_HOP, U)
    want = dmrg.wft_right(Lenl, Renl, Q, psi, Uf, d.right[r], d.right_U[r], Ln, Rn)
    # the same U in the device layout: per left sector its eigenvector matrix (kept columns first)
    Us = np.concatenate([Uq.ravel() for _, Uq in density.rho_eig(rho)])
    ca, cb = new_ctx(), new_ctx()
    try:
        DmrgLoader(ca, Lenl, Renl, T_HOP)
        DmrgLoader(cb, Ln, Rn, T_HOP)
        n2 = lib.tdmrg_sector_size(cb, Q)
        assert n2 == len(want)
        out = dev(np.full(n2, np.nan + 0j))
        Vh, kept_next = _eig_layout_of_V(d.right_U[r], Rn, d.right[r])
        lib.tdmrg_wft_right(ca, Q, dev(psi), dev(Us), counts, dev(Vh), kept_next, cb, out)
        assert np.abs(host(out) - want).max() < 1e-13
        # the projection keeps exactly the kept weight and the right expansion is an isometry
        assert abs(np.linalg.norm(host(out)) ** 2 - (1.0 - disc)) < 1e-12
    finally:
        lib.tdmrg_destroy(ca)
        lib.tdmrg_destroy(cb)


def test_wft_left_matches_oracle(lib, run_object):
    """The centre ground state moved one site to the left (rho_R truncation to m = 32 on the right, the
    left block expanded in the next left enlarged block) against the oracle's transformation: 1e-13;
    squared norm 1 - discarded weight."""
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = run_object
    Q = (L // 2, L // 2)
    l = L // 2 - 1
    rho = density.rho_right(sb, [(Q, psi)], [1.0])
    K, counts, lam, disc, Uf = dmrg.truncate(Renl, rho, M)
    Ln = dmrg.enlarge(d.left[l - 1], "L", T_HOP, U)
    Rn = dmrg.enlarge(K, "R", T_HOP, U)
    want = dmrg.wft_left(Lenl, Renl, Q, psi, Uf, d.left[l], d.left_U[l], Ln, Rn)
    Us = np.concatenate([Uq.ravel() for _, Uq in density.rho_eig(rho)])
    Vh, kept_next = _eig_layout_of_V(d.left_U[l], Ln, d.left[l])
    ca, cb = new_ctx(), new_ctx()
    try:
        DmrgLoader(ca, Lenl, Renl, T_HOP)
        DmrgLoader(cb, Ln, Rn, T_HOP)
        n2 = lib.tdmrg_sector_size(cb, Q)
        assert n2 == len(want)
        out = dev(np.full(n2, np.nan + 0j))
        lib.tdmrg_wft_left(ca, Q, dev(psi), dev(Us), counts, dev(Vh), kept_next, cb, out)
        assert np.abs(host(out) - want).max() < 1e-13
        assert abs(np.linalg.norm(host(out)) ** 2 - (1.0 - disc)) < 1e-12
    finally:
        lib.tdmrg_destroy(ca)
        lib.tdmrg_destroy(cb)


def test_rho_right_matches_oracle(lib, run_object):
    """rho_R of the ground state and three random targets in another sector (weights of time-step
    targeting) against the oracle's, 1e-14; its device eigenvalues against numpy's, 1e-14."""
    d, (Lenl, Renl, sb, HL, HR, conns, e, psi) = run_object
    Q0, Q1 = (L // 2, L // 2), (L // 2 + 1, L // 2)
    rng = np.random.default_rng(9)
    n1 = sb.size(Q1)
    xs = [rng.standard_normal(n1) + 1j * rng.standard_normal(n1) for _ in range(3)]
    w = [0.25, 0.25, 0.25, 0.25]
    want = density.rho_right(sb, [(Q0, psi)] + [(Q1, x) for x in xs], w)
    ctx = new_ctx()
    try:
        DmrgLoader(ctx, Lenl, Renl, T_HOP)
        nr, ne = lib.tdmrg_rho_size(ctx, 1)
        rho = dev(np.zeros(nr))
        lib.tdmrg_density_matrix(ctx, [(Q0, dev(psi))] + [(Q1, dev(x)) for x in xs], w, rho, side=1)
        got = host(rho)
        assert np.abs(got - np.concatenate([r.ravel() for r in want])).max() < 1e-14
        torch = torch_cuda()
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U = dev(np.zeros(nr))
        lib.tdmrg_rho_eig(ctx, rho, ev, U, side=1)
        ref = np.concatenate([lam for lam, _ in density.rho_eig(want)])
        assert np.abs(ev.cpu().numpy() - ref).max() < 1e-14
    finally:
        lib.tdmrg_destroy(ctx)
