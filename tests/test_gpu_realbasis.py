"""Real-basis variant (row f2): real operators are detected and their imaginary products skipped.

  - exact L=8 chain (every block operator real): H psi against the oracle on both paths; the FP64
    plan's flops are half those of the same operators stored with a 1e-300 imaginary part (complex),
    and the tensor path's executed flops drop (stage-2 tasks use the real half of K);
  - the c^dag trajectory on the FP64 real path against ED (n_i(t) <= 1e-8);
  - Re rho_L of complex targets (tdmrg_set_real_basis) against the oracle's real-basis rho_L (1e-14),
    its eigenvectors exactly real, and H_L renormalised with them exactly real."""
import numpy as np
import pytest

from oracle import density, ed, krylov, superblock
from tests.gpu_util import ExactLoader, dev, host, new_ctx, rel_err, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


class _Complexified(ExactLoader):
    """The same operators with a 1e-300 imaginary part: numerically equal, but not real."""

    def add(self, side, op):
        from oracle import blocks as oblocks
        op = oblocks.BlockOp({k: b + 1e-300j for k, b in op.blocks.items()}, op.odd)
        return super().add(side, op)


@pytest.mark.parametrize("slices", [0, 4])
def test_real_operators_half_the_work(lib, c1_problem, slices):
    p = c1_problem
    Q = (5, 4)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(p.sb.size(Q)) + 1j * rng.standard_normal(p.sb.size(Q))
    ref = superblock.apply_h(p.sb, p.HL, p.HR, p.conns, Q, x)
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=slices) if slices else {}
    res = {}
    for name, loader in (("real", ExactLoader), ("complex", _Complexified)):
        ctx = new_ctx(**kw)
        try:
            loader(ctx, p)
            out = dev(np.zeros(len(x)))
            lib.tdmrg_apply_h(ctx, Q, dev(x), out)
            assert rel_err(host(out), ref) < (1e-12 if not slices else 140.0 * 2.0 ** -28), name
            res[name] = (lib.tdmrg_hpsi_flops(ctx, Q), lib.tdmrg_hpsi_tensor_flops(ctx, Q))
        finally:
            lib.tdmrg_destroy(ctx)
    assert res["real"][0] == 0.5 * res["complex"][0]
    if slices:
        assert res["real"][1] < res["complex"][1]


def test_real_path_trajectory_against_ed(lib, c1_problem, c1_ground):
    p = c1_problem
    e, psi = c1_ground
    Q1 = (5, 4)
    sec = ed.Sector(8, *Q1)
    H = ed.hamiltonian(sec, ed.chain_hopping(8), 4.0)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    times = krylov.target_times(0.1, 4)
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        oL, oR = ld.local("cdag", 4, 0)
        nops = [[ld.local("n", site, s) for s in (0, 1)] for site in range(8)]
        n = lib.tdmrg_sector_size(ctx, Q1)
        phi = dev(np.zeros(n))
        lib.tdmrg_apply_op(ctx, oL, oR, p.Q, dev(psi), Q1, phi)
        phif = np.zeros(sec.dim, complex)
        phif[perm] = host(phi)
        tg = [dev(np.zeros(n)) for _ in range(3)] + [phi]
        out = dev(np.zeros(1))
        for s in range(10):
            lib.tdmrg_evolve(ctx, Q1, phi, times, 12, tg)
            ex = ed.evolve(H, phif, [(s + 1) * 0.1])[0]
            for site in (0, 3, 4, 7):
                d = 0.0
                for a, b in nops[site]:
                    lib.tdmrg_expect(ctx, a, b, Q1, phi, out)
                    d += host(out)[0].real
                assert abs(d - ed.density(ex, sec, site, 0) - ed.density(ex, sec, site, 1)) < 1e-8
    finally:
        lib.tdmrg_destroy(ctx)


def test_real_basis_rho_and_real_renormalisation(lib, c1_problem, c1_ground):
    torch = torch_cuda()
    p = c1_problem
    e, psi = c1_ground
    Q1 = (5, 4)
    times = krylov.target_times(0.1, 4)
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        oL, oR = ld.local("cdag", 4, 0)
        n = lib.tdmrg_sector_size(ctx, Q1)
        phi = dev(np.zeros(n))
        lib.tdmrg_apply_op(ctx, oL, oR, p.Q, dev(psi), Q1, phi)
        tg = [dev(np.zeros(n)) for _ in range(4)]
        lib.tdmrg_evolve(ctx, Q1, phi, times, 12, tg)          # complex targets
        wgs, w = lib.tdmrg_tst_weights(4)
        lib.tdmrg_set_real_basis(ctx, 1)
        nr, ne = lib.tdmrg_rho_size(ctx)
        rho = dev(np.zeros(nr))
        sts = [(p.Q, dev(psi))] + [(Q1, t) for t in tg]
        lib.tdmrg_density_matrix(ctx, sts, [wgs] + w, rho)
        got = [host(t) for t in tg]
        assert max(np.abs(g.imag).max() for g in got) > 1e-3   # the targets are complex
        ref = density.rho_left(p.sb, [(p.Q, psi)] + [(Q1, g) for g in got], [wgs] + w, real_basis=True)
        rho_h = host(rho)
        off = 0
        for qi, d in enumerate(p.sb.ldim):
            assert np.abs(rho_h[off: off + d * d].reshape(d, d) - ref[qi]).max() < 1e-14
            off += d * d
        ev = torch.zeros(ne, dtype=torch.float64, device="cuda")
        U = dev(np.zeros(nr))
        lib.tdmrg_rho_eig(ctx, rho, ev, U)
        U_h = host(U)
        assert np.abs(U_h.imag).max() == 0.0                    # real eigenvectors
        lam = np.concatenate([l for l, _ in density.rho_eig(ref)])
        assert np.abs(ev.cpu().numpy() - lam).max() < 1e-13
        kept = [min(d, 6) for d in p.sb.ldim]
        hl = ld.add(0, p.HL)
        size = sum(kept[qo] * kept[qi] for (qo, qi) in p.HL.blocks if kept[qo] and kept[qi])
        out = dev(np.zeros(size))
        lib.tdmrg_renormalize_op(ctx, 0, hl, U, kept, out)
        assert np.abs(host(out).imag).max() == 0.0              # the operator stays real
    finally:
        lib.tdmrg_destroy(ctx)
