"""GPU parity of the Krylov advance (Sec. II.A Eq. lanczosevolution, Sec. II.C Eq. lanczosevolution2)
against the oracle (<= 1e-10 on psi per step, FP64 path) and of the physical trajectory against ED
(<= 1e-8 on n_i(t))."""
import numpy as np
import pytest

from oracle import ed, krylov, models, superblock
from tests.gpu_util import ExactLoader, dev, host, new_ctx, oracle_ops_of_synthetic, rel_err
from workloads import sectors as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def test_c1_trajectory(lib, c1_problem, c1_ground):
    """L=8 chain, U=4, c^dag_{4 up} on the ground state, tau=0.1, n_v=4, n_K=12, 20 steps to t=2."""
    p = c1_problem
    e, psi = c1_ground
    Q1 = (5, 4)
    tau, nv, nk, steps = 0.1, 4, 12, 20
    times = krylov.target_times(tau, nv)
    sec = ed.Sector(8, *Q1)
    H = ed.hamiltonian(sec, ed.chain_hopping(8), 4.0)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    ctx = new_ctx()
    try:
        ld = ExactLoader(ctx, p)
        oL, oR = ld.local("cdag", 4, 0)
        nops = [[ld.local("n", site, s) for s in (0, 1)] for site in range(8)]
        n = lib.tdmrg_sector_size(ctx, Q1)
        phi_d = dev(np.zeros(n))
        lib.tdmrg_apply_op(ctx, oL, oR, p.Q, dev(psi), Q1, phi_d)
        phi_o = p.apply_local("cdag", 4, 0, p.Q, psi, Q1)
        assert rel_err(host(phi_d), phi_o) < 1e-13
        phif = np.zeros(sec.dim, complex); phif[perm] = phi_o
        tg = [dev(np.zeros(n)) for _ in range(nv)]
        cur_o = phi_o
        exp_d = dev(np.zeros(1))
        for s in range(steps):
            src = phi_d if s == 0 else tg[-1]
            lib.tdmrg_evolve(ctx, Q1, src, times, nk, tg)
            targets_o, n_used, err_o = krylov.evolve(p.apply_h(Q1), cur_o, times, nk)
            n_gpu, err_gpu, alpha, beta = lib.tdmrg_evolve_info(ctx)
            assert n_gpu == n_used
            assert abs(err_gpu - err_o) <= 1e-6 * err_o + 1e-13     # the estimate is at rounding level here
            for x in range(nv):
                assert rel_err(host(tg[x]), targets_o[x]) < 1e-10
            cur_o = targets_o[-1]
            if s % 5 == 4 or s == steps - 1:
                ex = ed.evolve(H, phif, [(s + 1) * tau])[0]
                for site in range(8):
                    d = 0.0
                    for (a, b) in nops[site]:
                        lib.tdmrg_expect(ctx, a, b, Q1, tg[-1], exp_d)
                        d += host(exp_d)[0].real
                    d_ed = ed.density(ex, sec, site, 0) + ed.density(ex, sec, site, 1)
                    assert abs(d - d_ed) < 1e-8
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("L,m,nb,nk,nv,tau", [(32, 400, 1, 10, 4, 0.05), (16, 150, 2, 12, 3, 0.1)])
def test_synthetic_evolve(lib, L, m, nb, nk, nv, tau):
    """One advance of the L=32 m=400 chain (and a ragged ladder twin) against the oracle."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(L, m, 4.0, nbonds=nb, seed=S.SEED_BASE + 1)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    times = krylov.target_times(tau, nv)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        phi = dev(ss.phi)
        tg = [dev(np.zeros(n)) for _ in range(nv)]
        lib.tdmrg_evolve(ctx, ss.Q1, phi, times, nk, tg)
        hf = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
        V, alpha, beta, b0, bn = krylov.lanczos(hf, ss.phi, nk)
        ref, n_used, err = krylov.evolve(hf, ss.phi, times, nk)
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == n_used == nk
        # the same a-posteriori error estimate; the absolute floor covers an estimate at rounding level
        assert abs(err_gpu - err) <= 1e-6 * err + 1e-15 * np.linalg.norm(ss.phi)
        assert np.abs(a_g - alpha).max() < 1e-10 * np.abs(alpha).max()
        assert np.abs(b_g[:-1] - beta).max() < 1e-10 * np.abs(beta).max()
        for x in range(nv):
            assert rel_err(host(tg[x]), ref[x]) < 1e-10
        # norm conservation of the FP64 Krylov propagator
        assert abs(np.linalg.norm(host(tg[-1])) - np.linalg.norm(ss.phi)) < 1e-12
    finally:
        lib.tdmrg_destroy(ctx)


def test_breakdown_and_alias(lib):
    """Krylov space exhausted before n_K (tiny sector): same n_used and targets as the oracle;
    the last target may overwrite phi in place."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(6, 6, 4.0, nbonds=1, seed=21)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        sizes = {(a, b): sb.size((a, b)) for a in range(0, 8) for b in range(0, 8)}
        Q = min((q for q, v in sizes.items() if 2 <= v <= 6), key=lambda q: sizes[q])
        n = sizes[Q]
        rng = np.random.default_rng(3)
        phi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        hf = lambda v: superblock.apply_h(sb, HL, HR, conns, Q, v)
        times = [0.0, 0.4, 0.8]
        ref, n_used, err = krylov.evolve(hf, phi, times, 12)
        assert n_used <= n
        phi_d = dev(phi)
        t0, t1 = dev(np.zeros(n)), dev(np.zeros(n))
        lib.tdmrg_evolve(ctx, Q, phi_d, times, 12, [t0, t1, phi_d])
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == n_used
        for got, want in zip((t0, t1, phi_d), ref):
            assert rel_err(host(got), want) < 1e-10
    finally:
        lib.tdmrg_destroy(ctx)


def test_unordered_times(lib):
    """Targets at unsorted, repeated and zero times, one of them far enough for several
    substeps of the propagation on the tridiagonal: same targets and error estimate as the oracle's
    e^{-iTt} from the eigendecomposition of T (Eq. lanczosevolution)."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 150, 4.0, nbonds=2, seed=S.SEED_BASE + 1)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    times = [0.3, 0.2, 0.0, 0.3, 1.5, 0.05]
    nk = 12
    ctx = new_ctx()
    try:
        problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        tg = [dev(np.zeros(n)) for _ in times]
        lib.tdmrg_evolve(ctx, ss.Q1, dev(ss.phi), times, nk, tg)
        hf = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
        ref, n_used, err = krylov.evolve(hf, ss.phi, times, nk)
        n_gpu, err_gpu, a_g, b_g = lib.tdmrg_evolve_info(ctx)
        assert n_gpu == n_used
        for x in range(len(times)):
            assert rel_err(host(tg[x]), ref[x]) < 1e-10, times[x]
        assert abs(err_gpu - err) <= 1e-8 * err + 1e-300
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("mixed", [False, True])
def test_time_dependent_hamiltonian(lib, mixed):
    """H(t) driven from the host: one time step under H, then the boundary hopping is changed to a
    weaker, Peierls-phased amplitude a = 0.5 t e^{0.7 i} (its Hermitian partner -conj(a)) by setting
    the Hamiltonian again, and a second step follows.  Both steps against the oracle with the same
    coefficients (the plans are rebuilt for the new terms)."""
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 120, 4.0, nbonds=1, seed=S.SEED_BASE + 8)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    a = 0.5 * ss.coeff_t * np.exp(0.7j)
    conns2 = [((a if i % 2 == 0 else -np.conj(a)), A, B) for i, (_, A, B) in enumerate(conns)]
    times = krylov.target_times(0.05, 4)
    h1 = lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v)
    h2 = lambda v: superblock.apply_h(sb, HL, HR, conns2, ss.Q1, v)
    ref1, _, _ = krylov.evolve(h1, ss.phi, times, 10)
    ref2, _, _ = krylov.evolve(h2, ref1[-1], times, 10)
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=5) if mixed else {}
    ctx = new_ctx(**kw)
    try:
        gconns = problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        phi = dev(ss.phi)
        tg = [dev(np.zeros(n)) for _ in times]
        lib.tdmrg_evolve(ctx, ss.Q1, phi, times, 10, tg)
        assert rel_err(host(tg[-1]), ref1[-1]) < (1e-8 if mixed else 1e-10)
        lib.tdmrg_set_hamiltonian(ctx, problem.OP_H, problem.OP_H,
                                  [(l, r, (a if i % 2 == 0 else -np.conj(a))) for i, (l, r, _) in enumerate(gconns)])
        tg2 = [dev(np.zeros(n)) for _ in times]
        lib.tdmrg_evolve(ctx, ss.Q1, tg[-1], times, 10, tg2)
        for x in range(len(times)):
            assert rel_err(host(tg2[x]), ref2[x]) < (1e-8 if mixed else 1e-10), x
        # the pulse changed the dynamics: the second step differs from evolving under the old H
        ref_old, _, _ = krylov.evolve(h1, ref1[-1], times, 10)
        assert rel_err(ref2[-1], ref_old[-1]) > 1e-4
    finally:
        lib.tdmrg_destroy(ctx)
