"""One finite sweep with time-step targeting on the GPU (Sec. II.B-II.D) against the oracle's sweep, step
by step, on the FP64 path.

L=10 Hubbard chain (U=4, half filling), m=20..24, n_v=4 targets, tau=0.1, n_K=10, three schedules of
Eq. b (c^dag_{5 up} at once; c_{7 dn} c^dag_{5 up} completed two steps later; c^dag_{8 dn} reached on the
left pass after ground-state targeting); the 2 x 5 ladder (t_leg = 1, t_rung = 0.5, U=4; Sec. III), m=28
and 32, two schedules, whose blocks carry their two edge sites and whose cuts are crossed by two or three
bonds; both sweeps start from the same stored blocks (the oracle's ground-state DMRG).  The device runs every step through the C ABI: ground state by restarted Lanczos, the
excitation operators, Krylov
advance, rho_L or rho_R, its eigendecomposition, truncation, renormalisation, enlargement of both blocks
and the wave-function transformation of all five targets, left and right.  Compared per step (quantities
that do not depend on eigenvector phases): the ground-state energy (1e-10), the kept counts (equal), all
eigenvalues of rho and the discarded weight (1e-12), and for every target its norm, <H>, the densities of
the two central sites and the bond <c^dag_l c_{l+1}> (1e-10)."""
import copy

import numpy as np
import pytest

from oracle import dmrg, tst
from tests.gpu_util import dev, torch_cuda

pytestmark = pytest.mark.gpu
L, U, T_HOP, M = 10, 4.0, 1.0, 24


def _blockops(blk, dense, odd):
    secs, _, _ = blk.sectors()
    bo = blk.blockop(dense, odd)
    qns = [tuple(secs[qo]) + tuple(secs[qi]) for (qo, qi) in bo.blocks]
    data = np.concatenate([b.ravel() for b in bo.blocks.values()]) if bo.blocks else np.zeros(0, complex)   # H = 0: one site at U = 0
    return qns, data


def _eig_layout(Ufull, enl, K):
    """The oracle's kept states (columns of Ufull over the enlarged block enl, grouped by K's sectors) in
    the layout of tdmrg_rho_eig: per sector of enl a dim x dim matrix whose first columns are K's states."""
    esecs, edims, estarts = enl.sectors()
    ksecs, kdims, kstarts = K.sectors()
    parts, kept = [], []
    for q, dq, s0 in zip(esecs, edims, estarts):
        M_ = np.zeros((dq, dq), complex)
        if q in ksecs:
            j = ksecs.index(q)
            M_[:, :kdims[j]] = Ufull[s0: s0 + dq, kstarts[j]: kstarts[j] + kdims[j]]
            kept.append(kdims[j])
        else:
            kept.append(0)
        parts.append(M_.ravel())
    return np.concatenate(parts), kept


def _device_blocks(d, sweep_mod):
    left, right = {}, {}
    for store, ustore, side, out in ((d.left, d.left_U, "L", left), (d.right, d.right_U, "R", right)):
        for n, blk in store.items():
            secs, dims, _ = blk.sectors()
            hq, hd = _blockops(blk, blk.H, False)
            cd = [_blockops(blk, blk.cdag[s], True) for s in range(2)]
            cd2 = None
            if blk.cdag2 is not None:
                cd2 = [(q, dev(x)) for q, x in (_blockops(blk, blk.cdag2[s], True) for s in range(2))]
            V = kept = None
            if n in ustore:   # (a block older than its smaller neighbour has no usable V; the sweep remakes it first)
                enl = dmrg.enlarge(store[n - 1], side, d.t, d.U, d.geom)
                if ustore[n].shape[0] == enl.dim:
                    Vh, kept = _eig_layout(ustore[n], enl, blk)
                    V = dev(Vh)
            out[n] = sweep_mod.Block(secs, dims, (hq, dev(hd)), [(q, dev(x)) for q, x in cd], V, kept,
                                     nsites=blk.nsites, cdag2=cd2)
    return left, right


# (m, advance_every, excitations of Eq. b, ladder); m is chosen per case so that no cut of the sweep falls
# inside a cluster of eigenvalues closer than 1e-7 lambda_max (checked on the oracle's records below)
CASES = [
    (24, 2, [(5, "cdag", 0)], False),
    (20, 1, [(5, "cdag", 0), (7, "c", 1)], False),   # partial product for two steps, completed at sites (6, 7)
    (24, 1, [(8, "cdag", 1)], False),                # ground-state targeting until the left pass reaches site 8
    (32, 2, [(5, "cdag", 0)], True),                 # 2 x 5 ladder: cuts after odd sites cross a rung
    (28, 1, [(4, "c", 1)], True),
]
T_RUNG = 0.5


@pytest.fixture(scope="module", params=range(len(CASES)))
def sweeps(request):
    m, every, exc, ladder = CASES[request.param]
    torch_cuda()
    from paper_1103_5391_gb300 import sweep as S
    d = dmrg.ChainDMRG(L, T_HOP, U, m, geom=dmrg.Geometry(2, T_HOP, T_RUNG) if ladder else None)
    d.run(sweeps=1)
    left, right = _device_blocks(d, S)
    want = tst.TSTSweep(copy.deepcopy(d), m, n_v=4, tau=0.1, nk=10, advance_every=every, excitations=exc).run()
    got = S.TSTSweep(L, T_HOP, U, m, left, right, n_v=4, tau=0.1, nk=10, advance_every=every, excitations=exc,
                     lattice=S.Lattice(2, T_HOP, T_RUNG) if ladder else None).run()
    return m, want, got


def test_sweep_cuts_are_clean(sweeps):
    m, want, _ = sweeps
    for r in want:
        if r["move"] is None:
            continue
        lam = np.sort(np.concatenate(r["evals"]))[::-1]
        if len(lam) > m:
            assert lam[m - 1] - lam[m] > 1e-7 * lam[0]


def test_sweep_matches_oracle_step_by_step(sweeps):
    m, want, got = sweeps
    _same_sweep(want, got)


def _same_sweep(want, got, tol=1e-10, tol_rho=1e-12):
    assert len(want) == len(got) == len(tst.sweep_path(L))
    for w, g in zip(want, got):
        assert (g["l"], g["move"], g["action"], g["applied"], tuple(g["Q1"])) == \
            (w["l"], w["move"], w["action"], w["applied"], tuple(w["Q1"]))
        assert abs(g["t"] - w["t"]) < 1e-15
        assert abs(g["energy"] - w["energy"]) < tol, (w["l"], w["move"])
        if w["move"] is not None:
            assert g["kept"] == list(w["kept"])
            assert abs(g["discarded"] - w["discarded"]) < tol_rho
            for a, b in zip(g["evals"], w["evals"]):
                assert np.abs(a - b).max() < tol_rho
        assert len(g["targets"]) == len(w["targets"])
        for a, b in zip(g["targets"], w["targets"]):
            for key in ("norm2", "energy", "n_left", "n_right", "bond"):
                assert abs(a[key] - b[key]) < tol, (w["l"], w["move"], key, a[key], b[key])


@pytest.mark.parametrize("ladder,m", [(False, 24), (True, 40)])
def test_device_infinite_algorithm_then_sweep(ladder, m):
    """The infinite algorithm on the device (site blocks made from the vacuum block, both blocks enlarged,
    the superblock's ground state, both cuts) against the oracle's: every step's ground-state energy
    (1e-10) and every kept block's sector dimensions; then one sweep with time-step targeting from each
    one's blocks, step by step as above.  m is chosen so that no cut of the infinite algorithm or the sweep
    lies within 1e-6 lambda_max of its neighbour (checked on the oracle: 1.9e-6 and 1.1e-6 for the chain,
    8.8e-6 and 4.1e-6 for the ladder).  The two starts are not the same blocks: each side converges its own
    ground states (the oracle here to residual 1e-12, the device its fixed restarts to rounding), and a
    cut a few 1e-6 lambda_max from its neighbour turns that into kept states that differ at ~1e-12 / 1e-6;
    hence energies and observables 1e-9, rho's eigenvalues and discarded weight 1e-10 (with the oracle's
    default residual 1e-9 the ladder's energies differed by 1e-9 at the end of the infinite stage)."""
    torch_cuda()
    from paper_1103_5391_gb300 import sweep as S
    geom = dmrg.Geometry(2, T_HOP, T_RUNG) if ladder else None
    lattice = S.Lattice(2, T_HOP, T_RUNG) if ladder else None
    d = dmrg.ChainDMRG(L, T_HOP, U, m, geom=geom, gs_resid=1e-12)
    d.infinite()
    left, right, energies = S.infinite(L, T_HOP, U, m, lattice=lattice)
    want_e = [(n, e) for kind, n, e in d.energies if kind == "infinite"]
    assert [n for n, _ in energies] == [n for n, _ in want_e]
    for (n, e), (_, we) in zip(energies, want_e):
        assert abs(e - we) < 1e-9, (n, e, we)
    for mine, theirs in ((left, d.left), (right, d.right)):
        assert sorted(mine) == sorted(theirs)
        for k, blk in theirs.items():
            secs, dims, _ = blk.sectors()
            assert mine[k].qn == [tuple(q) for q in secs] and mine[k].dim == list(dims), k
    exc = [(5, "cdag", 0)]
    want = tst.TSTSweep(copy.deepcopy(d), m, n_v=4, tau=0.1, nk=10, advance_every=2, excitations=exc).run()
    got = S.TSTSweep(L, T_HOP, U, m, left, right, n_v=4, tau=0.1, nk=10, advance_every=2, excitations=exc,
                     lattice=lattice).run()
    _same_sweep(want, got, tol=1e-9, tol_rho=1e-10)


def test_sweep_on_the_tensor_path():
    """The same sweep (first schedule) with every superblock product on the tensor cores (4 bf16 slices;
    Lanczos, rho, eigendecomposition and transformations in FP64) against the oracle's FP64 sweep: the
    kept counts equal; the discarded weight and every target's norm, densities and bond within 1e-8, the
    observable accuracy target of the mixed-precision path (measured 1.5e-11 and 6.7e-9); energies (the
    ground state's and every target's <H>) and the eigenvalues of rho (all <= 1), which carry the
    product's own error to first order, within the H psi slicing bound 140 2^-28 (relative for the
    energies; measured 1.8e-8 and 1.1e-8).  Rounding-level changes of the Krylov vectors move the bf16
    digits, so these values vary between builds within that bound."""
    torch_cuda()
    from paper_1103_5391_gb300 import sweep as S
    from paper_1103_5391_gb300 import tdmrg as T
    m, every, exc, _ = CASES[0]
    d = dmrg.ChainDMRG(L, T_HOP, U, m)
    d.run(sweeps=1)
    left, right = _device_blocks(d, S)
    want = tst.TSTSweep(copy.deepcopy(d), m, n_v=4, tau=0.1, nk=10, advance_every=every, excitations=exc).run()
    got = S.TSTSweep(L, T_HOP, U, m, left, right, n_v=4, tau=0.1, nk=10, advance_every=every, excitations=exc,
                     prec=T.TDMRG_OZAKI_BF16, ozaki_slices=4).run()
    worst = {"energy_rel": 0.0, "evals": 0.0, "discarded": 0.0, "observables": 0.0}
    for w, g in zip(want, got):
        assert (g["l"], g["move"], g["action"]) == (w["l"], w["move"], w["action"])
        worst["energy_rel"] = max(worst["energy_rel"], abs(g["energy"] - w["energy"]) / abs(w["energy"]))
        if w["move"] is not None:
            assert g["kept"] == list(w["kept"])
            worst["discarded"] = max(worst["discarded"], abs(g["discarded"] - w["discarded"]))
            for a, b in zip(g["evals"], w["evals"]):
                worst["evals"] = max(worst["evals"], float(np.abs(a - b).max()))
        for a, b in zip(g["targets"], w["targets"]):
            worst["energy_rel"] = max(worst["energy_rel"], abs(a["energy"] - b["energy"]) / abs(b["energy"]))
            for key in ("norm2", "n_left", "n_right", "bond"):
                worst["observables"] = max(worst["observables"], abs(a[key] - b[key]))
    assert worst["energy_rel"] < 140.0 * 2.0 ** -28, worst
    assert worst["evals"] < 140.0 * 2.0 ** -28, worst
    assert max(worst["discarded"], worst["observables"]) < 1e-8, worst
