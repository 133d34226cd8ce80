"""Sec. III.A, Fig. 2: the one-site hole excitation of the tight-binding chain (b) and two-leg ladder (a),
reproduced by a finite sweep with time-step targeting on the GPU and compared with the exact result of
App. A.

16-site chain, H_0 = -sum_<ij> sigma (c^dag c + h.c.) (U = 0), half filling, m = 200 (the paper's value for
the chain).  Everything runs on the device: the infinite algorithm, one finite ground-state sweep (W_gs,
its discarded weight, enters the energy bound), then the sweep with time-step targeting.  The hole is
created by c_{8 up} on the ground state (i = 8: b = 1, B = c_up in Eq. b) at the
sweep's first step, whose central sites are 7 and 8; n_v = 4 targets, tau = 0.1, n_K = 12, the targets
advanced at every other step (Sec. II.C).  At every step the device measures <n_{l up}> and <n_{l+1 up}>
of every target (l, l + 1: the new sites of the two enlarged blocks), normalised, so for target x at time
t = t_step + x tau / 3
    X_{8j}(t) = <phi|phi> <n_{j up}>(t),   <phi|phi> = <psi|n_{8 up}|psi> = R_8,
and the closed form X_ij(t) = R_i R_j - |T_ij(t)|^2 (oracle.closed_forms.hole_x, pinned against ED)
gives the expected density X_{8j}(t) / R_8.

The arithmetic is FP64 throughout, so the deviations are the method's truncation error, bounded by the
sweep's total discarded weight W = sum_k eps_k (eps_k the discarded weight of the weighted rho of step k
as the sweep reports it) and the targeting weights w (ground state 1/4, targets 1/4, 1/8, 1/8, 1/4):
eps_k = sum_x w_x ||(1 - P_k) phi_x||^2, so a cut removes at most eps_k / w_x of target x's squared norm
and these losses add up.  Hence every target's norm lies within W / min w of R_8; the ground-state
energy, variational, lies above the exact free-fermion energy by at most (W / w_gs) |E_0|; and a
density, not variational, errs at most at the order of the amplitude error sqrt(W / min w).  Measured
at m = 200: W = 2.3e-6; energy 1.1e-5 above (bound 1.8e-4), norm 1.1e-6 (bound 1.9e-5), densities
6.7e-4 over 200 points up to t = 1.2 (bound 4.3e-3).

Ladder, Fig. 2(a): 8 x 2 sites (rung-first labels, site 8 = leg 0 of rung 4), m = 400 (the paper's value
for the ladder), the same excitation and schedule.  The paper does not give the rung hopping of this
figure; with t_rung = t_leg the half-filled U=0 ladder has two levels at the Fermi energy, a degenerate
ground state for which App. A's X_ij is not defined, so t_rung = 0.5 (the value of Sec. III.B) is used,
which leaves a gap of 0.31.  The device runs the infinite algorithm and two ground-state sweeps (W_gs: the
last one's discarded weight).  Measured: W = 6.8e-4; energy 5.7e-3 above (bound 5.3e-2), densities 7.9e-3
(bound 7.4e-2): a ladder needs far more states than a chain for the same accuracy, as its cut crosses
two legs."""
import numpy as np
import pytest

from oracle import closed_forms, ed
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu
L, M, M_LADDER, I_SITE, TAU, N_V, T_RUNG = 16, 200, 400, 8, 0.1, 4, 0.5
HOP = -np.eye(L, k=1) - np.eye(L, k=-1)


def _check(records, hop, nsites, w_gs_sweep=0.0):
    """Energies, norms and densities of a sweep's records against App. A; returns (W, worst, points)."""
    from paper_1103_5391_gb300 import tdmrg as T
    e_exact = 2.0 * np.linalg.eigvalsh(hop)[: nsites // 2].sum()
    r8 = closed_forms.ground_density(hop, nsites // 2)[I_SITE]
    assert records[0]["action"] == "excite"
    worst = {"energy": 0.0, "norm": 0.0, "density": 0.0}
    npoints = 0
    for rec in records:
        worst["energy"] = max(worst["energy"], abs(rec["energy"] - e_exact))
        l = rec["l"]
        for x, tg in enumerate(rec["targets"]):
            t = rec["t"] + x * TAU / (N_V - 1)
            worst["norm"] = max(worst["norm"], abs(tg["norm2"] - r8))
            for site, key in ((l, "n_left"), (l + 1, "n_right")):
                want = closed_forms.hole_x(hop, nsites // 2, I_SITE, site, t) / r8
                worst["density"] = max(worst["density"], abs(tg[key].real - want))
                npoints += 1
    W = sum(rec.get("discarded", 0.0) for rec in records)
    w_gs, w = T.tdmrg_tst_weights(N_V)
    print("fig2:", npoints, "points, t up to %.2f, W = %.2e, W_gs = %.2e," % (records[-1]["t"], W, w_gs_sweep), worst)
    assert npoints > 150 and records[-1]["t"] >= 1.0
    assert min(rec["energy"] for rec in records) > e_exact - 1e-9   # variational: the cuts are projections
    assert worst["energy"] < (W / w_gs + w_gs_sweep) * abs(e_exact), (W, worst)
    assert worst["norm"] < W / min(w), (W, worst)
    assert worst["density"] < np.sqrt(W / min(w)), (W, worst)
    return W, worst


def _device_run(lattice, m, gs_sweeps):
    """Infinite algorithm, ground-state sweeps and the sweep with the hole c_{8 up}, all on the device."""
    torch_cuda()
    from paper_1103_5391_gb300 import sweep as S
    lat = None if lattice is None else S.Lattice(*lattice)
    left, right, _ = S.infinite(L, 1.0, 0.0, m, lattice=lat)
    w_gs_sweep = 0.0
    for _ in range(gs_sweeps):
        gs = S.TSTSweep(L, 1.0, 0.0, m, left, right, excitations=[], lattice=lat)
        w_gs_sweep = sum(r.get("discarded", 0.0) for r in gs.run())
        left, right = gs.left, gs.right
    records = S.TSTSweep(L, 1.0, 0.0, m, left, right, n_v=N_V, tau=TAU, nk=12, advance_every=2,
                         excitations=[(I_SITE, "c", 0)], lattice=lat).run()
    return records, w_gs_sweep


def test_chain_hole_excitation_matches_app_a():
    records, w_gs_sweep = _device_run(None, M, 1)
    W, _ = _check(records, HOP, L, w_gs_sweep)
    assert W < 1e-5   # m = 200 resolves the chain's targets: the bounds are tight


def test_ladder_hole_excitation_matches_app_a():
    records, w_gs_sweep = _device_run((2, 1.0, T_RUNG), M_LADDER, 2)
    _check(records, ed.ladder_hopping(L // 2, 1.0, T_RUNG), L, w_gs_sweep)
