"""Pins of the oracle against the paper's closed forms: App. A (one-site
excitation at U=0), Eq. nd and Sec. III.B.2 (holon-doublon at t=0), and the
small-time expansion of Sec. III.B.1."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import closed_forms, ed, krylov, models, superblock


def test_hole_formula_against_ed():
    """App. A's X_ij(t) = R_i R_j - |T_ij(t)|^2 against ED (U=0, 8-site chain, half filling)."""
    hop = ed.chain_hopping(8)
    s44, s34 = ed.Sector(8, 4, 4), ed.Sector(8, 3, 4)
    e, psi = ed.ground_state(ed.hamiltonian(s44, hop, 0.0))
    H34 = ed.hamiltonian(s34, hop, 0.0)
    i = 3
    phi = ed.apply_site_op(psi, s44, s34, [("c", ed.mode(i, 0))])
    for t in (0.0, 0.4, 1.3):
        pt = ed.evolve(H34, phi, [t])[0]
        for j in range(8):
            occ = np.array([(int(s) >> ed.mode(j, 0)) & 1 for s in s34.states])
            x_ed = float(np.dot(occ, np.abs(pt) ** 2))       # unnormalised, as in Eq. xij
            assert abs(x_ed - closed_forms.hole_x(hop, 4, i, j, t)) < 1e-10
    # Sec. III.A: X_ii(0) = 0; X_ij(0) = 1/4 - |G_ij|^2, 1/4 only where G_ij = 0
    assert abs(closed_forms.hole_x(hop, 4, i, i, 0.0)) < 1e-14
    assert abs(closed_forms.hole_x(hop, 4, i, i + 2, 0.0) - 0.25) < 1e-14


def test_c1_u0_trajectory_against_closed_form():
    """Oracle Krylov on the exact-block superblock (U=0) reproduces the particle closed form to 1e-8."""
    p = models.chain(8, U=0.0)
    e, psi = p.ground_state()
    Q1 = (5, 4)
    phi = p.apply_local("cdag", 4, 0, p.Q, psi, Q1)
    hop = ed.chain_hopping(8)
    Eone = np.linalg.eigvalsh(hop)
    assert Eone[4] - Eone[3] > 1e-6                          # non-degenerate Fermi level
    rdn = closed_forms.ground_density(hop, 4)
    tau = 0.1
    traj = krylov.time_steps(p.apply_h(Q1), phi, tau, 10, n_v=4, nk=12)
    for s, (targets, n_used, err) in enumerate(traj):
        t = (s + 1) * tau
        v = targets[-1]
        for j in range(8):
            n_up = p.density(v, Q1, j, sigma=0)
            n_dn = p.density(v, Q1, j, sigma=1)
            xp = closed_forms.particle_x(hop, 4, 4, j, t) / (1.0 - rdn[4])
            assert abs(n_up - xp) < 1e-8
            assert abs(n_dn - rdn[j]) < 1e-8


@pytest.fixture(scope="module")
def ladder_hd():
    """2x4 ladder, t_x=1, t_y=0.5, 4 up 4 down, holon at i=2, doublon at j=4 (Sec. III.B, Figs. 3-5)."""
    out = {}
    for U in (0.0, 10.0):
        p = models.ladder(4, t_leg=1.0, t_rung=0.5, U=U)
        e, psi = p.ground_state()
        # phi = c_{i up}(1 - n_{i dn}) c^dag_{j up} n_{j dn} psi  (sigma = sigma' = up)
        Q = p.Q
        x = p.apply_local("n", 4, 1, Q, psi, Q)
        x = p.apply_local("cdag", 4, 0, Q, x, (5, 4))
        x = x - p.apply_local("n", 2, 1, (5, 4), x, (5, 4))
        phi = p.apply_local("c", 2, 0, (5, 4), x, Q)
        out[U] = (p, phi)
    return out


@pytest.mark.parametrize("U", [0.0, 10.0])
def test_holon_doublon_t0(ladder_hd, U):
    """Eq. nd: density 0 at i, 2 at j, 1 elsewhere; N_d = 0 at i and 1 at j (Sec. III.B.2)."""
    p, phi = ladder_hd[U]
    dens = [p.density(phi, p.Q, s) for s in range(8)]
    assert np.abs(np.array(dens) - closed_forms.holon_doublon_t0(8, 2, 4)).max() < 1e-10
    assert abs(p.double_occupation(phi, p.Q, 2)) < 1e-12
    assert abs(p.double_occupation(phi, p.Q, 4) - 1.0) < 1e-10


def test_holon_doublon_against_ed(ladder_hd):
    """Full O_{j,i,p}(t) and N_d at U=10 against ED on the 2x4 ladder."""
    p, phi = ladder_hd[10.0]
    sec = ed.Sector(8, 4, 4)
    H = ed.hamiltonian(sec, ed.ladder_hopping(4, 1.0, 0.5), 10.0)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    phif = np.zeros(sec.dim, complex); phif[perm] = phi
    traj = krylov.time_steps(p.apply_h(p.Q), phi, 0.05, 6, n_v=3, nk=12)
    for s, (targets, n_used, err) in enumerate(traj):
        t = (s + 1) * 0.05
        ex = ed.evolve(H, phif, [t])[0]
        for site in (0, 2, 4, 7):
            d_ed = ed.density(ex, sec, site, 0) + ed.density(ex, sec, site, 1)
            assert abs(p.density(targets[-1], p.Q, site) - d_ed) < 1e-9
            assert abs(p.double_occupation(targets[-1], p.Q, site) - ed.double_occupation(ex, sec, site)) < 1e-9


def _fock_state(p, phi):
    sec = ed.Sector(8, *p.Q)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    phif = np.zeros(sec.dim, complex)
    phif[perm] = phi
    return sec, phif


@pytest.mark.parametrize("site", [2, 4, 5])
def test_small_time_coefficient_against_ed_curvature(ladder_hd, site):
    """closed_forms.small_time_coefficient against the curvature of the exact density: O(t) from
    exact evolution (ED, expm) at t = 0, +-h, +-h/2, and a = O''(0) / 2 by central differences with
    one Richardson step (error O(h^4)); U = 10 ladder, holon-doublon state (Sec. III.B.1).  A sign or
    ordering slip in the formula (H n H + H^2 n, or n H^2 for H n H) fails by orders of magnitude."""
    p, phi = ladder_hd[10.0]
    sec, phif = _fock_state(p, phi)
    H = ed.hamiltonian(sec, ed.ladder_hopping(4, 1.0, 0.5), 10.0)
    occ = np.array([((int(s) >> ed.mode(site, 0)) & 1) + ((int(s) >> ed.mode(site, 1)) & 1)
                    for s in sec.states], dtype=float)
    n_p = sp.diags(occ)
    a = closed_forms.small_time_coefficient(H, n_p, phif)

    def O(t):
        v = ed.evolve(H, phif, [t])[0]
        return float(np.dot(occ, np.abs(v) ** 2) / np.vdot(v, v).real)

    def curv(h):
        return (O(h) - 2.0 * O(0.0) + O(-h)) / (2.0 * h * h)

    h = 2e-3
    a_fd = (4.0 * curv(h / 2) - curv(h)) / 3.0
    assert abs(a - a_fd) < 1e-6 * max(1.0, abs(a)), (a, a_fd)
    assert abs(a) > 1e-3                       # the pin is not vacuous at this site


def test_small_time_expansion(ladder_hd):
    """O(t) - O(0) = a t^2 + O(t^4) with a from closed_forms.small_time_coefficient applied to the
    block-basis H psi of the oracle, at U = 10 (Sec. III.B.1)."""
    p, phi = ladder_hd[10.0]
    Hf = p.apply_h(p.Q)
    n = len(phi)
    Hop = spla.LinearOperator((n, n), matvec=Hf, dtype=complex)
    for site in (2, 4, 5):
        side, n_up = p.op("n", site, 0)
        side, n_dn = p.op("n", site, 1)

        def nop(v):
            out = 0
            for o in (n_up, n_dn):
                A, B = (o, None) if side == 0 else (None, o)
                out = out + superblock.apply_op(p.sb, A, B, p.Q, v, p.Q)
            return out

        a = closed_forms.small_time_coefficient(Hop, spla.LinearOperator((n, n), matvec=nop, dtype=complex), phi)
        O0 = p.density(phi, p.Q, site)
        for t in (0.005, 0.01, 0.02):
            targets, n_used, err = krylov.evolve(Hf, phi, [t], nk=12)
            resid = p.density(targets[0], p.Q, site) - O0 - a * t * t
            assert abs(resid) < 50.0 * t ** 4 * max(1.0, abs(a)) ** 2
