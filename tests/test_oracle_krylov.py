"""Pins of the oracle's Krylov advance (Sec. II.A Eq. lanczosevolution, Sec. II.C
Eq. lanczosevolution2) against dense matrix exponentials, exact diagonalisation and
conservation laws."""
import numpy as np
import scipy.linalg as sla

from oracle import ed, krylov, superblock


def _rand_herm(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (X + X.conj().T) / 2


def test_full_krylov_space_is_exact_expm():
    """With n_K = dimension the Krylov propagator is exp(-iHt) itself."""
    H = _rand_herm(9, 0)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    times = [0.0, 0.3, 0.7, 1.1]
    targets, n_used, err = krylov.evolve(lambda v: H @ v, phi, times, nk=9)
    for t, y in zip(times, targets):
        assert np.abs(y - sla.expm(-1j * H * t) @ phi).max() < 1e-12


def test_coefficients_equal_expm_of_t():
    """c = ||phi|| exp(-iTt) e_0: pins the orientation of S in T = S^dag D S."""
    rng = np.random.default_rng(2)
    alpha = rng.standard_normal(7)
    beta = rng.uniform(0.2, 1.0, 6)
    T = krylov.tridiagonal(alpha, beta)
    for t in (0.1, 0.9):
        c = krylov.krylov_coefficients(alpha, beta, 2.5, [t])[0]
        assert np.abs(c - 2.5 * sla.expm(-1j * T * t)[:, 0]).max() < 1e-13


def test_lanczos_relation_and_orthonormality():
    H = _rand_herm(60, 3)
    rng = np.random.default_rng(4)
    phi = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    V, alpha, beta, b0, bn = krylov.lanczos(lambda v: H @ v, phi, 12)
    Vm = np.array(V)
    assert np.abs(Vm.conj() @ Vm.T - np.eye(len(V))).max() < 1e-13
    T = krylov.tridiagonal(alpha, beta)
    assert np.abs(Vm.conj() @ H @ Vm.T - T).max() < 1e-12
    assert abs(b0 - np.linalg.norm(phi)) < 1e-13


def test_breakdown_on_invariant_subspace():
    """phi in a 3-dimensional invariant subspace: Lanczos stops at 3 and is exact."""
    H = _rand_herm(20, 5)
    w, U = np.linalg.eigh(H)
    phi = U[:, 2] + 0.5 * U[:, 7] - 0.25j * U[:, 11]
    targets, n_used, err = krylov.evolve(lambda v: H @ v, phi, [0.0, 2.0], nk=10)
    assert n_used == 3
    assert np.abs(targets[1] - sla.expm(-2j * H) @ phi).max() < 1e-12


def test_c1_trajectory_against_ed(c1_problem, c1_ground):
    """L=8, U=4 chain, c^dag_{4 up} excitation, tau=0.1, n_K=12: every step matches ED."""
    p = c1_problem
    e, psi = c1_ground
    Q1 = (5, 4)
    phi = p.apply_local("cdag", 4, 0, p.Q, psi, Q1)
    sec = ed.Sector(8, *Q1)
    H = ed.hamiltonian(sec, ed.chain_hopping(8), 4.0)
    perm = superblock.fock_to_psi(p.cut, sec, np.arange(sec.dim) + 0j).real.astype(int)
    phif = np.zeros(sec.dim, complex); phif[perm] = phi
    tau, steps = 0.1, 8
    traj = krylov.time_steps(p.apply_h(Q1), phi, tau, steps, n_v=4, nk=12)
    hphi = p.apply_h(Q1)
    n0, e0 = np.vdot(phi, phi).real, np.vdot(phi, hphi(phi)).real
    for s, (targets, n_used, err) in enumerate(traj):
        for x, tx in enumerate(krylov.target_times(tau, 4)):
            exact = ed.evolve(H, phif, [s * tau + tx])[0][perm]
            assert np.abs(targets[x] - exact).max() < 1e-10
        last = targets[-1]
        assert abs(np.vdot(last, last).real - n0) < 1e-12
        assert abs(np.vdot(last, hphi(last)).real - e0) < 1e-10 * max(1, abs(e0))
        assert err < 1e-8


def test_error_estimate_bounds_the_true_error():
    """The a-posteriori estimate ||phi|| beta_n |[e^{-iT t}]_{n-1,0}| (Saad) against the exact error
    from expm on a random Hermitian matrix with spectrum in about [-1, 1]: it stays above the true
    error and within a factor 30 of it, for several times and Krylov dimensions."""
    import scipy.linalg as sl
    rng = np.random.default_rng(2)
    n = 300
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (A + A.conj().T) / np.sqrt(8 * n)
    phi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for t in (0.5, 1.0, 2.0):
        exact = sl.expm(-1j * H * t) @ phi
        for nk in (6, 8, 10, 12):
            targets, n_used, err = krylov.evolve(lambda v: H @ v, phi, [0.0, t], nk)
            true = np.linalg.norm(targets[-1] - exact)
            assert true <= err <= 30.0 * true, (t, nk, err, true)
