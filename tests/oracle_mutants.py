"""Plausible mistakes planted in the oracle, one at a time, to show that its pins catch each of them.

Test infrastructure only.  This module is a pytest plugin that the mutation test loads into a child
pytest process (`-p tests.oracle_mutants`, environment variable ORACLE_MUTANT = the mistake's name); it
replaces one function of `oracle/` (or two, for a mistake that sits in a pair) by a wrong variant for that
process alone.  The main test session never loads it.  Each entry of MUTANTS gives the mistake, the
oracle attributes it replaces and the pin tests (node ids) of which at least one must fail.

The mistakes are those the pins are chosen against: a dropped term or factor, a wrong sign, a wrong or
shifted index, a transposed or conjugated operand, a wrong ordering, a wrong constant.
"""
import importlib
import os

import numpy as np

K = "tests/test_oracle_krylov.py::"
D = "tests/test_oracle_density.py::"
H = "tests/test_oracle_hpsi.py::"
C = "tests/test_oracle_closed_forms.py::"
G = "tests/test_oracle_dmrg.py::"
LAD = "tests/test_oracle_ladder.py::"
T = "tests/test_oracle_tst.py::"


# ---------------------------------------------------------------- Krylov (Sec. II.A, II.C)
def _time_sign(orig):
    """e^{+iTt} in place of e^{-iTt}."""
    return lambda alpha, beta, beta0, times: orig(alpha, beta, beta0, [-t for t in times])


def _s_untransposed(orig):
    """The columns of eigh's eigenvector matrix taken as the rows of S (T = S^dag D S)."""
    from oracle import krylov

    def f(alpha, beta, beta0, times):
        d, S = np.linalg.eigh(krylov.tridiagonal(alpha, beta))
        return np.array([beta0 * (S.conj().T @ (np.exp(-1j * d * t) * S[:, 0])) for t in times])
    return f


def _tridiag_shift(orig):
    """beta_j placed one row too low (off-by-one in the coupling index)."""
    return lambda alpha, beta: orig(alpha, np.roll(np.asarray(beta, dtype=float), 1))


def _norm_dropped(orig):
    """||phi|| lost: the expansion starts from the unit vector v_0 alone."""
    def f(*a, **k):
        V, alpha, beta, beta0, beta_n = orig(*a, **k)
        return V, alpha, beta, 1.0, beta_n
    return f


def _no_breakdown(orig):
    """The breakdown test never fires: the recursion runs on from a vector at rounding level."""
    return lambda apply_h, phi, nk, tol=1e-12: orig(apply_h, phi, nk, -1.0)


def _err_first_component(orig):
    """Saad's estimate with the first component of e^{-iTt} e_0 in place of the last."""
    from oracle import krylov

    def f(alpha, beta, beta0, beta_n, tau):
        c = krylov.krylov_coefficients(alpha, beta, 1.0, [tau])[0]
        return beta0 * beta_n * abs(c[0])
    return f


def _err_no_beta(orig):
    """Saad's estimate without the factor beta_n."""
    return lambda alpha, beta, beta0, beta_n, tau: orig(alpha, beta, beta0, 1.0, tau)


def _times_denominator(orig):
    """t_x = x tau / n_v: the last target falls short of tau."""
    return lambda tau, n_v: [x * tau / n_v for x in range(n_v)]


# ---------------------------------------------------------------- weights and rho (Sec. II.B, II.C)
def _omega(orig):
    """Omega = 1 / (n + 2) in place of 1 / (n + 3) (n = n_v + 1 targeted states)."""
    def f(n_v):
        gs, w = orig(n_v)
        s = (n_v + 4) / (n_v + 3)
        return gs * s, [x * s for x in w]
    return f


def _gs_weight(orig):
    """The ground state weighted Omega instead of 2 Omega."""
    def f(n_v):
        gs, w = orig(n_v)
        return gs / 2, w
    return f


def _rho_unnormalised(orig):
    """Targets not normalised before they enter rho."""
    def f(sb, states, weights, real_basis=False):
        return orig(sb, states, [w * np.vdot(v, v).real for (_, v), w in zip(states, weights)], real_basis)
    return f


def _rho_conjugated(orig):
    """rho^T (= conj(rho)) in place of rho: the dagger on the other factor."""
    return lambda sb, states, weights, real_basis=False: [r.conj() for r in orig(sb, states, weights, real_basis)]


def _dmrg_rho_conjugated(orig):
    return lambda sb, Q, psi: [r.conj() for r in orig(sb, Q, psi)]


def _eig_ascending(orig):
    """Eigenpairs in ascending order."""
    return lambda rho: [(lam[::-1], U[:, ::-1]) for lam, U in orig(rho)]


# ---------------------------------------------------------------- sector-pair products (Sec. IV)
def _parity_dropped(orig):
    """P_L left out of A P_L (x) B for odd B."""
    return lambda sb, qi: 1.0


def _dagger_no_conj(orig):
    """The adjoint of a block operator as its transpose only."""
    from oracle.blocks import BlockOp
    return lambda self: BlockOp({(qi, qo): b.T for (qo, qi), b in self.blocks.items()}, self.odd)


def _hc_sign(orig):
    """h (c^dag_i c_j + h.c.) written as h c^dag_i c_j + h c_i c^dag_j (the anticommutation sign lost)."""
    return lambda self: [(-c if k % 2 else c, A, B) for k, (c, A, B) in enumerate(orig(self))]


# ---------------------------------------------------------------- closed forms (App. A, Sec. III.B.1)
def _small_time_plus(orig):
    """a = <H n H + H^2 n> (sign of the second term)."""
    def f(H, n_p, phi):
        Hphi = H @ phi
        a = np.vdot(Hphi, n_p @ Hphi) + np.vdot(phi, H @ (H @ (n_p @ phi)))
        return (a / np.vdot(phi, phi)).real
    return f


def _small_time_order(orig):
    """a = <n H^2 - H^2 n> (n H^2 for H n H)."""
    def f(H, n_p, phi):
        a = np.vdot(phi, n_p @ (H @ (H @ phi))) - np.vdot(phi, H @ (H @ (n_p @ phi)))
        return (a / np.vdot(phi, phi)).real
    return f


def _hole_levels(orig):
    """One level too many in the primed (occupied) sums."""
    return lambda hop, nocc, i, j, t: orig(hop, nocc + 1, i, j, t)


def _hole_abs(orig):
    """|T_ij(t)| in place of |T_ij(t)|^2."""
    from oracle import closed_forms

    def f(hop, nocc, i, j, t):
        E, U = closed_forms.one_particle(hop)
        R = (np.abs(U[:, :nocc]) ** 2).sum(axis=1)
        Tij = (U[i, :nocc].conj() * U[j, :nocc] * np.exp(-1j * E[:nocc] * t)).sum()
        return R[i] * R[j] - abs(Tij)
    return f


def _particle_levels(orig):
    """The double-primed (empty) sum started one level too low."""
    return lambda hop, nocc, i, j, t: orig(hop, nocc - 1, i, j, t)


# ---------------------------------------------------------------- exact diagonalisation
def _no_jw(orig):
    """Fermion operators without the Jordan-Wigner sign."""
    def f(s, m):
        sign, s2 = orig(s, m)
        return abs(sign), s2
    return f


def _half_u(orig):
    """U/2 in the on-site term."""
    return lambda sector, hop, U: orig(sector, hop, 0.5 * U)


def _density_spin(orig):
    """The density of the other spin species."""
    return lambda vec, sector, i, sigma: orig(vec, sector, i, 1 - sigma)


# ---------------------------------------------------------------- exact blocks
def _block_half_u(orig):
    """U/2 in an exact block's Hamiltonian."""
    return lambda self, hop, U: orig(self, hop, 0.5 * U)


def _no_string(orig):
    """A block's c^dag / c without the Jordan-Wigner string of the sites before it."""
    from oracle import blocks

    def f(self, i, sigma, dagger):
        cd = blocks.SITE_CDAG_UP if sigma == 0 else blocks.SITE_CDAG_DN
        return self.kron_op([np.eye(4)] * i + [cd if dagger else cd.T] + [np.eye(4)] * (self.nsites - i - 1))
    return f


# ---------------------------------------------------------------- DMRG (Sec. I) and the sweep (Sec. II.B-II.D)
def _kept_smallest(orig):
    """The m smallest eigenvalues kept."""
    return lambda evals, m, *a, **k: orig([-np.asarray(e) for e in evals], m, *a, **k)


def _enlarge_half_u(orig):
    """U/2 on the new site of an enlarged block."""
    return lambda blk, side, t, U, geom=None: orig(blk, side, t, 0.5 * U, geom)


def _superblock_bond_halved(orig):
    """The hopping across the cut counted with half its amplitude (both of its terms)."""
    def f(*a, **k):
        sb, HL, HR, conns = orig(*a, **k)
        return sb, HL, HR, [(0.5 * c, A, B) for c, A, B in conns]
    return f


def _discarded_kept(orig):
    """The discarded weight reported as the kept weight."""
    def f(*a, **k):
        K, counts, lams, disc, U = orig(*a, **k)
        return K, counts, lams, float(sum(np.sum(x) for x in lams)) - disc, U
    return f


def _wft_u_conj(orig):
    """The kept states' projection with U^T (no conjugation) in a wave-function transformation."""
    return lambda Lenl, Renl, Q, psi, U, *rest: orig(Lenl, Renl, Q, psi, U.conj(), *rest)


def _wft_v_conj(orig):
    """The expansion of the other block's states with conj(V)."""
    return lambda Lenl, Renl, Q, psi, U, blk, V, *rest: orig(Lenl, Renl, Q, psi, U, blk, V.conj(), *rest)


def _ladder_bonds_swapped(orig):
    """A new ladder site bonded to the second site with the rung amplitude and to the edge with the leg's."""
    def f(self, k):
        a, b = orig(self, k)
        return (b, a) if self.legs == 2 else (a, b)
    return f


def _ladder_rung_dropped(orig):
    """The rung across the cut left out of the superblock."""
    return lambda self, l: [x for x in orig(self, l) if not (self.legs == 2 and tuple(x[:2]) == (0, 0))]


def _delta_sign(orig):
    """c and c^dag change the sector the other way."""
    return lambda kind, sigma: [-x for x in orig(kind, sigma)]


# name -> ([(module, attribute path)], factory, pins)
MUTANTS = {
    "krylov_time_sign": ([("oracle.krylov", "krylov_coefficients")], _time_sign,
                         [K + "test_coefficients_equal_expm_of_t", K + "test_full_krylov_space_is_exact_expm"]),
    "krylov_S_untransposed": ([("oracle.krylov", "krylov_coefficients")], _s_untransposed,
                              [K + "test_coefficients_equal_expm_of_t", K + "test_full_krylov_space_is_exact_expm"]),
    "tridiagonal_index": ([("oracle.krylov", "tridiagonal")], _tridiag_shift,
                          [K + "test_lanczos_relation_and_orthonormality", K + "test_full_krylov_space_is_exact_expm"]),
    "lanczos_norm_dropped": ([("oracle.krylov", "lanczos")], _norm_dropped,
                             [K + "test_full_krylov_space_is_exact_expm"]),
    "lanczos_no_breakdown": ([("oracle.krylov", "lanczos")], _no_breakdown,
                             [K + "test_breakdown_on_invariant_subspace"]),
    "error_estimate_component": ([("oracle.krylov", "error_estimate")], _err_first_component,
                                 [K + "test_error_estimate_bounds_the_true_error"]),
    "error_estimate_beta": ([("oracle.krylov", "error_estimate")], _err_no_beta,
                            [K + "test_error_estimate_bounds_the_true_error"]),
    "target_times": ([("oracle.krylov", "target_times")], _times_denominator,
                     [K + "test_c1_trajectory_against_ed"]),
    "weights_omega": ([("oracle.density", "tst_weights")], _omega, [D + "test_weights"]),
    "weights_ground_state": ([("oracle.density", "tst_weights")], _gs_weight, [D + "test_weights"]),
    "rho_unnormalised": ([("oracle.density", "rho_left")], _rho_unnormalised,
                         [D + "test_single_target_spectrum_is_schmidt", D + "test_mixed_sector_rho_properties"]),
    "rho_left_conjugated": ([("oracle.density", "rho_left")], _rho_conjugated,
                            [D + "test_mixed_sector_rho_properties"]),
    "rho_right_conjugated": ([("oracle.density", "rho_right")], _rho_conjugated,
                             [D + "test_rho_right_is_the_partial_trace"]),
    "dmrg_rho_right_conjugated": ([("oracle.dmrg", "rho_right")], _dmrg_rho_conjugated,
                                  [D + "test_rho_right_is_the_partial_trace"]),
    "rho_eig_ascending": ([("oracle.density", "rho_eig")], _eig_ascending,
                          [D + "test_mixed_sector_rho_properties"]),
    "parity_dropped": ([("oracle.superblock", "left_parity")], _parity_dropped,
                       [H + "test_exact_cut_hpsi_equals_ed"]),
    "dagger_no_conj": ([("oracle.blocks", "BlockOp.dagger")], _dagger_no_conj,
                       [H + "test_sector_hpsi_matches_dense_kron"]),
    "connection_hc_sign": ([("oracle.blocks", "Cut.connections")], _hc_sign,
                           [H + "test_exact_cut_hpsi_equals_ed"]),
    "small_time_sign": ([("oracle.closed_forms", "small_time_coefficient")], _small_time_plus,
                        [C + "test_small_time_coefficient_against_ed_curvature"]),
    "small_time_order": ([("oracle.closed_forms", "small_time_coefficient")], _small_time_order,
                         [C + "test_small_time_coefficient_against_ed_curvature"]),
    "hole_levels": ([("oracle.closed_forms", "hole_x")], _hole_levels, [C + "test_hole_formula_against_ed"]),
    "hole_not_squared": ([("oracle.closed_forms", "hole_x")], _hole_abs, [C + "test_hole_formula_against_ed"]),
    "particle_levels": ([("oracle.closed_forms", "particle_x")], _particle_levels,
                        [C + "test_c1_u0_trajectory_against_closed_form"]),
    "ed_no_jordan_wigner": ([("oracle.ed", "apply_c"), ("oracle.ed", "apply_cdag")], _no_jw,
                            [C + "test_hole_formula_against_ed", C + "test_c1_u0_trajectory_against_closed_form"]),
    "ed_half_u": ([("oracle.ed", "hamiltonian")], _half_u, [H + "test_exact_cut_hpsi_equals_ed"]),
    "ed_density_spin": ([("oracle.ed", "density")], _density_spin, [G + "test_dmrg_superblock_dynamics_match_ed"]),
    "block_half_u": ([("oracle.blocks", "Block.hubbard_h")], _block_half_u, [H + "test_exact_cut_hpsi_equals_ed"]),
    "block_no_jw_string": ([("oracle.blocks", "Block.site_fermion")], _no_string,
                           [H + "test_local_operators_equal_ed"]),
    "discarded_weight": ([("oracle.dmrg", "truncate")], _discarded_kept, [T + "test_truncated_sweep_invariants"]),
    "kept_smallest": ([("oracle.dmrg", "kept_counts")], _kept_smallest,
                      [G + "test_kept_counts_brute_force_small"]),
    "dmrg_eig_ascending": ([("oracle.dmrg", "eig_desc")], _eig_ascending,
                           [G + "test_dmrg_energy_variational_in_m"]),
    "enlarge_half_u": ([("oracle.dmrg", "enlarge")], _enlarge_half_u, [G + "test_dmrg_exact_blocks_match_ed"]),
    "superblock_bond_halved": ([("oracle.dmrg", "superblock_of")], _superblock_bond_halved,
                           [G + "test_dmrg_exact_blocks_match_ed"]),
    "wft_right_projection_conj": ([("oracle.dmrg", "wft_right")], _wft_u_conj,
                                  [T + "test_exact_sweep_is_exact_time_evolution"]),
    "wft_left_projection_conj": ([("oracle.dmrg", "wft_left")], _wft_u_conj,
                                 [T + "test_exact_sweep_is_exact_time_evolution"]),
    "wft_right_expansion_conj": ([("oracle.dmrg", "wft_right")], _wft_v_conj,
                                 [T + "test_exact_sweep_is_exact_time_evolution"]),
    "wft_left_expansion_conj": ([("oracle.dmrg", "wft_left")], _wft_v_conj,
                                [T + "test_exact_sweep_is_exact_time_evolution"]),
    "ladder_bonds_swapped": ([("oracle.dmrg", "Geometry.new_site_bonds")], _ladder_bonds_swapped,
                             [LAD + "test_geometry_is_the_lattice"]),
    "ladder_rung_dropped": ([("oracle.dmrg", "Geometry.cut_bonds")], _ladder_rung_dropped,
                            [LAD + "test_ladder_exact_sweep_is_exact_time_evolution"]),
    "sweep_sector_shift": ([("oracle.tst", "_delta")], _delta_sign,
                           [T + "test_exact_sweep_is_exact_time_evolution"]),
}


def _plant(name):
    targets, factory, _ = MUTANTS[name]
    for modname, path in targets:
        owner = importlib.import_module(modname)
        *outer, attr = path.split(".")
        for part in outer:
            owner = getattr(owner, part)
        setattr(owner, attr, factory(getattr(owner, attr)))


def pytest_configure(config):
    name = os.environ.get("ORACLE_MUTANT")
    if name:
        if name not in MUTANTS:
            raise ValueError(f"unknown oracle mutant {name!r}")
        _plant(name)
