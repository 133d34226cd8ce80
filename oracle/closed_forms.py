"""Closed forms used to pin the oracle (oracle; test infrastructure).

App. A (Sec. III.A, Eq. xij): for the tight-binding H_0 = sum t_ij c^dag c with
one-particle eigenvectors U[:, lam] and energies E_lam, the hole excitation
c_i|psi> gives
    X_ij(t) = R_i R_j - |T_ij(t)|^2,
    R_i = sum'_lam |U_{i lam}|^2,   T_ij(t) = sum'_lam conj(U_{i lam}) U_{j lam} e^{-i E_lam t},
with primed sums over the occupied levels.  The same Wick contraction for the
particle excitation c^dag_i|psi> gives
    X+_ij(t) = (1 - R_i) R_j + |sum''_lam U_{i lam} conj(U_{j lam}) e^{-i E_lam t}|^2,
with the double-primed sum over the empty levels; <phi|phi> = 1 - R_i.
Both are unnormalised expectation values of n_{j sigma} for the excited spin.

App. B, Eq. nd (Sec. III.B.1): the holon-doublon state at half filling has
density 0 at the holon site i, 2 at the doublon site j and 1 elsewhere at t=0;
Sec. III.B.2: its double occupation is 0 at i and 1 at j at t = 0.

Small-time expansion (Sec. III.B.1): O(t) = O(0) + a t^2 + O(t^4) with
a = <phi|H n_p H - H^2 n_p|phi> / <phi|phi> (real for real H and real phi).
"""
import numpy as np


def one_particle(hop):
    E, U = np.linalg.eigh(hop)
    return E, U


def hole_x(hop, nocc, i, j, t):
    """X_ij(t) of App. A (hole created at i), nocc lowest levels filled."""
    E, U = one_particle(hop)
    occ = slice(0, nocc)
    R = (np.abs(U[:, occ]) ** 2).sum(axis=1)
    T = (U[i, occ].conj() * U[j, occ] * np.exp(-1j * E[occ] * t)).sum()
    return R[i] * R[j] - abs(T) ** 2


def particle_x(hop, nocc, i, j, t):
    """X+_ij(t): particle created at i (same Wick derivation as App. A)."""
    E, U = one_particle(hop)
    occ, emp = slice(0, nocc), slice(nocc, None)
    R = (np.abs(U[:, occ]) ** 2).sum(axis=1)
    G = (U[i, emp] * U[j, emp].conj() * np.exp(-1j * E[emp] * t)).sum()
    return (1.0 - R[i]) * R[j] + abs(G) ** 2


def ground_density(hop, nocc):
    E, U = one_particle(hop)
    return (np.abs(U[:, :nocc]) ** 2).sum(axis=1)


def holon_doublon_t0(nsites, i, j):
    """Eq. nd: total density at t=0 at half filling."""
    out = np.ones(nsites)
    out[i] = 0.0
    out[j] = 2.0
    return out


def small_time_coefficient(H, n_p, phi):
    """a = <phi|H n H - H^2 n|phi>/<phi|phi> with dense or sparse H, n."""
    Hphi = H @ phi
    a = np.vdot(Hphi, n_p @ Hphi) - np.vdot(phi, H @ (H @ (n_p @ phi)))
    return (a / np.vdot(phi, phi)).real
