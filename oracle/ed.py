"""Exact diagonalisation of the Hubbard model in the Fock basis (oracle; test infrastructure).

Independent checker for everything built on blocks: states are bit strings
over 2N fermion modes, mode(i, sigma) = 2*i + sigma (up = 0, down = 1), so the
up mode of a site precedes its down mode and sites are ordered left to right.
A basis state is c^dag_{m1} c^dag_{m2} ... |0> with m1 < m2 < ..., and the
Jordan-Wigner sign of c_m is (-1)^(number of occupied modes below m).

Hamiltonian (Sec. III.A tight-binding part and Sec. III.B Hubbard term):
    H = sum_{i,j,sigma} t_ij c^dag_{i sigma} c_{j sigma} + U sum_i n_{i up} n_{i dn}
with a symmetric hopping matrix t_ij.  The lattices used here (open chain,
two-leg ladder) carry hopping -t on each bond.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def mode(i, sigma):
    return 2 * i + sigma


def sector_states(nsites, nup, ndn):
    """All Fock states with nup up and ndn down electrons, ascending integer order."""
    up_modes = [mode(i, 0) for i in range(nsites)]
    dn_modes = [mode(i, 1) for i in range(nsites)]
    states = []
    for ups in itertools.combinations(up_modes, nup):
        for dns in itertools.combinations(dn_modes, ndn):
            s = 0
            for m in ups + dns:
                s |= 1 << m
            states.append(s)
    return np.array(sorted(states), dtype=np.int64)


def _popcount_below(s, m):
    return bin(s & ((1 << m) - 1)).count("1")


def apply_c(s, m):
    """c_m |s> = sign |s'>; returns (sign, s') or (0, None)."""
    if not (s >> m) & 1:
        return 0, None
    return (-1) ** _popcount_below(s, m), s & ~(1 << m)


def apply_cdag(s, m):
    """c^dag_m |s> = sign |s'>; returns (sign, s') or (0, None)."""
    if (s >> m) & 1:
        return 0, None
    return (-1) ** _popcount_below(s, m), s | (1 << m)


def chain_hopping(nsites, t=1.0):
    """Open chain: -t on nearest-neighbour bonds, sites labelled 0..N-1 from the left."""
    h = np.zeros((nsites, nsites))
    for i in range(nsites - 1):
        h[i, i + 1] = h[i + 1, i] = -t
    return h


def ladder_hopping(lx, t_leg=1.0, t_rung=1.0):
    """Two-leg ladder, site i = 2x + y (rung-first zig-zag), legs along x, rungs along y."""
    n = 2 * lx
    h = np.zeros((n, n))
    for x in range(lx):
        a, b = 2 * x, 2 * x + 1
        h[a, b] = h[b, a] = -t_rung
        if x + 1 < lx:
            for y in range(2):
                i, j = 2 * x + y, 2 * (x + 1) + y
                h[i, j] = h[j, i] = -t_leg
    return h


class Sector:
    """Fock sector (N_up, N_dn) of an N-site lattice with index lookup."""

    def __init__(self, nsites, nup, ndn):
        self.nsites, self.nup, self.ndn = nsites, nup, ndn
        self.states = sector_states(nsites, nup, ndn)
        self.index = {int(s): k for k, s in enumerate(self.states)}

    @property
    def dim(self):
        return len(self.states)


def hamiltonian(sector, hop, U):
    """Sparse H in a Fock sector (real symmetric)."""
    rows, cols, vals = [], [], []
    n = sector.nsites
    for k, s in enumerate(sector.states):
        s = int(s)
        diag = 0.0
        for i in range(n):
            if (s >> mode(i, 0)) & 1 and (s >> mode(i, 1)) & 1:
                diag += U
        if diag != 0.0:
            rows.append(k); cols.append(k); vals.append(diag)
        for i in range(n):
            for j in range(n):
                if hop[i, j] == 0.0:
                    continue
                for sig in (0, 1):
                    s1, t1 = apply_c(s, mode(j, sig))
                    if s1 == 0:
                        continue
                    s2, t2 = apply_cdag(t1, mode(i, sig))
                    if s2 == 0:
                        continue
                    rows.append(sector.index[t2]); cols.append(k); vals.append(hop[i, j] * s1 * s2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(sector.dim, sector.dim))


def apply_site_op(vec, src, dst, ops):
    """Apply a product of mode operators to a sector vector.

    ops: list of (kind, mode) applied right to left, i.e. ops[-1] acts first;
    kind in {'c', 'cdag', 'n'}.
    """
    out = np.zeros(dst.dim, dtype=complex)
    for k, s in enumerate(src.states):
        amp = vec[k]
        if amp == 0:
            continue
        sign, cur = 1, int(s)
        for kind, m in reversed(ops):
            if kind == "n":
                if not (cur >> m) & 1:
                    sign = 0
                    break
                continue
            f = apply_c if kind == "c" else apply_cdag
            sg, cur2 = f(cur, m)
            if sg == 0:
                sign = 0
                break
            sign *= sg
            cur = cur2
        if sign != 0:
            out[dst.index[cur]] += sign * amp
    return out


def density(vec, sector, i, sigma):
    """<vec| n_{i sigma} |vec> / <vec|vec>."""
    occ = np.array([(int(s) >> mode(i, sigma)) & 1 for s in sector.states], dtype=float)
    p = np.abs(vec) ** 2
    return float(np.dot(occ, p) / p.sum())


def double_occupation(vec, sector, i):
    occ = np.array([((int(s) >> mode(i, 0)) & 1) * ((int(s) >> mode(i, 1)) & 1)
                    for s in sector.states], dtype=float)
    p = np.abs(vec) ** 2
    return float(np.dot(occ, p) / p.sum())


def ground_state(H):
    """Lowest eigenpair of a sparse Hermitian H (ARPACK, converged to machine precision)."""
    if H.shape[0] <= 400:
        w, v = np.linalg.eigh(H.toarray())
        return w[0], v[:, 0].astype(complex)
    w, v = spla.eigsh(H, k=1, which="SA", tol=0.0, ncv=40)
    return w[0], v[:, 0].astype(complex)


def evolve(H, vec, times):
    """exp(-i H t) vec for each t (scipy's expm_multiply, truncated Taylor at unit roundoff)."""
    times = list(times)
    out = []
    for t in times:
        out.append(spla.expm_multiply(-1j * t * H, vec) if t != 0 else vec.copy())
    return out
