"""Workload assembly from the Hubbard model for the exact (fixed-cut) configurations (oracle; test infrastructure).

Geometry and conventions: chain sites 0..L-1 from the left (Sec. III.A, Fig. 2
caption); two-leg ladder site i = 2x + y with legs along x and rungs along y;
fixed central cut (left block = sites 0..L/2-1).  Hamiltonian
H = -t sum_<ij> sigma (c^dag c + h.c.) + U sum n_up n_dn (Sec. III.B).
"""
import numpy as np

from . import blocks, ed, krylov, superblock


class ExactProblem:
    """Hubbard model on a lattice small enough that both halves are exact blocks."""

    def __init__(self, hop, U, nup, ndn):
        self.hop = np.asarray(hop, dtype=float)
        self.U = U
        self.nsites = self.hop.shape[0]
        self.Q = (nup, ndn)
        self.cut = blocks.Cut(self.hop, U, self.nsites // 2)
        self.sb = superblock.exact_superblock(self.cut)
        self.HL = self.cut.block_h(0)
        self.HR = self.cut.block_h(1)
        self.conns = self.cut.connections()

    def apply_h(self, Q):
        return lambda v: superblock.apply_h(self.sb, self.HL, self.HR, self.conns, Q, v)

    def ground_state(self, nk=200, tol=1e-14):
        """Ground state in sector Q by Lanczos restarts on the block-sector H psi (FP64)."""
        Q = self.Q
        n = self.sb.size(Q)
        rng = np.random.default_rng(11035391)
        v = rng.standard_normal(n) + 0j
        v /= np.linalg.norm(v)
        e_old = None
        for _ in range(30):
            V, alpha, beta, b0, bn = krylov.lanczos(self.apply_h(Q), v, min(nk, n), tol=1e-14)
            T = krylov.tridiagonal(alpha, beta)
            d, S = np.linalg.eigh(T)
            v = sum(S[k, 0] * V[k] for k in range(len(V)))
            v /= np.linalg.norm(v)
            # fix the global phase: largest entry real positive
            k = np.argmax(np.abs(v))
            v *= abs(v[k]) / v[k]
            if e_old is not None and abs(d[0] - e_old) < tol * max(1.0, abs(d[0])):
                resid = np.linalg.norm(self.apply_h(Q)(v) - d[0] * v)
                if resid < 1e-10:
                    return d[0], v
            e_old = d[0]
        return d[0], v

    def op(self, kind, site, sigma=0):
        """(side, BlockOp) for 'cdag', 'c', 'n', 'nn' (double occupation)."""
        if kind == "cdag":
            return self.cut.fermion(site, sigma, True)
        if kind == "c":
            return self.cut.fermion(site, sigma, False)
        if kind == "n":
            return self.cut.number(site, sigma)
        if kind == "nn":
            return self.cut.double_occ(site)
        raise ValueError(kind)

    def apply_local(self, kind, site, sigma, Q_in, psi, Q_out):
        side, o = self.op(kind, site, sigma)
        A, B = (o, None) if side == 0 else (None, o)
        return superblock.apply_op(self.sb, A, B, Q_in, psi, Q_out)

    def density(self, psi, Q, site, sigma=None):
        sig = (0, 1) if sigma is None else (sigma,)
        out = 0.0
        for s in sig:
            side, o = self.op("n", site, s)
            A, B = (o, None) if side == 0 else (None, o)
            out += superblock.expect(self.sb, A, B, Q, psi).real
        return out

    def double_occupation(self, psi, Q, site):
        side, o = self.op("nn", site)
        A, B = (o, None) if side == 0 else (None, o)
        return superblock.expect(self.sb, A, B, Q, psi).real


def chain(L, t=1.0, U=4.0, nup=None, ndn=None):
    nup = L // 2 if nup is None else nup
    ndn = L // 2 if ndn is None else ndn
    return ExactProblem(ed.chain_hopping(L, t), U, nup, ndn)


def ladder(lx, t_leg=1.0, t_rung=1.0, U=0.0, nup=None, ndn=None):
    n = 2 * lx
    nup = n // 2 if nup is None else nup
    ndn = n // 2 if ndn is None else ndn
    return ExactProblem(ed.ladder_hopping(lx, t_leg, t_rung), U, nup, ndn)
