"""Textbook two-site DMRG for the open Hubbard chain and two-leg ladder: infinite, then finite algorithm
(oracle; test infrastructure only).

Sec. I: a block keeps the m most probable states of its reduced density matrix, computed from the
superblock's targeted state, and every block operator is carried into the kept basis, O -> U^dag O U.
The superblock is (left block + one site) + (one site + right block); the two enlarged blocks are the
L and R blocks of the superblock product (Sec. II.B: alpha in L, beta in R).

Conventions (the same as the exact blocks of blocks.py and the superblock of superblock.py):
  - chain sites 0..L-1 from the left; H = -t sum_<ij> sigma (c^dag c + h.c.) + U sum n_up n_dn;
  - fermion order: left block string, then right block string; inside an enlarged block the sites in
    lattice order, so an odd operator of a later factor picks up the parity of the earlier factor;
  - a block basis is sorted by its quantum number (n_up, n_dn), lexicographically, stably;
  - every block operator is a dense matrix over the block basis (plain Kronecker products, then the
    sector permutation); sector blocks are cut from it for the superblock product.
A block carries its Hamiltonian and c^dag_{edge, sigma} of the site that bonds to the rest of the chain
(the last site of a left block, the first site of a right block).

Ladder (Sec. III: 8 x 2 and 2 x 4 ladders): sites i = 2x + y in rung-first order, so site i bonds to
i - 1 across a rung when i is odd and to i - 2 along a leg; a ladder block also carries c^dag of its
second site from the edge (cdag2), since a new site bonds to both.  The ladder with an even number of
sites is symmetric under reflection i -> N - 1 - i (which exchanges the legs), so a right block of r sites
has the bonds of a left block of r sites and the same rule (Geometry) builds both.

Truncation (the reading of the silent paper): the eigenvalues of rho of all sectors are sorted in
descending order; the m largest are kept; eigenvalues within 1e-12 lambda_max of the m-th largest are
ties, broken by (sector index ascending, eigen index ascending).  Within a sector the kept states are
then always the leading eigenvectors.

Algorithm:
  infinite: blocks of l sites on both sides grow one site per step (superblock of 2l + 2 sites at half
            filling) until the superblock has L sites;
  finite:   sweeps left to right and back over the stored blocks at fixed L (half filling), each step
            a ground state by Lanczos with restarts, then truncation of the growing side.
"""
import numpy as np

from . import blocks, density, krylov, superblock

# single-site basis in sector order (n_up, n_dn): |0>, |dn>, |up>, |up dn>; blocks.py uses
# (|0>, |up>, |dn>, |up dn>), so the operators are permuted from there
SITE_QN = [(0, 0), (0, 1), (1, 0), (1, 1)]
_PERM = [0, 2, 1, 3]
SITE_CDAG = [blocks.SITE_CDAG_UP[np.ix_(_PERM, _PERM)].astype(complex),
             blocks.SITE_CDAG_DN[np.ix_(_PERM, _PERM)].astype(complex)]
SITE_P = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
SITE_NN = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
TIE_REL = 1e-12


class Geometry:
    """Bonds of the open chain (legs = 1, hopping t_leg) or of the two-leg ladder (legs = 2) with
    rung-first labels, H_0 = -sum_bonds t (c^dag c + h.c.)."""

    def __init__(self, legs=1, t_leg=1.0, t_rung=1.0):
        assert legs in (1, 2)
        self.legs, self.t_leg, self.t_rung = legs, t_leg, t_rung

    def new_site_bonds(self, k):
        """Hopping of a new site with k sites between it and the block's open end to the block's edge
        (the site k - 1 from that end) and to the second site from the edge (k - 2)."""
        if self.legs == 1:
            return (self.t_leg if k >= 1 else 0.0), 0.0
        return (self.t_rung if k % 2 == 1 else 0.0), (self.t_leg if k >= 2 else 0.0)

    def cut_bonds(self, l):
        """Bonds between the left enlarged block (sites 0..l) and the right one (sites l + 1 ...), as
        (left edge index, right edge index, t); edge 0 is the site at the cut, edge 1 the next one."""
        if self.legs == 1:
            return [(0, 0, self.t_leg)]
        return ([(0, 0, self.t_rung)] if l % 2 == 0 else []) + [(1, 0, self.t_leg), (0, 1, self.t_leg)]

    def hopping(self, nsites):
        """The matrix h of H_0 = sum_ij h_ij c^dag_i c_j (h_ij = -t on bonds)."""
        h = np.zeros((nsites, nsites))
        for j in range(nsites):
            for d, tb in zip((1, 2), self.new_site_bonds(j)):
                if tb != 0.0 and j - d >= 0:
                    h[j - d, j] = h[j, j - d] = -tb
        return h


class DBlock:
    """A block: basis quantum numbers (sorted), dense H, c^dag of the edge site per spin, site count, and
    on a ladder c^dag of the second site from the edge per spin (cdag2; None on a chain)."""

    def __init__(self, qn, H, cdag, nsites, cdag2=None):
        self.qn = [tuple(q) for q in qn]
        self.H = H
        self.cdag = cdag
        self.cdag2 = cdag2
        self.nsites = nsites

    @property
    def dim(self):
        return len(self.qn)

    def parity(self):
        return np.diag([(-1.0) ** (a + b) for a, b in self.qn]).astype(complex)

    def sectors(self):
        """(sector list, dims, start offsets) of the sorted basis."""
        secs, dims, starts = [], [], []
        for k, q in enumerate(self.qn):
            if not secs or secs[-1] != q:
                secs.append(q)
                dims.append(0)
                starts.append(k)
            dims[-1] += 1
        return secs, dims, starts

    def blockop(self, M, odd):
        """Nonzero sector blocks of a dense operator on this block."""
        secs, dims, starts = self.sectors()
        out = {}
        for a, (sa, da) in enumerate(zip(starts, dims)):
            for b, (sb, db) in enumerate(zip(starts, dims)):
                blk = M[sa: sa + da, sb: sb + db]
                if np.any(blk != 0):
                    out[(a, b)] = blk.copy()
        return blocks.BlockOp(out, odd)


def site_block(U):
    return DBlock(SITE_QN, U * SITE_NN, [c.copy() for c in SITE_CDAG], 1)


def _sorted(qn, mats):
    order = sorted(range(len(qn)), key=lambda k: qn[k])   # stable: ties keep Kronecker order
    ix = np.ix_(order, order)
    return [qn[k] for k in order], [m[ix] for m in mats], order


def enlarge(blk, side, t, U, geom=None):
    """Left block + site (side 'L') or site + right block (side 'R'), with the bond between the block's
    edge site and the new site (hopping t); the new site becomes the edge.  With a geometry, the new
    site's bonds to the edge and to the second site from the edge come from it, and on a ladder the old
    edge is carried as the new block's second site from the edge."""
    t0, t1 = (t, 0.0) if geom is None else geom.new_site_bonds(blk.nsites)
    keep = geom is not None and geom.legs == 2
    s = site_block(U)
    Ib, I4 = np.eye(blk.dim, dtype=complex), np.eye(4, dtype=complex)
    edges = [(blk.cdag, t0), (blk.cdag2, t1)]
    if side == "L":     # block string first: an odd site operator picks up the block parity
        Pb = blk.parity()
        H = np.kron(blk.H, I4) + np.kron(Ib, s.H)
        cd_new, carried = [], []
        for sig in range(2):
            cs = np.kron(Pb, s.cdag[sig])
            for cdK, tb in edges:
                if cdK is not None and tb != 0.0:
                    cb = np.kron(cdK[sig], I4)
                    H = H - tb * (cb @ cs.conj().T + cs @ cb.conj().T)
            cd_new.append(cs)
            carried.append(np.kron(blk.cdag[sig], I4))
        qn = [(a + c, b + d) for (a, b) in blk.qn for (c, d) in SITE_QN]
    else:               # site string first: an odd block operator picks up the site parity
        H = np.kron(s.H, Ib) + np.kron(I4, blk.H)
        cd_new, carried = [], []
        for sig in range(2):
            cs = np.kron(s.cdag[sig], Ib)
            for cdK, tb in edges:
                if cdK is not None and tb != 0.0:
                    cb = np.kron(SITE_P, cdK[sig])
                    H = H - tb * (cs @ cb.conj().T + cb @ cs.conj().T)
            cd_new.append(cs)
            carried.append(np.kron(SITE_P, blk.cdag[sig]))
        qn = [(c + a, d + b) for (c, d) in SITE_QN for (a, b) in blk.qn]
    qn, mats, order = _sorted(qn, [H] + cd_new + (carried if keep else []))
    out = DBlock(qn, mats[0], mats[1:3], blk.nsites + 1, cdag2=mats[3:5] if keep else None)
    out.perm = order   # Kronecker index of each basis state: a * 4 + s (side 'L') or s * dim + a (side 'R')
    return out


def superblock_of(L, R, t, geom=None):
    """Superblock, H_L, H_R and the boundary terms -t (c^dag_L c_R + h.c.) of every bond across the cut as
    fermionic products (left operator first): -t c^dag_L c_R and +t c_L c^dag_R.  Without a geometry the
    one bond of the chain (hopping t) between the two edges."""
    lsec, ldim, _ = L.sectors()
    rsec, rdim, _ = R.sectors()
    sb = superblock.Superblock(lsec, ldim, rsec, rdim)
    HL, HR = L.blockop(L.H, False), R.blockop(R.H, False)
    conns = []
    bonds = [(0, 0, t)] if geom is None else geom.cut_bonds(L.nsites - 1)
    for eL, eR, tb in bonds:
        if tb == 0.0:
            continue
        opL = L.cdag if eL == 0 else L.cdag2
        opR = R.cdag if eR == 0 else R.cdag2
        for sig in range(2):
            cdL, cdR = L.blockop(opL[sig], True), R.blockop(opR[sig], True)
            conns.append((-tb, cdL, cdR.dagger()))
            conns.append((tb, cdL.dagger(), cdR))
    return sb, HL, HR, conns


def ground_state(apply_h, n, seed=11035391, nk=120, resid_tol=1e-9):
    """Lowest eigenpair by Lanczos with restarts (full re-orthogonalisation), FP64: stops when the energy
    is stationary to 1e-13 and ||H v - E v|| < resid_tol."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 0j
    v /= np.linalg.norm(v)
    e_old = None
    for _ in range(60):
        V, alpha, beta, b0, bn = krylov.lanczos(apply_h, v, min(nk, n), tol=1e-14)
        d, S = np.linalg.eigh(krylov.tridiagonal(alpha, beta))
        v = sum(S[k, 0] * V[k] for k in range(len(V)))
        v /= np.linalg.norm(v)
        k = np.argmax(np.abs(v))
        v *= abs(v[k]) / v[k]
        if e_old is not None and abs(d[0] - e_old) < 1e-13 * max(1.0, abs(d[0])):
            if np.linalg.norm(apply_h(v) - d[0] * v) < resid_tol:
                return d[0], v
        e_old = d[0]
    return d[0], v


def kept_counts(evals, m, tie_rel=TIE_REL):
    """Number of kept states per sector: the m largest eigenvalues over all sectors (each sector's list
    in descending order), ties within tie_rel * lambda_max of the m-th largest broken by (sector index,
    eigen index) ascending."""
    allv = [(lam, s, k) for s, ev in enumerate(evals) for k, lam in enumerate(ev)]
    counts = [0] * len(evals)
    if len(allv) <= m:
        return [len(ev) for ev in evals]
    srt = sorted(allv, key=lambda x: -x[0])
    lam_m = srt[m - 1][0]
    tol = tie_rel * max(srt[0][0], 0.0)
    above = [x for x in allv if x[0] > lam_m + tol]
    tied = sorted([x for x in allv if abs(x[0] - lam_m) <= tol], key=lambda x: (x[1], x[2]))
    for lam, s, k in above + tied[: m - len(above)]:
        counts[s] += 1
    return counts


def rho_right(sb, Q, psi):
    """rho_R per right sector: sum over alpha of Psi[alpha, beta] conj(Psi[alpha, beta'])."""
    rho = [np.zeros((d, d), dtype=complex) for d in sb.rdim]
    for qi, ri, off, dl, dr in sb.pairs(Q):
        X = psi[off: off + dl * dr].reshape(dl, dr)
        rho[ri] += X.T @ X.conj()
    return rho


def eig_desc(rho):
    """Per sector (eigenvalues descending, eigenvectors as columns)."""
    return density.rho_eig(rho)


def truncate(blk, rho, m):
    """Kept basis of an enlarged block from its reduced density matrix (list per sector): the block with
    every operator renormalised, O -> U^dag O U, plus (kept counts, eigenvalues, discarded weight, U),
    U (block dim x kept) holding the kept states in the enlarged block's basis, sector by sector."""
    eig = eig_desc(rho)
    counts = kept_counts([lam for lam, _ in eig], m)
    secs, dims, starts = blk.sectors()
    cols = []
    qn = []
    for s, ((lam, Uq), k) in enumerate(zip(eig, counts)):
        if k == 0:
            continue
        Ufull = np.zeros((blk.dim, k), dtype=complex)
        Ufull[starts[s]: starts[s] + dims[s], :] = Uq[:, :k]
        cols.append(Ufull)
        qn.extend([secs[s]] * k)
    U = np.concatenate(cols, axis=1)
    ren = lambda M: U.conj().T @ M @ U
    discarded = sum(float(np.sum(lam[k:])) for (lam, _), k in zip(eig, counts))
    cdag2 = None if blk.cdag2 is None else [ren(c) for c in blk.cdag2]
    return (DBlock(qn, ren(blk.H), [ren(c) for c in blk.cdag], blk.nsites, cdag2=cdag2), counts,
            [lam for lam, _ in eig], discarded, U)


class ChainDMRG:
    """Infinite + finite two-site DMRG of the open Hubbard chain of L sites (L even) at half filling, or
    of the two-leg ladder of L sites (geom = Geometry(2, t_leg, t_rung); the superblocks of the infinite
    algorithm are ladders of 2l + 2 sites)."""

    def __init__(self, L, t, U, m, geom=None, gs_resid=1e-9):
        assert L % 2 == 0 and L >= 4
        self.L, self.t, self.U, self.m, self.geom = L, t, U, m, geom
        self.gs_resid = gs_resid   # residual bound of every step's ground state
        self.left = {1: site_block(U)}
        self.right = {1: site_block(U)}
        self.right_U = {}   # right block of r sites: its kept states (columns) in the enlarged block of r - 1 sites
        self.left_U = {}    # the same for the left blocks
        self.energies = []

    def _step(self, l, r, Q):
        Lenl = enlarge(self.left[l], "L", self.t, self.U, self.geom)
        Renl = enlarge(self.right[r], "R", self.t, self.U, self.geom)
        sb, HL, HR, conns = superblock_of(Lenl, Renl, self.t, self.geom)
        e, psi = ground_state(lambda v: superblock.apply_h(sb, HL, HR, conns, Q, v), sb.size(Q),
                              resid_tol=self.gs_resid)
        return Lenl, Renl, sb, e, psi

    def infinite(self):
        l = 1
        while 2 * l + 2 <= self.L:
            Q = (l + 1, l + 1)
            Lenl, Renl, sb, e, psi = self._step(l, l, Q)
            self.energies.append(("infinite", 2 * l + 2, e))
            self.left[l + 1], *_, self.left_U[l + 1] = truncate(Lenl, density.rho_left(sb, [(Q, psi)], [1.0]), self.m)
            self.right[l + 1], *_, self.right_U[l + 1] = truncate(Renl, rho_right(sb, Q, psi), self.m)
            l += 1

    def sweep(self):
        """One finite sweep: left to right (new left blocks), right to left (new right blocks), then left
        to right back to the centre.  At left-block size l the right block has L - 2 - l sites."""
        L, h = self.L, self.L // 2
        Q = (h, h)
        rho_l = lambda sb, psi: density.rho_left(sb, [(Q, psi)], [1.0])
        for l in range(h - 1, L - 2):
            Lenl, Renl, sb, e, psi = self._step(l, L - 2 - l, Q)
            self.energies.append(("sweep right", l, e))
            if l + 1 <= L - 3:
                self.left[l + 1], *_, self.left_U[l + 1] = truncate(Lenl, rho_l(sb, psi), self.m)
        for r in range(1, L - 2):
            Lenl, Renl, sb, e, psi = self._step(L - 2 - r, r, Q)
            self.energies.append(("sweep left", L - 2 - r, e))
            if r + 1 <= L - 3:
                self.right[r + 1], *_, self.right_U[r + 1] = truncate(Renl, rho_right(sb, Q, psi), self.m)
        for l in range(1, h - 1):
            Lenl, Renl, sb, e, psi = self._step(l, L - 2 - l, Q)
            self.energies.append(("sweep right", l, e))
            self.left[l + 1], *_, self.left_U[l + 1] = truncate(Lenl, rho_l(sb, psi), self.m)

    def run(self, sweeps=2):
        """Infinite algorithm, `sweeps` finite sweeps, then the superblock at the central cut: returns
        (Lenl, Renl, sb, HL, HR, conns, energy, psi) with Q = (L/2, L/2)."""
        self.infinite()
        for _ in range(sweeps):
            self.sweep()
        h = self.L // 2
        Lenl, Renl, sb, e, psi = self._step(h - 1, h - 1, (h, h))
        sb, HL, HR, conns = superblock_of(Lenl, Renl, self.t, self.geom)
        return Lenl, Renl, sb, HL, HR, conns, e, psi


def dense_psi(sb, Q, psi):
    """The sector-blocked wave function as the dense matrix Psi[alpha, beta] over both block bases."""
    loff = np.concatenate([[0], np.cumsum(sb.ldim)])
    roff = np.concatenate([[0], np.cumsum(sb.rdim)])
    M = np.zeros((loff[-1], roff[-1]), dtype=complex)
    for qi, ri, off, dl, dr in sb.pairs(Q):
        M[loff[qi]: loff[qi] + dl, roff[ri]: roff[ri] + dr] = psi[off: off + dl * dr].reshape(dl, dr)
    return M


def blocks_of_dense(sb, Q, M):
    """Inverse of dense_psi: the sector-Q vector of a dense Psi."""
    loff = np.concatenate([[0], np.cumsum(sb.ldim)])
    roff = np.concatenate([[0], np.cumsum(sb.rdim)])
    out = np.zeros(sb.size(Q), dtype=complex)
    for qi, ri, off, dl, dr in sb.pairs(Q):
        out[off: off + dl * dr] = M[loff[qi]: loff[qi] + dl, roff[ri]: roff[ri] + dr].ravel()
    return out


def wft_right(Lenl, Renl, Q, psi, U, Rblk, V, Lenl_next, Renl_next):
    """Wave-function transformation (Sec. II.B) when the centre moves one site to the right: psi on
    (Lenl, Renl) with Renl = site + Rblk, to (Lenl_next, Renl_next) with Lenl_next = kept(Lenl) + site and
    Rblk the kept basis of Renl_next (|b> = sum_c V[c, b] |c>).  Left: projection on the kept states,
    Psi1 = U^dag Psi; right: each right-block state expanded in Renl_next; the moved site changes block
    but not its place in the lattice order of the fermions, so no sign arises."""
    sbA = superblock.Superblock(*Lenl.sectors()[:2], *Renl.sectors()[:2])
    sbB = superblock.Superblock(*Lenl_next.sectors()[:2], *Renl_next.sectors()[:2])
    P1 = U.conj().T @ dense_psi(sbA, Q, psi)                     # (kept, Renl)
    m, Db = P1.shape[0], Rblk.dim
    T = np.zeros((m, 4, Db), dtype=complex)
    for p, kidx in enumerate(Renl.perm):                         # Renl position p <- (site s, block b)
        s, b = divmod(kidx, Db)
        T[:, s, b] = P1[:, p]
    T2 = np.einsum("asb,cb->asc", T, V)                           # right block state b -> states c of Renl_next
    out = np.zeros((Lenl_next.dim, Renl_next.dim), dtype=complex)
    for p, kidx in enumerate(Lenl_next.perm):                    # Lenl_next position p <- (kept a, site s)
        a, s = divmod(kidx, 4)
        out[p, :] = T2[a, s, :]
    return blocks_of_dense(sbB, Q, out)


def wft_left(Lenl, Renl, Q, psi, U, Lblk, V, Lenl_next, Renl_next):
    """Wave-function transformation (Sec. II.B) when the centre moves one site to the left: psi on
    (Lenl, Renl) with Lenl = Lblk + site, to (Lenl_next, Renl_next) with Renl_next = site + kept(Renl) and
    Lblk the kept basis of Lenl_next (|a> = sum_c V[c, a] |c>).  Right: projection on the kept states
    |u_k> = sum_b U[b, k] |b>, Psi1 = Psi conj(U); left: each left-block state expanded in Lenl_next; no
    sign (the moved site keeps its place in the lattice order)."""
    sbA = superblock.Superblock(*Lenl.sectors()[:2], *Renl.sectors()[:2])
    sbB = superblock.Superblock(*Lenl_next.sectors()[:2], *Renl_next.sectors()[:2])
    P1 = dense_psi(sbA, Q, psi) @ U.conj()                        # (Lenl, kept)
    Da, k = Lblk.dim, P1.shape[1]
    T = np.zeros((Da, 4, k), dtype=complex)
    for p, kidx in enumerate(Lenl.perm):                          # Lenl position p <- (block a, site s)
        a, s = divmod(kidx, 4)
        T[a, s, :] = P1[p, :]
    T2 = np.einsum("ca,ask->csk", V, T)                           # left block state a -> states c of Lenl_next
    out = np.zeros((Lenl_next.dim, Renl_next.dim), dtype=complex)
    for p, kidx in enumerate(Renl_next.perm):                     # Renl_next position p <- (site s, kept k)
        s, kk = divmod(kidx, k)
        out[:, p] = T2[:, s, kk]
    return blocks_of_dense(sbB, Q, out)
