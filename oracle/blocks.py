"""Exact block operators at a fixed left/right cut (oracle; test infrastructure).

A block of l sites is the tensor product of l Hubbard sites.  Site basis
{|0>, |up>, |dn>, |up dn>} with |up dn> = c^dag_up c^dag_dn |0> (up before
down), so c^dag_dn carries the intra-site sign (-1)^{n_up}.  Site operators are
placed in the block with a Jordan-Wigner parity string on the sites to their
left (Sec. II.B: fermionic operators reorder "yielding at most a minus sign").

Block states are grouped into sectors q = (n_up, n_dn) in ascending
lexicographic order; inside a sector states are ordered by their Fock bit
string (bit 2*i = up mode of local site i, bit 2*i+1 = down mode).  A block
operator is kept as a dict {(q_out, q_in): dense block} of its nonzero sector
blocks, plus its fermion parity.

The superblock basis is |alpha>_L |beta>_R = (left creation string)(right
creation string)|0>, the Fock order of the whole lattice when the left block
holds sites 0..l-1.
"""
import numpy as np

# site operators in the basis (|0>, |up>, |dn>, |up dn>)
SITE_CDAG_UP = np.zeros((4, 4)); SITE_CDAG_UP[1, 0] = 1.0; SITE_CDAG_UP[3, 2] = 1.0
SITE_CDAG_DN = np.zeros((4, 4)); SITE_CDAG_DN[2, 0] = 1.0; SITE_CDAG_DN[3, 1] = -1.0
SITE_P = np.diag([1.0, -1.0, -1.0, 1.0])
SITE_NUP = np.diag([0.0, 1.0, 0.0, 1.0])
SITE_NDN = np.diag([0.0, 0.0, 1.0, 1.0])
SITE_UP_OF = np.array([0, 1, 0, 1])
SITE_DN_OF = np.array([0, 0, 1, 1])


class BlockOp:
    """Sector-block operator on one block: blocks {(q_out, q_in): ndarray}, fermion parity `odd`."""

    def __init__(self, blocks, odd):
        self.blocks = blocks
        self.odd = bool(odd)

    def dagger(self):
        return BlockOp({(qi, qo): b.conj().T for (qo, qi), b in self.blocks.items()}, self.odd)


class Block:
    """Exact l-site block: sector table, kron-to-sector permutation, operator builders."""

    def __init__(self, nsites):
        self.nsites = nsites
        dim = 4 ** nsites
        # site occupations of every kron index (first site is the most significant base-4 digit)
        digits = np.array([[(k // 4 ** (nsites - 1 - i)) % 4 for i in range(nsites)] for k in range(dim)],
                          dtype=np.int64).reshape(dim, nsites)
        nup = SITE_UP_OF[digits].sum(axis=1)
        ndn = SITE_DN_OF[digits].sum(axis=1)
        fock = np.zeros(dim, dtype=np.int64)
        for i in range(nsites):
            fock |= digits[:, i] << (2 * i)
        self.sectors = sorted(set(zip(nup.tolist(), ndn.tolist())))
        self.sector_index = {q: k for k, q in enumerate(self.sectors)}
        self.perm = []          # kron indices of the states of each sector, in Fock order
        for q in self.sectors:
            ks = np.nonzero((nup == q[0]) & (ndn == q[1]))[0]
            ks = ks[np.argsort(fock[ks])]
            self.perm.append(ks)
        self.dims = [len(p) for p in self.perm]
        self.fock = fock
        self.digits = digits

    def kron_op(self, site_ops):
        """Dense 4^l x 4^l matrix of a product of site matrices (list of length l)."""
        out = np.array([[1.0]])
        for m in site_ops:
            out = np.kron(out, m)
        return out

    def site_fermion(self, i, sigma, dagger):
        """c^dag_{i sigma} (dagger=True) or c_{i sigma} as a dense block matrix with its JW string."""
        cd = SITE_CDAG_UP if sigma == 0 else SITE_CDAG_DN
        m = cd if dagger else cd.T
        ops = [SITE_P] * i + [m] + [np.eye(4)] * (self.nsites - i - 1)
        return self.kron_op(ops)

    def site_number(self, i, sigma):
        ops = [np.eye(4)] * self.nsites
        ops[i] = SITE_NUP if sigma == 0 else SITE_NDN
        return self.kron_op(ops)

    def parity(self):
        return self.kron_op([SITE_P] * self.nsites)

    def to_sectors(self, dense, odd, tol=0.0):
        """Cut a dense block matrix into its nonzero sector blocks."""
        blocks = {}
        for a, pa in enumerate(self.perm):
            for b, pb in enumerate(self.perm):
                blk = dense[np.ix_(pa, pb)]
                if np.any(np.abs(blk) > tol):
                    blocks[(a, b)] = blk.astype(complex)
        return BlockOp(blocks, odd)

    def hubbard_h(self, hop, U):
        """Block Hamiltonian sum_{ij in block} hop_ij c^dag_i c_j + U sum_i n_up n_dn (dense)."""
        n = self.nsites
        dim = 4 ** n
        h = np.zeros((dim, dim))
        for i in range(n):
            h += U * self.site_number(i, 0) @ self.site_number(i, 1)
            for j in range(n):
                if hop[i, j] != 0.0:
                    for s in (0, 1):
                        h += hop[i, j] * self.site_fermion(i, s, True) @ self.site_fermion(j, s, False)
        return h


class Cut:
    """Exact superblock of an L-site lattice cut into sites 0..l-1 (left) and l..L-1 (right)."""

    def __init__(self, hop, U, lsites):
        self.hop = np.asarray(hop, dtype=float)
        self.U = U
        self.nsites = self.hop.shape[0]
        self.lsites = lsites
        self.left = Block(lsites)
        self.right = Block(self.nsites - lsites)

    def block_h(self, side):
        if side == 0:
            h = self.hop[: self.lsites, : self.lsites]
            return self.left.to_sectors(self.left.hubbard_h(h, self.U), odd=False)
        h = self.hop[self.lsites:, self.lsites:]
        return self.right.to_sectors(self.right.hubbard_h(h, self.U), odd=False)

    def fermion(self, site, sigma, dagger):
        """c^dag / c of a lattice site as an operator of the block that holds it: (side, BlockOp)."""
        if site < self.lsites:
            return 0, self.left.to_sectors(self.left.site_fermion(site, sigma, dagger), odd=True)
        k = site - self.lsites
        return 1, self.right.to_sectors(self.right.site_fermion(k, sigma, dagger), odd=True)

    def number(self, site, sigma):
        if site < self.lsites:
            return 0, self.left.to_sectors(self.left.site_number(site, sigma), odd=False)
        k = site - self.lsites
        return 1, self.right.to_sectors(self.right.site_number(k, sigma), odd=False)

    def double_occ(self, site):
        blk = self.left if site < self.lsites else self.right
        k = site if site < self.lsites else site - self.lsites
        side = 0 if site < self.lsites else 1
        return side, blk.to_sectors(blk.site_number(k, 0) @ blk.site_number(k, 1), odd=False)

    def connections(self):
        """Hopping terms across the cut as fermionic products (coeff, A_left, B_right).

        For a bond (i in L, j in R) with amplitude h_ij:
            h_ij (c^dag_i c_j + c^dag_j c_i) = h_ij c^dag_i c_j - h_ij c_i c^dag_j,
        each written with the left operator first (anticommuting c^dag_j past c_i).
        """
        terms = []
        for i in range(self.lsites):
            for j in range(self.lsites, self.nsites):
                hij = self.hop[i, j]
                if hij == 0.0:
                    continue
                for s in (0, 1):
                    _, cd_i = self.fermion(i, s, True)
                    _, c_j = self.fermion(j, s, False)
                    _, c_i = self.fermion(i, s, False)
                    _, cd_j = self.fermion(j, s, True)
                    terms.append((hij, cd_i, c_j))
                    terms.append((-hij, c_i, cd_j))
        return terms
