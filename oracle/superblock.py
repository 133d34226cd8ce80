"""Superblock L u R with (N_up, N_dn) sectors and the sector-pair H psi (oracle; test infrastructure).

The wave function of a superblock sector Q is the matrix Psi[alpha, beta],
alpha in L, beta in R, split by the left quantum number q (Eq. rdensitymatrix
labels alpha, beta; Sec. II.B).  Storage: for ascending q (lexicographic) with
partner r = Q - q present on the right, the block Psi_q of shape
dL(q) x dR(r) row-major; the blocks are concatenated into one complex vector.

A superblock term is a fermionic product coeff * A_L B_R of a left-block
operator A and a right-block operator B (either may be the identity).  In the
basis |alpha>|beta> = (L string)(R string)|0>, moving an odd B_R past the left
string costs (-1)^{N_L}, so the term acts as coeff * (A P_L) (x) B, with
P_L = diag((-1)^{n_up+n_dn}) on the left block; for a sector block this is
    Psi'_{q_out} += coeff * s(q_in) * A[q_out <- q_in] Psi_{q_in} B[r_out <- r_in]^T
with s(q_in) = (-1)^{N(q_in)} when B is odd, else 1.  H psi is the sum over
H_L (x) 1, 1 (x) H_R and the connection terms across the cut, which is the
"Hamiltonian connections" computation of Sec. IV.
"""
import numpy as np


class Superblock:
    """Sector tables of the two blocks: lists of (n_up, n_dn) and dims."""

    def __init__(self, lsec, ldim, rsec, rdim):
        self.lsec = [tuple(q) for q in lsec]
        self.rsec = [tuple(q) for q in rsec]
        self.ldim = list(ldim)
        self.rdim = list(rdim)
        self.lidx = {q: k for k, q in enumerate(self.lsec)}
        self.ridx = {q: k for k, q in enumerate(self.rsec)}

    def pairs(self, Q):
        """[(q index, r index, offset, dL, dR)] in storage order for sector Q."""
        out, off = [], 0
        for qi in sorted(range(len(self.lsec)), key=lambda k: self.lsec[k]):
            q = self.lsec[qi]
            r = (Q[0] - q[0], Q[1] - q[1])
            ri = self.ridx.get(r)
            if ri is None:
                continue
            dl, dr = self.ldim[qi], self.rdim[ri]
            out.append((qi, ri, off, dl, dr))
            off += dl * dr
        return out

    def size(self, Q):
        return sum(p[3] * p[4] for p in self.pairs(Q))

    def blocks_of(self, Q, psi):
        """dict q index -> view of Psi_q."""
        return {qi: psi[off: off + dl * dr].reshape(dl, dr) for qi, ri, off, dl, dr in self.pairs(Q)}


def left_parity(sb, qi):
    n = sb.lsec[qi][0] + sb.lsec[qi][1]
    return -1.0 if n % 2 else 1.0


def apply_terms(sb, terms, Q_in, psi, Q_out):
    """sum_k coeff_k (A_k P_L^{odd(B_k)}) (x) B_k applied to psi in sector Q_in, result in Q_out.

    terms: list of (coeff, A or None, B or None); None is the identity.
    """
    pin = sb.blocks_of(Q_in, psi)
    pairs_out = sb.pairs(Q_out)
    out = np.zeros(sb.size(Q_out), dtype=complex)
    oblk = {qi: out[off: off + dl * dr].reshape(dl, dr) for qi, ri, off, dl, dr in pairs_out}
    out_r = {qi: ri for qi, ri, off, dl, dr in pairs_out}
    for qi, ri, off, dl, dr in sb.pairs(Q_in):
        X = pin[qi]
        for coeff, A, B in terms:
            sign = left_parity(sb, qi) if (B is not None and B.odd) else 1.0
            a_list = [(qi, None)] if A is None else [(qo, blk) for (qo, qq), blk in A.blocks.items() if qq == qi]
            b_list = [(ri, None)] if B is None else [(ro, blk) for (ro, rr), blk in B.blocks.items() if rr == ri]
            for qo, ablk in a_list:
                if qo not in oblk:
                    continue
                for ro, bblk in b_list:
                    if out_r[qo] != ro:
                        continue
                    Y = X if ablk is None else ablk @ X
                    Y = Y if bblk is None else Y @ bblk.T
                    oblk[qo] += coeff * sign * Y
    return out


def hamiltonian_terms(HL, HR, conns):
    """Term list of H = H_L (x) 1 + 1 (x) H_R + sum_k coeff_k A_k B_k."""
    terms = []
    if HL is not None:
        terms.append((1.0, HL, None))
    if HR is not None:
        terms.append((1.0, None, HR))
    terms.extend(conns)
    return terms


def apply_h(sb, HL, HR, conns, Q, psi):
    return apply_terms(sb, hamiltonian_terms(HL, HR, conns), Q, psi, Q)


def apply_op(sb, A, B, Q_in, psi, Q_out):
    """Excitation operator (A P_L^{odd(B)}) (x) B (Eq. b with one or two local factors)."""
    return apply_terms(sb, [(1.0, A, B)], Q_in, psi, Q_out)


def expect(sb, A, B, Q, psi):
    """<psi| A B |psi> / <psi|psi> for a sector-preserving product."""
    y = apply_op(sb, A, B, Q, psi, Q)
    return np.vdot(psi, y) / np.vdot(psi, psi).real


# ---------------------------------------------------------------- brute force
def dense_op(sb, A, side):
    """Full dense matrix of a block operator over the whole block basis (sector order)."""
    dims = sb.ldim if side == 0 else sb.rdim
    offs = np.concatenate([[0], np.cumsum(dims)])
    M = np.zeros((offs[-1], offs[-1]), dtype=complex)
    for (qo, qi), blk in A.blocks.items():
        M[offs[qo]: offs[qo + 1], offs[qi]: offs[qi + 1]] = blk
    return M


def dense_parity(sb):
    return np.concatenate([[left_parity(sb, qi)] * d for qi, d in enumerate(sb.ldim)])


def superblock_index(sb, Q):
    """Flat indices, in the full kron(L, R) basis, of the entries of the sector-Q vector."""
    loff = np.concatenate([[0], np.cumsum(sb.ldim)])
    roff = np.concatenate([[0], np.cumsum(sb.rdim)])
    DR = roff[-1]
    idx = []
    for qi, ri, off, dl, dr in sb.pairs(Q):
        a = loff[qi] + np.arange(dl)
        b = roff[ri] + np.arange(dr)
        idx.append((a[:, None] * DR + b[None, :]).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def dense_terms(sb, terms, Q_in, Q_out):
    """Dense matrix of sum_k coeff_k (A P_L^odd) kron B restricted to Q_out x Q_in (np.kron)."""
    DL, DR = sum(sb.ldim), sum(sb.rdim)
    P = np.diag(dense_parity(sb))
    M = np.zeros((DL * DR, DL * DR), dtype=complex)
    for coeff, A, B in terms:
        a = np.eye(DL) if A is None else dense_op(sb, A, 0)
        b = np.eye(DR) if B is None else dense_op(sb, B, 1)
        if B is not None and B.odd:
            a = a @ P
        M += coeff * np.kron(a, b)
    io, ii = superblock_index(sb, Q_out), superblock_index(sb, Q_in)
    return M[np.ix_(io, ii)]


# ---------------------------------------------------------------- ED mapping
def fock_to_psi(cut, sector, vec):
    """Map an ED sector vector (Fock basis) onto the sector-blocked Psi of the exact cut.

    Both bases are the canonical Fock order of the lattice, so this is a pure
    permutation (no signs): Fock state s = s_L | (s_R << 2 l).
    """
    L, R = cut.left, cut.right
    sb = exact_superblock(cut)
    Q = (sector.nup, sector.ndn)
    pos = {}
    for qi, ri, off, dl, dr in sb.pairs(Q):
        pos[qi] = (off, dr)
    lmask = (1 << (2 * cut.lsites)) - 1
    lloc = _local_index(L)
    rloc = _local_index(R)
    out = np.zeros(sb.size(Q), dtype=complex)
    for k, s in enumerate(sector.states):
        s = int(s)
        qa, a = lloc[s & lmask]
        qb, b = rloc[s >> (2 * cut.lsites)]
        off, dr = pos[qa]
        out[off + a * dr + b] = vec[k]
    return out


def _local_index(block):
    """Fock bits of a block state -> (sector index, index within sector)."""
    m = {}
    for qi, ks in enumerate(block.perm):
        for a, k in enumerate(ks):
            m[int(block.fock[k])] = (qi, a)
    return m


def exact_superblock(cut):
    return Superblock(cut.left.sectors, cut.left.dims, cut.right.sectors, cut.right.dims)
