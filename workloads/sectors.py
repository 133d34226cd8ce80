"""Gaussian sector model of a truncated DMRG superblock (seeded).

A left block is a renormalised block of l_b sites keeping m states, tensored
with one explicit site; the right block mirrors it.  The renormalised block
holds sectors (n_up, n_dn) with n_sigma within +-5 of l_b/2 and dimension
proportional to exp(-((n_up - l_b/2)^2 + (n_dn - l_b/2)^2) / 8), rounded and at
least 1, summing to about m.  Tensoring with one site (states 0, up, dn, updn)
gives the block sector table.

Operators drawn here:
  H_L, H_R      block diagonal, each sector block Hermitian (complex Gaussian),
                scaled so that the spectrum spans about +-l (2t + U/4);
  c^dag_{i s}   on the left, one per bond and spin: blocks (q + e_s <- q),
                complex Gaussian with variance 1/d_in; the annihilator is its
                conjugate transpose;
  c_{j s}       on the right, likewise with blocks (r - e_s <- r);
  n_op          diagonal number-like observables with entries in [0, 1].
Wave functions are complex Gaussian, normalised.  Seed: 11035391 + config index.
"""
import numpy as np

SEED_BASE = 11035391


def gaussian_block_sectors(lb, m, spread=5, width=8.0):
    """Sector table of a renormalised l_b-site block with about m states."""
    c = lb / 2.0
    lo, hi = int(np.floor(c)) - spread, int(np.floor(c)) + spread
    lo, hi = max(lo, 0), min(hi, lb)
    qs, ws = [], []
    for a in range(lo, hi + 1):
        for b in range(lo, hi + 1):
            qs.append((a, b))
            ws.append(np.exp(-((a - c) ** 2 + (b - c) ** 2) / width))
    ws = np.array(ws) / np.sum(ws) * m
    dims = np.maximum(1, np.rint(ws)).astype(int)
    return qs, dims.tolist()


def tensor_site(qs, dims):
    """Sector table of (block) x (one site); sectors sorted lexicographically."""
    acc = {}
    for (a, b), d in zip(qs, dims):
        for su, sd in ((0, 0), (1, 0), (0, 1), (1, 1)):
            key = (a + su, b + sd)
            acc[key] = acc.get(key, 0) + d
    keys = sorted(acc)
    return keys, [acc[k] for k in keys]


class SyntheticSuperblock:
    """Container of one synthetic superblock problem (all arrays complex128 / int)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    def sector_size(self, Q):
        ridx = {q: k for k, q in enumerate(self.rsec)}
        n = 0
        for qi, q in enumerate(self.lsec):
            ri = ridx.get((Q[0] - q[0], Q[1] - q[1]))
            if ri is not None:
                n += self.ldim[qi] * self.rdim[ri]
        return n


def _cgauss(rng, shape, scale=1.0):
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _hermitian_blocks(rng, sec, dims, radius):
    out = {}
    for k, d in enumerate(dims):
        X = _cgauss(rng, (d, d))
        Hq = (X + X.conj().T) / 2.0
        # GUE with unit-variance entries has spectral radius ~ 2 sqrt(d)
        out[(k, k)] = Hq * (radius / (2.0 * np.sqrt(d)))
    return out


def _shift_blocks(rng, sec, dims, shift):
    """Random blocks of an operator mapping sector q to q + shift (both present)."""
    idx = {q: k for k, q in enumerate(sec)}
    out = {}
    for k, q in enumerate(sec):
        qo = (q[0] + shift[0], q[1] + shift[1])
        ko = idx.get(qo)
        if ko is None:
            continue
        out[(ko, k)] = _cgauss(rng, (dims[ko], dims[k]), 1.0 / np.sqrt(dims[k]))
    return out


def _diag_blocks(rng, dims):
    return {(k, k): np.diag(rng.uniform(0.0, 1.0, d)).astype(complex) for k, d in enumerate(dims)}


def make_synthetic(L, m, U, t=1.0, nbonds=1, seed=SEED_BASE, N=None):
    """Synthetic superblock of an L-site lattice (half filling) with nbonds bonds across the cut.

    Returns a SyntheticSuperblock with fields:
      lsec, ldim, rsec, rdim        sector tables (sorted)
      HL, HR                        {(q_out, q_in): block}
      cdagL[b][s], cR[b][s]         creation op on the left / annihilation op on the right, bond b, spin s
      coeff_t                       hopping amplitude (-t)
      Q0, Q1                        ground-state sector (N, N) and excited sector (N+1, N)
      psi_gs (in Q0), phi (in Q1)   random normalised wave functions
      cdag_exc                      right-block creation op c^dag_{j up} of the first right site
      nL, nR                        diagonal number-like observables on each side
    """
    rng = np.random.default_rng(seed)
    half = L // 2
    lb = half - 1
    bq, bd = gaussian_block_sectors(lb, m)
    lsec, ldim = tensor_site(bq, bd)
    rsec, rdim = list(lsec), list(ldim)
    radius = half * (2.0 * t + U / 4.0)
    HL = _hermitian_blocks(rng, lsec, ldim, radius)
    HR = _hermitian_blocks(rng, rsec, rdim, radius)
    cdagL = [[_shift_blocks(rng, lsec, ldim, (1, 0)), _shift_blocks(rng, lsec, ldim, (0, 1))] for _ in range(nbonds)]
    cR = [[_shift_blocks(rng, rsec, rdim, (-1, 0)), _shift_blocks(rng, rsec, rdim, (0, -1))] for _ in range(nbonds)]
    cdag_exc = _shift_blocks(rng, rsec, rdim, (1, 0))
    nL, nR = _diag_blocks(rng, ldim), _diag_blocks(rng, rdim)
    Nh = L // 2 if N is None else N
    ss = SyntheticSuperblock(lsec=lsec, ldim=ldim, rsec=rsec, rdim=rdim)
    Q0, Q1 = (Nh, Nh), (Nh + 1, Nh)
    psi = _cgauss(rng, ss.sector_size(Q0)); psi /= np.linalg.norm(psi)
    phi = _cgauss(rng, ss.sector_size(Q1)); phi /= np.linalg.norm(phi)
    ss.__dict__.update(HL=HL, HR=HR, cdagL=cdagL, cR=cR, coeff_t=-t, Q0=Q0, Q1=Q1, psi_gs=psi, phi=phi,
                       cdag_exc=cdag_exc, nL=nL, nR=nR, L=L, m=m, U=U, nbonds=nbonds, seed=seed)
    return ss


def chain_config(L=32, m=400, U=4.0, index=1):
    """1D Hubbard chain at half filling, one bond across the central cut."""
    return make_synthetic(L, m, U, nbonds=1, seed=SEED_BASE + index)


def ladder_config(Lx=16, m=800, U=8.0, index=2):
    """Two-leg ladder 2 x Lx at half filling, two leg bonds across the central cut."""
    return make_synthetic(2 * Lx, m, U, nbonds=2, seed=SEED_BASE + index)
