"""Finite DMRG sweeps with time-step targeting on the device (Sec. I; Sec. II.B-II.D), driven through
the C ABI of libtdmrg.  Every arithmetic step (ground state, excitation, Krylov advance, reduced density
matrix, its eigendecomposition, truncation, renormalisation, enlargement, wave-function transformation,
observables) runs in the library's kernels; this module keeps the block tables (host) and the blocks'
device buffers (torch tensors) and calls the entry points in the order of the method.

A kept block K (Block) holds its sector table, H_K and the edge-site c^dag_s as device sector blocks,
and -- when it was cut from an enlarged block -- its states in that block's basis (V, the layout of
tdmrg_rho_eig) with the kept counts, which the wave-function transformation needs.  Enlarged blocks
(Enlarged) add the new site's densities.  Operator ids inside a superblock context: 0 = H, 10 + s =
c^dag_{edge s}, 30 + s = its adjoint, 50 + s = n_{edge s}; the boundary terms are -t c^dag_L c_R and
+t c_L c^dag_R per spin and bond.

Ladders (Sec. III: the 8 x 2 ladder of Fig. 2, the 2 x 4 ladders of Figs. 3-4; Lattice): sites i = 2x + y
in rung-first order, site i bonds to i - 1 across a rung when i is odd and to i - 2 along a leg, so a block
also carries c^dag of its second site from the edge (20 + s, adjoint 40 + s), the enlargement bonds the
new site to both (tdmrg_enlarge_bonds) and the central cut is crossed by two legs and, when the left
enlarged block ends on the first site of a rung, by that rung.

Excitation (Eq. b): phi = B_{b-1} ... B_0 psi with local c^dag / c operators on sites in the order the
sweep reaches them; B_i is applied at the first step whose central pair of sites (l, the new site of the
left enlarged block, and l + 1, the new site of the right one) holds its site.  Before B_0 only the
ground state is targeted; while the product is partial it takes the places of all n_v targets; at the
step that completes it the targets phi(t_x) are built.

Start: the stored blocks of an infinite-system DMRG, on the device (`infinite`) or from elsewhere.

Schedule of one sweep (the paper leaves it open): from the centre of the chain move right to the right
end (right block of one site), left to the left end, and right back to the centre; the targets advance by
tau at every `advance_every`-th step after the one that completed phi (Sec. II.C: the targets are
wave-function transformed at every other step).
"""
import numpy as np
import torch

from . import tdmrg as T

H_ID, CDAG_ID, CDAG2_ID, C_ID, C2_ID, N_ID = 0, 10, 20, 30, 40, 50


def _zeros(n, dev):
    return torch.zeros(max(int(n), 1), dtype=torch.complex128, device=dev)


class Lattice:
    """Bonds of the lattice (host tables): the open chain (legs = 1, hopping t_leg between neighbours) or
    the two-leg ladder with rung-first labels (legs = 2).  An even number of sites makes the ladder
    symmetric under reflection i -> N - 1 - i (which exchanges the legs), so a right block of r sites bonds
    like a left block of r sites."""

    def __init__(self, legs=1, t_leg=1.0, t_rung=1.0):
        if legs not in (1, 2):
            raise ValueError("Lattice: legs must be 1 (chain) or 2 (ladder)")
        self.legs, self.t_leg, self.t_rung = legs, float(t_leg), float(t_rung)

    def new_site_bonds(self, k):
        """Hoppings of a new site with k sites between it and the block's open end to the block's edge
        site and to its second site from the edge."""
        if self.legs == 1:
            return (self.t_leg if k >= 1 else 0.0), 0.0
        return (self.t_rung if k % 2 == 1 else 0.0), (self.t_leg if k >= 2 else 0.0)

    def cut_bonds(self, l):
        """(left edge index, right edge index, hopping) of the bonds between the left enlarged block (sites
        0..l) and the right one; edge 0 is the site at the cut, edge 1 the next one."""
        if self.legs == 1:
            return [(0, 0, self.t_leg)]
        return ([(0, 0, self.t_rung)] if l % 2 == 0 else []) + [(1, 0, self.t_leg), (0, 1, self.t_leg)]


class Block:
    """A kept block on the device."""

    def __init__(self, qn, dim, H, cdag, V=None, kept_V=None, nsites=None, cdag2=None):
        self.qn = [tuple(int(x) for x in q) for q in qn]
        self.dim = [int(x) for x in dim]
        self.H = H            # (block quantum numbers, device data)
        self.cdag = cdag      # [(qns, data), (qns, data)] for up, down
        self.V = V            # its states in the enlarged block it was cut from (tdmrg_rho_eig layout), or None
        self.kept_V = kept_V  # kept counts per sector of that enlarged block
        self.nsites = nsites  # sites in the block (needed on a ladder)
        self.cdag2 = cdag2    # ladder: c^dag of the second site from the edge, like cdag; None on a chain


class Enlarged:
    """K + site or site + K on the device, with the new site's densities."""

    def __init__(self, qn, dim, H, cdag, n, nsites=None, cdag2=None):
        self.qn, self.dim, self.H, self.cdag, self.n = qn, dim, H, cdag, n
        self.nsites, self.cdag2 = nsites, cdag2


def enlarge(ctx, blk, side, t, U, dev, lattice=None):
    """blk + site (side 0) or site + blk (side 1).  Chain: the bond -t between blk's edge and the new site.
    lattice: the new site's bonds from it; on a ladder blk's edge is carried as the second site from the
    enlarged block's edge."""
    qn, dim, nb, ent = T.tdmrg_enlarge_size(side, blk.qn, blk.dim)
    qn = [tuple(int(x) for x in q) for q in qn]
    dim = [int(x) for x in dim]
    H = _zeros(ent[0], dev)
    cd = [_zeros(ent[1 + s], dev) for s in range(2)]
    n = [_zeros(ent[0], dev) for _ in range(2)]
    hq = [q + q for q in qn]
    nsites = None if blk.nsites is None else blk.nsites + 1
    if lattice is None or lattice.legs == 1:
        tb = t if lattice is None else lattice.new_site_bonds(blk.nsites if blk.nsites is not None else 1)[0]
        cq = T.tdmrg_enlarge(ctx, side, blk.qn, blk.dim, blk.H, blk.cdag, tb, U, H, cd, n)
        return Enlarged(qn, dim, (hq, H), [(cq[s], cd[s]) for s in range(2)], [(hq, n[s]) for s in range(2)], nsites)
    t0, t1 = lattice.new_site_bonds(blk.nsites)
    edges, ts = [blk.cdag], [t0]
    if blk.cdag2 is not None:
        edges.append(blk.cdag2)
        ts.append(t1)
    carry = [_zeros(ent[1 + s], dev) for s in range(2)]
    cq = T.tdmrg_enlarge_bonds(ctx, side, blk.qn, blk.dim, blk.H, edges, ts, U, H, cd, n, carry)
    return Enlarged(qn, dim, (hq, H), [(cq[s], cd[s]) for s in range(2)], [(hq, n[s]) for s in range(2)], nsites,
                    [(cq[s], carry[s]) for s in range(2)])


def load(ctx, Lenl, Renl, t, lattice=None, l=None):
    """The superblock (Lenl, Renl) with the Hubbard bonds across the cut: the one between the two edge sites
    (hopping t) without a lattice, else the lattice's bonds at the cut after site l."""
    for side, b in enumerate((Lenl, Renl)):
        T.tdmrg_set_block(ctx, side, b.qn, b.dim)
    for side, b in enumerate((Lenl, Renl)):
        T.tdmrg_set_op_device(ctx, side, H_ID, 0, *b.H)
        for s in range(2):
            T.tdmrg_set_op_device(ctx, side, CDAG_ID + s, 1, *b.cdag[s])
            T.tdmrg_set_op_adjoint(ctx, side, C_ID + s, CDAG_ID + s)
            T.tdmrg_set_op_device(ctx, side, N_ID + s, 0, *b.n[s])
            if b.cdag2 is not None:
                T.tdmrg_set_op_device(ctx, side, CDAG2_ID + s, 1, *b.cdag2[s])
                T.tdmrg_set_op_adjoint(ctx, side, C2_ID + s, CDAG2_ID + s)
    bonds = [(0, 0, t)] if lattice is None else [x for x in lattice.cut_bonds(l) if x[2] != 0.0]
    cd_id = lambda e: CDAG_ID if e == 0 else CDAG2_ID
    c_id = lambda e: C_ID if e == 0 else C2_ID
    conns = [(cd_id(eL) + s, c_id(eR) + s, -tb) for eL, eR, tb in bonds for s in range(2)]
    conns += [(c_id(eL) + s, cd_id(eR) + s, tb) for eL, eR, tb in bonds for s in range(2)]
    T.tdmrg_set_hamiltonian(ctx, H_ID, H_ID, conns)


def _kept_blocks(qns, kept_of):
    """Blocks of an operator that survive the truncation (both sectors kept), in the order they were set."""
    return [q for q in qns if kept_of.get(tuple(q[:2]), 0) > 0 and kept_of.get(tuple(q[2:]), 0) > 0]


def truncate_block(ctx, side, enl, states, weights, m, real_basis, dev):
    """Reduced density matrix of one block of the superblock in ctx from the weighted targets, its
    eigendecomposition and the m-state truncation, then H and the edge c^dag renormalised into the kept
    basis.  Returns (Block K, host record {kept, evals, discarded}, U)."""
    nr, ne = T.tdmrg_rho_size(ctx, side)
    rho = _zeros(nr, dev)
    T.tdmrg_set_real_basis(ctx, real_basis)
    evals = torch.zeros(ne, dtype=torch.float64, device=dev)
    U = _zeros(nr, dev)
    T.tdmrg_density_eig(ctx, states, weights, rho, evals, U, side=side)
    kept_d = torch.zeros(len(enl.dim), dtype=torch.int32, device=dev)
    disc = torch.zeros(1, dtype=torch.float64, device=dev)
    T.tdmrg_truncate(ctx, evals, m, kept_d, disc, side=side)
    kept = [int(x) for x in kept_d.cpu().numpy()]
    kept_of = dict(zip(enl.qn, kept))
    kq = [q for q, k in zip(enl.qn, kept) if k > 0]
    kd = [k for k in kept if k > 0]
    ops = []
    todo = [(H_ID, enl.H[0]), (CDAG_ID, enl.cdag[0][0]), (CDAG_ID + 1, enl.cdag[1][0])]
    if enl.cdag2 is not None:
        todo += [(CDAG2_ID, enl.cdag2[0][0]), (CDAG2_ID + 1, enl.cdag2[1][0])]
    for op_id, qns in todo:
        out = _zeros(sum(enl.dim[enl.qn.index(tuple(q[:2]))] * enl.dim[enl.qn.index(tuple(q[2:]))] for q in qns), dev)
        nb = T.tdmrg_renormalize_op(ctx, side, op_id, U, kept, out)
        kb = _kept_blocks(qns, kept_of)
        assert nb == len(kb)
        ops.append((kb, out))
    K = Block(kq, kd, ops[0], ops[1:3], V=U, kept_V=kept, nsites=enl.nsites,
              cdag2=ops[3:5] if enl.cdag2 is not None else None)
    ev = evals.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(enl.dim)])
    rec = {"kept": kept, "evals": [ev[off[i]: off[i + 1]] for i in range(len(enl.dim))],
           "discarded": float(disc.cpu().numpy()[0])}
    return K, rec, U


def site_block(ctx, U, dev, lattice=None):
    """One Hubbard site as a Block, made on the device: the one-state vacuum block (sector (0, 0), H = 0,
    no c^dag blocks) enlarged by a site, so H = U n_up n_dn and c^dag_s are the site's (on a ladder with a
    zero second edge)."""
    vac = Block([(0, 0)], [1], ([], _zeros(1, dev)), [([], _zeros(1, dev)), ([], _zeros(1, dev))], nsites=0)
    e = enlarge(ctx, vac, 0, 0.0, U, dev, lattice)
    return Block(e.qn, e.dim, e.H, e.cdag, nsites=1, cdag2=e.cdag2)


def infinite(L, t, U, m, lattice=None, device=None, gs_nk=32, gs_restarts=40):
    """Infinite-system DMRG on the device (Sec. I): both blocks grow by one site per step; the superblock
    of 2l + 2 sites (l sites per block, the lattice's bonds at the cut after site l) at half filling, its
    ground state by restarted Lanczos from a seeded vector, and both enlarged blocks cut to their m most
    probable states (rho_L and rho_R of the ground state alone).  On a ladder the rung-first labels make
    every intermediate superblock a ladder of l + 1 rungs and the right block the reflection of the left
    one.  Returns ({sites: left Block}, {sites: right Block}, [(superblock sites, energy)]); the blocks of
    two or more sites carry their states in the enlarged block they were cut from, as TSTSweep needs."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    mk = lambda: T.tdmrg_create(device=dev.index, stream=torch.cuda.current_stream(dev).cuda_stream,
                                nk_max=max(32, gs_nk), prec=T.TDMRG_FP64)
    work, cur = mk(), mk()
    try:
        site = site_block(work, U, dev, lattice)
        left, right, energies = {1: site}, {1: site}, []
        l = 1
        while 2 * l + 2 <= L:
            Lenl = enlarge(work, left[l], 0, t, U, dev, lattice)
            Renl = enlarge(work, right[l], 1, t, U, dev, lattice)
            load(cur, Lenl, Renl, t, lattice, l)
            Q = (l + 1, l + 1)
            n = T.tdmrg_sector_size(cur, Q)
            g = torch.Generator().manual_seed(11035391 + l)
            psi = torch.complex(torch.randn(n, generator=g, dtype=torch.float64),
                                torch.randn(n, generator=g, dtype=torch.float64)).to(dev)
            energies.append((2 * l + 2, T.tdmrg_ground_state(cur, Q, psi, gs_nk, gs_restarts)))
            left[l + 1], _, _ = truncate_block(cur, 0, Lenl, [(Q, psi)], [1.0], m, False, dev)
            right[l + 1], _, _ = truncate_block(cur, 1, Renl, [(Q, psi)], [1.0], m, False, dev)
            l += 1
        return left, right, energies
    finally:
        for c in (work, cur):
            T.tdmrg_destroy(c)


class TSTSweep:
    """One finite sweep of the L-site Hubbard chain or two-leg ladder (half filling) with time-step
    targeting, on the device.

    left, right: dicts {number of sites: Block} of the stored blocks the sweep starts from (each block of
    two or more sites with its V and kept counts); they are replaced by the blocks the sweep makes."""

    def __init__(self, L, t, U, m, left, right, n_v=4, tau=0.1, nk=12, advance_every=2, gs_nk=32, gs_restarts=40,
                 real_basis=False, device=None, excitations=None, prec=None, ozaki_slices=4, lattice=None):
        """prec: arithmetic of the superblock products (T.TDMRG_FP64, the default, or T.TDMRG_OZAKI_BF16
        with ozaki_slices slices); everything else stays FP64.  lattice: a Lattice (default: the chain with
        hopping t); on a ladder every stored block carries its nsites and cdag2."""
        self.L, self.t, self.U, self.m = L, t, U, m
        self.lattice = lattice
        self.prec = T.TDMRG_FP64 if prec is None else prec
        self.ozaki_slices = ozaki_slices
        self.left, self.right = dict(left), dict(right)
        self.n_v, self.tau, self.nk, self.advance_every = n_v, tau, nk, advance_every
        self.gs_nk, self.gs_restarts = gs_nk, gs_restarts
        self.real_basis = real_basis
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.times = [x * tau / (n_v - 1) for x in range(n_v)]
        self.w_gs, self.w = T.tdmrg_tst_weights(n_v)
        # excitations: [(site, 'cdag' | 'c', sigma)] in sweep order; [] targets the ground state alone (a
        # finite DMRG sweep); None: c^dag_{L/2, up}
        self.excitations = list(excitations) if excitations is not None else [(L // 2, "cdag", 0)]

    def path(self):
        h, L = self.L // 2 - 1, self.L
        p = [(l, "R") for l in range(h, L - 3)] + [(l, "L") for l in range(L - 3, 1, -1)] + [(l, "R") for l in range(1, h)]
        return p + [(h, None)]

    def _ctx(self):
        return T.tdmrg_create(device=self.dev.index, stream=torch.cuda.current_stream(self.dev).cuda_stream,
                              nk_max=max(32, self.nk, self.gs_nk), prec=self.prec, ozaki_slices=self.ozaki_slices)

    def _observe(self, ctx, Q, x):
        n = T.tdmrg_sector_size(ctx, Q)
        out = _zeros(5, self.dev)
        hx = _zeros(n, self.dev)
        T.tdmrg_overlap_op(ctx, -1, -1, Q, x, Q, x, out[0:1])
        T.tdmrg_apply_h(ctx, Q, x, hx)
        T.tdmrg_overlap_op(ctx, -1, -1, Q, x, Q, hx, out[1:2])
        T.tdmrg_expect(ctx, N_ID, -1, Q, x, out[2:3])
        T.tdmrg_expect(ctx, -1, N_ID, Q, x, out[3:4])
        T.tdmrg_expect(ctx, CDAG_ID, C_ID, Q, x, out[4:5])
        o = out.cpu().numpy()
        return {"norm2": o[0].real, "energy": o[1].real / o[0].real, "n_left": o[2], "n_right": o[3], "bond": o[4]}

    def run(self, psi0=None):
        """Runs the sweep; returns the per-step records (host)."""
        L, h = self.L, self.L // 2
        Q0, Q1 = (h, h), (h + 1, h)
        work, cur, nxt = self._ctx(), self._ctx(), self._ctx()
        records = []
        psi, targets, t_now = None, None, 0.0
        try:
            path = self.path()
            l0 = path[0][0]
            Lenl = enlarge(work, self.left[l0], 0, self.t, self.U, self.dev, self.lattice)
            Renl = enlarge(work, self.right[L - 2 - l0], 1, self.t, self.U, self.dev, self.lattice)
            load(cur, Lenl, Renl, self.t, self.lattice, l0)
            if psi0 is None:
                n0 = T.tdmrg_sector_size(cur, Q0)
                g = torch.Generator().manual_seed(11035391)
                psi = torch.complex(torch.randn(n0, generator=g, dtype=torch.float64),
                                    torch.randn(n0, generator=g, dtype=torch.float64)).to(self.dev)
            else:
                psi = psi0
            phi, Q1, pending, done_step = None, Q0, list(self.excitations), None
            for step, (l, move) in enumerate(path):
                r = L - 2 - l
                e = T.tdmrg_ground_state(cur, Q0, psi, self.gs_nk, self.gs_restarts)
                action = "ground" if phi is None else ("partial" if pending else "keep")
                applied = False
                while pending and pending[0][0] in (l, l + 1):   # operators of Eq. b reached here
                    site, kind, sigma = pending.pop(0)
                    op = (CDAG_ID if kind == "cdag" else C_ID) + sigma
                    opL, opR = (op, -1) if site == l else (-1, op)
                    dq = [0, 0]
                    dq[sigma] = 1 if kind == "cdag" else -1
                    Qn = (Q1[0] + dq[0], Q1[1] + dq[1])
                    out = _zeros(T.tdmrg_sector_size(cur, Qn), self.dev)
                    T.tdmrg_apply_op(cur, opL, opR, Q1, psi if phi is None else phi, Qn, out)
                    phi, Q1, applied = out, Qn, True
                if applied and not pending:
                    targets = [torch.empty_like(phi) for _ in range(self.n_v)]
                    T.tdmrg_evolve(cur, Q1, phi, self.times, self.nk, targets)
                    action, done_step = "excite", step
                elif applied:
                    targets, action = [phi] * self.n_v, "partial"
                elif done_step is not None and (step - done_step) % self.advance_every == 0:
                    new = [torch.empty_like(targets[0]) for _ in range(self.n_v)]
                    T.tdmrg_evolve(cur, Q1, targets[-1], self.times, self.nk, new)
                    targets = new
                    t_now += self.tau
                    action = "advance"
                rec = {"l": l, "move": move, "action": action, "t": t_now, "energy": e, "Q1": Q1,
                       "applied": len(self.excitations) - len(pending),
                       "targets": [self._observe(cur, Q1, x) for x in targets or []]}
                if move is not None:
                    if targets is None:   # before the first operator of Eq. b: the ground state alone
                        states, weights = [(Q0, psi)], [1.0]
                    else:
                        states = [(Q0, psi)] + [(Q1, x) for x in targets]
                        weights = [self.w_gs] + list(self.w)
                    side = 0 if move == "R" else 1
                    K, trec, Uk = truncate_block(cur, side, Lenl if side == 0 else Renl, states, weights, self.m,
                                                 self.real_basis, self.dev)
                    rec.update(trec)
                    if move == "R":
                        nL = enlarge(work, K, 0, self.t, self.U, self.dev, self.lattice)
                        nR = enlarge(work, self.right[r - 1], 1, self.t, self.U, self.dev, self.lattice)
                        load(nxt, nL, nR, self.t, self.lattice, l + 1)
                        Rb = self.right[r]
                        moved = []
                        for Q, v in states:
                            o = _zeros(T.tdmrg_sector_size(nxt, Q), self.dev)
                            T.tdmrg_wft_right(cur, Q, v, Uk, trec["kept"], Rb.V, Rb.kept_V, nxt, o)
                            moved.append(o)
                        self.left[l + 1] = K
                    else:
                        nL = enlarge(work, self.left[l - 1], 0, self.t, self.U, self.dev, self.lattice)
                        nR = enlarge(work, K, 1, self.t, self.U, self.dev, self.lattice)
                        load(nxt, nL, nR, self.t, self.lattice, l - 1)
                        Lb = self.left[l]
                        moved = []
                        for Q, v in states:
                            o = _zeros(T.tdmrg_sector_size(nxt, Q), self.dev)
                            T.tdmrg_wft_left(cur, Q, v, Uk, trec["kept"], Lb.V, Lb.kept_V, nxt, o)
                            moved.append(o)
                        self.right[r + 1] = K
                    psi = moved[0]
                    if targets is not None:
                        targets = moved[1:]
                        if pending:   # the partial product is every target
                            phi = targets[0]
                    Lenl, Renl = nL, nR
                    cur, nxt = nxt, cur
                records.append(rec)
        finally:
            for c in (work, cur, nxt):
                T.tdmrg_destroy(c)
        return records
