"""Time-step targeting during finite DMRG sweeps (oracle; test infrastructure only).

Sec. II.B-II.D: at every step of a finite sweep the ground state of the superblock is found first; then
the time targets are produced or carried over (the evolve call of Sec. II.D):
  - at the step where the centre first reaches the excitation site, phi = B psi (Eq. b) and the targets
    phi(t_x) = exp(-i H t_x) phi, x = 0..n_v-1 (Eq. lanczosevolution; t_0 = 0, t_{n_v-1} = tau);
  - at an advance step, the targets are rebuilt from the last one, phi(t + tau + t_x) =
    exp(-i H t_x) phi(t + tau) (Eq. lanczosevolution2), and the time moves on by tau;
  - at every other step the targets are only wave-function transformed (Sec. II.B, II.C);
then the reduced density matrix of the growing block is formed from the ground state and the targets with
the weights of Sec. II.C (2 Omega for the ground state and the first and last target, Omega for the
others, Omega = 1 / (n_v + 4)), the block is truncated to its m most probable states, and every target is
transported to the next superblock.

Excitation (Eq. b): phi = B_{b-1} ... B_1 B_0 psi with local operators (c^dag or c of one spin) on sites
in the order in which the sweep reaches them; B_i is applied at the first step whose central pair of
sites (the new site l of the left enlarged block, the new site l+1 of the right one) holds its site,
to the partial state transported so far.  Before B_0 only the ground state is targeted (weight 1); while
the product is partial, the partial state takes the places of all n_v time targets; at the step that
completes phi, the targets phi(t_x) are built.

Schedule (the reading of a silent paper): one finite sweep starting at the centre of the chain moving
right, turning at the right end (right block of one site) and at the left end (left block of one site),
and ending back at the centre; the time advances at every `advance_every`-th step after the one that
completed phi.  Per step the record
holds quantities that do not depend on the phases of eigenvectors (so that two implementations can be
compared): the ground-state energy, the kept counts, rho's eigenvalues and the discarded weight, and per
target its squared norm, <H>, the densities of the two central sites and the bond <c^dag_{l up} c_{l+1 up}>.
"""
import numpy as np

from . import density, dmrg, krylov, superblock


def sweep_path(L):
    """(left-block size l, move) of every step of one finite sweep from the centre: 'R', 'L', and a final
    ('R' ... ) step at the centre marked None (no move)."""
    h = L // 2 - 1
    path = [(l, "R") for l in range(h, L - 3)]
    path += [(l, "L") for l in range(L - 3, 1, -1)]
    path += [(l, "R") for l in range(1, h)]
    return path + [(h, None)]


def _delta(kind, sigma):
    d = [0, 0]
    d[sigma] = 1 if kind == "cdag" else -1
    return d


class TSTSweep:
    def __init__(self, d, m, n_v=4, tau=0.1, nk=12, advance_every=2, real_basis=False, gs_resid=1e-11,
                 excitations=None):
        """d: a ChainDMRG that has run (its blocks and their kept bases are the sweep's start); m: states
        kept per block during the sweep; gs_resid: the ground state's residual bound (the excitation and
        the ground-state target inherit its error to first order); excitations: [(site, 'cdag' | 'c',
        sigma)] in the order the sweep reaches them ([]: the ground state alone, a finite DMRG sweep; default
        c^dag_{L/2, up}, reached at once)."""
        self.gs_resid = gs_resid
        self.d, self.m, self.n_v, self.tau, self.nk = d, m, n_v, tau, nk
        self.advance_every = advance_every
        self.real_basis = real_basis
        self.times = krylov.target_times(tau, n_v)
        self.w_gs, self.w = density.tst_weights(n_v)
        self.excitations = list(excitations) if excitations is not None else [(d.L // 2, "cdag", 0)]

    def _blocks(self, l):
        d = self.d
        r = d.L - 2 - l
        Lenl = dmrg.enlarge(d.left[l], "L", d.t, d.U, d.geom)
        Renl = dmrg.enlarge(d.right[r], "R", d.t, d.U, d.geom)
        return Lenl, Renl, r

    @staticmethod
    def _local(Lenl, Renl, l, site, kind, sigma):
        """(A, B) of the superblock product for a local c^dag / c on site l (left edge) or l + 1 (right)."""
        blk = Lenl if site == l else Renl
        M = blk.cdag[sigma] if kind == "cdag" else blk.cdag[sigma].conj().T
        op = blk.blockop(M, True)
        return (op, None) if site == l else (None, op)

    def run(self):
        d = self.d
        h = d.L // 2
        Q0 = (h, h)
        records = []
        psi, targets, t_now = None, None, 0.0
        phi, Q1, pending, done_step = None, Q0, list(self.excitations), None
        for step, (l, move) in enumerate(sweep_path(d.L)):
            Lenl, Renl, r = self._blocks(l)
            sb, HL, HR, conns = dmrg.superblock_of(Lenl, Renl, d.t, d.geom)
            hq = lambda Q: (lambda v: superblock.apply_h(sb, HL, HR, conns, Q, v))
            e, psi = dmrg.ground_state(hq(Q0), sb.size(Q0), resid_tol=self.gs_resid)
            # the evolve call: apply the operators of Eq. b reached here, then excite, advance or keep
            action = "ground" if phi is None else ("partial" if pending else "keep")
            applied = False
            while pending and pending[0][0] in (l, l + 1):
                site, kind, sigma = pending.pop(0)
                A, B = self._local(Lenl, Renl, l, site, kind, sigma)
                src = psi if phi is None else phi
                dq = _delta(kind, sigma)
                Qn = (Q1[0] + dq[0], Q1[1] + dq[1])
                phi = superblock.apply_op(sb, A, B, Q1, src, Qn)
                Q1 = Qn
                applied = True
            if applied and not pending:
                targets, _, _ = krylov.evolve(hq(Q1), phi, self.times, self.nk)
                action, done_step = "excite", step
            elif applied:
                targets, action = [phi] * self.n_v, "partial"
            elif done_step is not None and (step - done_step) % self.advance_every == 0:
                targets, _, _ = krylov.evolve(hq(Q1), targets[-1], self.times, self.nk)
                t_now += self.tau
                action = "advance"
            rec = {"l": l, "move": move, "action": action, "t": t_now, "energy": e, "Q1": Q1,
                   "applied": len(self.excitations) - len(pending),
                   "targets": [self._observe(sb, HL, HR, conns, Lenl, Renl, Q1, x) for x in targets or []]}
            if move is not None:
                if targets is None:
                    states, weights = [(Q0, psi)], [1.0]
                else:
                    states = [(Q0, psi)] + [(Q1, x) for x in targets]
                    weights = [self.w_gs] + list(self.w)
                if move == "R":
                    rho = density.rho_left(sb, states, weights, self.real_basis)
                    K, counts, lams, disc, U = dmrg.truncate(Lenl, rho, self.m)
                    Ln = dmrg.enlarge(K, "L", d.t, d.U, d.geom)
                    Rn = dmrg.enlarge(d.right[r - 1], "R", d.t, d.U, d.geom)
                    moved = [dmrg.wft_right(Lenl, Renl, Q, v, U, d.right[r], d.right_U[r], Ln, Rn)
                             for Q, v in states]
                    d.left[l + 1], d.left_U[l + 1] = K, U
                else:
                    rho = density.rho_right(sb, states, weights, self.real_basis)
                    K, counts, lams, disc, U = dmrg.truncate(Renl, rho, self.m)
                    Ln = dmrg.enlarge(d.left[l - 1], "L", d.t, d.U, d.geom)
                    Rn = dmrg.enlarge(K, "R", d.t, d.U, d.geom)
                    moved = [dmrg.wft_left(Lenl, Renl, Q, v, U, d.left[l], d.left_U[l], Ln, Rn)
                             for Q, v in states]
                    d.right[r + 1], d.right_U[r + 1] = K, U
                rec.update(kept=list(counts), evals=[np.asarray(x) for x in lams], discarded=disc)
                psi = moved[0]
                if targets is not None:
                    targets = moved[1:]
                    if pending:   # the partial product is every target
                        phi = targets[0]
            records.append(rec)
        return records

    @staticmethod
    def _observe(sb, HL, HR, conns, Lenl, Renl, Q, x):
        nrm2 = np.vdot(x, x).real
        hx = superblock.apply_h(sb, HL, HR, conns, Q, x)
        cdL = Lenl.blockop(Lenl.cdag[0], True)
        cR = Renl.blockop(Renl.cdag[0].conj().T, True)
        nL = Lenl.blockop(Lenl.cdag[0] @ Lenl.cdag[0].conj().T, False)
        nR = Renl.blockop(Renl.cdag[0] @ Renl.cdag[0].conj().T, False)
        return {"norm2": nrm2, "energy": np.vdot(x, hx).real / nrm2,
                "n_left": superblock.expect(sb, nL, None, Q, x), "n_right": superblock.expect(sb, None, nR, Q, x),
                "bond": np.vdot(x, superblock.apply_op(sb, cdL, cR, Q, x, Q)) / nrm2}
