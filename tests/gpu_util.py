"""Helpers of the GPU parity tests: load oracle problems into libtdmrg and compare."""
import numpy as np
import pytest

from oracle import blocks as oblocks
from oracle import superblock


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


def new_ctx(**kw):
    from paper_1103_5391_gb300 import tdmrg as T
    torch = torch_cuda()
    return T.tdmrg_create(device=torch.cuda.current_device(),
                          stream=torch.cuda.current_stream().cuda_stream, **kw)


def dev(x):
    torch = torch_cuda()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(t):
    return t.cpu().numpy()


def oracle_ops_of_synthetic(ss):
    HL = oblocks.BlockOp(ss.HL, False)
    HR = oblocks.BlockOp(ss.HR, False)
    conns = []
    for b in range(ss.nbonds):
        for s in range(2):
            A = oblocks.BlockOp(ss.cdagL[b][s], True)
            B = oblocks.BlockOp(ss.cR[b][s], True)
            conns.append((ss.coeff_t, A, B))
            conns.append((-ss.coeff_t, A.dagger(), B.dagger()))
    sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
    return sb, HL, HR, conns


class ExactLoader:
    """Loads an oracle.models.ExactProblem: H and arbitrary local operators by id."""

    def __init__(self, ctx, prob):
        from paper_1103_5391_gb300 import tdmrg as T
        self.T, self.ctx, self.p = T, ctx, prob
        T.tdmrg_set_block(ctx, 0, prob.sb.lsec, prob.sb.ldim)
        T.tdmrg_set_block(ctx, 1, prob.sb.rsec, prob.sb.rdim)
        self.next_id = [100, 100]
        hl = self.add(0, prob.HL)
        hr = self.add(1, prob.HR)
        conns = []
        for coeff, A, B in prob.conns:
            conns.append((self.add(0, A), self.add(1, B), coeff))
        T.tdmrg_set_hamiltonian(ctx, hl, hr, conns)

    def add(self, side, op):
        sec = self.p.sb.lsec if side == 0 else self.p.sb.rsec
        i = self.next_id[side]
        self.next_id[side] += 1
        blks = [(sec[qo], sec[qi], b) for (qo, qi), b in op.blocks.items()]
        self.T.tdmrg_set_op(self.ctx, side, i, op.odd, blks)
        return i

    def local(self, kind, site, sigma=0):
        side, op = self.p.op(kind, site, sigma)
        i = self.add(side, op)
        return (i, -1) if side == 0 else (-1, i)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


class DmrgLoader:
    """Loads the central-cut superblock of an oracle DMRG run (oracle.dmrg enlarged blocks) into libtdmrg:
    ids 0 = H, 10 + s = c^dag_{edge s}, 30 + s = its adjoint, 50 + s = n_{edge s} on both sides; the
    Hamiltonian's boundary terms -t c^dag_L c_R + t c_L c^dag_R per spin."""

    def __init__(self, ctx, Lenl, Renl, t):
        from paper_1103_5391_gb300 import tdmrg as T
        self.T, self.ctx = T, ctx
        self.blk = (Lenl, Renl)
        for side, b in enumerate(self.blk):
            secs, dims, _ = b.sectors()
            T.tdmrg_set_block(ctx, side, secs, dims)
            self.add(side, 0, b.H, False)
            for s in range(2):
                self.add(side, 10 + s, b.cdag[s], True)
                self.add(side, 30 + s, b.cdag[s].conj().T, True)
                self.add(side, 50 + s, b.cdag[s] @ b.cdag[s].conj().T, False)
        conns = []
        for s in range(2):
            conns += [(10 + s, 30 + s, -t), (30 + s, 10 + s, t)]
        T.tdmrg_set_hamiltonian(ctx, 0, 0, conns)

    def add(self, side, op_id, dense, odd):
        b = self.blk[side]
        secs, _, _ = b.sectors()
        bo = b.blockop(dense, odd)
        self.T.tdmrg_set_op(self.ctx, side, op_id, odd, [(secs[qo], secs[qi], blk) for (qo, qi), blk in bo.blocks.items()])
        return bo
