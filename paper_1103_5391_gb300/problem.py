"""Loads a superblock problem into a libtdmrg context (marshalling only).

Operator ids used for the synthetic Gaussian-sector superblocks:
  left : 0 = H_L, 10 + 2b + s = c^dag_{b s}, 30 + 2b + s = c_{b s} (its adjoint), 50 = n_L
  right: 0 = H_R, 10 + 2b + s = c_{b s},     30 + 2b + s = c^dag_{b s},           49 = c^dag_exc, 50 = n_R
where b is the bond across the cut and s the spin.  The Hamiltonian is
H_L (x) 1 + 1 (x) H_R + sum_{b,s} [ -t c^dag_{Lbs} c_{Rbs} + t c_{Lbs} c^dag_{Rbs} ]
(fermionic products written left operator first; Sec. IV, Sec. III.B).
"""
import numpy as np

from . import tdmrg as T

OP_H, OP_CDAG, OP_C, OP_EXC, OP_N = 0, 10, 30, 49, 50


def _blocks(sec, blocks, adjoint=False):
    out = []
    for (qo, qi), b in blocks.items():
        if adjoint:
            out.append((sec[qi], sec[qo], np.asarray(b).conj().T))
        else:
            out.append((sec[qo], sec[qi], b))
    return out


def load_synthetic(ctx, ss):
    """Set blocks, operators and the Hamiltonian of a workloads.SyntheticSuperblock."""
    T.tdmrg_set_block(ctx, T.TDMRG_LEFT, ss.lsec, ss.ldim)
    T.tdmrg_set_block(ctx, T.TDMRG_RIGHT, ss.rsec, ss.rdim)
    T.tdmrg_set_op(ctx, 0, OP_H, 0, _blocks(ss.lsec, ss.HL))
    T.tdmrg_set_op(ctx, 1, OP_H, 0, _blocks(ss.rsec, ss.HR))
    conns = []
    for b in range(ss.nbonds):
        for s in range(2):
            k = 2 * b + s
            T.tdmrg_set_op(ctx, 0, OP_CDAG + k, 1, _blocks(ss.lsec, ss.cdagL[b][s]))
            T.tdmrg_set_op(ctx, 0, OP_C + k, 1, _blocks(ss.lsec, ss.cdagL[b][s], adjoint=True))
            T.tdmrg_set_op(ctx, 1, OP_CDAG + k, 1, _blocks(ss.rsec, ss.cR[b][s]))
            T.tdmrg_set_op(ctx, 1, OP_C + k, 1, _blocks(ss.rsec, ss.cR[b][s], adjoint=True))
            conns.append((OP_CDAG + k, OP_CDAG + k, ss.coeff_t))
            conns.append((OP_C + k, OP_C + k, -ss.coeff_t))
    T.tdmrg_set_op(ctx, 1, OP_EXC, 1, _blocks(ss.rsec, ss.cdag_exc))
    T.tdmrg_set_op(ctx, 0, OP_N, 0, _blocks(ss.lsec, ss.nL))
    T.tdmrg_set_op(ctx, 1, OP_N, 0, _blocks(ss.rsec, ss.nR))
    T.tdmrg_set_hamiltonian(ctx, OP_H, OP_H, conns)
    return conns
