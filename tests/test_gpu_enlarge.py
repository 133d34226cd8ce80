"""Block enlargement K + site / site + K on the GPU (Sec. I: the blocks grow by one site per step) and
the adjoint of a block operator, against the oracle DMRG's enlargement of the same blocks.

  - the enlarged sector table, H' and the new edge c^dag'_s of left and right blocks of 1, 3 and 4 sites
    of the L=10 m=32 run: every block equal to the oracle's (scaled copies: 1e-15);
  - the same on the 2 x 5 ladder (blocks of 1 to 4 sites) with the two bonds of the new site and K's edge
    carried as the second site from the edge (tdmrg_enlarge_bonds);
  - the adjoint c = (c^dag)^dag defined on the device against the explicitly loaded adjoint (bit-equal
    products);
  - a superblock assembled only from device outputs (enlarged blocks, their edge operators and adjoints)
    against the oracle's superblock H psi: 1e-12."""
import numpy as np
import pytest

from oracle import dmrg, superblock
from tests.gpu_util import DmrgLoader, dev, host, new_ctx, rel_err

pytestmark = pytest.mark.gpu
L, U, T_HOP, M = 10, 4.0, 1.0, 32


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


@pytest.fixture(scope="module")
def run():
    d = dmrg.ChainDMRG(L, T_HOP, U, M)
    d.run(sweeps=1)
    return d


def _blocks(blk, dense, odd):
    secs, _, _ = blk.sectors()
    bo = blk.blockop(dense, odd)
    qns = [tuple(secs[qo]) + tuple(secs[qi]) for (qo, qi) in bo.blocks]
    data = np.concatenate([b.ravel() for b in bo.blocks.values()]) if bo.blocks else np.zeros(1, complex)
    return qns, data


def _device_enlarge(lib, ctx, blk, side):
    secs, dims, _ = blk.sectors()
    qn_o, dim_o, nb, ent = lib.tdmrg_enlarge_size(side, secs, dims)
    hq, hd = _blocks(blk, blk.H, False)
    cd = [_blocks(blk, blk.cdag[s], True) for s in range(2)]
    H_out = dev(np.zeros(int(ent[0])))
    c_out = [dev(np.zeros(max(int(ent[1 + s]), 1))) for s in range(2)]
    cq = lib.tdmrg_enlarge(ctx, side, secs, dims, (hq, dev(hd)), [(q, dev(x)) for q, x in cd], T_HOP, U, H_out, c_out)
    qn_o = [tuple(int(x) for x in q) for q in qn_o]
    return qn_o, [int(x) for x in dim_o], H_out, c_out, cq


def _unpack(qn_o, dim_o, data, qns):
    """Dense blocks keyed by (out sector, in sector) from packed device output."""
    d = dict(zip(qn_o, dim_o))
    out, off = {}, 0
    for b in qns:
        qo, qi = tuple(b[:2]), tuple(b[2:])
        n = d[qo] * d[qi]
        out[(qo, qi)] = data[off: off + n].reshape(d[qo], d[qi])
        off += n
    return out


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("nsites", [1, 3, 4])
def test_enlarge_matches_oracle(lib, run, side, nsites):
    blk = (run.left if side == 0 else run.right)[nsites]
    want = dmrg.enlarge(blk, "L" if side == 0 else "R", T_HOP, U)
    wsecs, wdims, _ = want.sectors()
    ctx = new_ctx()
    try:
        qn_o, dim_o, H_out, c_out, cq = _device_enlarge(lib, ctx, blk, side)
        assert qn_o == [tuple(q) for q in wsecs] and dim_o == list(wdims)
        got_h = _unpack(qn_o, dim_o, host(H_out), [q + q for q in qn_o])
        want_h = want.blockop(want.H, False).blocks
        for (a, b), blkw in want_h.items():
            assert a == b
            assert np.abs(got_h[(wsecs[a], wsecs[a])] - blkw).max() <= 1e-15
        for q, g in got_h.items():   # sector blocks the oracle omits are zero
            if (wsecs.index(q[0]), wsecs.index(q[0])) not in want_h:
                assert not np.any(g)
        for s in range(2):
            got_c = _unpack(qn_o, dim_o, host(c_out[s]), [tuple(int(x) for x in b) for b in cq[s]])
            want_c = {(wsecs[a], wsecs[b]): m for (a, b), m in want.blockop(want.cdag[s], True).blocks.items()}
            assert set(got_c) == set(want_c)
            for k, m in want_c.items():
                assert np.array_equal(got_c[k], m)
    finally:
        lib.tdmrg_destroy(ctx)


LADDER = dmrg.Geometry(2, 1.0, 0.5)


@pytest.fixture(scope="module")
def ladder_run():
    d = dmrg.ChainDMRG(L, T_HOP, U, M, geom=LADDER)
    d.run(sweeps=1)
    return d


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("nsites", [1, 2, 3, 4])
def test_ladder_enlarge_matches_oracle(lib, ladder_run, side, nsites):
    """2 x 5 ladder blocks (Sec. III): the new site bonded to K's edge (a rung when K has an odd number of
    sites) and to the second site from the edge (a leg, K of two or more sites), the second bond added by
    the accumulating launch; K's edge carried as the enlarged block's second site from the edge.  H' to
    1e-15, the new and the carried c^dag bit-equal to the oracle's."""
    blk = (ladder_run.left if side == 0 else ladder_run.right)[nsites]
    want = dmrg.enlarge(blk, "L" if side == 0 else "R", T_HOP, U, LADDER)
    wsecs, wdims, _ = want.sectors()
    secs, dims, _ = blk.sectors()
    qn_o, dim_o, nb, ent = lib.tdmrg_enlarge_size(side, secs, dims)
    qn_o = [tuple(int(x) for x in q) for q in qn_o]
    dim_o = [int(x) for x in dim_o]
    hq, hd = _blocks(blk, blk.H, False)
    edges = [[(q, dev(x)) for q, x in (_blocks(blk, blk.cdag[s], True) for s in range(2))]]
    t0, t1 = LADDER.new_site_bonds(nsites)
    ts = [t0]
    if blk.cdag2 is not None:
        edges.append([(q, dev(x)) for q, x in (_blocks(blk, blk.cdag2[s], True) for s in range(2))])
        ts.append(t1)
    assert (blk.cdag2 is None) == (nsites == 1)
    ctx = new_ctx()
    try:
        H_out = dev(np.zeros(int(ent[0])))
        c_out = [dev(np.zeros(max(int(ent[1 + s]), 1))) for s in range(2)]
        k_out = [dev(np.zeros(max(int(ent[1 + s]), 1))) for s in range(2)]
        cq = lib.tdmrg_enlarge_bonds(ctx, side, secs, dims, (hq, dev(hd)), edges, ts, U, H_out, c_out, None, k_out)
        assert qn_o == [tuple(q) for q in wsecs] and dim_o == list(wdims)
        got_h = _unpack(qn_o, dim_o, host(H_out), [q + q for q in qn_o])
        want_h = want.blockop(want.H, False).blocks
        for (a, b), blkw in want_h.items():
            assert np.abs(got_h[(wsecs[a], wsecs[a])] - blkw).max() <= 1e-15
        for q, g in got_h.items():
            if (wsecs.index(q[0]), wsecs.index(q[0])) not in want_h:
                assert not np.any(g)
        for s in range(2):
            for out, op in ((c_out[s], want.cdag[s]), (k_out[s], want.cdag2[s])):
                got_c = _unpack(qn_o, dim_o, host(out), [tuple(int(x) for x in b) for b in cq[s]])
                want_c = {(wsecs[a], wsecs[b]): m for (a, b), m in want.blockop(op, True).blocks.items()}
                assert set(want_c) <= set(got_c)
                for k, m in got_c.items():
                    assert np.array_equal(m, want_c[k]) if k in want_c else not np.any(m)
    finally:
        lib.tdmrg_destroy(ctx)


def test_adjoint_operator(lib, run):
    Lenl = dmrg.enlarge(run.left[4], "L", T_HOP, U)
    Renl = dmrg.enlarge(run.right[4], "R", T_HOP, U)
    Q, Q1 = (L // 2, L // 2), (L // 2 + 1, L // 2)
    ctx = new_ctx()
    try:
        DmrgLoader(ctx, Lenl, Renl, T_HOP)
        for side in (0, 1):
            lib.tdmrg_set_op_adjoint(ctx, side, 70, 10)   # c_{edge up} from c^dag_{edge up}
            n = lib.tdmrg_sector_size(ctx, Q1)
            x = dev(np.random.default_rng(side).standard_normal(n) + 0j)
            a, b = dev(np.zeros(lib.tdmrg_sector_size(ctx, Q))), dev(np.zeros(lib.tdmrg_sector_size(ctx, Q)))
            ops = (70, -1) if side == 0 else (-1, 70)
            ref = (30, -1) if side == 0 else (-1, 30)
            lib.tdmrg_apply_op(ctx, *ops, Q1, x, Q, a)
            lib.tdmrg_apply_op(ctx, *ref, Q1, x, Q, b)
            assert np.array_equal(host(a), host(b))
    finally:
        lib.tdmrg_destroy(ctx)


def test_superblock_from_device_enlargement(lib, run):
    """(K_L + site) + (site + K_R) with K_L, K_R the 4-site blocks: every operator of the superblock comes
    from tdmrg_enlarge, the boundary c from tdmrg_set_op_adjoint."""
    Lenl = dmrg.enlarge(run.left[4], "L", T_HOP, U)
    Renl = dmrg.enlarge(run.right[4], "R", T_HOP, U)
    sb, HL, HR, conns = dmrg.superblock_of(Lenl, Renl, T_HOP)
    Q = (L // 2, L // 2)
    work = new_ctx()
    ctx = new_ctx()
    try:
        outs = [_device_enlarge(lib, work, b, side) for side, b in ((0, run.left[4]), (1, run.right[4]))]
        for side, (qn_o, dim_o, H_out, c_out, cq) in enumerate(outs):
            lib.tdmrg_set_block(ctx, side, qn_o, dim_o)
        for side, (qn_o, dim_o, H_out, c_out, cq) in enumerate(outs):
            lib.tdmrg_set_op_device(ctx, side, 0, 0, [(q[0], q[1], q[0], q[1]) for q in qn_o], H_out)
            for s in range(2):
                lib.tdmrg_set_op_device(ctx, side, 10 + s, 1, [tuple(int(x) for x in b) for b in cq[s]], c_out[s])
                lib.tdmrg_set_op_adjoint(ctx, side, 30 + s, 10 + s)
        lib.tdmrg_set_hamiltonian(ctx, 0, 0, [(10 + s, 30 + s, -T_HOP) for s in range(2)] +
                                  [(30 + s, 10 + s, T_HOP) for s in range(2)])
        n = lib.tdmrg_sector_size(ctx, Q)
        assert n == sb.size(Q)
        x = np.random.default_rng(3).standard_normal(n) + 1j * np.random.default_rng(4).standard_normal(n)
        y = dev(np.zeros(n))
        lib.tdmrg_apply_h(ctx, Q, dev(x), y)
        assert rel_err(host(y), superblock.apply_h(sb, HL, HR, conns, Q, x)) < 1e-12
    finally:
        lib.tdmrg_destroy(ctx)
        lib.tdmrg_destroy(work)
