// Pieces of a finite sweep on the GPU beyond truncation (Sec. I, Sec. II.B): the wave-function
// transformation of the targets when the centre moves one site to the right.
//
// The superblock before the move is (L_enl, R_enl) with R_enl = site + R_b; after it, (L_enl', R_enl')
// with L_enl' = K + site, K the kept states of L_enl, and R_b the kept basis of R_enl'.  Block bases are
// Kronecker products sorted stably by quantum number, so inside a sector of R_enl the states run over the
// site states in order (0,0), (0,1), (1,0), (1,1) and, for each, over the states of R_b in its order; inside
// a sector of L_enl' they run over the states of K in order, each with the one site state that completes
// the sector.  The moved site keeps its place in the lattice order of the fermions, so no sign arises:
//   stage A (per left sector q of L_enl):  P1_q = U_q[:, :k_q]^dag Psi_q                 (k_q x dim R_enl(Q-q))
//   stage B (per q and site state s):       Psi'[q + s] rows of K_q  =  P1_q[:, s-columns] V_{q_b}^T
// with q_b = Q - q - s, V_{q_b} the states of R_b (columns) in the basis of R_enl' (rows).  Both stages are
// grouped FP64 launches; blocks of Psi' that no (q, s) reaches are zero.
#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "internal.h"

namespace tdmrg {
namespace {

const int kSiteQ[4][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};   // site sectors in sorted order

struct PairL { int qi, ri; int64_t off; int dl, dr; };

std::vector<PairL> pairs_Q(const tdmrg_ctx* c, int a, int b) {
    std::vector<PairL> out;
    const Side& L = c->side[0];
    const Side& R = c->side[1];
    int64_t off = 0;
    for (size_t qi = 0; qi < L.dim.size(); ++qi) {
        const int ri = R.find(a - L.nup[qi], b - L.ndn[qi]);
        if (ri < 0) continue;
        out.push_back({(int)qi, ri, off, L.dim[qi], R.dim[ri]});
        off += (int64_t)L.dim[qi] * R.dim[ri];
    }
    return out;
}

}  // namespace
}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_wft_right(tdmrg_ctx* from, int a, int b, const tdmrg_c64* psi, const tdmrg_c64* U, const int32_t* kept,
                               int rb_nsec, const int32_t* rb_qn, const int32_t* rb_dim, const tdmrg_c64* V, tdmrg_ctx* to,
                               tdmrg_c64* out) {
    if (!from || !to) return fail(nullptr, TDMRG_EINVAL, "wft_right: null context");
    if (!psi || !U || !kept || !V || !out || rb_nsec < 1 || !rb_qn || !rb_dim)
        return fail(from, TDMRG_EINVAL, "wft_right: bad argument");
    if (!from->side[0].set || !from->side[1].set || !to->side[0].set || !to->side[1].set)
        return fail(from, TDMRG_ESTATE, "wft_right: blocks not set");
    if (from->opts.device != to->opts.device) return fail(from, TDMRG_EINVAL, "wft_right: contexts on different devices");
    const Side& fL = from->side[0];
    const Side& fR = from->side[1];
    const Side& tL = to->side[0];
    const Side& tR = to->side[1];
    // R_b: sector table and the offsets of its V blocks
    std::map<std::pair<int, int>, int> rbi;
    std::vector<int64_t> voff(rb_nsec);
    int64_t vo = 0;
    for (int s = 0; s < rb_nsec; ++s) {
        rbi[{rb_qn[2 * s], rb_qn[2 * s + 1]}] = s;
        const int ti = tR.find(rb_qn[2 * s], rb_qn[2 * s + 1]);
        if (ti < 0 || rb_dim[s] < 1 || rb_dim[s] > tR.dim[ti])
            return fail(from, TDMRG_ESECTOR, "wft_right: a sector of R_b is missing from the next right block");
        voff[s] = vo;
        vo += (int64_t)tR.dim[ti] * rb_dim[s];
    }
    auto rb_find = [&](int x, int y) { auto it = rbi.find({x, y}); return it == rbi.end() ? -1 : it->second; };
    // R_enl = site + R_b: column offset of site state s inside each sector of R_enl
    std::vector<std::array<int, 4>> coff(fR.dim.size());
    for (size_t q = 0; q < fR.dim.size(); ++q) {
        int o = 0;
        for (int s = 0; s < 4; ++s) {
            coff[q][s] = o;
            const int bi = rb_find(fR.nup[q] - kSiteQ[s][0], fR.ndn[q] - kSiteQ[s][1]);
            if (bi >= 0) o += rb_dim[bi];
        }
        if (o != fR.dim[q]) return fail(from, TDMRG_ESECTOR, "wft_right: the right block is not site + R_b");
    }
    // L_enl' = K + site: row offset of (kept sector q, site state s) inside each sector of L_enl'
    std::map<std::pair<int, int>, int> roff;   // (q of L_enl, s) -> row offset in sector q + s of L_enl'
    std::vector<int> fill(tL.dim.size(), 0);
    for (size_t q = 0; q < fL.dim.size(); ++q) {
        if (kept[q] < 0 || kept[q] > fL.dim[q]) return fail(from, TDMRG_EINVAL, "wft_right: kept count outside 0..dim");
        if (kept[q] == 0) continue;
        for (int s = 0; s < 4; ++s) {
            const int ti = tL.find(fL.nup[q] + kSiteQ[s][0], fL.ndn[q] + kSiteQ[s][1]);
            if (ti < 0) return fail(from, TDMRG_ESECTOR, "wft_right: the next left block is not K + site");
            roff[{(int)q, s}] = fill[ti];
            fill[ti] += kept[q];
        }
    }
    for (size_t t = 0; t < tL.dim.size(); ++t)
        if (fill[t] != tL.dim[t]) return fail(from, TDMRG_ESECTOR, "wft_right: the next left block is not K + site");
    std::vector<int64_t> uoff(fL.dim.size());
    int64_t uo = 0;
    for (size_t q = 0; q < fL.dim.size(); ++q) { uoff[q] = uo; uo += (int64_t)fL.dim[q] * fL.dim[q]; }
    const std::vector<PairL> pf = pairs_Q(from, a, b), pt = pairs_Q(to, a, b);
    std::map<int, const PairL*> pt_of_l;
    for (const PairL& p : pt) pt_of_l[p.qi] = &p;
    const int64_t nout = pt.empty() ? 0 : pt.back().off + (int64_t)pt.back().dl * pt.back().dr;
    if (nout == 0) return fail(from, TDMRG_ESECTOR, "wft_right: empty sector in the next superblock");
    // the two stages
    const int8_t BU = BUF_EXTRA0, BV = BUF_EXTRA0 + 1;
    TaskList s1, s2;
    int64_t scr = 0;
    for (const PairL& p : pf) {
        const int k = kept[p.qi];
        if (k == 0) continue;
        Task t1{};
        t1.c_off = scr; t1.c_buf = BUF_SCRATCH; t1.ldc = p.dr; t1.M = k; t1.N = p.dr;
        t1.seg_begin = (int)s1.segs.size();
        Seg g1{};
        g1.a_off = uoff[p.qi]; g1.a_buf = BU; g1.lda = p.dl; g1.opa = 2;   // U^dag
        g1.b_off = p.off; g1.b_buf = BUF_IN; g1.ldb = p.dr; g1.opb = OPB_N;
        g1.K = p.dl; g1.scale = make_double2(1.0, 0.0); g1.dscale = -1;
        s1.segs.push_back(g1);
        t1.seg_end = (int)s1.segs.size();
        s1.tasks.push_back(t1);
        for (int s = 0; s < 4; ++s) {
            const int bi = rb_find(fR.nup[p.ri] - kSiteQ[s][0], fR.ndn[p.ri] - kSiteQ[s][1]);
            if (bi < 0) continue;
            const int tl = tL.find(fL.nup[p.qi] + kSiteQ[s][0], fL.ndn[p.qi] + kSiteQ[s][1]);
            auto it = pt_of_l.find(tl);
            if (it == pt_of_l.end()) continue;
            const PairL& q2 = *it->second;
            const int tr = tR.find(rb_qn[2 * bi], rb_qn[2 * bi + 1]);
            if (q2.ri != tr) return fail(from, TDMRG_ESECTOR, "wft_right: inconsistent sectors");
            Task t2{};
            t2.c_off = q2.off + (int64_t)roff[{p.qi, s}] * q2.dr; t2.c_buf = BUF_OUT; t2.ldc = q2.dr;
            t2.M = k; t2.N = q2.dr;
            t2.seg_begin = (int)s2.segs.size();
            Seg g2{};
            g2.a_off = scr + coff[p.ri][s]; g2.a_buf = BUF_SCRATCH; g2.lda = p.dr;
            g2.b_off = voff[bi]; g2.b_buf = BV; g2.ldb = rb_dim[bi]; g2.opb = OPB_T;   // V^T
            g2.K = rb_dim[bi]; g2.scale = make_double2(1.0, 0.0); g2.dscale = -1;
            s2.segs.push_back(g2);
            t2.seg_end = (int)s2.segs.size();
            s2.tasks.push_back(t2);
        }
        scr += (int64_t)k * p.dr;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != from->opts.device) cudaSetDevice(from->opts.device);
    make_tiles(s1, kTileF64, kTileF64, kSplitK);
    make_tiles(s2, kTileF64, kTileF64, kSplitK);
    cplx* P1 = nullptr;
    int rc = dev_alloc(from, (void**)&P1, (size_t)std::max<int64_t>(scr, 1) * sizeof(cplx), "wft scratch");
    if (!rc) rc = upload(from, s1);
    if (!rc) rc = upload(from, s2);
    if (!rc) rc = cuda_check(from, cudaMemsetAsync(out, 0, (size_t)nout * sizeof(cplx), from->stream), "wft clear");
    if (!rc) {
        GemmArgs g{};
        g.bufs[BUF_IN] = (cplx*)psi;
        g.bufs[BUF_SCRATCH] = P1;
        g.bufs[BUF_OUT] = (cplx*)out;
        g.bufs[BU] = (cplx*)U;
        g.bufs[BV] = (cplx*)V;
        g.dscale = from->dscale;
        for (TaskList* tl : {&s1, &s2}) {
            if (tl->tiles.empty()) continue;
            g.tasks = tl->d_tasks; g.segs = tl->d_segs; g.tiles = tl->d_tiles; g.ntiles = (int)tl->tiles.size();
            g.partials = tl->d_partials; g.counters = tl->d_counters;
            from->launches++;
            rc = cuda_check(from, launch_gemm_f64(g, from->stream, nullptr, 0), "wft launch");
            if (rc) break;
        }
    }
    const int rc2 = cuda_check(from, cudaStreamSynchronize(from->stream), "wft");
    release(from, s1);
    release(from, s2);
    dev_free(from, P1, (size_t)std::max<int64_t>(scr, 1) * sizeof(cplx));
    if (prev >= 0 && prev != from->opts.device) cudaSetDevice(prev);
    return rc ? rc : rc2;
}
