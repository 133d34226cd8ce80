// Wave-function transformation of the targets when the centre of a finite sweep moves one site
// (Sec. I; Sec. II.B: the targets are transported from one superblock to the next).
//
// Block bases are Kronecker products sorted stably by quantum number: inside a sector of an enlarged
// left block K + site the states run over K's sectors in order (each with the one site state that
// completes the sector); inside a sector of an enlarged right block site + K they run over the site states
// (0,0), (0,1), (1,0), (1,1) in order, each followed by the states of K's matching sector.  The moved site
// keeps its place in the lattice order of the fermions, so no sign arises.
//
// Move right: (L_enl, R_enl = site + R_b) -> (L_enl' = K + site, R_enl'), K the kept states of L_enl
// (columns of U), R_b the kept basis of R_enl' (columns of V):
//   stage A (per left sector q of L_enl):  P1_q = U_q[:, :k_q]^dag Psi_q               (k_q x dim R_enl(Q-q))
//   stage B (per q, site state s):          Psi'[q + s] rows of K_q  =  P1_q[:, s-columns] V_{q_b}^T
// with q_b = Q - q - s.
// Move left: (L_enl = L_b + site, R_enl) -> (L_enl', R_enl' = site + K), K the kept states of R_enl
// (columns of U), L_b the kept basis of L_enl' (columns of V):
//   stage A (per right sector r of R_enl): P1_r = Psi_r conj(U_r[:, :k_r])              (dim L_enl(Q-r) x k_r)
//   stage B (per r, site state s):          Psi'[q_b] columns (s, K_r) = V_{q_b} P1_r[s-rows]
// with q_b = Q - r - s.  Both stages are grouped FP64 launches; blocks of Psi' that nothing reaches are zero.
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

std::vector<int64_t> square_offsets(const Side& S) {
    std::vector<int64_t> o(S.dim.size());
    int64_t x = 0;
    for (size_t q = 0; q < S.dim.size(); ++q) { o[q] = x; x += (int64_t)S.dim[q] * S.dim[q]; }
    return o;
}

// Offsets of the runs of an enlarged block built from a kept basis (sectors of `base` with kept > 0,
// kept[q] states each) and one site: runs[q][s] = offset inside sector (q + s) of `enl`, -1 when absent.
// site_first: runs ordered by site state (site + K), else by K's sector (K + site).
int enlarged_runs(const Side& base, const int32_t* kept, const Side& enl, bool site_first,
                  std::vector<std::array<int, 4>>& runs) {
    runs.assign(base.dim.size(), {-1, -1, -1, -1});
    std::vector<int> fill(enl.dim.size(), 0);
    auto place = [&](size_t q, int s) {
        const int t = enl.find(base.nup[q] + kSiteQ[s][0], base.ndn[q] + kSiteQ[s][1]);
        if (t < 0) return false;
        runs[q][s] = fill[t];
        fill[t] += kept[q];
        return true;
    };
    if (site_first) {
        for (int s = 0; s < 4; ++s)
            for (size_t q = 0; q < base.dim.size(); ++q)
                if (kept[q] > 0 && !place(q, s)) return TDMRG_ESECTOR;
    } else {
        for (size_t q = 0; q < base.dim.size(); ++q)
            for (int s = 0; s < 4; ++s)
                if (kept[q] > 0 && !place(q, s)) return TDMRG_ESECTOR;
    }
    for (size_t t = 0; t < enl.dim.size(); ++t)
        if (fill[t] != enl.dim[t]) return TDMRG_ESECTOR;
    return TDMRG_OK;
}

int check_kept(tdmrg_ctx* c, const Side& S, const int32_t* kept) {
    for (size_t q = 0; q < S.dim.size(); ++q)
        if (kept[q] < 0 || kept[q] > S.dim[q]) return fail(c, TDMRG_EINVAL, "wft: kept count outside 0..dim");
    return TDMRG_OK;
}

int run_stages(tdmrg_ctx* from, TaskList& s1, TaskList& s2, int64_t scr, const tdmrg_c64* psi, const tdmrg_c64* U,
               const tdmrg_c64* V, tdmrg_c64* out, int64_t nout) {
    const int8_t BU = BUF_EXTRA0, BV = BUF_EXTRA0 + 1;
    DeviceGuard g(from->opts.device);
    make_tiles(s1, kTileF64, kTileF64, kSplitK);
    make_tiles(s2, kTileF64, kTileF64, kSplitK);
    cplx* P1 = nullptr;
    const size_t sb = (size_t)std::max<int64_t>(scr, 1) * sizeof(cplx);
    int rc = dev_alloc(from, (void**)&P1, sb, "wft scratch");
    if (!rc) rc = upload(from, s1);
    if (!rc) rc = upload(from, s2);
    if (!rc) rc = cuda_check(from, cudaMemsetAsync(out, 0, (size_t)nout * sizeof(cplx), from->stream), "wft clear");
    if (!rc) {
        GemmArgs ga{};
        ga.bufs[BUF_IN] = (cplx*)psi;
        ga.bufs[BUF_SCRATCH] = P1;
        ga.bufs[BUF_OUT] = (cplx*)out;
        ga.bufs[BU] = (cplx*)U;
        ga.bufs[BV] = (cplx*)V;
        ga.dscale = from->dscale;
        for (TaskList* tl : {&s1, &s2}) {
            if (tl->tiles.empty()) continue;
            ga.tasks = tl->d_tasks; ga.segs = tl->d_segs; ga.tiles = tl->d_tiles; ga.ntiles = (int)tl->tiles.size();
            ga.partials = tl->d_partials; ga.counters = tl->d_counters;
            from->launches++;
            rc = cuda_check(from, launch_gemm_f64(ga, from->stream, nullptr, 0), "wft launch");
            if (rc) break;
        }
    }
    const int rc2 = cuda_check(from, cudaStreamSynchronize(from->stream), "wft");
    release(from, s1);
    release(from, s2);
    dev_free(from, P1, sb);
    return rc ? rc : rc2;
}

Seg seg(int64_t a_off, int8_t a_buf, int lda, int opa, int64_t b_off, int8_t b_buf, int ldb, int8_t opb, int K) {
    Seg g{};
    g.a_off = a_off; g.a_buf = a_buf; g.lda = lda; g.opa = (int8_t)opa;
    g.b_off = b_off; g.b_buf = b_buf; g.ldb = ldb; g.opb = opb;
    g.K = K; g.scale = make_double2(1.0, 0.0); g.dscale = -1;
    return g;
}

void add_task(TaskList& tl, int64_t c_off, int8_t c_buf, int ldc, int M, int N, const Seg& g) {
    Task t{};
    t.c_off = c_off; t.c_buf = c_buf; t.ldc = ldc; t.M = M; t.N = N;
    t.seg_begin = (int)tl.segs.size();
    tl.segs.push_back(g);
    t.seg_end = (int)tl.segs.size();
    tl.tasks.push_back(t);
}

int check_pair(tdmrg_ctx* from, tdmrg_ctx* to, const tdmrg_c64* psi, const tdmrg_c64* U, const int32_t* kept,
               const tdmrg_c64* V, const int32_t* kept_next, const tdmrg_c64* out) {
    if (!from || !to) return fail(nullptr, TDMRG_EINVAL, "wft: null context");
    if (!psi || !U || !kept || !V || !kept_next || !out) return fail(from, TDMRG_EINVAL, "wft: bad argument");
    if (!from->side[0].set || !from->side[1].set || !to->side[0].set || !to->side[1].set)
        return fail(from, TDMRG_ESTATE, "wft: blocks not set");
    if (from->opts.device != to->opts.device) return fail(from, TDMRG_EINVAL, "wft: contexts on different devices");
    return TDMRG_OK;
}

}  // namespace
}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_wft_right(tdmrg_ctx* from, int a, int b, const tdmrg_c64* psi, const tdmrg_c64* U, const int32_t* kept,
                               const tdmrg_c64* V, const int32_t* kept_next, tdmrg_ctx* to, tdmrg_c64* out) {
    int rc = check_pair(from, to, psi, U, kept, V, kept_next, out);
    if (rc) return rc;
    const Side& fL = from->side[0];
    const Side& fR = from->side[1];
    const Side& tL = to->side[0];
    const Side& tR = to->side[1];
    if ((rc = check_kept(from, fL, kept)) || (rc = check_kept(from, tR, kept_next))) return rc;
    // R_enl = site + R_b with R_b = the kept states of R_enl'; L_enl' = K + site
    std::vector<std::array<int, 4>> rrun, lrun;
    if (enlarged_runs(tR, kept_next, fR, true, rrun))
        return fail(from, TDMRG_ESECTOR, "wft_right: the right block is not site + the kept basis of the next one");
    if (enlarged_runs(fL, kept, tL, false, lrun))
        return fail(from, TDMRG_ESECTOR, "wft_right: the next left block is not the kept states + site");
    const std::vector<int64_t> uoff = square_offsets(fL), voff = square_offsets(tR);
    const std::vector<PairL> pf = pairs_Q(from, a, b), pt = pairs_Q(to, a, b);
    std::map<int, const PairL*> pt_of_l;
    for (const PairL& p : pt) pt_of_l[p.qi] = &p;
    const int64_t nout = pt.empty() ? 0 : pt.back().off + (int64_t)pt.back().dl * pt.back().dr;
    if (nout == 0) return fail(from, TDMRG_ESECTOR, "wft_right: empty sector in the next superblock");
    const int8_t BU = BUF_EXTRA0, BV = BUF_EXTRA0 + 1;
    TaskList s1, s2;
    int64_t scr = 0;
    for (const PairL& p : pf) {
        const int k = kept[p.qi];
        if (k == 0) continue;
        add_task(s1, scr, BUF_SCRATCH, p.dr, k, p.dr,
                 seg(uoff[p.qi], BU, p.dl, 2, p.off, BUF_IN, p.dr, OPB_N, p.dl));   // U^dag Psi
        for (size_t t = 0; t < tR.dim.size(); ++t) {   // R_b sector t, site state s with q + s + t = Q
            if (kept_next[t] == 0) continue;
            for (int s = 0; s < 4; ++s) {
                const int co = rrun[t][s];
                if (co < 0 || fR.nup[p.ri] != tR.nup[t] + kSiteQ[s][0] || fR.ndn[p.ri] != tR.ndn[t] + kSiteQ[s][1]) continue;
                const int tl = tL.find(fL.nup[p.qi] + kSiteQ[s][0], fL.ndn[p.qi] + kSiteQ[s][1]);
                auto it = pt_of_l.find(tl);
                if (it == pt_of_l.end()) continue;
                const PairL& q2 = *it->second;
                if (q2.ri != (int)t) return fail(from, TDMRG_ESECTOR, "wft_right: inconsistent sectors");
                add_task(s2, q2.off + (int64_t)lrun[p.qi][s] * q2.dr, BUF_OUT, q2.dr, k, q2.dr,
                         seg(scr + co, BUF_SCRATCH, p.dr, 0, voff[t], BV, tR.dim[t], OPB_T, kept_next[t]));   // V^T
            }
        }
        scr += (int64_t)k * p.dr;
    }
    return run_stages(from, s1, s2, scr, psi, U, V, out, nout);
}

extern "C" int tdmrg_wft_left(tdmrg_ctx* from, int a, int b, const tdmrg_c64* psi, const tdmrg_c64* U, const int32_t* kept,
                              const tdmrg_c64* V, const int32_t* kept_next, tdmrg_ctx* to, tdmrg_c64* out) {
    int rc = check_pair(from, to, psi, U, kept, V, kept_next, out);
    if (rc) return rc;
    const Side& fL = from->side[0];
    const Side& fR = from->side[1];
    const Side& tL = to->side[0];
    const Side& tR = to->side[1];
    if ((rc = check_kept(from, fR, kept)) || (rc = check_kept(from, tL, kept_next))) return rc;
    // L_enl = L_b + site with L_b = the kept states of L_enl'; R_enl' = site + K
    std::vector<std::array<int, 4>> lrun, rrun;
    if (enlarged_runs(tL, kept_next, fL, false, lrun))
        return fail(from, TDMRG_ESECTOR, "wft_left: the left block is not the kept basis of the next one + site");
    if (enlarged_runs(fR, kept, tR, true, rrun))
        return fail(from, TDMRG_ESECTOR, "wft_left: the next right block is not site + the kept states");
    const std::vector<int64_t> uoff = square_offsets(fR), voff = square_offsets(tL);
    const std::vector<PairL> pf = pairs_Q(from, a, b), pt = pairs_Q(to, a, b);
    std::map<int, const PairL*> pt_of_l;
    for (const PairL& p : pt) pt_of_l[p.qi] = &p;
    const int64_t nout = pt.empty() ? 0 : pt.back().off + (int64_t)pt.back().dl * pt.back().dr;
    if (nout == 0) return fail(from, TDMRG_ESECTOR, "wft_left: empty sector in the next superblock");
    const int8_t BU = BUF_EXTRA0, BV = BUF_EXTRA0 + 1;
    TaskList s1, s2;
    int64_t scr = 0;
    for (const PairL& p : pf) {
        const int k = kept[p.ri];
        if (k == 0) continue;
        add_task(s1, scr, BUF_SCRATCH, k, p.dl, k,
                 seg(p.off, BUF_IN, p.dr, 0, uoff[p.ri], BU, p.dr, OPB_CN, p.dr));   // Psi conj(U)
        for (size_t t = 0; t < tL.dim.size(); ++t) {   // L_b sector t, site state s with t + s = q
            if (kept_next[t] == 0) continue;
            for (int s = 0; s < 4; ++s) {
                const int ro = lrun[t][s];
                if (ro < 0 || fL.nup[p.qi] != tL.nup[t] + kSiteQ[s][0] || fL.ndn[p.qi] != tL.ndn[t] + kSiteQ[s][1]) continue;
                auto it = pt_of_l.find((int)t);
                if (it == pt_of_l.end()) continue;
                const PairL& q2 = *it->second;
                if (q2.ri != tR.find(fR.nup[p.ri] + kSiteQ[s][0], fR.ndn[p.ri] + kSiteQ[s][1]))
                    return fail(from, TDMRG_ESECTOR, "wft_left: inconsistent sectors");
                add_task(s2, q2.off + rrun[p.ri][s], BUF_OUT, q2.dr, q2.dl, k,
                         seg(voff[t], BV, tL.dim[t], 0, scr + (int64_t)ro * k, BUF_SCRATCH, k, OPB_N, kept_next[t]));   // V P1
            }
        }
        scr += (int64_t)p.dl * k;
    }
    return run_stages(from, s1, s2, scr, psi, U, V, out, nout);
}
