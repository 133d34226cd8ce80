// Block enlargement of the DMRG (Sec. I: the blocks grow by one site per step; Sec. II.B: the superblock
// is (block + site) + (site + block)) and the adjoint of a block operator.
//
// Hubbard site, states in quantum-number order s = 0..3: |0> (0,0), |dn> (0,1), |up> (1,0), |up dn> (1,1),
// created as c^dag_up c^dag_dn |0> (up before down), so
//   c^dag_up: |0> -> |up>, |dn> -> |up dn>;   c^dag_dn: |0> -> |dn>, |up> -> -|up dn>;
// site parity p(s) = (-1)^{n_up + n_dn}, site energy U n_up n_dn.
//
// Left enlargement L' = K + site (K's fermions first in the creation string):
//   H' = H_K x 1 + 1 x U n_up n_dn - t sum_sigma [ (c^dag_K P_K) x c_site + (P_K c_K) x c^dag_site ],
//   c^dag'_sigma = P_K x c^dag_site          (the new site is the edge that bonds to the right);
// right enlargement R' = site + K (the site's fermions first):
//   H' = U n_up n_dn x 1 + 1 x H_K - t sum_sigma [ (c^dag_site P_site) x c_K + (P_site c_site) x c^dag_K ],
//   c^dag'_sigma = c^dag_site x 1.
// The enlarged basis is the Kronecker basis sorted stably by quantum number.  Inside a sector of L' the
// states run over K's sectors in order, each once (with the one site state that completes the sector);
// inside a sector of R' they run over the site states in order.  Every sector block of an output is a set
// of disjoint sub-blocks ("runs" pairs), each a scaled copy, scaled adjoint or scaled identity of a block
// of K, so one launch places all of them into zeroed outputs (no sub-block is written twice: the U term
// rides on the H_K copy's diagonal).
//
// Ladders (Sec. III): the new site also bonds to the second site from K's edge (a leg when the edge bond is
// a rung or absent), whose bond terms fall on the same sub-blocks of H' as the edge's, so they are added by
// a second launch; and K's edge becomes the enlarged block's second site from the edge, carried as
// c^dag_K x 1 (left) or P_site x c^dag_K (right) with the block layout of the new edge's c^dag'.
#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "internal.h"

namespace tdmrg {
namespace {

const int kSq[4][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};
const int kParity[4] = {1, -1, -1, 1};
struct SiteHop { int from, to; double v; };
const SiteHop kCdag[2][2] = {{{0, 2, 1.0}, {1, 3, 1.0}},     // c^dag_up
                             {{0, 1, 1.0}, {2, 3, -1.0}}};   // c^dag_dn

enum { MODE_COPY = 0, MODE_ADJ = 1, MODE_EYE = 2 };
constexpr int kPT = 32;   // placement tile edge

struct Place {
    int64_t dst, src;       // element offsets in the destination / source buffer
    int ldd, lds;
    int rows, cols;         // destination extent
    int8_t dbuf, sbuf, mode;
    int8_t acc;             // add to the destination instead of writing it
    double2 scale;
    double diag;            // added on the diagonal (MODE_COPY, MODE_ADJ)
};
struct PlaceTile { int item, r0, c0; };
struct PlaceBufs { cplx* d[5]; const cplx* s[3]; };

// One CTA of 32 x 8 threads per 32 x 32 destination tile; a transposed source goes through shared memory
// so that both the read and the write are coalesced.
__global__ void __launch_bounds__(256) k_place(const Place* __restrict__ items, const PlaceTile* __restrict__ tiles,
                                               PlaceBufs b) {
    pdl_enter();
    __shared__ cplx sm[kPT][kPT + 1];
    const PlaceTile tl = tiles[blockIdx.x];
    const Place it = items[tl.item];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    cplx* dst = b.d[it.dbuf] + it.dst;
    if (it.mode == MODE_ADJ) {
        const cplx* src = b.s[it.sbuf] + it.src;
        for (int r = ty; r < kPT; r += 8) {   // source rows = destination columns
            const int sr = tl.c0 + r, sc = tl.r0 + tx;
            sm[r][tx] = (sr < it.cols && sc < it.rows) ? src[(int64_t)sr * it.lds + sc] : make_double2(0.0, 0.0);
        }
        __syncthreads();
    }
    for (int r = ty; r < kPT; r += 8) {
        const int i = tl.r0 + r, j = tl.c0 + tx;
        if (i >= it.rows || j >= it.cols) continue;
        cplx x;
        if (it.mode == MODE_COPY) {
            x = b.s[it.sbuf][it.src + (int64_t)i * it.lds + j];
        } else if (it.mode == MODE_ADJ) {
            x = sm[tx][r];
            x.y = -x.y;
        } else {
            x = make_double2(i == j ? 1.0 : 0.0, 0.0);
        }
        cplx y = make_double2(it.scale.x * x.x - it.scale.y * x.y, it.scale.x * x.y + it.scale.y * x.x);
        if (i == j && it.mode != MODE_EYE) y.x += it.diag;
        if (it.acc) { const cplx o = dst[(int64_t)i * it.ldd + j]; y.x += o.x; y.y += o.y; }
        dst[(int64_t)i * it.ldd + j] = y;
    }
}

// Sector table of an enlarged block and the place of every (K sector, site state) run in it.
struct Layout {
    std::vector<std::pair<int, int>> qn;    // output sectors, ascending
    std::vector<int> dim;
    std::vector<std::array<int, 4>> osec;   // per K sector and site state: output sector
    std::vector<std::array<int, 4>> roff;   // ... and the run's offset inside it
    std::vector<int64_t> hoff;              // H' block offsets (every output sector, dim x dim)
    int64_t nH = 0;
    std::vector<std::pair<int, int>> cblk[2];   // c^dag'_sigma blocks (out, in sector index), in-sector order
    std::vector<int64_t> coff[2];
    int64_t nC[2] = {0, 0};
};

int make_layout(int side, int nsec, const int32_t* qn, const int32_t* dim, Layout& L) {
    std::map<std::pair<int, int>, int> idx;
    for (int q = 0; q < nsec; ++q)
        for (int s = 0; s < 4; ++s) idx[{qn[2 * q] + kSq[s][0], qn[2 * q + 1] + kSq[s][1]}] = 0;
    for (auto& kv : idx) { kv.second = (int)L.qn.size(); L.qn.push_back(kv.first); }
    L.dim.assign(L.qn.size(), 0);
    L.osec.assign(nsec, {0, 0, 0, 0});
    L.roff.assign(nsec, {0, 0, 0, 0});
    if (side == 0) {   // runs ordered by K sector
        for (int q = 0; q < nsec; ++q)
            for (int s = 0; s < 4; ++s) {
                const int o = idx[{qn[2 * q] + kSq[s][0], qn[2 * q + 1] + kSq[s][1]}];
                L.osec[q][s] = o; L.roff[q][s] = L.dim[o]; L.dim[o] += dim[q];
            }
    } else {           // runs ordered by site state
        for (int s = 0; s < 4; ++s)
            for (int q = 0; q < nsec; ++q) {
                const int o = idx[{qn[2 * q] + kSq[s][0], qn[2 * q + 1] + kSq[s][1]}];
                L.osec[q][s] = o; L.roff[q][s] = L.dim[o]; L.dim[o] += dim[q];
            }
    }
    L.hoff.resize(L.qn.size());
    for (size_t o = 0; o < L.qn.size(); ++o) { L.hoff[o] = L.nH; L.nH += (int64_t)L.dim[o] * L.dim[o]; }
    for (int sg = 0; sg < 2; ++sg) {
        std::vector<int> tgt(L.qn.size(), -1);   // in sector -> out sector of c^dag'_sigma
        for (int q = 0; q < nsec; ++q)
            for (const SiteHop& h : kCdag[sg]) tgt[L.osec[q][h.from]] = L.osec[q][h.to];
        for (size_t o = 0; o < L.qn.size(); ++o) {
            if (tgt[o] < 0) continue;
            L.cblk[sg].push_back({tgt[o], (int)o});
            L.coff[sg].push_back(L.nC[sg]);
            L.nC[sg] += (int64_t)L.dim[tgt[o]] * L.dim[o];
        }
    }
    return TDMRG_OK;
}

int check_block_table(int nsec, const int32_t* qn, const int32_t* dim) {
    if (nsec < 1 || !qn || !dim) return TDMRG_EINVAL;
    for (int q = 0; q < nsec; ++q) {
        if (dim[q] < 1) return TDMRG_ESECTOR;
        if (q > 0 && std::make_pair(qn[2 * q - 2], qn[2 * q - 1]) >= std::make_pair(qn[2 * q], qn[2 * q + 1]))
            return TDMRG_ESECTOR;
    }
    return TDMRG_OK;
}

int launch_places(tdmrg_ctx* c, const std::vector<Place>& items, const PlaceBufs& pb) {
    std::vector<PlaceTile> tiles;
    for (size_t k = 0; k < items.size(); ++k)
        for (int r = 0; r < items[k].rows; r += kPT)
            for (int q = 0; q < items[k].cols; q += kPT) tiles.push_back({(int)k, r, q});
    if (tiles.empty()) return TDMRG_OK;
    const size_t bi = items.size() * sizeof(Place), bt = tiles.size() * sizeof(PlaceTile);
    void* d = nullptr;
    int rc = dev_alloc(c, &d, bi + bt, "placement list");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(d, items.data(), bi, cudaMemcpyHostToDevice, c->stream), "placement upload");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync((char*)d + bi, tiles.data(), bt, cudaMemcpyHostToDevice, c->stream),
                             "placement upload");
    if (!rc) {
        c->launches++;
        rc = cuda_check(c, launch_pdl(k_place, (unsigned)tiles.size(), 256, 0, c->stream, (const Place*)d,
                                      (const PlaceTile*)((char*)d + bi), pb), "placement launch");
    }
    const int rc2 = cuda_check(c, cudaStreamSynchronize(c->stream), "placement");
    dev_free(c, d, bi + bt);
    return rc ? rc : rc2;
}

}  // namespace
}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_enlarge_size(int side, int nsec, const int32_t* qn, const int32_t* dim, int cap, int* nsec_out,
                                  int32_t* qn_out, int32_t* dim_out, int32_t* nblk_cdag, int64_t* entries) {
    if (side != 0 && side != 1) return fail(nullptr, TDMRG_EINVAL, "enlarge_size: side must be 0 or 1");
    int rc = check_block_table(nsec, qn, dim);
    if (rc) return fail(nullptr, rc, "enlarge_size: bad sector table (ascending, dims >= 1)");
    Layout L;
    make_layout(side, nsec, qn, dim, L);
    if (nsec_out) *nsec_out = (int)L.qn.size();
    if ((qn_out || dim_out) && cap < (int)L.qn.size())
        return fail(nullptr, TDMRG_EINVAL, "enlarge_size: capacity below the number of enlarged sectors");
    for (size_t o = 0; o < L.qn.size(); ++o) {
        if (qn_out) { qn_out[2 * o] = L.qn[o].first; qn_out[2 * o + 1] = L.qn[o].second; }
        if (dim_out) dim_out[o] = L.dim[o];
    }
    if (nblk_cdag) { nblk_cdag[0] = (int)L.cblk[0].size(); nblk_cdag[1] = (int)L.cblk[1].size(); }
    if (entries) { entries[0] = L.nH; entries[1] = L.nC[0]; entries[2] = L.nC[1]; }
    return TDMRG_OK;
}

namespace tdmrg {
namespace {

// The enlargement with nedge (1 or 2) bonds of the new site: edge e of K with c^dag cdag[2e + s] and
// hopping t[e]; carry_out (nullable): K's edge carried as the enlarged block's second site from the edge.
int enlarge_impl(tdmrg_ctx* c, int side, int nsec, const int32_t* qn, const int32_t* dim, const tdmrg_blocks* H,
                 int nedge, const tdmrg_blocks* cdag, const double* t, double U, tdmrg_c64* H_out,
                 tdmrg_c64* const* cdag_out, int32_t* const* cdag_qn_out, tdmrg_c64* const* n_out,
                 tdmrg_c64* const* carry_out) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if ((side != 0 && side != 1) || !H || !cdag || !t || nedge < 1 || nedge > 2 || !H_out || !cdag_out ||
        !cdag_out[0] || !cdag_out[1] || (carry_out && (!carry_out[0] || !carry_out[1])))
        return fail(c, TDMRG_EINVAL, "enlarge: bad argument");
    int rc = check_block_table(nsec, qn, dim);
    if (rc) return fail(c, rc, "enlarge: bad sector table (ascending, dims >= 1)");
    std::map<std::pair<int, int>, int> kidx;
    for (int q = 0; q < nsec; ++q) kidx[{qn[2 * q], qn[2 * q + 1]}] = q;
    auto kfind = [&](int a, int b) { auto it = kidx.find({a, b}); return it == kidx.end() ? -1 : it->second; };
    Layout L;
    make_layout(side, nsec, qn, dim, L);
    // input blocks: H_K must be sector-diagonal, c^dag_sigma must raise n_sigma by one
    std::vector<int64_t> hsrc(nsec, -1);
    if (H->nblk < 0 || (H->nblk > 0 && (!H->blk_qn || !H->data_d)))
        return fail(c, TDMRG_EINVAL, "enlarge: H blocks without data");
    {
        int64_t o = 0;
        for (int k = 0; k < H->nblk; ++k) {
            const int32_t* b = H->blk_qn + 4 * k;
            const int qo = kfind(b[0], b[1]), qi = kfind(b[2], b[3]);
            if (qo < 0 || qi < 0 || qo != qi) return fail(c, TDMRG_ESECTOR, "enlarge: H block off the sector diagonal");
            if (hsrc[qo] >= 0) return fail(c, TDMRG_ESECTOR, "enlarge: duplicate H block");
            hsrc[qo] = o;
            o += (int64_t)dim[qo] * dim[qo];
        }
    }
    std::vector<Place> items;
    auto hsec = [&](int q, int s) { return L.osec[q][s]; };
    const int8_t OH = 0, OC0 = 1;
    for (int q = 0; q < nsec; ++q)
        for (int s = 0; s < 4; ++s) {
            const int o = hsec(q, s), r = L.roff[q][s];
            const double u = s == 3 ? U : 0.0;
            Place p{};
            p.dst = L.hoff[o] + (int64_t)r * L.dim[o] + r; p.ldd = L.dim[o]; p.rows = p.cols = dim[q]; p.dbuf = OH;
            if (hsrc[q] >= 0) {
                p.mode = MODE_COPY; p.sbuf = 0; p.src = hsrc[q]; p.lds = dim[q]; p.scale = make_double2(1.0, 0.0); p.diag = u;
            } else if (u != 0.0) {
                p.mode = MODE_EYE; p.scale = make_double2(u, 0.0);
            } else {
                continue;
            }
            items.push_back(p);
        }
    // bond terms of edge e (first bonded edge: into the first launch; the other: added by a second one)
    std::vector<Place> bond_items[2];
    int first_bond = -1;
    for (int e = 0; e < nedge; ++e)
        if (t[e] != 0.0 && first_bond < 0) first_bond = e;
    for (int e = 0; e < nedge; ++e)
    for (int sg = 0; sg < 2; ++sg) {
        const tdmrg_blocks& C = cdag[2 * e + sg];
        if (C.nblk < 0 || (C.nblk > 0 && (!C.blk_qn || !C.data_d)))
            return fail(c, TDMRG_EINVAL, "enlarge: c^dag blocks without data");
        if (t[e] == 0.0) continue;
        std::vector<Place>& dst_items = e == first_bond ? items : bond_items[e];
        const double te = t[e];
        const int8_t acc = e == first_bond ? 0 : 1;
        int64_t so = 0;
        for (int k = 0; k < C.nblk; ++k) {
            const int32_t* b = C.blk_qn + 4 * k;
            const int qo = kfind(b[0], b[1]), qi = kfind(b[2], b[3]);
            if (qo < 0 || qi < 0 || b[0] - b[2] != kSq[sg == 0 ? 2 : 1][0] || b[1] - b[3] != kSq[sg == 0 ? 2 : 1][1])
                return fail(c, TDMRG_ESECTOR, "enlarge: c^dag block does not raise n_sigma by one");
            const int nq = qn[2 * qi] + qn[2 * qi + 1];   // particles of the lower K sector q
            const double pk = (nq & 1) ? -1.0 : 1.0;
            for (const SiteHop& h : kCdag[sg]) {
                // K-raising, site-lowering: (q, to) -> (q + e, from); K-lowering, site-raising: (q + e, from) -> (q, to)
                Place a{}, d{};
                if (side == 0) {   // -t (c^dag_K P_K) x c_site and -t (P_K c_K) x c^dag_site, P_K on sector q
                    a.scale = make_double2(-te * pk * h.v, 0.0);
                    d.scale = a.scale;
                } else {           // -t (P_site c_site) x c^dag_K and -t (c^dag_site P_site) x c_K, p(from)
                    a.scale = make_double2(-te * kParity[h.from] * h.v, 0.0);
                    d.scale = a.scale;
                }
                a.acc = d.acc = acc;
                const int oa = hsec(qo, h.from), ob = hsec(qi, h.to);
                if (oa != ob) return fail(c, TDMRG_ESECTOR, "enlarge: inconsistent sectors");
                a.mode = MODE_COPY; a.sbuf = (int8_t)(1 + sg); a.src = so; a.lds = dim[qi];
                a.dst = L.hoff[oa] + (int64_t)L.roff[qo][h.from] * L.dim[oa] + L.roff[qi][h.to];
                a.ldd = L.dim[oa]; a.rows = dim[qo]; a.cols = dim[qi]; a.dbuf = OH;
                d.mode = MODE_ADJ; d.sbuf = (int8_t)(1 + sg); d.src = so; d.lds = dim[qi];
                d.dst = L.hoff[oa] + (int64_t)L.roff[qi][h.to] * L.dim[oa] + L.roff[qo][h.from];
                d.ldd = L.dim[oa]; d.rows = dim[qi]; d.cols = dim[qo]; d.dbuf = OH;
                dst_items.push_back(a);
                dst_items.push_back(d);
            }
            so += (int64_t)dim[qo] * dim[qi];
        }
    }
    // K's edge carried: its blocks (q_o, q_i) copied to the runs (q_o, s) x (q_i, s) of every site state s,
    // scaled by the site parity on the right (the site's fermion comes first)
    std::vector<Place> carry_items;
    if (carry_out)
        for (int sg = 0; sg < 2; ++sg) {
            std::map<int, size_t> blk_of_in;
            for (size_t k = 0; k < L.cblk[sg].size(); ++k) blk_of_in[L.cblk[sg][k].second] = k;
            const tdmrg_blocks& C = cdag[sg];
            int64_t so = 0;
            for (int k = 0; k < C.nblk; ++k) {
                const int32_t* b = C.blk_qn + 4 * k;
                const int qo = kfind(b[0], b[1]), qi = kfind(b[2], b[3]);
                for (int st = 0; st < 4; ++st) {
                    const int oi = hsec(qi, st), oo = hsec(qo, st);
                    const auto it = blk_of_in.find(oi);
                    if (it == blk_of_in.end() || L.cblk[sg][it->second].first != oo)
                        return fail(c, TDMRG_ESECTOR, "enlarge: inconsistent carried edge sectors");
                    Place p{};
                    p.mode = MODE_COPY; p.sbuf = (int8_t)(1 + sg); p.src = so; p.lds = dim[qi];
                    p.scale = make_double2(side == 0 ? 1.0 : (double)kParity[st], 0.0);
                    p.dst = L.coff[sg][it->second] + (int64_t)L.roff[qo][st] * L.dim[oi] + L.roff[qi][st];
                    p.ldd = L.dim[oi]; p.rows = dim[qo]; p.cols = dim[qi]; p.dbuf = (int8_t)sg;
                    carry_items.push_back(p);
                }
                so += (int64_t)dim[qo] * dim[qi];
            }
        }
    // the new edge operators: scaled identities between the runs (q, from) and (q, to)
    for (int sg = 0; sg < 2; ++sg) {
        std::map<int, size_t> blk_of_in;
        for (size_t k = 0; k < L.cblk[sg].size(); ++k) blk_of_in[L.cblk[sg][k].second] = k;
        for (int q = 0; q < nsec; ++q) {
            const int nq = qn[2 * q] + qn[2 * q + 1];
            for (const SiteHop& h : kCdag[sg]) {
                const int oi = hsec(q, h.from), oo = hsec(q, h.to);
                const size_t k = blk_of_in.at(oi);
                Place p{};
                p.mode = MODE_EYE;
                p.scale = make_double2(side == 0 ? ((nq & 1) ? -h.v : h.v) : h.v, 0.0);
                p.dst = L.coff[sg][k] + (int64_t)L.roff[q][h.to] * L.dim[oi] + L.roff[q][h.from];
                p.ldd = L.dim[oi]; p.rows = p.cols = dim[q]; p.dbuf = (int8_t)(OC0 + sg);
                if (L.cblk[sg][k].first != oo) return fail(c, TDMRG_ESECTOR, "enlarge: inconsistent edge sectors");
                items.push_back(p);
            }
        }
        if (cdag_qn_out && cdag_qn_out[sg])
            for (size_t k = 0; k < L.cblk[sg].size(); ++k) {
                int32_t* b = cdag_qn_out[sg] + 4 * k;
                b[0] = L.qn[L.cblk[sg][k].first].first; b[1] = L.qn[L.cblk[sg][k].first].second;
                b[2] = L.qn[L.cblk[sg][k].second].first; b[3] = L.qn[L.cblk[sg][k].second].second;
            }
    }
    // densities of the new site: identity runs where the site state holds a particle of that spin
    for (int sg = 0; sg < 2; ++sg) {
        if (!n_out || !n_out[sg]) continue;
        for (int q = 0; q < nsec; ++q)
            for (int s = 0; s < 4; ++s) {
                if (!kSq[s][sg == 0 ? 0 : 1]) continue;
                const int o = hsec(q, s), r = L.roff[q][s];
                Place p{};
                p.mode = MODE_EYE; p.scale = make_double2(1.0, 0.0);
                p.dst = L.hoff[o] + (int64_t)r * L.dim[o] + r; p.ldd = L.dim[o]; p.rows = p.cols = dim[q];
                p.dbuf = (int8_t)(3 + sg);
                items.push_back(p);
            }
    }
    DeviceGuard g(c->opts.device);
    rc = cuda_check(c, cudaMemsetAsync(H_out, 0, (size_t)L.nH * sizeof(cplx), c->stream), "enlarge clear");
    for (int sg = 0; sg < 2 && !rc; ++sg)
        if (n_out && n_out[sg])
            rc = cuda_check(c, cudaMemsetAsync(n_out[sg], 0, (size_t)L.nH * sizeof(cplx), c->stream), "enlarge clear");
    for (int sg = 0; sg < 2 && !rc; ++sg)
        if (L.nC[sg]) rc = cuda_check(c, cudaMemsetAsync(cdag_out[sg], 0, (size_t)L.nC[sg] * sizeof(cplx), c->stream),
                                      "enlarge clear");
    for (int sg = 0; sg < 2 && !rc && carry_out; ++sg)
        if (L.nC[sg]) rc = cuda_check(c, cudaMemsetAsync(carry_out[sg], 0, (size_t)L.nC[sg] * sizeof(cplx), c->stream),
                                      "enlarge clear");
    if (rc) return rc;
    const int e0 = first_bond < 0 ? 0 : first_bond;
    PlaceBufs pb{};
    pb.d[0] = (cplx*)H_out; pb.d[1] = (cplx*)cdag_out[0]; pb.d[2] = (cplx*)cdag_out[1];
    pb.d[3] = n_out ? (cplx*)n_out[0] : nullptr; pb.d[4] = n_out ? (cplx*)n_out[1] : nullptr;
    pb.s[0] = (const cplx*)H->data_d;
    pb.s[1] = (const cplx*)cdag[2 * e0].data_d; pb.s[2] = (const cplx*)cdag[2 * e0 + 1].data_d;
    rc = launch_places(c, items, pb);
    for (int e = 0; e < nedge && !rc; ++e) {
        if (bond_items[e].empty()) continue;
        PlaceBufs pe{};
        pe.d[0] = (cplx*)H_out;
        pe.s[1] = (const cplx*)cdag[2 * e].data_d; pe.s[2] = (const cplx*)cdag[2 * e + 1].data_d;
        rc = launch_places(c, bond_items[e], pe);
    }
    if (!rc && !carry_items.empty()) {
        PlaceBufs pc{};
        pc.d[0] = (cplx*)carry_out[0]; pc.d[1] = (cplx*)carry_out[1];
        pc.s[1] = (const cplx*)cdag[0].data_d; pc.s[2] = (const cplx*)cdag[1].data_d;
        rc = launch_places(c, carry_items, pc);
    }
    return rc;
}

}  // namespace
}  // namespace tdmrg

extern "C" int tdmrg_enlarge(tdmrg_ctx* c, int side, int nsec, const int32_t* qn, const int32_t* dim,
                             const tdmrg_blocks* H, const tdmrg_blocks* cdag, double t, double U, tdmrg_c64* H_out,
                             tdmrg_c64* const* cdag_out, int32_t* const* cdag_qn_out, tdmrg_c64* const* n_out) {
    return enlarge_impl(c, side, nsec, qn, dim, H, 1, cdag, &t, U, H_out, cdag_out, cdag_qn_out, n_out, nullptr);
}

extern "C" int tdmrg_enlarge_bonds(tdmrg_ctx* c, int side, int nsec, const int32_t* qn, const int32_t* dim,
                                   const tdmrg_blocks* H, int nedge, const tdmrg_blocks* cdag, const double* t, double U,
                                   tdmrg_c64* H_out, tdmrg_c64* const* cdag_out, int32_t* const* cdag_qn_out,
                                   tdmrg_c64* const* n_out, tdmrg_c64* const* carry_out) {
    return enlarge_impl(c, side, nsec, qn, dim, H, nedge, cdag, t, U, H_out, cdag_out, cdag_qn_out, n_out, carry_out);
}

extern "C" int tdmrg_set_op_adjoint(tdmrg_ctx* c, int side, int op_id, int src_id) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if ((side != 0 && side != 1) || op_id < 0 || op_id == src_id) return fail(c, TDMRG_EINVAL, "set_op_adjoint: bad argument");
    auto it = c->ops[side].find(src_id);
    if (it == c->ops[side].end()) return fail(c, TDMRG_EINVAL, "set_op_adjoint: unknown source operator");
    const BlockOp src = it->second;
    const Side& S = c->side[side];
    std::vector<int32_t> bq;
    std::vector<Place> items;
    int64_t n = 0;
    for (const auto& b : src.blocks) {
        const int qo = std::get<0>(b), qi = std::get<1>(b);
        bq.insert(bq.end(), {S.nup[qi], S.ndn[qi], S.nup[qo], S.ndn[qo]});
        Place p{};
        p.mode = MODE_ADJ; p.sbuf = 0; p.src = std::get<2>(b); p.lds = S.dim[qi];
        p.dst = n; p.ldd = S.dim[qo]; p.rows = S.dim[qi]; p.cols = S.dim[qo]; p.dbuf = 0;
        p.scale = make_double2(1.0, 0.0);
        items.push_back(p);
        n += (int64_t)S.dim[qo] * S.dim[qi];
    }
    DeviceGuard g(c->opts.device);
    cplx* tmp = nullptr;
    int rc = dev_alloc(c, (void**)&tmp, (size_t)std::max<int64_t>(n, 1) * sizeof(cplx), "adjoint scratch");
    if (rc) return rc;
    PlaceBufs pb{};
    pb.d[0] = tmp;
    pb.s[0] = c->pool;
    rc = launch_places(c, items, pb);
    if (!rc) rc = tdmrg_set_op(c, side, op_id, src.odd, (int)src.blocks.size(), bq.data(), (const tdmrg_c64*)tmp, 1);
    cudaStreamSynchronize(c->stream);
    dev_free(c, tmp, (size_t)std::max<int64_t>(n, 1) * sizeof(cplx));
    return rc;
}
