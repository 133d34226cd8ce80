// Sector bookkeeping: compiles a superblock product sum_k coeff_k (A_k P_L^{odd B_k}) (x) B_k from
// sector Q_in to Q_out into two grouped lists of small complex GEMMs (Sec. IV, the "Hamiltonian
// connections" between the two blocks; superblock sectors of Sec. II.B).
//
// For an input pair (q', r' = Q_in - q') and a term with blocks A[q <- q'] and B[r <- r'] such that
// (q, r) is a pair of Q_out, the contribution is
//     Psi'_q += coeff * s(q') * A Psi_{q'} B^T,     s(q') = (-1)^{N(q')} if B is odd, else 1.
// Stage 1 (right products):   T = Psi_{q'} B^T  into scratch, or straight into Psi'_q when A = 1;
// stage 2 (left products):    Psi'_q = [stage-1 value] + sum coeff s A T  (and A Psi_{q'} when B = 1).
// Each stage-2 output block owns one task whose segments are all its left products, so every
// output tile accumulates all of its terms in registers before a single store (no atomics).
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace tdmrg {

int upload(tdmrg_ctx* c, TaskList& tl) {
    release(c, tl);
    struct { void** dst; const void* src; size_t bytes; } parts[3] = {
        {(void**)&tl.d_tasks, tl.tasks.data(), tl.tasks.size() * sizeof(Task)},
        {(void**)&tl.d_segs, tl.segs.data(), tl.segs.size() * sizeof(Seg)},
        {(void**)&tl.d_tiles, tl.tiles.data(), tl.tiles.size() * sizeof(Tile)}};
    for (auto& pt : parts) {
        if (!pt.bytes) continue;
        int rc = dev_alloc(c, pt.dst, pt.bytes, "task list");
        if (rc) return rc;
        // synchronous copy: the host vectors may be rebuilt before the stream reaches this point
        rc = cuda_check(c, cudaMemcpy(*pt.dst, pt.src, pt.bytes, cudaMemcpyHostToDevice), "task list upload");
        if (rc) return rc;
    }
    if (tl.nsplit) {
        int rc = dev_alloc(c, (void**)&tl.d_partials, (size_t)tl.npartial * kTileF64 * kTileF64 * sizeof(cplx),
                           "split-K partials");
        if (!rc) rc = dev_alloc(c, (void**)&tl.d_counters, (size_t)tl.nsplit * sizeof(int), "split-K tickets");
        if (!rc) rc = cuda_check(c, cudaMemset(tl.d_counters, 0, (size_t)tl.nsplit * sizeof(int)), "split-K tickets");
        if (rc) return rc;
    }
    tl.bytes = tl.tasks.size() * sizeof(Task) + tl.segs.size() * sizeof(Seg) + tl.tiles.size() * sizeof(Tile) +
               (size_t)tl.npartial * kTileF64 * kTileF64 * sizeof(cplx) + (size_t)tl.nsplit * sizeof(int);
    return TDMRG_OK;
}

void release(tdmrg_ctx* c, TaskList& tl) {
    if (tl.d_tasks) dev_free(c, tl.d_tasks, tl.tasks.size() * sizeof(Task));
    if (tl.d_segs) dev_free(c, tl.d_segs, tl.segs.size() * sizeof(Seg));
    if (tl.d_tiles) dev_free(c, tl.d_tiles, tl.tiles.size() * sizeof(Tile));
    if (tl.d_partials) dev_free(c, tl.d_partials, (size_t)tl.npartial * kTileF64 * kTileF64 * sizeof(cplx));
    if (tl.d_counters) dev_free(c, tl.d_counters, (size_t)tl.nsplit * sizeof(int));
    tl.d_tasks = nullptr; tl.d_segs = nullptr; tl.d_tiles = nullptr; tl.d_partials = nullptr; tl.d_counters = nullptr;
}

int64_t sector_size(const tdmrg_ctx* c, int n_up, int n_dn) {
    const Side& L = c->side[0];
    const Side& R = c->side[1];
    int64_t n = 0;
    for (size_t qi = 0; qi < L.dim.size(); ++qi) {
        int ri = R.find(n_up - L.nup[qi], n_dn - L.ndn[qi]);
        if (ri >= 0) n += (int64_t)L.dim[qi] * R.dim[ri];
    }
    return n;
}

void make_tiles(TaskList& tl, int tm, int tn, int ksplit) {
    tl.tiles.clear();
    tl.flops = 0.0;
    tl.nsplit = 0;
    tl.npartial = 0;
    for (size_t t = 0; t < tl.tasks.size(); ++t) {
        const Task& k = tl.tasks[t];
        int64_t ksum = 0;
        for (int s = k.seg_begin; s < k.seg_end; ++s) {
            ksum += tl.segs[s].K;
            // 8 real flops per complex multiply-add, 4 when one operand is real
            tl.flops += (tl.segs[s].rflags ? 4.0 : 8.0) * (double)k.M * k.N * (double)tl.segs[s].K;
        }
        // split long K along segment boundaries into parts of about ksplit
        std::vector<std::pair<int, int>> parts;
        const int nseg = k.seg_end - k.seg_begin;
        int want = (int)std::min<int64_t>({(ksum + ksplit - 1) / std::max(ksplit, 1), (int64_t)nseg, (int64_t)8});
        if (ksplit <= 0 || want <= 1) {
            parts.push_back({k.seg_begin, k.seg_end});
        } else {
            const double target = (double)ksum / want;
            int lo = k.seg_begin;
            int64_t acc = 0;
            for (int s = k.seg_begin; s < k.seg_end; ++s) {
                acc += tl.segs[s].K;
                const bool room = (int)parts.size() < want - 1;
                if (room && acc >= target * (parts.size() + 1) && s + 1 < k.seg_end) {
                    parts.push_back({lo, s + 1});
                    lo = s + 1;
                }
            }
            parts.push_back({lo, k.seg_end});
        }
        for (int m0 = 0; m0 < std::max(k.M, 1); m0 += tm)
            for (int n0 = 0; n0 < std::max(k.N, 1); n0 += tn) {
                if (m0 >= k.M || n0 >= k.N) continue;
                if (k.herm && n0 > m0) continue;   // upper tiles are written as mirrors of the lower ones
                int mm = std::min(tm, k.M - m0), nn = std::min(tn, k.N - n0);
                const int np = (int)parts.size();
                const int split = np > 1 ? tl.nsplit++ : -1;
                const int base = np > 1 ? tl.npartial : 0;
                if (np > 1) tl.npartial += np;
                for (int p = 0; p < np; ++p) {
                    int64_t kp = 0;
                    for (int s = parts[p].first; s < parts[p].second; ++s) kp += tl.segs[s].K;
                    int64_t cost = (int64_t)mm * nn * std::max<int64_t>(kp, 1);
                    Tile tile{};
                    tile.task = (int32_t)t; tile.m0 = m0; tile.n0 = n0;
                    tile.cost = (int32_t)std::min<int64_t>(cost, 0x7fffffff);
                    tile.seg_lo = parts[p].first; tile.seg_hi = parts[p].second;
                    tile.split = split; tile.part = p; tile.nparts = np; tile.split_base = base;
                    tl.tiles.push_back(tile);
                }
            }
    }
    // longest tiles first: the grid drains big work before the tail of small tiles
    std::stable_sort(tl.tiles.begin(), tl.tiles.end(),
                     [](const Tile& a, const Tile& b) { return a.cost > b.cost; });
}

namespace {

struct PairInfo {
    int qi, ri;
    int64_t off;
    int dl, dr;
};

std::vector<PairInfo> pairs_of(const tdmrg_ctx* c, int a, int b) {
    std::vector<PairInfo> out;
    const Side& L = c->side[0];
    const Side& R = c->side[1];
    int64_t off = 0;
    for (size_t qi = 0; qi < L.dim.size(); ++qi) {
        int ri = R.find(a - L.nup[qi], b - L.ndn[qi]);
        if (ri < 0) continue;
        out.push_back({(int)qi, ri, off, L.dim[qi], R.dim[ri]});
        off += (int64_t)L.dim[qi] * R.dim[ri];
    }
    return out;
}

}  // namespace

int build_plan(tdmrg_ctx* c, const std::vector<Term>& terms, int qa, int qb, int oa, int ob, Plan* p, bool to_device) {
    const Side& L = c->side[0];
    p->qin[0] = qa; p->qin[1] = qb; p->qout[0] = oa; p->qout[1] = ob;
    std::vector<PairInfo> pin = pairs_of(c, qa, qb), pout = pairs_of(c, oa, ob);
    p->n_in = pin.empty() ? 0 : pin.back().off + (int64_t)pin.back().dl * pin.back().dr;
    p->n_out = pout.empty() ? 0 : pout.back().off + (int64_t)pout.back().dl * pout.back().dr;
    std::vector<int> out_of_q(L.dim.size(), -1);
    for (size_t k = 0; k < pout.size(); ++k) out_of_q[pout[k].qi] = (int)k;

    std::vector<std::vector<Seg>> direct(pout.size()), left(pout.size());
    std::vector<Task> s1_inter;
    std::vector<Seg> s1_inter_seg;
    int64_t scr = 0;
    const cplx one = make_double2(1.0, 0.0);

    for (const PairInfo& pi : pin) {
        int nparity = (L.nup[pi.qi] + L.ndn[pi.qi]) & 1;
        for (const Term& t : terms) {
            const BlockOp* A = t.opL >= 0 ? &c->ops[0].at(t.opL) : nullptr;
            const BlockOp* B = t.opR >= 0 ? &c->ops[1].at(t.opR) : nullptr;
            double sgn = (B && B->odd && nparity) ? -1.0 : 1.0;
            // a connection's coefficient is either folded into the segment or read at run time from the
            // caller's device array (tdmrg_set_coefficients); the fermion sign stays static
            const bool run_time = c->dcoef != nullptr && t.conn >= 0;
            cplx sc = run_time ? make_double2(sgn, 0.0) : make_double2(sgn * t.coeff.x, sgn * t.coeff.y);
            const int dcoef = run_time ? t.conn : -1;
            // real operands skip their imaginary products: A (left operator) with a real static factor,
            // B (right operator) always (its factor goes on A in the FP64 kernel)
            const int8_t a_real = (A && A->real && sc.y == 0.0 && dcoef < 0) ? 1 : 0;
            const int8_t b_real = (B && B->real) ? 2 : 0;
            std::vector<std::pair<int, int64_t>> al, bl;
            if (!A) al.push_back({pi.qi, -1});
            else for (auto& blk : A->blocks) if (std::get<1>(blk) == pi.qi) al.push_back({std::get<0>(blk), std::get<2>(blk)});
            if (!B) bl.push_back({pi.ri, -1});
            else for (auto& blk : B->blocks) if (std::get<1>(blk) == pi.ri) bl.push_back({std::get<0>(blk), std::get<2>(blk)});
            for (auto& a : al) {
                int ko = out_of_q[a.first];
                if (ko < 0) continue;
                const PairInfo& po = pout[ko];
                for (auto& b : bl) {
                    if (b.first != po.ri) continue;
                    if (!A && !B) return fail(c, TDMRG_EINVAL, "a term needs an operator on at least one block");
                    if (!A) {          // Psi'_q += sc * Psi_q B^T, written by stage 1
                        Seg s{};
                        s.a_off = pi.off; s.a_buf = BUF_IN; s.lda = pi.dr;
                        s.b_off = b.second; s.b_buf = BUF_OPS; s.ldb = pi.dr; s.opb = OPB_T;
                        s.K = pi.dr; s.scale = sc; s.dscale = -1; s.dcoef = dcoef;
                        s.rflags = b_real;
                        direct[ko].push_back(s);
                    } else if (!B) {   // Psi'_q += sc * A Psi_{q'}
                        Seg s{};
                        s.a_off = a.second; s.a_buf = BUF_OPS; s.lda = pi.dl;
                        s.b_off = pi.off; s.b_buf = BUF_IN; s.ldb = pi.dr; s.opb = OPB_N;
                        s.K = pi.dl; s.scale = sc; s.dscale = -1; s.dcoef = dcoef;
                        s.rflags = a_real;
                        left[ko].push_back(s);
                    } else {           // T = Psi_{q'} B^T (scratch, stored as T^T), then Psi'_q += sc * A T
                        // T^T rows are the columns of T: the stage-1 stores and the stage-2 operand
                        // reads (slicing of the columns of T) run along contiguous memory
                        Task tk{};
                        tk.c_off = scr; tk.c_buf = BUF_SCRATCH; tk.ldc = pi.dl; tk.M = pi.dl; tk.N = po.dr;
                        tk.beta = 0; tk.trans = 1;
                        Seg s{};
                        s.a_off = pi.off; s.a_buf = BUF_IN; s.lda = pi.dr;
                        s.b_off = b.second; s.b_buf = BUF_OPS; s.ldb = pi.dr; s.opb = OPB_T;
                        s.K = pi.dr; s.scale = one; s.dscale = -1;
                        s.rflags = b_real;
                        s1_inter.push_back(tk);
                        s1_inter_seg.push_back(s);
                        Seg s2{};
                        s2.a_off = a.second; s2.a_buf = BUF_OPS; s2.lda = pi.dl;
                        s2.b_off = scr; s2.b_buf = BUF_SCRATCH; s2.ldb = pi.dl; s2.opb = OPB_T;
                        s2.K = pi.dl; s2.scale = sc; s2.dscale = -1; s2.dcoef = dcoef;
                        s2.rflags = a_real;
                        left[ko].push_back(s2);
                        scr += (int64_t)pi.dl * po.dr;
                    }
                }
            }
        }
    }
    // stage 1: direct writes into the output, then scratch intermediates
    TaskList& s1 = p->stage1;
    TaskList& s2 = p->stage2;
    release(c, s1); release(c, s2);
    s1.tasks.clear(); s1.segs.clear(); s2.tasks.clear(); s2.segs.clear();
    for (size_t k = 0; k < pout.size(); ++k) {
        if (direct[k].empty()) continue;
        Task tk{};
        tk.c_off = pout[k].off; tk.c_buf = BUF_OUT; tk.ldc = pout[k].dr; tk.M = pout[k].dl; tk.N = pout[k].dr;
        tk.beta = 0;
        tk.seg_begin = (int)s1.segs.size();
        for (auto& s : direct[k]) s1.segs.push_back(s);
        tk.seg_end = (int)s1.segs.size();
        s1.tasks.push_back(tk);
    }
    for (size_t k = 0; k < s1_inter.size(); ++k) {
        Task tk = s1_inter[k];
        tk.seg_begin = (int)s1.segs.size();
        s1.segs.push_back(s1_inter_seg[k]);
        tk.seg_end = (int)s1.segs.size();
        s1.tasks.push_back(tk);
    }
    // stage 2: one task per output block that still needs left products or a zero fill
    for (size_t k = 0; k < pout.size(); ++k) {
        bool has_direct = !direct[k].empty();
        if (has_direct && left[k].empty()) continue;
        Task tk{};
        tk.c_off = pout[k].off; tk.c_buf = BUF_OUT; tk.ldc = pout[k].dr; tk.M = pout[k].dl; tk.N = pout[k].dr;
        tk.beta = has_direct ? 1 : 0;
        tk.seg_begin = (int)s2.segs.size();
        for (auto& s : left[k]) s2.segs.push_back(s);
        tk.seg_end = (int)s2.segs.size();
        s2.tasks.push_back(tk);
    }
    make_tiles(s1, kTileF64, kTileF64, kSplitK);
    make_tiles(s2, kTileF64, kTileF64, kSplitK);
    p->scratch = scr;
    p->flops = s1.flops + s2.flops;
    if (!to_device) return TDMRG_OK;   // host task lists only (merged into a larger launch by the caller)
    int urc = upload(c, s1);
    if (!urc) urc = upload(c, s2);
    if (urc) return urc;
    if (scr > c->scratch_cap) {
        if (c->scratch) dev_free(c, c->scratch, c->scratch_cap * sizeof(cplx));
        c->scratch = nullptr;
        c->scratch_cap = 0;
        int rc = dev_alloc(c, (void**)&c->scratch, scr * sizeof(cplx), "superblock scratch");
        if (rc) return rc;
        c->scratch_cap = scr;
    }
    return cuda_check(c, cudaGetLastError(), "plan upload");
}

int run_plan(tdmrg_ctx* c, const Plan& p, const cplx* in, cplx* out, const int* skip_flag, int skip_step) {
    if (p.oz.ready) return run_oz(c, p, in, out, skip_flag, skip_step);
    GemmArgs a{};
    a.bufs[BUF_OPS] = c->pool;
    a.bufs[BUF_IN] = const_cast<cplx*>(in);
    a.bufs[BUF_SCRATCH] = c->scratch;
    a.bufs[BUF_OUT] = out;
    a.dscale = c->dscale;
    a.dcoef = c->dcoef;
    for (const TaskList* tl : {&p.stage1, &p.stage2}) {
        if (tl->tiles.empty()) continue;
        a.tasks = tl->d_tasks; a.segs = tl->d_segs; a.tiles = tl->d_tiles; a.ntiles = (int)tl->tiles.size();
        a.partials = tl->d_partials; a.counters = tl->d_counters;
        cudaError_t e = launch_gemm_f64(a, c->stream, skip_flag, skip_step);
        c->launches++;
        int rc = cuda_check(c, e, "superblock product launch");
        if (rc) return rc;
    }
    return TDMRG_OK;
}

}  // namespace tdmrg
