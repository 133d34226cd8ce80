// Correlation grid <phi1| A_i B_j |phi2> over a list of left operators A_i and right operators B_j: the
// two-state form of Eq. generalcorrelation with one local operator per block, e.g. the Green's function
// G_ij(t) = <phi(t)| c_i c^dag_j |psi(t)> (Sec. I) measured on device-resident states.
//
// Every product W_ij = (A_i P_L^{odd B_j}) (x) B_j phi2 is compiled by the sector bookkeeping of a
// superblock product (plan.cu); the products of the whole grid are merged into one pair of task lists,
// so the grid costs two grouped FP64 launches (right products into per-product scratch, left products
// into per-product vectors of sector Q1), then a fixed-order reduction of <phi1|W_ij> per entry
// (partials over kCorrChunks chunks, summed in chunk order).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int CT = 256;

// part[p * kCorrChunks + chunk] = sum over the chunk of conj(phi1) W_p
__global__ void __launch_bounds__(CT) k_corr_dots(const cplx* __restrict__ phi1, const cplx* __restrict__ W, int64_t n,
                                                  double2* __restrict__ part) {
    pdl_enter();
    const int p = blockIdx.x, ch = blockIdx.y;
    const int64_t len = (n + kCorrChunks - 1) / kCorrChunks;
    const int64_t lo = min(n, (int64_t)ch * len), hi = min(n, lo + len);
    const cplx* __restrict__ w = W + (int64_t)p * n;
    double sr = 0.0, si = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += CT) {
        const double2 a = phi1[i], b = w[i];
        sr = fma(a.x, b.x, fma(a.y, b.y, sr));
        si = fma(a.x, b.y, fma(-a.y, b.x, si));
    }
    __shared__ double2 sh[CT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_double2(sr, si);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < CT / 32; ++k) { t.x += sh[k].x; t.y += sh[k].y; }
        part[(int64_t)p * kCorrChunks + ch] = t;
    }
}

__global__ void k_corr_final(const double2* __restrict__ part, int npairs, cplx* __restrict__ out) {
    pdl_enter();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    double2 t = make_double2(0.0, 0.0);
    for (int k = 0; k < kCorrChunks; ++k) { t.x += part[(int64_t)p * kCorrChunks + k].x; t.y += part[(int64_t)p * kCorrChunks + k].y; }
    out[p] = t;
}

void free_corr(tdmrg_ctx* c, CorrPlan& cp) {
    release(c, cp.s1);
    release(c, cp.s2);
    dev_free(c, cp.T, (size_t)cp.scratch * sizeof(cplx));
    dev_free(c, cp.W, (size_t)cp.npairs * cp.n1 * sizeof(cplx));
    dev_free(c, cp.part, (size_t)cp.npairs * kCorrChunks * sizeof(double2));
}

// Appends the task lists of one product to the merged lists, its scratch at `sbase` and its output
// vector at `obase` (element offsets).
void append(TaskList& dst, const TaskList& src, int64_t sbase, int64_t obase) {
    const int seg0 = (int)dst.segs.size();
    for (Seg s : src.segs) {
        if (s.a_buf == BUF_SCRATCH) s.a_off += sbase;
        if (s.b_buf == BUF_SCRATCH) s.b_off += sbase;
        dst.segs.push_back(s);
    }
    for (Task t : src.tasks) {
        t.c_off += t.c_buf == BUF_SCRATCH ? sbase : obase;
        t.seg_begin += seg0;
        t.seg_end += seg0;
        dst.tasks.push_back(t);
    }
}

}  // namespace

void release_corr(tdmrg_ctx* c) {
    for (auto& kv : c->corr_plans) free_corr(c, *kv.second);
    c->corr_plans.clear();
}

}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_correlation(tdmrg_ctx* c, int nL, const int32_t* opL, int nR, const int32_t* opR, int a1, int b1,
                                 const tdmrg_c64* phi1, int a2, int b2, const tdmrg_c64* phi2, tdmrg_c64* out) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if (nL < 1 || nR < 1 || !opL || !opR || !phi1 || !phi2 || !out) return fail(c, TDMRG_EINVAL, "correlation: bad argument");
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "correlation: blocks not set");
    for (int i = 0; i < nL; ++i)
        if (opL[i] >= 0 && !c->ops[0].count(opL[i])) return fail(c, TDMRG_EINVAL, "correlation: left op id not set");
    for (int j = 0; j < nR; ++j)
        if (opR[j] >= 0 && !c->ops[1].count(opR[j])) return fail(c, TDMRG_EINVAL, "correlation: right op id not set");
    for (int i = 0; i < nL; ++i)
        for (int j = 0; j < nR; ++j)
            if (opL[i] < 0 && opR[j] < 0) return fail(c, TDMRG_EINVAL, "correlation: a product with two identities");
    const int64_t n1 = sector_size(c, a1, b1);
    if (n1 == 0 || sector_size(c, a2, b2) == 0) return fail(c, TDMRG_ESECTOR, "correlation: empty sector");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->opts.device) cudaSetDevice(c->opts.device);
    std::vector<int> key{nL, nR, a1, b1, a2, b2};
    key.insert(key.end(), opL, opL + nL);
    key.insert(key.end(), opR, opR + nR);
    auto it = c->corr_plans.find(key);
    int rc = TDMRG_OK;
    if (it == c->corr_plans.end()) {   // compile every product of the grid, merged into two task lists
        std::unique_ptr<CorrPlan> cp(new CorrPlan());
        cp->npairs = nL * nR;
        cp->n1 = n1;
        for (int i = 0; i < nL && !rc; ++i)
            for (int j = 0; j < nR && !rc; ++j) {
                Plan p;
                std::vector<Term> terms{{opL[i], opR[j], make_double2(1.0, 0.0)}};
                rc = build_plan(c, terms, a2, b2, a1, b1, &p, false);
                if (rc) break;
                append(cp->s1, p.stage1, cp->scratch, (int64_t)(i * nR + j) * n1);
                append(cp->s2, p.stage2, cp->scratch, (int64_t)(i * nR + j) * n1);
                cp->scratch += p.scratch;
            }
        if (!rc) {
            make_tiles(cp->s1, kTileF64, kTileF64, kSplitK);
            make_tiles(cp->s2, kTileF64, kTileF64, kSplitK);
            rc = upload(c, cp->s1);
            if (!rc) rc = upload(c, cp->s2);
            if (!rc) rc = dev_alloc(c, (void**)&cp->T, (size_t)std::max<int64_t>(cp->scratch, 1) * sizeof(cplx), "correlation scratch");
            if (!rc) rc = dev_alloc(c, (void**)&cp->W, (size_t)cp->npairs * n1 * sizeof(cplx), "correlation vectors");
            if (!rc) rc = dev_alloc(c, (void**)&cp->part, (size_t)cp->npairs * kCorrChunks * sizeof(double2), "correlation partials");
        }
        if (rc) {
            free_corr(c, *cp);
            if (prev >= 0 && prev != c->opts.device) cudaSetDevice(prev);
            return rc;
        }
        it = c->corr_plans.emplace(key, std::move(cp)).first;
    }
    CorrPlan& cp = *it->second;
    GemmArgs g{};
    g.bufs[BUF_OPS] = c->pool;
    g.bufs[BUF_IN] = (cplx*)phi2;
    g.bufs[BUF_SCRATCH] = cp.T;
    g.bufs[BUF_OUT] = cp.W;
    g.dscale = c->dscale;
    for (TaskList* tl : {&cp.s1, &cp.s2}) {
        if (tl->tiles.empty() || rc) continue;
        g.tasks = tl->d_tasks; g.segs = tl->d_segs; g.tiles = tl->d_tiles; g.ntiles = (int)tl->tiles.size();
        g.partials = tl->d_partials; g.counters = tl->d_counters;
        c->launches++;
        rc = cuda_check(c, launch_gemm_f64(g, c->stream, nullptr, 0), "correlation products");
    }
    if (!rc) {
        launch_pdl(k_corr_dots, dim3(cp.npairs, kCorrChunks), CT, 0, c->stream, (const cplx*)phi1, (const cplx*)cp.W, n1, cp.part);
        launch_pdl(k_corr_final, (cp.npairs + 127) / 128, 128, 0, c->stream, (const double2*)cp.part, cp.npairs, (cplx*)out);
        c->launches += 2;
        rc = cuda_check(c, cudaGetLastError(), "correlation dots");
    }
    if (prev >= 0 && prev != c->opts.device) cudaSetDevice(prev);
    return rc;
}
