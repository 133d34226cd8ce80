// Weighted reduced density matrix of the targeted states (Eq. rdensitymatrix; weights of
// Sec. II.C) and its eigendecomposition, which feeds the truncation of Sec. II.B.
//
// rho_L(q) = sum_l w_l / <psi_l|psi_l> Psi_l(q) Psi_l(q)^dag, with Psi_l(q) the dL(q) x dR(Q_l - q)
// block of target l in its own sector Q_l.  Each left sector is one task of the grouped FP64 GEMM
// (segments A = Psi_l(q), op(B) = Psi_l(q)^dag, real device scale w_l / ||psi_l||^2), so all sectors
// and all targets go in one launch.  The right block's matrix (the block truncated when the sweep moves
// left) is rho_R(r) = sum_l w_l / <psi_l|psi_l> sum_{q: Q_l - q = r} Psi_l(q)^T conj(Psi_l(q)), i.e.
// rho_R[b, b'] = sum_a Psi[a, b] conj(Psi[a, b']): one task per right sector, segments A = Psi_l(q)^T,
// op(B) = conj(Psi_l(q)).  The eigendecomposition is in eig.cu.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int NB = kRedBlocks;

struct Weights { double w[12]; };

__global__ void k_weight_scale(const double2* __restrict__ part, int nt, double* __restrict__ dscale, Weights ws) {
    pdl_enter();
    // one warp per target: dscale[l] = w_l / ||psi_l||^2 (0 for a zero state)
    const int l = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (l >= nt) return;
    double s = 0.0;
    for (int b = lane; b < NB; b += 32) s += part[(int64_t)l * NB + b].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dscale[l] = s > 0.0 ? ws.w[l] / s : 0.0;
}

// Real-basis variant: Re rho_L = sum_l w_l (Re Psi_l Re Psi_l^T + Im Psi_l Im Psi_l^T) / <psi_l|psi_l>, the
// real part of the Hermitian rho_L (each target's real and imaginary parts targeted apart).
__global__ void k_real_part(cplx* __restrict__ rho, int64_t n) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rho[i].y = 0.0;
}

// Direct sum of superblocks: each target is normalised per source, dscale[l * nsrc + k] = w_l / ||psi_l^(k)||^2
// with psi_l^(k) the elements of source k (one block per (target, source), fixed-order block sum).
struct SegNorm { int64_t lo, hi; int l, k; };
struct TargetList { const cplx* p[12]; };
__global__ void __launch_bounds__(256) k_seg_weight(const SegNorm* __restrict__ segs, TargetList tl, Weights ws, int nsrc,
                                                    double* __restrict__ dscale) {
    pdl_enter();
    __shared__ double sh[8];
    const SegNorm sg = segs[blockIdx.x];
    const cplx* x = tl.p[sg.l];
    double s = 0.0;
    for (int64_t i = sg.lo + threadIdx.x; i < sg.hi; i += 256) { const double2 v = x[i]; s += v.x * v.x + v.y * v.y; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[k];
        dscale[sg.l * nsrc + sg.k] = t > 0.0 ? ws.w[sg.l] / t : 0.0;
    }
}

}  // namespace

int density_matrix(tdmrg_ctx* c, int side, int nt, const int32_t* Q, const cplx* const* psi, const double* w, cplx* rho,
                   bool grouped) {
    const Side& L = c->side[0];
    const Side& R = c->side[1];
    cudaStream_t s = c->stream;
    Weights wl{};
    for (int l = 0; l < nt; ++l) wl.w[l] = w[l];
    const int nsrc = c->dsum_nsrc;   // > 0: a direct sum, normalised per source
    double* dscale = c->dscale;
    if (nsrc > 0) {
        const size_t need = (size_t)nt * nsrc * sizeof(double);
        if (c->dsum_dscale_bytes < need) {
            dev_free(c, c->dsum_dscale, c->dsum_dscale_bytes);
            c->dsum_dscale = nullptr;
            c->dsum_dscale_bytes = 0;
            int rc = dev_alloc(c, (void**)&c->dsum_dscale, need, "direct sum scales");
            if (rc) return rc;
            c->dsum_dscale_bytes = need;
        }
        dscale = c->dsum_dscale;
        // the ranges of every (target, source) pair, built once per set of target sectors (outside any
        // stream capture: the first call of a captured step runs directly)
        std::vector<int> nkey(Q, Q + 2 * nt);
        auto nit = c->dsum_norms.find(nkey);
        if (nit == c->dsum_norms.end()) {
            std::vector<SegNorm> segs;
            for (int l = 0; l < nt; ++l) {   // pairs come by left sector, and the left sectors by source
                std::vector<int64_t> lo(nsrc, -1), hi(nsrc, -1);
                int64_t off = 0;
                for (size_t qi = 0; qi < L.dim.size(); ++qi) {
                    const int ri = R.find(Q[2 * l] - L.nup[qi], Q[2 * l + 1] - L.ndn[qi]);
                    if (ri < 0) continue;
                    const int k = c->dsum_src[0][qi];
                    if (lo[k] < 0) lo[k] = off;
                    off += (int64_t)L.dim[qi] * R.dim[ri];
                    hi[k] = off;
                }
                if (off == 0) return fail(c, TDMRG_ESECTOR, "density_matrix: target in an empty sector");
                for (int k = 0; k < nsrc; ++k) segs.push_back({lo[k] < 0 ? 0 : lo[k], lo[k] < 0 ? 0 : hi[k], l, k});
            }
            tdmrg_ctx::DsumNorms dn;
            dn.bytes = segs.size() * sizeof(SegNorm);
            dn.count = (int)segs.size();
            int rc = dev_alloc(c, &dn.d, dn.bytes, "direct sum norms");
            if (!rc) rc = cuda_check(c, cudaMemcpyAsync(dn.d, segs.data(), dn.bytes, cudaMemcpyHostToDevice, s), "direct sum norms");
            if (!rc) rc = cuda_check(c, cudaStreamSynchronize(s), "direct sum norms");
            if (rc) { dev_free(c, dn.d, dn.bytes); return rc; }
            nit = c->dsum_norms.emplace(nkey, dn).first;
        }
        TargetList tl{};
        for (int l = 0; l < nt; ++l) tl.p[l] = psi[l];
        c->launches++;
        int rc = cuda_check(c, launch_pdl(k_seg_weight, nit->second.count, 256, 0, s, (const SegNorm*)nit->second.d, tl, wl,
                                          nsrc, dscale), "direct sum norms");
        if (rc) return rc;
    } else {
        // norms of the targets -> dscale[l] = w_l / ||psi_l||^2; partials in the upper half of the reduction
        // workspace, apart from those of tdmrg_expect / tdmrg_overlap_op (which may run beside on another stream)
        double2* nred = c->red + 64 * (int64_t)NB;
        for (int l = 0; l < nt; ++l) {
            const int64_t nl = sector_size(c, Q[2 * l], Q[2 * l + 1]);
            if (nl == 0) return fail(c, TDMRG_ESECTOR, "density_matrix: target in an empty sector");
            cudaError_t e = launch_norm2(psi[l], nl, nred + (int64_t)l * NB, NB, s);
            c->launches++;
            if (e != cudaSuccess) return cuda_check(c, e, "density_matrix norms");
        }
        launch_pdl(k_weight_scale, 1, 32 * 12, 0, s, nred, nt, c->dscale, wl);
        c->launches++;
    }
    // task list: one task per sector of the side, compiled once per (side, set of target sectors, order);
    // grouped: the eigensolver's first group's sectors first, so that their tiles form one launch
    const EigWork& ew = c->eig[side];
    grouped = grouped && ew.ready && ew.ngroups == 2;
    const int nsec = (int)c->side[side].dim.size();
    std::vector<int> order;
    if (grouped) {
        order = ew.grp[0].sel;
        order.insert(order.end(), ew.grp[1].sel.begin(), ew.grp[1].sel.end());
    } else {
        for (int q = 0; q < nsec; ++q) order.push_back(q);
    }
    const int nfirst = grouped ? (int)ew.grp[0].sel.size() : 0;
    std::vector<int> key(Q, Q + 2 * nt);
    key.push_back(side);
    key.push_back(nsrc);
    key.push_back(grouped ? 1 : 0);
    auto it = c->rho_plans.find(key);
    if (it == c->rho_plans.end() && side == 1) {
        std::unique_ptr<TaskList> tl(new TaskList());
        std::vector<std::vector<Seg>> segs(R.dim.size());
        for (int l = 0; l < nt; ++l) {
            int64_t po = 0;   // offset of Psi_l(q) inside target l
            for (size_t qi = 0; qi < L.dim.size(); ++qi) {
                const int ri = R.find(Q[2 * l] - L.nup[qi], Q[2 * l + 1] - L.ndn[qi]);
                if (ri < 0) continue;
                Seg sg{};
                sg.a_off = po; sg.a_buf = (int8_t)(BUF_EXTRA0 + l); sg.lda = R.dim[ri]; sg.opa = 1;   // Psi^T
                sg.b_off = po; sg.b_buf = (int8_t)(BUF_EXTRA0 + l); sg.ldb = R.dim[ri]; sg.opb = OPB_CN;
                sg.K = L.dim[qi]; sg.scale = make_double2(1.0, 0.0);
                sg.dscale = nsrc > 0 ? l * nsrc + c->dsum_src[0][qi] : l;
                segs[ri].push_back(sg);
                po += (int64_t)L.dim[qi] * R.dim[ri];
            }
        }
        std::vector<int64_t> roff(R.dim.size() + 1, 0);
        for (size_t ri = 0; ri < R.dim.size(); ++ri) roff[ri + 1] = roff[ri] + (int64_t)R.dim[ri] * R.dim[ri];
        for (int ri : order) {
            Task tk{};
            tk.c_off = roff[ri]; tk.c_buf = BUF_OUT; tk.ldc = R.dim[ri]; tk.M = R.dim[ri]; tk.N = R.dim[ri]; tk.beta = 0;
            tk.herm = 1;
            tk.seg_begin = (int)tl->segs.size();
            tl->segs.insert(tl->segs.end(), segs[ri].begin(), segs[ri].end());
            tk.seg_end = (int)tl->segs.size();
            tl->tasks.push_back(tk);
        }
        make_tiles(*tl, kTileF64, kTileF64, kSplitK);
        for (const Tile& t : tl->tiles) tl->ntiles_first += t.task < nfirst ? 1 : 0;
        int rc = upload(c, *tl);
        if (rc) { release(c, *tl); return rc; }
        it = c->rho_plans.emplace(key, std::move(tl)).first;
    }
    if (it == c->rho_plans.end()) {
        std::unique_ptr<TaskList> tl(new TaskList());
        std::vector<int64_t> loff(L.dim.size() + 1, 0);
        for (size_t qi = 0; qi < L.dim.size(); ++qi) loff[qi + 1] = loff[qi] + (int64_t)L.dim[qi] * L.dim[qi];
        for (int qi : order) {
            Task tk{};
            tk.c_off = loff[qi]; tk.c_buf = BUF_OUT; tk.ldc = L.dim[qi]; tk.M = L.dim[qi]; tk.N = L.dim[qi]; tk.beta = 0;
            tk.herm = 1;   // rho_L(q) is Hermitian: lower tiles plus mirror (a batched HERK)
            tk.seg_begin = (int)tl->segs.size();
            for (int l = 0; l < nt; ++l) {
                int ri = R.find(Q[2 * l] - L.nup[qi], Q[2 * l + 1] - L.ndn[qi]);
                if (ri < 0) continue;
                int64_t po = 0;   // offset of Psi_l(q) inside target l
                for (size_t k = 0; k < qi; ++k) {
                    int rk = R.find(Q[2 * l] - L.nup[k], Q[2 * l + 1] - L.ndn[k]);
                    if (rk >= 0) po += (int64_t)L.dim[k] * R.dim[rk];
                }
                Seg sg{};
                sg.a_off = po; sg.a_buf = (int8_t)(BUF_EXTRA0 + l); sg.lda = R.dim[ri];
                sg.b_off = po; sg.b_buf = (int8_t)(BUF_EXTRA0 + l); sg.ldb = R.dim[ri]; sg.opb = OPB_C;
                sg.K = R.dim[ri]; sg.scale = make_double2(1.0, 0.0);
                sg.dscale = nsrc > 0 ? l * nsrc + c->dsum_src[0][qi] : l;
                tl->segs.push_back(sg);
            }
            tk.seg_end = (int)tl->segs.size();
            tl->tasks.push_back(tk);
        }
        make_tiles(*tl, kTileF64, kTileF64, kSplitK);
        for (const Tile& t : tl->tiles) tl->ntiles_first += t.task < nfirst ? 1 : 0;
        int rc = upload(c, *tl);
        if (rc) { release(c, *tl); return rc; }
        it = c->rho_plans.emplace(key, std::move(tl)).first;
    }
    const TaskList& tl = *it->second;
    GemmArgs a{};
    a.tasks = tl.d_tasks; a.segs = tl.d_segs; a.tiles = tl.d_tiles; a.ntiles = (int)tl.tiles.size();
    a.partials = tl.d_partials; a.counters = tl.d_counters;
    a.bufs[BUF_OPS] = c->pool;
    a.bufs[BUF_OUT] = rho;
    for (int l = 0; l < nt; ++l) a.bufs[BUF_EXTRA0 + l] = const_cast<cplx*>(psi[l]);
    a.dscale = dscale;
    cudaError_t e = cudaSuccess;
    if (grouped) {   // the first group's blocks on its stream, forked after the norms and weights
        e = cudaEventRecord(ew.fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ew.side, ew.fork, 0);
        GemmArgs a1 = a;
        a1.ntiles = tl.ntiles_first;
        if (e == cudaSuccess) e = launch_gemm_f64(a1, ew.side, nullptr, 0);
        a.tiles = tl.d_tiles + tl.ntiles_first;
        a.ntiles = (int)tl.tiles.size() - tl.ntiles_first;
        c->launches++;
    }
    if (e == cudaSuccess) e = launch_gemm_f64(a, s, nullptr, 0);
    c->launches++;
    if (e == cudaSuccess && c->real_basis) {
        int64_t nr = 0;
        for (int d : c->side[side].dim) nr += (int64_t)d * d;
        launch_pdl(k_real_part, (int)std::min<int64_t>((nr + 255) / 256, 4L * c->num_sms), 256, 0, s, rho, nr);
        c->launches++;
        e = cudaGetLastError();
    }
    return cuda_check(c, e, "density_matrix launch");
}

}  // namespace tdmrg
