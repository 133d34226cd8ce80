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

}  // namespace

int density_matrix(tdmrg_ctx* c, int side, int nt, const int32_t* Q, const cplx* const* psi, const double* w, cplx* rho) {
    const Side& L = c->side[0];
    const Side& R = c->side[1];
    cudaStream_t s = c->stream;
    // norms of the targets -> dscale[l] = w_l / ||psi_l||^2
    std::vector<int64_t> nl(nt);
    for (int l = 0; l < nt; ++l) {
        nl[l] = sector_size(c, Q[2 * l], Q[2 * l + 1]);
        if (nl[l] == 0) return fail(c, TDMRG_ESECTOR, "density_matrix: target in an empty sector");
        cudaError_t e = launch_norm2(psi[l], nl[l], c->red + (int64_t)l * NB, NB, s);
        c->launches++;
        if (e != cudaSuccess) return cuda_check(c, e, "density_matrix norms");
    }
    Weights wl{};
    for (int l = 0; l < nt; ++l) wl.w[l] = w[l];
    launch_pdl(k_weight_scale, 1, 32 * 12, 0, s, c->red, nt, c->dscale, wl);
    c->launches++;
    // task list: one task per sector of the side, compiled once per (side, set of target sectors)
    std::vector<int> key(Q, Q + 2 * nt);
    key.push_back(side);
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
                sg.K = L.dim[qi]; sg.scale = make_double2(1.0, 0.0); sg.dscale = l;
                segs[ri].push_back(sg);
                po += (int64_t)L.dim[qi] * R.dim[ri];
            }
        }
        int64_t off = 0;
        for (size_t ri = 0; ri < R.dim.size(); ++ri) {
            Task tk{};
            tk.c_off = off; tk.c_buf = BUF_OUT; tk.ldc = R.dim[ri]; tk.M = R.dim[ri]; tk.N = R.dim[ri]; tk.beta = 0;
            tk.herm = 1;
            tk.seg_begin = (int)tl->segs.size();
            tl->segs.insert(tl->segs.end(), segs[ri].begin(), segs[ri].end());
            tk.seg_end = (int)tl->segs.size();
            tl->tasks.push_back(tk);
            off += (int64_t)R.dim[ri] * R.dim[ri];
        }
        make_tiles(*tl, kTileF64, kTileF64, kSplitK);
        int rc = upload(c, *tl);
        if (rc) { release(c, *tl); return rc; }
        it = c->rho_plans.emplace(key, std::move(tl)).first;
    }
    if (it == c->rho_plans.end()) {
        std::unique_ptr<TaskList> tl(new TaskList());
        int64_t off = 0;
        for (size_t qi = 0; qi < L.dim.size(); ++qi) {
            Task tk{};
            tk.c_off = off; tk.c_buf = BUF_OUT; tk.ldc = L.dim[qi]; tk.M = L.dim[qi]; tk.N = L.dim[qi]; tk.beta = 0;
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
                sg.K = R.dim[ri]; sg.scale = make_double2(1.0, 0.0); sg.dscale = l;
                tl->segs.push_back(sg);
            }
            tk.seg_end = (int)tl->segs.size();
            tl->tasks.push_back(tk);
            off += (int64_t)L.dim[qi] * L.dim[qi];
        }
        make_tiles(*tl, kTileF64, kTileF64, kSplitK);
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
    a.dscale = c->dscale;
    cudaError_t e = launch_gemm_f64(a, s, nullptr, 0);
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
