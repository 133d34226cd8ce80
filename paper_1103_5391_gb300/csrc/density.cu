// Weighted reduced density matrix of the targeted states (Eq. rdensitymatrix; weights of
// Sec. II.C) and its eigendecomposition, which feeds the truncation of Sec. II.B.
//
// rho_L(q) = sum_l w_l / <psi_l|psi_l> Psi_l(q) Psi_l(q)^dag, with Psi_l(q) the dL(q) x dR(Q_l - q)
// block of target l in its own sector Q_l.  Each left sector is one task of the grouped FP64 GEMM
// (segments A = Psi_l(q), op(B) = Psi_l(q)^dag, real device scale w_l / ||psi_l||^2), so all sectors
// and all targets go in one launch.  The eigendecomposition is a batched two-sided cyclic Jacobi
// (one CTA per sector, parallel round-robin ordering of disjoint rotations), FP64 throughout.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int NB = kRedBlocks;

struct Weights { double w[12]; };

__global__ void k_weight_scale(const double2* __restrict__ part, int nt, double* __restrict__ dscale, Weights ws) {
    // one warp per target: dscale[l] = w_l / ||psi_l||^2 (0 for a zero state)
    const int l = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (l >= nt) return;
    double s = 0.0;
    for (int b = lane; b < NB; b += 32) s += part[(int64_t)l * NB + b].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dscale[l] = s > 0.0 ? ws.w[l] / s : 0.0;
}

// ---- batched Hermitian Jacobi -----------------------------------------------------------------
// A (n x n Hermitian) and V live in shared memory when 2 n^2 complex fit, else in global workspace.
constexpr int EIG_THREADS = 256;

struct EigArgs {
    const cplx* rho;
    double* evals;
    cplx* evecs;
    const int64_t* rho_off;   // per sector: offset of its n x n block
    const int64_t* ev_off;    // per sector: offset of its eigenvalues
    const int* dims;
    cplx* work;               // global fallback: 2 n^2 per sector at rho_off * 2
    int smem_max_n;
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void __launch_bounds__(EIG_THREADS) k_herm_jacobi(EigArgs ea) {
    extern __shared__ double2 smem[];
    const int sct = blockIdx.x;
    const int n = ea.dims[sct];
    const int tid = threadIdx.x;
    double2* A;
    double2* V;
    if (n <= ea.smem_max_n) {
        A = smem;
        V = smem + n * n;
    } else {
        A = ea.work + 2 * ea.rho_off[sct];
        V = A + (int64_t)n * n;
    }
    __shared__ int pp[128], qq[128];
    __shared__ double cs[128];
    __shared__ double2 sn[128];   // s * e^{i theta}
    __shared__ double red[EIG_THREADS / 32];
    __shared__ double stop_flag;
    const cplx* R = ea.rho + ea.rho_off[sct];
    for (int e = tid; e < n * n; e += EIG_THREADS) {
        const int r = e / n, c = e % n;
        A[e] = R[e];
        V[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    const int P = n + (n & 1);   // players of the round-robin (one dummy when n is odd)
    const int npair = P / 2;
    // threshold Jacobi: rotate only |a_pq| above 2 eps ||A||_F (smaller entries are set to zero);
    // stop after a sweep without rotations
    __shared__ int rotated;
    double fro = 0.0;
    for (int e = tid; e < n * n; e += EIG_THREADS) { const double2 a = A[e]; fro += a.x * a.x + a.y * a.y; }
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0) red[tid >> 5] = fro;
    __syncthreads();
    if (tid == 0) {
        double f = 0.0;
        for (int k = 0; k < EIG_THREADS / 32; ++k) f += red[k];
        stop_flag = 2.220446049250313e-16 * sqrt(f);
    }
    __syncthreads();
    const double thr = stop_flag;
    for (int sweep = 0; sweep < 30 && n > 1; ++sweep) {
        __syncthreads();
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < P - 1; ++round) {
            // circle method: player P-1 meets `round`; (round+k, round-k) mod (P-1) for k >= 1
            for (int i = tid; i < npair; i += EIG_THREADS) {
                int p, q;
                if (i == 0) { p = P - 1; q = round; }
                else { p = (round + i) % (P - 1); q = (round - i + (P - 1)) % (P - 1); }
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0;
                double2 s = make_double2(0.0, 0.0);
                if (q < n) {
                    const double2 b = A[p * n + q];
                    const double ab = sqrt(b.x * b.x + b.y * b.y);
                    if (ab <= thr) {
                        A[p * n + q] = make_double2(0.0, 0.0);
                        A[q * n + p] = make_double2(0.0, 0.0);
                    } else {
                        rotated = 1;
                        const double a = A[p * n + p].x, d = A[q * n + q].x;
                        const double tau = (d - a) / (2.0 * ab);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        const double sv = t * c;
                        s = make_double2(sv * b.x / ab, sv * b.y / ab);   // s e^{i theta}, b = |b| e^{i theta}
                    }
                }
                pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
            }
            __syncthreads();
            // rows: A <- J^H A,  new A_p. = c A_p. - s u A_q.,  new A_q. = conj(s u) A_p. + c A_q.
            for (int e = tid; e < npair * n; e += EIG_THREADS) {
                const int i = e / n, k = e % n;
                const int p = pp[i], q = qq[i];
                if (q >= n) continue;
                const double c = cs[i];
                const double2 s = sn[i];
                const double2 ap = A[p * n + k], aq = A[q * n + k];
                const double2 t1 = cm(s, aq), t2 = cm(cconj(s), ap);
                A[p * n + k] = make_double2(c * ap.x - t1.x, c * ap.y - t1.y);
                A[q * n + k] = make_double2(t2.x + c * aq.x, t2.y + c * aq.y);
            }
            __syncthreads();
            // columns: A <- A J and V <- V J,  new X_.p = c X_.p - conj(s u) X_.q,  new X_.q = s u X_.p + c X_.q
            for (int e = tid; e < npair * n; e += EIG_THREADS) {
                const int i = e / n, k = e % n;
                const int p = pp[i], q = qq[i];
                if (q >= n) continue;
                const double c = cs[i];
                const double2 s = sn[i], sc = cconj(s);
                double2 xp = A[k * n + p], xq = A[k * n + q];
                double2 t1 = cm(sc, xq), t2 = cm(s, xp);
                A[k * n + p] = make_double2(c * xp.x - t1.x, c * xp.y - t1.y);
                A[k * n + q] = make_double2(t2.x + c * xq.x, t2.y + c * xq.y);
                xp = V[k * n + p]; xq = V[k * n + q];
                t1 = cm(sc, xq); t2 = cm(s, xp);
                V[k * n + p] = make_double2(c * xp.x - t1.x, c * xp.y - t1.y);
                V[k * n + q] = make_double2(t2.x + c * xq.x, t2.y + c * xq.y);
            }
            __syncthreads();
        }
        __syncthreads();
        if (!rotated) break;
    }
    // sort descending by rank counting (ties broken by index), write eigenpairs
    double* ev = ea.evals + ea.ev_off[sct];
    cplx* U = ea.evecs + ea.rho_off[sct];
    for (int j = tid; j < n; j += EIG_THREADS) {
        const double lj = A[j * n + j].x;
        int rank = 0;
        for (int m = 0; m < n; ++m) {
            const double lm = A[m * n + m].x;
            rank += (lm > lj) || (lm == lj && m < j);
        }
        ev[rank] = lj;
        for (int r = 0; r < n; ++r) U[r * n + rank] = V[r * n + j];
    }
}

}  // namespace

int density_matrix(tdmrg_ctx* c, int nt, const int32_t* Q, const cplx* const* psi, const double* w, cplx* rho) {
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
    k_weight_scale<<<1, 32 * 12, 0, s>>>(c->red, nt, c->dscale, wl);
    c->launches++;
    // task list: one task per left sector
    TaskList tl;
    int64_t off = 0;
    for (size_t qi = 0; qi < L.dim.size(); ++qi) {
        Task tk{};
        tk.c_off = off; tk.c_buf = BUF_OUT; tk.ldc = L.dim[qi]; tk.M = L.dim[qi]; tk.N = L.dim[qi]; tk.beta = 0;
        tk.seg_begin = (int)tl.segs.size();
        for (int l = 0; l < nt; ++l) {
            int ri = R.find(Q[2 * l] - L.nup[qi], Q[2 * l + 1] - L.ndn[qi]);
            if (ri < 0) continue;
            // offset of Psi_l(q) inside target l
            int64_t po = 0;
            for (size_t k = 0; k < qi; ++k) {
                int rk = R.find(Q[2 * l] - L.nup[k], Q[2 * l + 1] - L.ndn[k]);
                if (rk >= 0) po += (int64_t)L.dim[k] * R.dim[rk];
            }
            Seg sg{};
            sg.a_off = po; sg.a_buf = (int8_t)(BUF_EXTRA0 + l); sg.lda = R.dim[ri];
            sg.b_off = po; sg.b_buf = (int8_t)(BUF_EXTRA0 + l); sg.ldb = R.dim[ri]; sg.opb = OPB_C;
            sg.K = R.dim[ri]; sg.scale = make_double2(1.0, 0.0); sg.dscale = l;
            tl.segs.push_back(sg);
        }
        tk.seg_end = (int)tl.segs.size();
        tl.tasks.push_back(tk);
        off += (int64_t)L.dim[qi] * L.dim[qi];
    }
    make_tiles(tl, kTileF64, kTileF64, kSplitK);
    int rc = upload(c, tl);
    if (rc) { release(c, tl); return rc; }
    GemmArgs a{};
    a.tasks = tl.d_tasks; a.segs = tl.d_segs; a.tiles = tl.d_tiles; a.ntiles = (int)tl.tiles.size();
    a.partials = tl.d_partials; a.counters = tl.d_counters;
    a.bufs[BUF_OPS] = c->pool;
    a.bufs[BUF_OUT] = rho;
    for (int l = 0; l < nt; ++l) a.bufs[BUF_EXTRA0 + l] = const_cast<cplx*>(psi[l]);
    a.dscale = c->dscale;
    cudaError_t e = launch_gemm_f64(a, s, nullptr, 0);
    c->launches++;
    // the task list is freed after the stream reaches this point
    cudaStreamSynchronize(s);
    release(c, tl);
    return cuda_check(c, e, "density_matrix launch");
}

int rho_eig(tdmrg_ctx* c, const cplx* rho, double* evals, cplx* evecs) {
    const Side& L = c->side[0];
    const int ns = (int)L.dim.size();
    std::vector<int64_t> ro(ns), eo(ns);
    int64_t r = 0, e = 0;
    int maxn = 0;
    for (int k = 0; k < ns; ++k) {
        ro[k] = r; eo[k] = e;
        r += (int64_t)L.dim[k] * L.dim[k];
        e += L.dim[k];
        maxn = std::max(maxn, L.dim[k]);
    }
    if (maxn > 2 * 128) return fail(c, TDMRG_EINVAL, "rho_eig: sector dimension above 256");
    const int smem_max_n = 82;   // A and V: 2 * 82^2 * 16 B = 210 KB of shared memory
    size_t smem = (size_t)2 * std::min(maxn, smem_max_n) * std::min(maxn, smem_max_n) * sizeof(cplx);
    int64_t* d_ro = nullptr;
    int64_t* d_eo = nullptr;
    int* d_dims = nullptr;
    cplx* work = nullptr;
    int rc = dev_alloc(c, (void**)&d_ro, ns * sizeof(int64_t), "rho_eig tables");
    if (!rc) rc = dev_alloc(c, (void**)&d_eo, ns * sizeof(int64_t), "rho_eig tables");
    if (!rc) rc = dev_alloc(c, (void**)&d_dims, ns * sizeof(int), "rho_eig tables");
    if (!rc && maxn > smem_max_n) rc = dev_alloc(c, (void**)&work, 2 * r * sizeof(cplx), "rho_eig workspace");
    if (!rc) rc = cuda_check(c, cudaMemcpy(d_ro, ro.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice), "rho_eig upload");
    if (!rc) rc = cuda_check(c, cudaMemcpy(d_eo, eo.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice), "rho_eig upload");
    if (!rc) rc = cuda_check(c, cudaMemcpy(d_dims, L.dim.data(), ns * sizeof(int), cudaMemcpyHostToDevice), "rho_eig upload");
    if (!rc) rc = cuda_check(c, cudaFuncSetAttribute(k_herm_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "rho_eig smem");
    if (!rc) {
        EigArgs ea{rho, evals, evecs, d_ro, d_eo, d_dims, work, smem_max_n};
        k_herm_jacobi<<<ns, EIG_THREADS, smem, c->stream>>>(ea);
        c->launches++;
        rc = cuda_check(c, cudaGetLastError(), "rho_eig launch");
        cudaStreamSynchronize(c->stream);
    }
    dev_free(c, d_ro, ns * sizeof(int64_t));
    dev_free(c, d_eo, ns * sizeof(int64_t));
    dev_free(c, d_dims, ns * sizeof(int));
    dev_free(c, work, 2 * r * sizeof(cplx));
    return rc;
}

}  // namespace tdmrg
