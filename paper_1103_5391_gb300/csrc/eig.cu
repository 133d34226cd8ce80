// Eigendecomposition of rho_L per left sector (truncation input of Sec. II.B), FP64 accurate.
//
// GB300 runs FP64 at about 1 TFLOP/s chip-wide (~7 GFLOP/s per SM), so an FP64 Jacobi on one SM per
// sector would take milliseconds for the largest sectors.  Instead:
//   1. seed: a cyclic two-sided Jacobi in FP32 per sector (one CTA per sector, parallel round-robin
//      ordering of disjoint rotations), giving eigenvectors X0 accurate to about 1e-6;
//   2. refine: iterative refinement for Hermitian eigenproblems (Ogita & Aishima, 2018), whose FP64
//      work is three grouped GEMMs per iteration spread over every SM:
//         G = X^H X,  S = X^H (rho X),  lambda_i = Re S_ii / Re G_ii,  R = I - G,
//         E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   if |lambda_i - lambda_j| > delta,
//         E_ij = R_ij / 2 otherwise (and on the diagonal),  delta = 2 (||S - diag(lambda)|| + ||rho|| ||R||),
//         X <- X (I + E);
//      convergence is quadratic; three iterations take the FP32 seed to FP64 accuracy, including
//      near-degenerate pairs that the first iteration treats as a cluster;
//   3. sort each sector's eigenpairs by descending eigenvalue.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int JT = 1024;  // threads of the FP32 Jacobi CTA (warps over rotation pairs, lanes over rows)
constexpr int kSmemMaxN = 112;
constexpr int kRefine = 3;       // refinement iterations   // A and V as float2 in shared memory: 2 * 112^2 * 8 B = 196 KB

struct EigTables {
    const int64_t* off;   // per sector: offset of its n x n block
    const int64_t* eoff;  // per sector: offset of its eigenvalues
    const int* dims;
};

__device__ __forceinline__ float2 cmf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// FP32 seed: X0 (unsorted columns) of each sector's rho block.
__global__ void __launch_bounds__(JT) k_jacobi32(const cplx* __restrict__ rho, cplx* __restrict__ X, EigTables tb,
                                                 float2* __restrict__ gwork) {
    extern __shared__ float2 fsm[];
    const int sct = blockIdx.x, n = tb.dims[sct], tid = threadIdx.x;
    const int64_t off = tb.off[sct];
    const int ld = n | 1;   // odd row stride: column accesses of a warp hit distinct banks
    float2* A;
    float2* V;
    if (n <= kSmemMaxN) { A = fsm; V = fsm + n * ld; }
    else { A = gwork + 4 * off; V = A + (int64_t)n * ld; }
    __shared__ int pp[256], qq[256];
    __shared__ float cs[256];
    __shared__ float2 sn[256];
    __shared__ float red[JT / 32];
    __shared__ float thr_s;
    __shared__ int rotated;
    const cplx* R = rho + off;
    for (int e = tid; e < n * n; e += JT) {
        const int r = e / n, cc = e % n;
        const double2 v = R[e];
        A[r * ld + cc] = make_float2((float)v.x, (float)v.y);
        V[r * ld + cc] = make_float2(r == cc ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    float fro = 0.f;
    for (int e = tid; e < n * n; e += JT) { const float2 a = A[(e / n) * ld + e % n]; fro += a.x * a.x + a.y * a.y; }
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0) red[tid >> 5] = fro;
    __syncthreads();
    if (tid == 0) {
        float f = 0.f;
        for (int k = 0; k < JT / 32; ++k) f += red[k];
        thr_s = 4.8e-7f * sqrtf(f);   // 4 eps_fp32 ||A||_F: above FP32 rounding noise, so sweeps terminate
    }
    __syncthreads();
    const float thr = thr_s;
    const int P = n + (n & 1), npair = P / 2;
    for (int sweep = 0; sweep < 12 && n > 1; ++sweep) {
        __syncthreads();
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < P - 1; ++round) {
            for (int i = tid; i < npair; i += JT) {
                int p, q;
                if (i == 0) { p = P - 1; q = round; }
                else { p = (round + i) % (P - 1); q = (round - i + (P - 1)) % (P - 1); }
                if (p > q) { int t = p; p = q; q = t; }
                float c = 1.f;
                float2 s = make_float2(0.f, 0.f);
                if (q < n) {
                    const float2 b = A[p * ld + q];
                    const float ab = sqrtf(b.x * b.x + b.y * b.y);
                    if (ab <= thr) {
                        A[p * ld + q] = make_float2(0.f, 0.f);
                        A[q * ld + p] = make_float2(0.f, 0.f);
                    } else {
                        rotated = 1;
                        const float a = A[p * ld + p].x, d = A[q * ld + q].x;
                        const float tau = (d - a) / (2.f * ab);
                        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
                        c = rsqrtf(1.f + t * t);
                        const float sv = t * c / ab;
                        s = make_float2(sv * b.x, sv * b.y);   // s e^{i theta}, b = |b| e^{i theta}
                    }
                }
                pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
            }
            __syncthreads();
            const int warp = tid >> 5, lane = tid & 31;
            for (int i = warp; i < npair; i += JT / 32) {   // rows: A <- J^H A
                const int p = pp[i], q = qq[i];
                if (q >= n) continue;
                const float c = cs[i];
                const float2 s = sn[i], sc = conjf2(s);
                for (int k = lane; k < n; k += 32) {
                    const float2 ap = A[p * ld + k], aq = A[q * ld + k];
                    const float2 t1 = cmf(s, aq), t2 = cmf(sc, ap);
                    A[p * ld + k] = make_float2(c * ap.x - t1.x, c * ap.y - t1.y);
                    A[q * ld + k] = make_float2(t2.x + c * aq.x, t2.y + c * aq.y);
                }
            }
            __syncthreads();
            for (int i = warp; i < npair; i += JT / 32) {   // columns: A <- A J, V <- V J
                const int p = pp[i], q = qq[i];
                if (q >= n) continue;
                const float c = cs[i];
                const float2 s = sn[i], sc = conjf2(s);
                for (int k = lane; k < n; k += 32) {
                    float2 xp = A[k * ld + p], xq = A[k * ld + q];
                    float2 t1 = cmf(sc, xq), t2 = cmf(s, xp);
                    A[k * ld + p] = make_float2(c * xp.x - t1.x, c * xp.y - t1.y);
                    A[k * ld + q] = make_float2(t2.x + c * xq.x, t2.y + c * xq.y);
                    xp = V[k * ld + p]; xq = V[k * ld + q];
                    t1 = cmf(sc, xq); t2 = cmf(s, xp);
                    V[k * ld + p] = make_float2(c * xp.x - t1.x, c * xp.y - t1.y);
                    V[k * ld + q] = make_float2(t2.x + c * xq.x, t2.y + c * xq.y);
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (!rotated) break;
    }
    cplx* Xs = X + off;
    for (int e = tid; e < n * n; e += JT) {
        const float2 v = V[(e / n) * ld + e % n];
        Xs[e] = make_double2(v.x, v.y);
    }
}

// Xh = X^H per sector.
__global__ void k_conj_transpose(const cplx* __restrict__ X, cplx* __restrict__ Xh, EigTables tb) {
    const int sct = blockIdx.x, n = tb.dims[sct];
    const int64_t off = tb.off[sct];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double2 v = X[off + (int64_t)j * n + i];
        Xh[off + e] = make_double2(v.x, -v.y);
    }
}

// One refinement step's correction: E1 = I + E from S, G; eigenvalue estimates into lam.
__global__ void __launch_bounds__(256) k_oa_update(const cplx* __restrict__ S, const cplx* __restrict__ G,
                                                   const double* __restrict__ rho_fro, cplx* __restrict__ E1,
                                                   double* __restrict__ lam, EigTables tb) {
    const int sct = blockIdx.x, n = tb.dims[sct], tid = threadIdx.x;
    const int64_t off = tb.off[sct];
    const int64_t eo = tb.eoff[sct];
    __shared__ double red[2][8];
    __shared__ double delta_s;
    for (int i = tid; i < n; i += blockDim.x) lam[eo + i] = S[off + (int64_t)i * n + i].x / G[off + (int64_t)i * n + i].x;
    __syncthreads();
    double offS = 0.0, rr = 0.0;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double2 s = S[off + e];
        if (i == j) s.x -= lam[eo + i];
        offS += s.x * s.x + s.y * s.y;
        double2 g = G[off + e];
        const double rx = (i == j ? 1.0 : 0.0) - g.x, ry = -g.y;
        rr += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) {
        offS += __shfl_xor_sync(0xffffffffu, offS, o);
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = offS; red[1][tid >> 5] = rr; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) { a += red[0][k]; b += red[1][k]; }
        delta_s = 2.0 * (sqrt(a) + rho_fro[sct] * sqrt(b));
    }
    __syncthreads();
    const double delta = delta_s;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double2 g = G[off + e];
        const double2 r = make_double2((i == j ? 1.0 : 0.0) - g.x, -g.y);
        double2 ev;
        const double li = lam[eo + i], lj = lam[eo + j];
        if (i != j && fabs(li - lj) > delta) {
            const double2 s = S[off + e];
            const double inv = 1.0 / (lj - li);
            ev = make_double2((s.x + lj * r.x) * inv, (s.y + lj * r.y) * inv);
        } else {
            ev = make_double2(0.5 * r.x, 0.5 * r.y);
        }
        if (i == j) ev.x += 1.0;
        E1[off + e] = ev;
    }
}

__global__ void k_rho_fro(const cplx* __restrict__ rho, double* __restrict__ fro, EigTables tb) {
    const int sct = blockIdx.x, n = tb.dims[sct];
    const int64_t off = tb.off[sct];
    double s = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) { const double2 v = rho[off + e]; s += v.x * v.x + v.y * v.y; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) a += red[k];
        fro[sct] = sqrt(a);
    }
}

// Descending order (ties by index); permute columns of X into U.
__global__ void k_eig_sort(const cplx* __restrict__ X, const double* __restrict__ lam, cplx* __restrict__ U,
                           double* __restrict__ evals, EigTables tb) {
    const int sct = blockIdx.x, n = tb.dims[sct];
    const int64_t off = tb.off[sct], eo = tb.eoff[sct];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double lj = lam[eo + j];
        int rank = 0;
        for (int m = 0; m < n; ++m) {
            const double lm = lam[eo + m];
            rank += (lm > lj) || (lm == lj && m < j);
        }
        evals[eo + rank] = lj;
        for (int r = 0; r < n; ++r) U[off + (int64_t)r * n + rank] = X[off + (int64_t)r * n + j];
    }
}

}  // namespace

// Buffer ids of the refinement GEMMs (all packed like rho).
enum { EB_RHO = BUF_EXTRA0, EB_X, EB_AX, EB_XH, EB_S, EB_G, EB_E, EB_Y };

int rho_eig(tdmrg_ctx* c, const cplx* rho, double* evals, cplx* evecs) {
    const Side& L = c->side[0];
    const int ns = (int)L.dim.size();
    EigWork& w = c->eig;
    cudaStream_t s = c->stream;
    if (!w.ready) {
        std::vector<int64_t> off(ns), eoff(ns);
        int64_t r = 0, e = 0;
        int maxn = 0;
        for (int k = 0; k < ns; ++k) {
            off[k] = r; eoff[k] = e;
            r += (int64_t)L.dim[k] * L.dim[k];
            e += L.dim[k];
            maxn = std::max(maxn, L.dim[k]);
        }
        if (maxn > 2 * 256) return fail(c, TDMRG_EINVAL, "rho_eig: sector dimension above 512");
        w.nrho = r; w.nev = e; w.maxn = maxn; w.ns = ns;
        int rc = dev_alloc(c, (void**)&w.tables, (size_t)ns * (2 * sizeof(int64_t) + sizeof(int)), "eig tables");
        if (!rc) rc = dev_alloc(c, (void**)&w.buf, (size_t)6 * r * sizeof(cplx), "eig workspace");
        if (!rc) rc = dev_alloc(c, (void**)&w.lam, (size_t)e * sizeof(double), "eig workspace");
        if (!rc) rc = dev_alloc(c, (void**)&w.fro, (size_t)ns * sizeof(double), "eig workspace");
        if (!rc && maxn > kSmemMaxN) rc = dev_alloc(c, (void**)&w.gwork, (size_t)4 * r * sizeof(float2), "eig workspace");
        if (rc) return rc;
        std::vector<unsigned char> host((size_t)ns * (2 * sizeof(int64_t) + sizeof(int)));
        memcpy(host.data(), off.data(), ns * sizeof(int64_t));
        memcpy(host.data() + ns * sizeof(int64_t), eoff.data(), ns * sizeof(int64_t));
        memcpy(host.data() + 2 * ns * sizeof(int64_t), L.dim.data(), ns * sizeof(int));
        rc = cuda_check(c, cudaMemcpy(w.tables, host.data(), host.size(), cudaMemcpyHostToDevice), "eig tables");
        if (rc) return rc;
        // task lists: AX = rho X; S = Xh AX and G = Xh X; Y = X E1
        auto one = [&](TaskList& tl, int cbuf, int abuf, int bbuf, int cbuf2, int abuf2, int bbuf2) {
            tl.tasks.clear(); tl.segs.clear();
            for (int k = 0; k < ns; ++k) {
                const int n = L.dim[k];
                for (int rep = 0; rep < (cbuf2 >= 0 ? 2 : 1); ++rep) {
                    Task t{};
                    t.c_off = off[k]; t.c_buf = (int8_t)(rep ? cbuf2 : cbuf); t.ldc = n; t.M = n; t.N = n; t.beta = 0;
                    t.seg_begin = (int)tl.segs.size();
                    Seg sg{};
                    sg.a_off = off[k]; sg.a_buf = (int8_t)(rep ? abuf2 : abuf); sg.lda = n;
                    sg.b_off = off[k]; sg.b_buf = (int8_t)(rep ? bbuf2 : bbuf); sg.ldb = n; sg.opb = OPB_N;
                    sg.K = n; sg.scale = make_double2(1.0, 0.0); sg.dscale = -1;
                    tl.segs.push_back(sg);
                    t.seg_end = (int)tl.segs.size();
                    tl.tasks.push_back(t);
                }
            }
            make_tiles(tl, kTileF64, kTileF64, kSplitK);
            return upload(c, tl);
        };
        // the opt-in is a property of the kernel on the device, shared by every context: always the maximum
        rc = cuda_check(c, cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)((size_t)2 * kSmemMaxN * (kSmemMaxN | 1) * sizeof(float2))),
                        "eig smem");
        if (!rc) rc = one(w.tl_ax, EB_AX, EB_RHO, EB_X, -1, -1, -1);
        if (!rc) rc = one(w.tl_sg, EB_S, EB_XH, EB_AX, EB_G, EB_XH, EB_X);
        if (!rc) rc = one(w.tl_y, EB_Y, EB_X, EB_E, -1, -1, -1);
        if (rc) return rc;
        w.ready = true;
    }
    EigTables tb{(const int64_t*)w.tables, (const int64_t*)w.tables + ns, (const int*)((const int64_t*)w.tables + 2 * ns)};
    cplx* X = w.buf;
    cplx* AX = w.buf + w.nrho;
    cplx* Xh = w.buf + 2 * w.nrho;
    cplx* S = w.buf + 3 * w.nrho;
    cplx* G = w.buf + 4 * w.nrho;
    cplx* E1 = w.buf + 5 * w.nrho;
    cplx* Y = evecs;   // ping-pong with the caller's output, which receives the sorted result at the end
    const int sm = std::min(w.maxn, kSmemMaxN);
    const size_t smem = (size_t)2 * sm * (sm | 1) * sizeof(float2);
    k_rho_fro<<<ns, 256, 0, s>>>(rho, w.fro, tb);
    k_jacobi32<<<ns, JT, smem, s>>>(rho, X, tb, w.gwork);
    c->launches += 2;
    GemmArgs a{};
    a.dscale = c->dscale;
    a.bufs[EB_RHO] = const_cast<cplx*>(rho);
    a.bufs[EB_AX] = AX; a.bufs[EB_XH] = Xh; a.bufs[EB_S] = S; a.bufs[EB_G] = G; a.bufs[EB_E] = E1;
    auto gemm = [&](TaskList& tl) {
        a.tasks = tl.d_tasks; a.segs = tl.d_segs; a.tiles = tl.d_tiles; a.ntiles = (int)tl.tiles.size();
        a.partials = tl.d_partials; a.counters = tl.d_counters;
        c->launches++;
        return launch_gemm_f64(a, s, nullptr, 0);
    };
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < kRefine && e == cudaSuccess; ++it) {
        a.bufs[EB_X] = X; a.bufs[EB_Y] = Y;
        e = gemm(w.tl_ax);
        k_conj_transpose<<<ns, 256, 0, s>>>(X, Xh, tb);
        if (e == cudaSuccess) e = gemm(w.tl_sg);
        k_oa_update<<<ns, 256, 0, s>>>(S, G, w.fro, E1, w.lam, tb);
        if (e == cudaSuccess) e = gemm(w.tl_y);
        c->launches += 2;
        std::swap(X, Y);
    }
    // X holds the refined vectors; with an odd number of swaps X == evecs, so sort from a copy
    if (X == evecs) {
        e = cudaMemcpyAsync(w.buf + 5 * w.nrho, evecs, (size_t)w.nrho * sizeof(cplx), cudaMemcpyDeviceToDevice, s);
        X = w.buf + 5 * w.nrho;
    }
    if (e == cudaSuccess) {
        k_eig_sort<<<ns, 128, 0, s>>>(X, w.lam, evecs, evals, tb);
        c->launches++;
        e = cudaGetLastError();
    }
    return cuda_check(c, e, "rho_eig launch");
}

void release_eig(tdmrg_ctx* c) {
    EigWork& w = c->eig;
    release(c, w.tl_ax); release(c, w.tl_sg); release(c, w.tl_y);
    const int ns = w.ns;
    dev_free(c, w.tables, (size_t)ns * (2 * sizeof(int64_t) + sizeof(int)));
    dev_free(c, w.buf, (size_t)6 * w.nrho * sizeof(cplx));
    dev_free(c, w.lam, (size_t)w.nev * sizeof(double));
    dev_free(c, w.fro, (size_t)ns * sizeof(double));
    dev_free(c, w.gwork, (size_t)4 * w.nrho * sizeof(float2));
    w = EigWork();
}

}  // namespace tdmrg
