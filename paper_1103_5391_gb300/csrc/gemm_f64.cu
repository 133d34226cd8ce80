// Grouped complex FP64 GEMM for the sector-pair products of H psi (Sec. IV, Hamiltonian
// connections), the excitation operators (Eq. b), and rho_L (Eq. rdensitymatrix).
//
// One CTA computes one 16 x 16 output tile of one task over a range of its segments:
//     C_tile = (beta ? C_tile : 0) + sum_segments scale * A_seg * op(B_seg)
// For a Hermitian result (rho_L and the Gram matrices of the eigen-refinement) only the tiles on and
// below the diagonal are computed and each off-diagonal tile is also stored conjugate-transposed.
// On GB300 FP64 runs at about 1 TFLOP/s for the whole chip (scalar DFMA and the FP64 MMA alike),
// i.e. about 7 GFLOP/s per SM, so the kernel is organised for balance rather than data reuse:
//   - small (16 x 16) tiles so that every sector pair spreads over many SMs;
//   - each of the four warps owns one 8 x 8 sub-block over the whole K range (no cross-warp sums),
//     and negated or conjugated operands are staged by integer sign flips, so that the FP64 pipe
//     runs the MMAs and little else;
//   - tasks with a long K (many segments) are split across CTAs along segment boundaries; each part
//     stores its partial tile and the last part to arrive (atomic ticket) sums all parts in index
//     order, so results do not depend on scheduling.
// Complex products use the FP64 tensor MMA (mma.sync m8n8k4 f64): four real MMAs per complex MMA.
//
// The correction mode (kCorr) serves the update W' = (I + D) W of the eigen-refinement, where D is small
// (|D| <= 1e-3, ~1e-7 in the last iteration): D W runs in FP32 (each CTA accumulates one K part of at
// most a few dozen terms; parts are summed in FP64), so its rounding is ~1e-7 of |D| |W|, and the
// epilogue adds W itself in FP64.  W is the B operand of the task's first segment.  FP32 accumulation
// is what limits the accuracy, so this mode suits small corrections only, not full products.
#include "internal.h"

namespace tdmrg {
namespace {

constexpr int TS = kTileF64;     // 16
constexpr int KC = 16;
constexpr int PAD = TS + 4;      // row stride of the staged planes (conflict-free fragment loads)

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// Sign flip of a double on the integer pipe: FP64 arithmetic is scarce on this GPU, so negated and
// conjugated operands are formed while staging instead of by FP64 instructions.
__device__ __forceinline__ double neg(double x) { return __longlong_as_double(__double_as_longlong(x) ^ (1ll << 63)); }

// acc += a * b for complex a = (ar, ai), b = (br, bi) in FP32
__device__ __forceinline__ void cfma32(float& cr, float& ci, float ar, float ai, float br, float bi) {
    cr = fmaf(ar, br, fmaf(-ai, bi, cr));
    ci = fmaf(ar, bi, fmaf(ai, br, ci));
}

template <bool kCorr>
__global__ void __launch_bounds__(128) gemm_f64_kernel(GemmArgs args, const int* skip_flag, int skip_step) {
    pdl_enter();
    if (skip_flag != nullptr && skip_step >= *skip_flag) return;   // Krylov space already complete
    __shared__ double Are[kCorr ? 1 : TS][PAD], Aim[kCorr ? 1 : TS][PAD], Ain[kCorr ? 1 : TS][PAD];   // Ain = -Aim
    __shared__ double Bre[kCorr ? 1 : KC][PAD], Bim[kCorr ? 1 : KC][PAD];
    // correction mode: FP32 operands, [0] real and [1] imaginary
    __shared__ float fA[2][kCorr ? TS : 1][PAD], fB[2][kCorr ? KC : 1][PAD];
    __shared__ int last;

    const Tile tile = args.tiles[blockIdx.x];
    const Task task = args.tasks[tile.task];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int m0 = tile.m0, n0 = tile.n0;
    const int Mt = min(TS, task.M - m0), Nt = min(TS, task.N - n0);
    // warp w owns the 8 x 8 sub-block (w / 2, w % 2) over the whole K range: no cross-warp sums
    const int bi = warp >> 1, bj = warp & 1;
    const bool active = (8 * bi < Mt) && (8 * bj < Nt);
    double cre[2] = {0.0, 0.0}, cim[2] = {0.0, 0.0};
    float fre[2] = {0.f, 0.f}, fim[2] = {0.f, 0.f};

    for (int s = tile.seg_lo; s < tile.seg_hi; ++s) {
        const Seg seg = args.segs[s];
        const cplx* __restrict__ A = args.bufs[seg.a_buf] + seg.a_off;
        const cplx* __restrict__ B = args.bufs[seg.b_buf] + seg.b_off;
        double sr = seg.scale.x, si = seg.scale.y;
        if (seg.dscale >= 0) {
            const double d = args.dscale[seg.dscale];
            sr *= d; si *= d;
        }
        if (seg.dcoef >= 0 && args.dcoef != nullptr) {   // run-time coefficient of a connection term
            const cplx d = args.dcoef[seg.dcoef];
            const double tr = sr * d.x - si * d.y;
            si = sr * d.y + si * d.x;
            sr = tr;
        }
        const bool scaled = !(sr == 1.0 && si == 0.0);
        const bool conj = seg.opb == OPB_C;
        const bool a_real = (seg.rflags & 1) != 0, b_real = (seg.rflags & 2) != 0;   // skip zero imaginary products
        for (int k0 = 0; k0 < seg.K; k0 += KC) {
            const int kc = min(KC, seg.K - k0);
#pragma unroll
            for (int u = 0; u < 2; ++u) {             // A chunk TS x KC: threads along k (along m when transposed)
                const int e = tid + 128 * u;
                const int r = seg.opa ? e % TS : e / KC, k = seg.opa ? e / TS : e % KC;
                double2 v = make_double2(0.0, 0.0);
                if (r < Mt && k < kc)
                    v = seg.opa ? A[(int64_t)(k0 + k) * seg.lda + m0 + r] : A[(int64_t)(m0 + r) * seg.lda + k0 + k];
                if (seg.opa == 2) v.y = neg(v.y);
                if (scaled) v = make_double2(sr * v.x - si * v.y, sr * v.y + si * v.x);
                if constexpr (kCorr) {
                    fA[0][r][k] = (float)v.x;
                    fA[1][r][k] = (float)v.y;
                } else {
                    Are[r][k] = v.x;
                    Aim[r][k] = v.y;
                    Ain[r][k] = neg(v.y);
                }
            }
            if (seg.opb == OPB_N || seg.opb == OPB_CN) {   // B[k][n] at B[k*ldb + n] (conjugated for 'CN'): threads along n
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = tid + 128 * u, k = e / TS, n = e % TS;
                    double2 v = make_double2(0.0, 0.0);
                    if (k < kc && n < Nt) v = B[(int64_t)(k0 + k) * seg.ldb + n0 + n];
                    if (seg.opb == OPB_CN) v.y = neg(v.y);
                    if constexpr (kCorr) {
                        fB[0][k][n] = (float)v.x;
                        fB[1][k][n] = (float)v.y;
                    } else {
                        Bre[k][n] = v.x;
                        Bim[k][n] = v.y;
                    }
                }
            } else {                                  // B[k][n] at B[n*ldb + k] (conjugated for 'C')
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = tid + 128 * u, n = e / KC, k = e % KC;
                    double2 v = make_double2(0.0, 0.0);
                    if (k < kc && n < Nt) v = B[(int64_t)(n0 + n) * seg.ldb + k0 + k];
                    if (conj) v.y = neg(v.y);
                    if constexpr (kCorr) {
                        fB[0][k][n] = (float)v.x;
                        fB[1][k][n] = (float)v.y;
                    } else {
                        Bre[k][n] = v.x;
                        Bim[k][n] = v.y;
                    }
                }
            }
            __syncthreads();
            if constexpr (kCorr) {
                if (active) {
                    const int rr = 8 * bi + gid;
                    for (int kk = 0; kk < kc; ++kk) {
                        const float ar = fA[0][rr][kk], ai = fA[1][rr][kk];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int cc = 8 * bj + 2 * tig + e;
                            cfma32(fre[e], fim[e], ar, ai, fB[0][kk][cc], fB[1][kk][cc]);
                        }
                    }
                }
            } else if (active) {
                if (a_real || b_real) {   // one operand real: two real MMAs per complex k-step
                    for (int kk = 0; kk < kc; kk += 4) {
                        const double ar = Are[8 * bi + gid][kk + tig], ai = Aim[8 * bi + gid][kk + tig];
                        const double br = Bre[kk + tig][8 * bj + gid], bm = Bim[kk + tig][8 * bj + gid];
                        dmma(cre[0], cre[1], ar, br);
                        if (a_real) dmma(cim[0], cim[1], ar, bm);
                        else dmma(cim[0], cim[1], ai, br);
                    }
                } else {
                    for (int kk = 0; kk < kc; kk += 4) {   // zero-padded beyond kc
                        const double ar = Are[8 * bi + gid][kk + tig], ai = Aim[8 * bi + gid][kk + tig];
                        const double an = Ain[8 * bi + gid][kk + tig];
                        const double br = Bre[kk + tig][8 * bj + gid], bm = Bim[kk + tig][8 * bj + gid];
                        dmma(cre[0], cre[1], ar, br);
                        dmma(cre[0], cre[1], an, bm);
                        dmma(cim[0], cim[1], ar, bm);
                        dmma(cim[0], cim[1], ai, br);
                    }
                }
            }
            __syncthreads();
        }
    }

    // this thread's two outputs: row 8 bi + gid, columns 8 bj + 2 tig + e
    const int r = 8 * bi + gid, col0 = 8 * bj + 2 * tig;
    double2 v[2] = {make_double2(cre[0], cim[0]), make_double2(cre[1], cim[1])};
    if constexpr (kCorr) {
        v[0] = make_double2((double)fre[0], (double)fim[0]);
        v[1] = make_double2((double)fre[1], (double)fim[1]);
    }
    if (tile.split >= 0) {
        // split-K: publish this part, the last part to arrive sums all parts in index order
        cplx* part = args.partials + ((int64_t)tile.split_base + tile.part) * (TS * TS);
        if (active) {
            part[r * TS + col0] = v[0];
            part[r * TS + col0 + 1] = v[1];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) last = (atomicAdd(args.counters + tile.split, 1) == tile.nparts - 1);
        __syncthreads();
        if (!last) return;
        __threadfence();
        if (active) {
            const cplx* base = args.partials + (int64_t)tile.split_base * (TS * TS);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                double2 t = make_double2(0.0, 0.0);
                for (int p = 0; p < tile.nparts; ++p) {
                    const double2 x = __ldcg(base + (int64_t)p * (TS * TS) + r * TS + col0 + e);
                    t.x += x.x; t.y += x.y;
                }
                v[e] = t;
            }
        }
        if (tid == 0) args.counters[tile.split] = 0;   // ready for the next launch
    }
    if (!active) return;
    cplx* __restrict__ C = args.bufs[task.c_buf] + task.c_off;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int col = col0 + e;
        if (r < Mt && col < Nt) {
            cplx* p = task.trans ? C + (int64_t)(n0 + col) * task.ldc + m0 + r : C + (int64_t)(m0 + r) * task.ldc + n0 + col;
            double2 x = v[e];
            if constexpr (kCorr) {   // (I + D) W: add W in FP64
                const Seg s0 = args.segs[task.seg_begin];
                const double2 w = args.bufs[s0.b_buf][s0.b_off + (int64_t)(m0 + r) * s0.ldb + n0 + col];
                x.x += w.x;
                x.y += w.y;
            }
            if (task.beta) {
                const double2 o = *p;
                x.x += o.x;
                x.y += o.y;
            }
            *p = x;
            if (task.herm && m0 != n0) C[(int64_t)(n0 + col) * task.ldc + m0 + r] = make_double2(x.x, neg(x.y));
        }
    }
}

}  // namespace

cudaError_t launch_gemm_f64(const GemmArgs& a, cudaStream_t s, const int* skip_flag, int skip_step, bool corr) {
    if (a.ntiles <= 0) return cudaSuccess;
    if (corr) launch_pdl(gemm_f64_kernel<true>, a.ntiles, 128, 0, s, a, skip_flag, skip_step);
    else launch_pdl(gemm_f64_kernel<false>, a.ntiles, 128, 0, s, a, skip_flag, skip_step);
    return cudaGetLastError();
}

}  // namespace tdmrg
